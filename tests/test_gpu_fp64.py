"""FP64 GPU path vs the FP64 oracle, stage by stage, through the C ABI.

Bar: relative Frobenius error <= 1e-10 on the Gram, the Cholesky factor,
G^-1, Recon and the images (the FP64 target of the workload definition).
Sizes are chosen so the oracle finishes in seconds while the GPU kernels
still run several 64-wide tiles and a ragged tail.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.pinv_oracle as O  # noqa: E402
from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402
from tests._ref import oracle_all, rel  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()


def _plan(p, **kw):
    from paper_2410_06129_gb300.plan import Plan
    kw.setdefault("keep_gram", True)
    return Plan.from_inputs(p, **kw)


def _check_all_stages(p, tol=TOL, **kw):
    ref = oracle_all(p)
    pl = _plan(p, **kw).build()
    G = pl.export(L.EXPORT_GRAM).cpu().numpy()
    Lg = pl.export(L.EXPORT_CHOL).cpu().numpy()
    Gi = pl.export(L.EXPORT_GINV).cpu().numpy()
    R = pl.export(L.EXPORT_RECON).cpu().numpy()
    d = torch.from_numpy(p.data).cuda()
    x = pl.apply(d).cpu().numpy()
    info = pl.info()
    assert abs(info["lambda_abs"] - ref.lam) <= 1e-12 * ref.lam
    assert rel(np.tril(G), np.tril(ref.G)) < tol
    assert rel(Lg, ref.L) < tol
    assert rel(Gi, ref.Ginv) < tol
    assert rel(R, ref.R) < tol
    assert rel(x, ref.images) < tol
    assert info["min_pivot"] ** 2 >= ref.lam * (1 - 1e-9)
    pl.close()
    return ref


def test_cfg1_reduced_ragged():
    """Single coil spiral, N = 400 (6 tiles of 64 + a tail of 16)."""
    p = synth.make_plan(20, 1, "spiral", 2, 1001, 1e-3, samples=800, interleaves=1)
    _check_all_stages(p)


def test_cfg1_full_size():
    """Workload 1 at its full size: 32x32, one spiral of 2048 samples."""
    _check_all_stages(synth.config(1))


def test_coils_and_b0():
    """8 coils (Hadamard coil epilogue) and a B0 map (per-readout time table)."""
    p = synth.make_plan(16, 8, "radial", 3, 1500, 1e-4, b0=True, spokes=24, per_spoke=40)
    _check_all_stages(p)


def test_cfg2_reduced():
    """Workload 2 shrunk to 24x24: 8 coils, 4 interleaved spirals, lambda_rel 1e-4."""
    _check_all_stages(synth.config(2, reduced=True))


def test_factor_only_apply_matches_recon():
    """Section 3.3: G^-1 (sum_c E_c^H d_c) without forming Recon."""
    p = synth.make_plan(16, 4, "spiral", 3, 1601, 1e-3, samples=512, interleaves=2, b0=True)
    ref = oracle_all(p)
    pl = _plan(p, recon_mode=L.RECON_NONE).build()
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    assert rel(x, ref.images) < TOL
    with pytest.raises(L.PinvError, match="UNSUPPORTED"):
        pl.export(L.EXPORT_RECON)


def test_complex64_data_path():
    p = synth.make_plan(16, 2, "spiral", 5, 1701, 1e-3, samples=512, interleaves=2)
    ref = oracle_all(p)
    pl = _plan(p).build()
    d32 = torch.from_numpy(p.data.astype(np.complex64)).cuda()
    x = pl.apply(d32)
    assert x.dtype == torch.complex64
    ref32 = O.reconstruct(ref.R, O.data_columns(p.data.astype(np.complex64))).T
    assert rel(x.cpu().numpy(), ref32) < 1e-6


def test_voxel_mask():
    """Explicit voxel list (circular field-of-view mask, Section 4.4)."""
    side = 16
    p = synth.make_plan(side, 2, "spiral", 2, 1801, 1e-3, samples=512, interleaves=2)
    r = synth.voxel_positions((side, side))
    keep = np.nonzero(np.sum(r ** 2, axis=1) <= 0.45 ** 2)[0]
    vox = O.voxel_positions((side, side))[keep]
    E = O.encode(p.traj, vox, p.coil_maps[:, keep], None, None)
    lam = O.lambda_abs(E, p.lambda_rel)
    Rm, _ = O.recon_matrix(E, lam)
    x_ref = O.reconstruct(Rm, O.data_columns(p.data)).T
    from paper_2410_06129_gb300.plan import Plan
    pl = Plan((side, side), p.traj, p.coil_maps[:, keep], lam=p.lambda_rel, voxel_index=keep).build()
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    assert x.shape == (2, keep.size)
    assert rel(x, x_ref) < TOL


def test_three_dimensional_grid():
    rng = np.random.default_rng(5)
    dims = (6, 5, 4)
    N = int(np.prod(dims))
    k = rng.uniform(-2.5, 2.5, size=(2 * N, 3))
    vox = O.voxel_positions(dims)
    E = O.encode(k, vox)
    lam = O.lambda_abs(E, 1e-3)
    Rm, _ = O.recon_matrix(E, lam)
    d = rng.standard_normal((2, 1, 2 * N)) + 1j * rng.standard_normal((2, 1, 2 * N))
    x_ref = O.reconstruct(Rm, O.data_columns(d)).T
    from paper_2410_06129_gb300.plan import Plan
    pl = Plan(dims, k, lam=1e-3).build()
    x = pl.apply(torch.from_numpy(d).cuda()).cpu().numpy()
    assert rel(x, x_ref) < TOL


def test_not_positive_definite_reported():
    """lambda = 0 and a voxel no coil sees: G has an exactly zero pivot -> NOT_PD, no fault."""
    from paper_2410_06129_gb300.plan import Plan
    p = synth.make_plan(12, 2, "spiral", 1, 1901, 0.0, samples=512, interleaves=1)
    maps = p.coil_maps.copy()
    maps[:, 70] = 0.0
    pl = Plan(p.dims, p.traj, maps, lam=0.0, lambda_mode=L.LAMBDA_ABS)
    with pytest.raises(L.PinvError, match="NOT_PD"):
        pl.build()
    assert pl.info()["info"] == 70
    with pytest.raises(L.PinvError, match="NOT_BUILT"):
        pl.apply(torch.zeros((1, 1024), dtype=torch.complex128, device="cuda"))


def test_zero_frames_and_rebuild():
    p = synth.make_plan(8, 1, "spiral", 1, 1902, 1e-3, samples=128, interleaves=1)
    pl = _plan(p).build()
    out = pl.apply(torch.zeros((0, 128), dtype=torch.complex128, device="cuda"))
    assert out.shape == (0, 64)
    x1 = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    pl.build()
    x2 = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    assert np.array_equal(x1, x2)
