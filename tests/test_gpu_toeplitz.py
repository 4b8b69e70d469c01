"""Exact Gram from the Toeplitz table, and the refinement residual r = E^H d - G x.

Without B0 and with voxels on the grid, (A^H A)[n][n'] depends only on the
grid offset between n and n' (from the encoding model, Eq. 2), so the plan
forms the exact Gram in FP64 from a (2n-1)-per-axis table. Bars: the exported
exact Gram equals the oracle's Gram, E^H E + lambda I from the explicit E, to
1e-13 relative (FP64 rounding, stored as double-float pairs); images after
refinement meet the mixed bar and agree with the E-generating double-float
residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.pinv_oracle as O  # noqa: E402
from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402
from tests._ref import oracle_all, rel  # noqa: E402

pytestmark = pytest.mark.gpu
GRAM_TOL = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _need_tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")


def _plan(*a, **kw):
    from paper_2410_06129_gb300.plan import Plan
    kw.setdefault("precision", L.MIXED_BF16X6)
    kw.setdefault("refine_residual", L.RESIDUAL_TOEPLITZ)
    return Plan(*a, **kw)


def _gram_ref(E, lam):
    return E.conj().T @ E + lam * np.eye(E.shape[1])


@pytest.mark.parametrize("side,coils,traj", [(20, 4, "spiral"), (16, 1, "radial"), (13, 3, "radial")])
def test_exact_gram_2d(side, coils, traj):
    """Ragged N (400, 256, 169), multi- and single-coil, spiral and radial."""
    p = synth.make_plan(side, coils, traj, 1, 2301 + side, 1e-3, samples=3 * side * side)
    ref = oracle_all(p)
    pl = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, refine_max_iters=1).build()
    G = pl.export(L.EXPORT_GRAM_EXACT).cpu().numpy()
    assert rel(G, _gram_ref(ref.E, ref.lam)) < GRAM_TOL
    assert rel(G, G.conj().T) < 1e-14


def test_exact_gram_3d_and_1d():
    rng = np.random.default_rng(7)
    for dims in [(6, 5, 4), (37,)]:
        N = int(np.prod(dims))
        k = rng.uniform(-0.5 * min(dims), 0.5 * min(dims), size=(2 * N, len(dims)))
        E = O.encode(k, O.voxel_positions(dims))
        lam = O.lambda_abs(E, 1e-3)
        pl = _plan(dims, k, lam=1e-3, refine_max_iters=1).build()
        G = pl.export(L.EXPORT_GRAM_EXACT).cpu().numpy()
        assert rel(G, _gram_ref(E, lam)) < GRAM_TOL, dims


def test_exact_gram_voxel_mask():
    side = 16
    p = synth.make_plan(side, 2, "spiral", 2, 2311, 1e-3, samples=512, interleaves=2)
    r = synth.voxel_positions((side, side))
    keep = np.nonzero(np.sum(r ** 2, axis=1) <= 0.45 ** 2)[0]
    E = O.encode(p.traj, O.voxel_positions((side, side))[keep], p.coil_maps[:, keep], None, None)
    lam = O.lambda_abs(E, p.lambda_rel)
    pl = _plan((side, side), p.traj, p.coil_maps[:, keep], lam=p.lambda_rel, voxel_index=keep,
               refine_max_iters=1).build()
    G = pl.export(L.EXPORT_GRAM_EXACT).cpu().numpy()
    assert rel(G, _gram_ref(E, lam)) < GRAM_TOL
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    Rm, _ = O.recon_matrix(E, lam)
    assert rel(x, O.reconstruct(Rm, O.data_columns(p.data)).T) <= 1e-4


@pytest.mark.parametrize("recon_mode", [L.RECON_STORE, L.RECON_NONE])
def test_images_cfg2_reduced(recon_mode):
    """Workload 2 shrunk to 24x24: the exact-Gram residual reaches the mixed bar
    and agrees with the E-generating double-float residual."""
    p = synth.config(2, reduced=True)
    ref = oracle_all(p)
    d = torch.from_numpy(p.data).cuda()
    pl = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, recon_mode=recon_mode,
               refine_max_iters=3).build()
    x = pl.apply(d).cpu().numpy()
    assert rel(x, ref.images) <= 1e-4
    pdf = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, recon_mode=recon_mode,
                refine_max_iters=3, refine_residual=L.RESIDUAL_DOUBLE_FLOAT).build()
    xdf = pdf.apply(d).cpu().numpy()
    assert rel(x, xdf) <= 1e-6


def test_stop_rule_uses_exact_residual():
    p = synth.config(2, reduced=True)
    ref = oracle_all(p)
    pl = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, refine_max_iters=8, refine_tol=1e-9).build()
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    info = pl.info()
    assert 1 <= info["last_refine_iters"] <= 8
    assert info["last_refine_resid"] <= 1e-9 or info["last_refine_iters"] == 8
    assert rel(x, ref.images) <= 1e-4


def test_toeplitz_needs_b0_free_plan():
    p = synth.make_plan(12, 2, "radial", 1, 2321, 1e-3, b0=True, spokes=12, per_spoke=24)
    with pytest.raises(L.PinvError, match="UNSUPPORTED"):
        _plan(p.dims, p.traj, p.coil_maps, p.b0_hz, p.times, lam=p.lambda_rel)
    pl = _plan(p.dims, p.traj, p.coil_maps, p.b0_hz, p.times, lam=p.lambda_rel,
               refine_residual=L.RESIDUAL_DOUBLE_FLOAT).build()
    with pytest.raises(L.PinvError, match="UNSUPPORTED"):
        pl.export(L.EXPORT_GRAM_EXACT)


def test_lean_plan_same_images_less_memory():
    """A lean plan drops G / L, the FP64 W and the double-float exact Gram after
    its build, and keeps no digit table of conj(A) (its E^H d forms the digits in
    every CTA): same images bit for bit, N^2 x 48 bytes plus the table's
    ceil(N / 128) x ceil(M_k / 16) x 48 KiB less device memory, no L / W /
    exact-Gram exports."""
    p = synth.config(2, reduced=True)
    d = torch.from_numpy(p.data).cuda()
    full = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, refine_max_iters=3).build()
    lean = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, refine_max_iters=3, lean=True).build()
    assert torch.equal(full.apply(d), lean.apply(d))
    N = p.n_vox
    table = -(-N // 128) * -(-p.n_samples // 16) * 6 * 8192
    assert full.info()["bytes_device"] - lean.info()["bytes_device"] == 48 * N * N + table
    for what in (L.EXPORT_CHOL, L.EXPORT_LINV, L.EXPORT_GINV, L.EXPORT_GRAM_EXACT):
        with pytest.raises(L.PinvError, match="UNSUPPORTED"):
            lean.export(what)
    lean.build()  # rebuild allocates the temporaries again
    assert torch.equal(full.apply(d), lean.apply(d))


@pytest.mark.parametrize("side,frames,samples", [(20, 40, 1200), (24, 16, 1152)])
def test_exact_tensor_core_adjoint_many_frames(side, frames, samples):
    """With 16 or more frames E^H d runs exactly on the tensor cores
    (fixed-point digits): ragged voxels (N = 400), frames (40 = 32 + 8) and
    samples. Images meet the mixed bar against the oracle and agree with the
    same frames applied a few at a time (double-float E^H d)."""
    p = synth.make_plan(side, 4, "spiral", frames, 2601 + side, 1e-4, samples=samples, interleaves=2)
    ref = oracle_all(p)
    pl = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, refine_max_iters=3).build()
    d = torch.from_numpy(p.data).cuda()
    x = pl.apply(d).cpu().numpy()
    assert rel(x, ref.images) <= 1e-5
    x_small = np.concatenate([pl.apply(d[i:i + 8]).cpu().numpy() for i in range(0, frames, 8)])
    assert rel(x, x_small) <= 1e-5


def test_exact_adjoint_digit_table_bit_identical(monkeypatch):
    """The digits of conj(A) written once per build and bulk-copied per stage are the
    digits the generating kernel forms in every CTA, summed in the same order: the
    images are the same bit for bit. 36 frames, ragged N = 400, 4 coils."""
    p = synth.make_plan(20, 4, "spiral", 36, 2609, 1e-4, samples=1000, interleaves=2)
    d = torch.from_numpy(p.data).cuda()

    def images():
        pl = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, refine_max_iters=3).build()
        return pl.apply(d).cpu().numpy()

    x_table = images()
    monkeypatch.setenv("PINV_ADJ_TABLE", "0")
    assert np.array_equal(images(), x_table)


@pytest.mark.parametrize("frames", [24, 150])
def test_tensor_core_recon_apply_matches_fp32_apply(frames):
    """Recon x data for 16 or more frames runs split-BF16 on the tensor cores
    (sample range split over tiles, frames in blocks of 128); without
    refinement it agrees with the FP32 SIMT product used for fewer frames."""
    p = synth.make_plan(20, 3, "spiral", frames, 2701, 1e-3, samples=1100, interleaves=2)
    pl = _plan(p.dims, p.traj, p.coil_maps, lam=p.lambda_rel, refine_max_iters=0).build()
    d = torch.from_numpy(p.data.astype(np.complex64)).cuda()
    x_tc = pl.apply(d).cpu().numpy()
    x_32 = np.concatenate([pl.apply(d[i:i + 8]).cpu().numpy() for i in range(0, frames, 8)])
    # both are FP32-class sums of M terms: bound sqrt(M) 2^-24 times the cancellation
    # ratio || |R| |d| || / || R d || of this product
    R = pl.export(L.EXPORT_RECON).cpu().numpy().astype(np.complex128)
    dd = p.data.astype(np.complex64).reshape(frames, -1).astype(np.complex128).T
    amp = np.linalg.norm(np.abs(R) @ np.abs(dd)) / np.linalg.norm(R @ dd)
    bound = 4 * np.sqrt(R.shape[1]) * 2.0 ** -24 * amp
    assert rel(x_tc, x_32) <= bound, (rel(x_tc, x_32), bound)
