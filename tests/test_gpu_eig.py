"""Gram eigendecomposition and truncated reconstruction (pinv_plan_eig,
pinv_tsvd_apply) against the oracle (Section 2.1).

Bars: FP64 plans: eigenvalues within 1e-12 of the largest; eigenvectors
orthonormal and reconstructing E^H E to 1e-12, and spanning the oracle's
eigenvectors (projector distance) where eigenvalues are well separated;
truncated images within 1e-10 (NRMSE) of the oracle's, ranks identical and
condition numbers within 1e-10. With every eigenvalue kept and the plan's
lambda as loading the truncated reconstruction is the plan's own Tikhonov
image. A mixed plan's kept Gram carries its split-BF16 rounding (about 2e-6
relative per entry), which bounds its eigenvalues through ||dG||_F (Weyl).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.pinv_oracle as O  # noqa: E402
from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402
from tests._ref import oracle_all, rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()


def _plan(p, **kw):
    from paper_2410_06129_gb300.plan import Plan
    return Plan.from_inputs(p, keep_gram=True, **kw).build()


def _check_eig(pl, E, mu_tol=1e-12, vec_tol=1e-12):
    mu, P, sweeps = pl.eig()
    mu, P = mu.cpu().numpy(), P.cpu().numpy()
    mu_ref, P_ref = O.gram_eig(E)
    scale = mu_ref[0]
    assert np.max(np.abs(mu - mu_ref)) < mu_tol * scale
    G0 = E.conj().T @ E
    assert np.max(np.abs(P.conj().T @ P - np.eye(len(mu)))) < vec_tol * 10
    assert np.max(np.abs(P @ np.diag(mu) @ P.conj().T - G0)) < vec_tol * scale
    # eigenvectors of isolated eigenvalues agree up to phase: |p_i^H p_ref_i| = 1
    gap = np.minimum(np.abs(np.diff(mu_ref, prepend=np.inf)), np.abs(np.diff(mu_ref, append=-np.inf)))
    iso = np.where(gap > 1e-3 * scale)[0]
    assert len(iso) > 0
    overlap = np.abs(np.sum(P[:, iso].conj() * P_ref[:, iso], axis=0))
    assert np.max(np.abs(overlap - 1.0)) < 1e-8
    assert 1 <= sweeps <= 30
    return mu, P


def test_eig_fp64_matches_oracle():
    p = synth.make_plan(16, 3, "spiral", 1, 2601, 1e-3, samples=768, interleaves=2, b0=True)
    E = O.plan_encode(p)
    _check_eig(_plan(p, precision=L.FP64), E)


def test_eig_odd_size_radial():
    """N = 225: an odd count leaves one index idle in every round."""
    p = synth.make_plan(15, 2, "radial", 1, 2602, 1e-3, spokes=16, per_spoke=30)
    _check_eig(_plan(p, precision=L.FP64), O.plan_encode(p))


@pytest.mark.parametrize("side,coils,b0", [(16, 3, True), (15, 2, False)])
def test_eigenvalues_only_tridiagonal_path(side, coils, b0):
    """Without eigenvectors the spectrum comes from Householder tridiagonalisation
    and bisection: the same eigenvalues to 1e-12 of mu_1 (even and odd N)."""
    p = synth.make_plan(side, coils, "spiral", 1, 2607 + side, 1e-3, samples=3 * side * side, interleaves=2, b0=b0)
    E = O.plan_encode(p)
    pl = _plan(p, precision=L.FP64)
    mu, P, sweeps = pl.eig(vectors=False)
    assert P is None and sweeps == 0
    mu_ref, _ = O.gram_eig(E)
    assert np.max(np.abs(mu.cpu().numpy() - mu_ref)) < 1e-12 * mu_ref[0]
    mu_j, _, _ = pl.eig()
    assert np.max(np.abs(mu.cpu().numpy() - mu_j.cpu().numpy())) < 1e-12 * mu_ref[0]


@pytest.mark.parametrize("energy", [0.9, 0.99])
def test_tsvd_matches_oracle(energy):
    p = synth.make_plan(14, 2, "spiral", 3, 2603, 1e-3, samples=400, interleaves=2)
    E = O.plan_encode(p)
    pl = _plan(p, precision=L.FP64)
    mu, P, _ = pl.eig()
    mu_ref, P_ref = O.gram_eig(E)
    r_ref = O.tsvd_rank(mu_ref, energy)
    b = E.conj().T @ O.data_columns(p.data)
    want = O.tsvd_solve(mu_ref, P_ref, b, r_ref).T
    for dt in (torch.complex128, torch.complex64):
        d = torch.from_numpy(p.data).cuda().to(dt)
        x, r, kappa = pl.tsvd_apply(mu, P, d, energy=energy)
        assert x.shape == want.shape
        assert r == r_ref
        assert abs(kappa - O.tsvd_condition(mu_ref, r_ref)) < 1e-10 * kappa
        tol = 1e-10 if dt == torch.complex128 else 1e-6
        assert rel(x.to(torch.complex128).cpu().numpy(), want) < tol


def test_tsvd_full_energy_with_loading_is_the_tikhonov_image():
    """Every eigenvalue kept and mu + lambda inverted: the truncated reconstruction
    is the normal-equation image of Eq. 6."""
    p = synth.make_plan(12, 2, "spiral", 2, 2604, 1e-3, samples=300, interleaves=1)
    ref = oracle_all(p)
    pl = _plan(p, precision=L.FP64)
    mu, P, _ = pl.eig()
    x, r, _ = pl.tsvd_apply(mu, P, torch.from_numpy(p.data).cuda(), energy=1.0, lam=pl.info()["lambda_abs"])
    assert x.shape == ref.images.shape
    assert r == pl.n_vox
    assert rel(x.cpu().numpy(), ref.images) < 1e-10


def test_eig_needs_kept_gram():
    from paper_2410_06129_gb300.plan import Plan
    p = synth.make_plan(8, 1, "spiral", 1, 2605, 1e-3, samples=128, interleaves=1)
    pl = Plan.from_inputs(p, precision=L.FP64).build()
    with pytest.raises(L.PinvError, match="UNSUPPORTED"):
        pl.eig()


def test_eig_mixed_plan_split_precision_bound():
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")
    p = synth.make_plan(16, 2, "spiral", 1, 2606, 1e-3, samples=512, interleaves=2)
    E = O.plan_encode(p)
    pl = _plan(p, precision=L.MIXED_BF16X6)
    mu, _, _ = pl.eig(vectors=False)
    mu_ref, _ = O.gram_eig(E)
    # Weyl: |d mu| <= ||dG||_2 <= ||dG||_F, and the split-BF16 Gram's entries carry a
    # relative error below about 2e-6 (3 x DRAIN x 2^-24 from the accumulation groups)
    assert np.max(np.abs(mu.cpu().numpy() - mu_ref)) < 4e-6 * np.linalg.norm(E.conj().T @ E)
