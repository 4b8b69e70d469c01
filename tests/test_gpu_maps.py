"""SRF and noise maps (pinv_plan_map) against the oracle's definitions.

The oracle forms SRF = Recon x Encode (Eq. 9) and X = Recon Psi Recon^H
(Eq. 10) as full matrices from its explicit E and Recon; the maps are their
diagonals. Bars: FP64 plans 1e-10 (relative to the map's largest value);
mixed plans with the exact Gram 1e-6 (their G^-1 is refined); mixed plans
without it carry their split-precision factor, bounded here by
kappa(G) x the split rounding.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.pinv_oracle as O  # noqa: E402
from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402
from tests._ref import oracle_all  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()


def _err(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def _ref_maps(ref, psi):
    srf = np.real(np.diag(O.srf(ref.R, ref.E)))
    white = np.real(np.diag(O.noise_matrix(ref.R, np.eye(ref.E.shape[0]))))
    Mk = ref.E.shape[0] // psi.shape[0]
    colored = np.real(np.diag(O.noise_matrix(ref.R, np.kron(psi, np.eye(Mk)))))
    return srf, white, colored


def _psi(C, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((C, C)) + 1j * rng.standard_normal((C, C))
    return A @ A.conj().T / C + np.eye(C)


def _plan(p, **kw):
    from paper_2410_06129_gb300.plan import Plan
    return Plan.from_inputs(p, **kw).build()


def test_maps_fp64_with_b0():
    p = synth.make_plan(14, 3, "radial", 1, 2501, 1e-3, b0=True, spokes=16, per_spoke=30)
    ref = oracle_all(p)
    psi = _psi(3, 1)
    srf, white, colored = _ref_maps(ref, psi)
    pl = _plan(p, precision=L.FP64)
    assert _err(pl.map(L.MAP_SRF).cpu().numpy(), srf) < 1e-10
    assert _err(pl.map(L.MAP_NOISE).cpu().numpy(), white) < 1e-10
    assert _err(pl.map(L.MAP_NOISE, psi=psi).cpu().numpy(), colored) < 1e-10
    assert np.all(srf <= 1.0 + 1e-12) and np.all(srf > 0.0)


def test_maps_mixed_exact_gram_refined():
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")
    p = synth.make_plan(20, 4, "spiral", 1, 2502, 1e-4, samples=1600, interleaves=2)
    ref = oracle_all(p)
    srf, white, _ = _ref_maps(ref, np.eye(4))
    pl = _plan(p, precision=L.MIXED_BF16X6, refine_residual=L.RESIDUAL_TOEPLITZ, refine_max_iters=3)
    assert _err(pl.map(L.MAP_SRF).cpu().numpy(), srf) < 1e-6
    assert _err(pl.map(L.MAP_NOISE).cpu().numpy(), white) < 1e-6


def test_maps_mixed_factor_precision_bound():
    """With B0 there is no exact Gram: the maps come from W^H W of the split
    factor, within kappa(G) x the BF16x6 rounding (first-order perturbation)."""
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")
    p = synth.make_plan(16, 2, "radial", 1, 2503, 1e-3, b0=True, spokes=16, per_spoke=32)
    ref = oracle_all(p)
    srf, white, _ = _ref_maps(ref, np.eye(2))
    kappa = np.linalg.cond(ref.G)
    bound = 2e-6 * kappa
    pl = _plan(p, precision=L.MIXED_BF16X6)
    assert _err(pl.map(L.MAP_SRF).cpu().numpy(), srf) < bound
    assert _err(pl.map(L.MAP_NOISE).cpu().numpy(), white) < bound


def test_colored_noise_needs_recon():
    p = synth.make_plan(12, 2, "spiral", 1, 2504, 1e-3, samples=300, interleaves=1)
    pl = _plan(p, precision=L.FP64, recon_mode=L.RECON_NONE)
    with pytest.raises(L.PinvError, match="UNSUPPORTED"):
        pl.map(L.MAP_NOISE, psi=np.eye(2))
    white = pl.map(L.MAP_NOISE).cpu().numpy()  # white noise needs only G^-1
    ref = oracle_all(p)
    assert _err(white, np.real(np.diag(O.noise_matrix(ref.R, np.eye(ref.E.shape[0]))))) < 1e-10
