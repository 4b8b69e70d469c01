"""The lambda / condition check of every build (Section 2.1: the condition number
of the inversion; Section 2.2: the Tikhonov load makes G positive definite).

kappa_est is Hager's estimate of kappa_1(G) = ||G||_1 ||G^-1||_1 from the factor
(mixed plans certify it against G itself). Against the oracle's G:
  * ||G||_1 matches np.linalg.norm(G, 1) (FP32 magnitudes, double-float sums);
  * kappa_est never exceeds np.linalg.cond(G, 1) beyond the rounding of its sums
    (1e-6 relative; 1e-4 for mixed plans without the exact Gram, whose ||G||_1 is
    read from the split-precision Gram) and is within a factor of 3 below it.
Plus the pivot check of the mixed path: a Gram with an exactly zero pivot is
reported as NOT_PD with the pivot's index, as on the FP64 path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.pinv_oracle as O  # noqa: E402
from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mixed_ok():
    return bool(L.load().pinv_tc_available())


def _oracle_gram(p):
    E = O.plan_encode(p)
    return O.gram(E, O.lambda_abs(E, p.lambda_rel))


CASES = [
    # (side, coils, traj, b0, lambda_rel, precision, residual, slack above kappa_1)
    (16, 3, "spiral", False, 1e-3, L.FP64, L.RESIDUAL_AUTO, 1e-6),
    (15, 2, "radial", True, 1e-4, L.FP64, L.RESIDUAL_AUTO, 1e-6),
    (16, 3, "spiral", False, 1e-3, L.MIXED_BF16X6, L.RESIDUAL_TOEPLITZ, 1e-6),
    (18, 4, "spiral", False, 1e-3, L.MIXED_BF16X3, L.RESIDUAL_TOEPLITZ, 1e-6),
    (16, 2, "radial", True, 1e-3, L.MIXED_BF16X6, L.RESIDUAL_DOUBLE_FLOAT, 1e-4),
    (14, 2, "spiral", False, 1e-3, L.MIXED_BF16X6, L.RESIDUAL_FP64, 1e-4),
]


@pytest.mark.parametrize("side,coils,traj,b0,lam,prec,res,slack", CASES)
def test_kappa_estimate_against_oracle(side, coils, traj, b0, lam, prec, res, slack):
    from paper_2410_06129_gb300.plan import Plan
    if prec != L.FP64 and not _mixed_ok():
        pytest.skip("tcgen05 kernels need sm_103a")
    kw = dict(samples=2 * side * side, interleaves=2) if traj == "spiral" else dict(spokes=2 * side, per_spoke=side + 3)
    p = synth.make_plan(side, coils, traj, 1, 2700 + side + coils, lam, b0=b0, **kw)
    G = _oracle_gram(p)
    k1 = np.linalg.cond(G, 1)
    n1 = np.linalg.norm(G, 1)
    with Plan.from_inputs(p, precision=prec, refine_residual=res) as pl:
        pl.build()
        inf = pl.info()
    exact_norm = prec == L.FP64 or res == L.RESIDUAL_TOEPLITZ  # else read from the split-precision Gram
    assert abs(inf["norm1_g"] - n1) <= (1e-6 if exact_norm else 1e-4) * n1
    k = inf["kappa_est"]
    assert np.isfinite(k) and k > 0
    assert k <= k1 * (1 + slack), (k, k1)
    assert k >= k1 / 3, (k, k1)


def test_kappa_estimate_lean_plan_and_rebuild():
    """A lean mixed plan (G, L and the FP64 W are build temporaries) gives the same
    estimate as a full one, and a second build the same value again."""
    from paper_2410_06129_gb300.plan import Plan
    if not _mixed_ok():
        pytest.skip("tcgen05 kernels need sm_103a")
    p = synth.make_plan(20, 3, "spiral", 1, 2751, 1e-3, samples=800, interleaves=2)
    k1 = np.linalg.cond(_oracle_gram(p), 1)
    with Plan.from_inputs(p, precision=L.MIXED_BF16X6, lean=True) as a, \
            Plan.from_inputs(p, precision=L.MIXED_BF16X6) as b:
        ka = a.build().info()["kappa_est"]
        kb = b.build().info()["kappa_est"]
        kb2 = b.build().info()["kappa_est"]
    assert ka == kb == kb2
    assert k1 / 3 <= ka <= k1 * (1 + 1e-6)


def test_mixed_not_positive_definite_reported():
    """lambda = 0 and a voxel no coil sees: the split-precision Gram keeps that
    row exactly zero (Hadamard coil epilogue), the double-float diagonal block
    finds a zero pivot and the build reports NOT_PD with its index."""
    from paper_2410_06129_gb300.plan import Plan
    if not _mixed_ok():
        pytest.skip("tcgen05 kernels need sm_103a")
    p = synth.make_plan(12, 2, "spiral", 1, 2752, 0.0, samples=512, interleaves=1)
    maps = p.coil_maps.copy()
    maps[:, 70] = 0.0
    for res in (L.RESIDUAL_TOEPLITZ, L.RESIDUAL_DOUBLE_FLOAT):
        pl = Plan(p.dims, p.traj, maps, lam=0.0, lambda_mode=L.LAMBDA_ABS, precision=L.MIXED_BF16X6,
                  refine_residual=res)
        with pytest.raises(L.PinvError, match="NOT_PD"):
            pl.build()
        assert pl.info()["info"] == 70
        with pytest.raises(L.PinvError, match="NOT_BUILT"):
            pl.apply(torch.zeros((1, 1024), dtype=torch.complex64, device="cuda"))
        pl.close()
