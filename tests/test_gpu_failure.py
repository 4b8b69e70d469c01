"""Failure handling on the GPU without a fault: bounded waits that run out.

Every pipeline wait of the tensor-core kernels is bounded. pinv_set_wait_limit
shortens the bound to a few thousand SM cycles, so real waits (a stage's bulk
copies landing, an MMA group finishing) run out during a build. The build must
report PINV_ERR_TIMEOUT without hanging or faulting; every aborted CTA must have
waited for its own MMAs and copies and freed its tensor memory. The next build
of the same plan, with the default bound, allocates tensor memory on the same
SMs: it succeeds and its images match the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402
from tests._ref import oracle_all, rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")


def test_wait_limit_rejects_negative():
    with pytest.raises(L.PinvError, match="INVALID_ARG"):
        L.check(L.load().pinv_set_wait_limit(-1))


# Both limits are below one stage's round trip from L2 (several hundred cycles), so the
# first pipeline wait of every tensor-core kernel of the build runs out. (At 2000 cycles
# the stages of this small plan's Gram and trailing updates can land in time, and
# whether the build times out depends on its other kernels.)
@pytest.mark.parametrize("cycles", [250, 500])
def test_expired_waits_report_timeout_and_next_build_succeeds(cycles):
    from paper_2410_06129_gb300.plan import Plan
    lib = L.load()
    p = synth.make_plan(24, 3, "spiral", 2, 2901, 1e-3, samples=1152, interleaves=2)
    ref = oracle_all(p)
    d = torch.from_numpy(p.data).cuda()
    with Plan.from_inputs(p, precision=L.MIXED_BF16X6, refine_max_iters=3, refine_tol=0.0) as pl:
        try:
            L.check(lib.pinv_set_wait_limit(cycles))
            with pytest.raises(L.PinvError, match="TIMEOUT"):
                pl.build()
        finally:
            L.check(lib.pinv_set_wait_limit(0))
        with pytest.raises(L.PinvError, match="NOT_BUILT"):
            pl.apply(d)
        pl.build()
        x = pl.apply(d).cpu().numpy()
    assert rel(x, ref.images) <= 1e-4
    torch.cuda.synchronize()


def test_non_finite_data_is_reported_with_the_stopping_rule():
    """A NaN in one frame's data: with the stopping rule the refinement reads the
    residual norms and ends the call with INVALID_ARG naming the frame, instead of
    returning NaN images; without it the other frames' images are unaffected."""
    from paper_2410_06129_gb300.plan import Plan
    p = synth.make_plan(16, 2, "spiral", 3, 2903, 1e-3, samples=512, interleaves=2)
    d = torch.from_numpy(p.data).cuda()
    d[1, 0, 5] = float("nan")
    with Plan.from_inputs(p, precision=L.MIXED_BF16X6, refine_max_iters=3, refine_tol=1e-12) as pl:
        pl.build()
        with pytest.raises(L.PinvError, match="non-finite .* frame 1"):
            pl.apply(d)
    with Plan.from_inputs(p, precision=L.MIXED_BF16X6, refine_max_iters=3, refine_tol=0.0) as pl:
        pl.build()
        x = pl.apply(d).cpu().numpy()
        ok = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()  # the same frames, frame 1 clean
    assert not np.isfinite(x[1]).all()
    assert np.array_equal(x[[0, 2]], ok[[0, 2]])
