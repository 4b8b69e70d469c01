"""Plan memory comes from the library's per-device pool, which keeps memory
between plans (so that creating a plan again maps nothing) and returns it when
the last plan is destroyed.

Checked here on a mixed plan with an exact-Gram residual and a Recon: creating,
building, applying and destroying the same plan again and again leaves the
device's free memory where one cycle left it (the pool reuses the memory instead
of growing), and the images of every cycle are bit-identical.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")


def test_plan_cycles_reuse_pool_memory():
    from paper_2410_06129_gb300.plan import Plan
    p = synth.make_plan(32, 4, "spiral", 32, 2701, 1e-3, samples=1024, interleaves=4)
    d = torch.from_numpy(p.data).to(torch.complex64).cuda()
    keep = Plan.from_inputs(p, precision=L.MIXED_BF16X6, refine_max_iters=2).build()  # one plan stays alive
    free, ref, footprint = [], None, None
    for cycle in range(4):
        with Plan.from_inputs(p, precision=L.MIXED_BF16X6, refine_max_iters=2, refine_tol=0.0) as pl:
            pl.build()
            x = pl.apply(d).clone()
            footprint = pl.info()["bytes_device"]
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        if ref is None:
            ref = x
        else:
            assert torch.equal(x, ref), cycle
    # after the first cycle the pool holds the plan's memory; later cycles reuse it
    assert max(free[1:]) - min(free[1:]) < 0.25 * footprint + (64 << 20), (free, footprint)
    keep.close()
