"""pinv_apply_noalloc gives the same images as pinv_apply.

pinv_apply_noalloc serves callers that cannot allocate device memory while
they reconstruct: a real-time loop under a fixed memory budget, or an
application whose device memory belongs to another allocator. Its scratch is
one fixed device array shared by all calls, which keeps the previous call's
contents, so the result is checked on two calls in a row. The file is named
to run last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()


def _noalloc(pl, data, out):
    dt = L.C128 if data.dtype == torch.complex128 else L.C64
    return L.load().pinv_apply_noalloc(pl._h, data.data_ptr(), out.data_ptr(), data.shape[0], dt,
                                       torch.cuda.current_stream().cuda_stream)


def _rel(a, b):
    return float(torch.linalg.norm((a - b).flatten()) / torch.linalg.norm(b.flatten()))


CASES = [
    ("fp64-explicit-c64", dict(precision=L.FP64), torch.complex64),
    ("fp64-factor-only-c128", dict(precision=L.FP64, recon_mode=L.RECON_NONE), torch.complex128),
    ("mixed-explicit-c128", dict(precision=L.MIXED_BF16X6, refine_max_iters=2, refine_tol=1e-14),
     torch.complex128),
    ("mixed-factor-only-c64", dict(precision=L.MIXED_BF16X3, recon_mode=L.RECON_NONE, refine_max_iters=1),
     torch.complex64),
]


@pytest.mark.parametrize("name,kw,dtype", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_apply_twice(name, kw, dtype):
    if kw["precision"] != L.FP64 and not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")
    from paper_2410_06129_gb300.plan import Plan
    p = synth.make_plan(16, 3, "spiral", 3, 2201, 1e-3, samples=600, interleaves=2, b0=True)
    with Plan.from_inputs(p, **kw).build() as pl:
        d = torch.from_numpy(p.data).to(dtype).cuda()
        ref = pl.apply(d).clone()
        for call in range(2):
            out = torch.full_like(ref, float("nan"))
            st = _noalloc(pl, d, out)
            assert st == L.OK, L.load().pinv_last_error()
            torch.cuda.synchronize()
            assert _rel(out, ref) <= TOL, (name, call)


def test_noalloc_rejects_more_frames_than_its_scratch_holds():
    """The size check happens on the host, before any kernel touches a buffer."""
    from paper_2410_06129_gb300.plan import Plan
    p = synth.make_plan(8, 1, "spiral", 1, 2202, 1e-3, samples=128, interleaves=1)
    with Plan.from_inputs(p).build() as pl:
        d = torch.zeros((1, 128), dtype=torch.complex64, device="cuda")
        x = torch.zeros((1, 64), dtype=torch.complex64, device="cuda")
        frames = L.NOALLOC_SCRATCH_BYTES // (16 * (128 + 64)) + 1
        st = L.load().pinv_apply_noalloc(pl._h, d.data_ptr(), x.data_ptr(), frames, L.C64,
                                         torch.cuda.current_stream().cuda_stream)
        assert st == L.ERR_INVALID_ARG
        assert b"scratch" in L.load().pinv_last_error()
        st = L.load().pinv_apply_noalloc(pl._h, d.data_ptr(), x.data_ptr(), 1, L.C64,
                                         torch.cuda.current_stream().cuda_stream)
        assert st == L.OK
