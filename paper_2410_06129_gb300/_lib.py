"""ctypes binding of libpinv.so (include/pinv.h). Argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy
host arrays and torch CUDA tensors into the pointers and sizes the C ABI
takes, and turns non-OK status codes into exceptions. There is no CPU
fallback: if the shared library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpinv.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_BUDGET, ERR_NOT_PD, ERR_NOT_BUILT, ERR_TIMEOUT, ERR_CUDA, \
    ERR_INTERNAL, ERR_UNSUPPORTED = range(10)
FP64, MIXED_BF16X3, MIXED_BF16X6 = 0, 1, 2
LAMBDA_ABS, LAMBDA_REL_MEAN_DIAG = 0, 1
C64, C128 = 0, 1
RECON_AUTO, RECON_NONE, RECON_STORE = -1, 0, 1
RESIDUAL_DOUBLE_FLOAT, RESIDUAL_FP64, RESIDUAL_TOEPLITZ = 0, 1, 2
RESIDUAL_AUTO = -1  # binding-side default: TOEPLITZ without B0, else DOUBLE_FLOAT
EXPORT_GRAM, EXPORT_CHOL, EXPORT_GINV, EXPORT_RECON, EXPORT_LINV, EXPORT_GRAM_EXACT = 0, 1, 2, 3, 4, 5

_STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "BUDGET", 4: "NOT_PD", 5: "NOT_BUILT",
                 6: "TIMEOUT", 7: "CUDA", 8: "INTERNAL", 9: "UNSUPPORTED"}


class PinvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pinv {_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("dims", C.c_int * 3), ("fov", C.c_double * 3),
        ("voxel_index", C.POINTER(C.c_int64)), ("n_vox", C.c_int64), ("n_samples", C.c_int64),
        ("traj", C.POINTER(C.c_double)), ("n_coils", C.c_int), ("coil_maps", C.POINTER(C.c_double)),
        ("b0_hz", C.POINTER(C.c_double)), ("times", C.POINTER(C.c_double)),
        ("lambda_", C.c_double), ("lambda_mode", C.c_int), ("precision", C.c_int),
        ("recon_mode", C.c_int), ("refine_max_iters", C.c_int), ("refine_tol", C.c_double),
        ("refine_residual", C.c_int), ("lean", C.c_int),
    ]


class PlanInfo(C.Structure):
    _fields_ = [
        ("n_vox", C.c_int64), ("n_samples", C.c_int64), ("n_rows", C.c_int64),
        ("n_coils", C.c_int), ("precision", C.c_int), ("has_recon", C.c_int),
        ("lambda_abs", C.c_double), ("min_pivot", C.c_double), ("max_pivot", C.c_double),
        ("bytes_device", C.c_size_t), ("bytes_recon", C.c_size_t),
        ("ms_tables", C.c_double), ("ms_gram", C.c_double), ("ms_chol", C.c_double),
        ("ms_inverse", C.c_double), ("ms_recon", C.c_double), ("info", C.c_int),
        ("last_refine_iters", C.c_int), ("last_refine_resid", C.c_double),
        ("ms_gram_kernel", C.c_double), ("kappa_est", C.c_double), ("norm1_g", C.c_double),
        ("ms_cond", C.c_double), ("last_refine_bound", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(C.Structure):
    _fields_ = [
        ("completed", C.c_uint64), ("failed", C.c_uint64), ("builds", C.c_uint64),
        ("evictions", C.c_uint64), ("frames", C.c_double), ("p50_ms", C.c_double),
        ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
        ("span_s", C.c_double), ("resident_bytes", C.c_size_t), ("resident_plans", C.c_int),
        ("queued", C.c_int), ("recon_drops", C.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


DONE_CB = C.CFUNCTYPE(None, C.c_uint64, C.c_int, C.c_void_p)

# Symbols declared in include/pinv.h: name -> (restype, argtypes)
_VP = C.c_void_p
SIGNATURES = {
    "pinv_version": (C.c_int, []),
    "pinv_kernel_launches": (C.c_ulonglong, []),
    "pinv_tc_available": (C.c_int, []),
    "pinv_last_error": (C.c_char_p, []),
    "pinv_set_wait_limit": (C.c_int, [C.c_int64]),
    "pinv_plan_create": (C.c_int, [C.POINTER(PlanDesc), _VP, C.POINTER(_VP)]),
    "pinv_build": (C.c_int, [_VP, _VP]),
    "pinv_plan_sync": (C.c_int, [_VP]),
    "pinv_apply": (C.c_int, [_VP, _VP, _VP, C.c_int64, C.c_int, _VP]),
    "pinv_plan_export": (C.c_int, [_VP, C.c_int, _VP, C.c_size_t, _VP]),
    "pinv_plan_keep_gram": (C.c_int, [_VP, C.c_int]),
    "pinv_plan_info": (C.c_int, [_VP, C.POINTER(PlanInfo)]),
    "pinv_plan_destroy": (None, [_VP]),
    "pinv_apply_noalloc": (C.c_int, [_VP, _VP, _VP, C.c_int64, C.c_int, _VP]),
    "pinv_plan_map": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_double), _VP, _VP]),
    "pinv_plan_eig": (C.c_int, [_VP, _VP, _VP, C.POINTER(C.c_int), _VP]),
    "pinv_tsvd_apply": (C.c_int, [_VP, _VP, _VP, C.c_double, C.c_double, _VP, _VP, C.c_int64, C.c_int,
                                  C.POINTER(C.c_int), C.POINTER(C.c_double), _VP]),
    "pinv_autotune_report": (C.c_size_t, [C.c_char_p, C.c_size_t]),
    "pinv_batch_create": (C.c_int, [C.POINTER(_VP), C.c_int, C.c_int, C.POINTER(_VP)]),
    "pinv_batch_build": (C.c_int, [_VP, _VP]),
    "pinv_batch_apply": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(C.c_int64), C.c_int, _VP]),
    "pinv_batch_sync": (C.c_int, [_VP, C.POINTER(C.c_int)]),
    "pinv_batch_destroy": (None, [_VP]),
    "pinv_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(_VP)]),
    "pinv_serve_register": (C.c_int, [_VP, C.POINTER(PlanDesc), C.POINTER(C.c_int)]),
    "pinv_serve_enqueue": (C.c_int, [_VP, C.c_int, _VP, _VP, C.c_int64, C.c_int, _VP, _VP,
                                     C.POINTER(C.c_uint64)]),
    "pinv_serve_poll": (C.c_int, [_VP, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pinv_serve_wait": (C.c_int, [_VP, C.c_uint64, C.c_double, C.POINTER(C.c_int)]),
    "pinv_serve_times": (C.c_int, [_VP, C.c_uint64, C.POINTER(C.c_double)]),
    "pinv_server_set_merge": (C.c_int, [_VP, C.c_int64]),
    "pinv_server_stats": (C.c_int, [_VP, C.POINTER(ServerStats)]),
    "pinv_server_destroy": (None, [_VP]),
}
NOALLOC_SCRATCH_BYTES = 64 << 20
BATCH_GRAPH = 1
MAP_SRF, MAP_NOISE = 0, 1

_lib = None


def load(path: str = LIB_PATH):
    """Load libpinv.so once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def autotune_report() -> str:
    buf = C.create_string_buffer(8192)
    load().pinv_autotune_report(buf, 8192)
    return buf.value.decode()


def check(status: int):
    if status != OK:
        raise PinvError(status, load().pinv_last_error().decode())


def _dptr(a: np.ndarray | None, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def make_desc(dims, traj, coil_maps=None, b0_hz=None, times=None, lam=1e-3,
              lambda_mode=LAMBDA_REL_MEAN_DIAG, precision=FP64, recon_mode=RECON_STORE,
              voxel_index=None, fov=None, refine_max_iters=0, refine_tol=0.0,
              refine_residual=RESIDUAL_AUTO, lean=False):
    """Build a PlanDesc plus the numpy arrays that must outlive the create call."""
    dims = [int(d) for d in dims]
    ndim = len(dims)
    keep = {}
    keep["traj"] = np.ascontiguousarray(traj, dtype=np.float64).reshape(-1, ndim)
    d = PlanDesc()
    d.ndim = ndim
    for i in range(3):
        d.dims[i] = dims[i] if i < ndim else 1
        d.fov[i] = (fov[i] if fov is not None else 1.0) if i < ndim else 1.0
    if voxel_index is not None:
        keep["vi"] = np.ascontiguousarray(voxel_index, dtype=np.int64)
        d.voxel_index = _dptr(keep["vi"], C.c_int64)
        d.n_vox = keep["vi"].shape[0]
    else:
        d.n_vox = int(np.prod(dims))
    d.n_samples = keep["traj"].shape[0]
    d.traj = _dptr(keep["traj"], C.c_double)
    if coil_maps is not None:
        keep["cm"] = np.ascontiguousarray(coil_maps, dtype=np.complex128)
        d.n_coils = keep["cm"].shape[0]
        d.coil_maps = keep["cm"].ctypes.data_as(C.POINTER(C.c_double))
    else:
        d.n_coils = 1
    if b0_hz is not None:
        keep["b0"] = np.ascontiguousarray(b0_hz, dtype=np.float64)
        keep["t"] = np.ascontiguousarray(times, dtype=np.float64)
        d.b0_hz = _dptr(keep["b0"], C.c_double)
        d.times = _dptr(keep["t"], C.c_double)
    d.lambda_ = float(lam)
    d.lambda_mode = int(lambda_mode)
    d.precision = int(precision)
    d.recon_mode = int(recon_mode)
    d.refine_max_iters = int(refine_max_iters)
    d.refine_tol = float(refine_tol)
    if refine_residual == RESIDUAL_AUTO:
        refine_residual = RESIDUAL_DOUBLE_FLOAT if b0_hz is not None else RESIDUAL_TOEPLITZ
    d.refine_residual = int(refine_residual)
    d.lean = 1 if lean else 0
    return d, keep
