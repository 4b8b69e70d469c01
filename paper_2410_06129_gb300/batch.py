"""Python front end of plan batches (pinv_batch_* in include/pinv.h).

A Batch builds and applies several plans of uneven size together: shared
persistent tensor-core launches for the Gram and Recon of all plans,
concurrent per-plan factorisations and applies, optionally replayed from a
CUDA graph. This module only marshals arguments.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from .plan import _stream_handle


class Batch:
    def __init__(self, plans, graph: bool = True):
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = C.c_void_p()
        L.check(L.load().pinv_batch_create(arr, len(self.plans), L.BATCH_GRAPH if graph else 0, C.byref(h)))
        self._h = h

    def build_async(self, stream=None) -> "Batch":
        L.check(L.load().pinv_batch_build(self._h, _stream_handle(stream)))
        return self

    def sync(self) -> "Batch":
        bad = C.c_int(-1)
        st = L.load().pinv_batch_sync(self._h, C.byref(bad))
        if st != L.OK:
            raise L.PinvError(st, f"plan {bad.value}: " + L.load().pinv_last_error().decode())
        return self

    def build(self, stream=None) -> "Batch":
        return self.build_async(stream).sync()

    def apply(self, datas, outs=None, stream=None):
        """datas[i]: [F_i][C_i][M_k,i] CUDA tensors of one complex dtype -> images [F_i][N_i]."""
        if len(datas) != len(self.plans):
            raise ValueError("one data tensor per plan")
        dt = datas[0].dtype
        datas = [d.contiguous() for d in datas]
        if outs is None:
            outs = [torch.empty((d.shape[0], p.n_vox), dtype=dt, device=d.device) for d, p in zip(datas, self.plans)]
        for d, o, p in zip(datas, outs, self.plans):
            if d.dtype != dt or o.dtype != dt or not d.is_cuda:
                raise ValueError("all data and images must be CUDA tensors of one dtype")
            if d.numel() != d.shape[0] * p.n_rows or o.numel() != d.shape[0] * p.n_vox:
                raise ValueError("data / image shape does not match its plan")
        n = len(self.plans)
        dp = (C.c_void_p * n)(*[d.data_ptr() for d in datas])
        op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        fr = (C.c_int64 * n)(*[d.shape[0] for d in datas])
        code = L.C128 if dt == torch.complex128 else L.C64
        L.check(L.load().pinv_batch_apply(self._h, dp, op, fr, code, _stream_handle(stream)))
        return outs

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().pinv_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
