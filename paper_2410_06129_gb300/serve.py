"""Python front end of the serving loop (pinv_server_* in include/pinv.h).

A Server keeps factored plans of registered encodings resident in device
memory under a byte budget and reconstructs requests as they arrive; all work
runs in libpinv.so's worker thread. This module only marshals arguments and
keeps each request's tensors alive until the request has finished.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


class Server:
    def __init__(self, budget_bytes: int, max_slots: int = 4):
        lib = L.load()
        h = C.c_void_p()
        L.check(lib.pinv_server_create(int(budget_bytes), int(max_slots), C.byref(h)))
        self._h = h
        self._live = {}      # ticket -> tensors the request reads or writes
        self._shapes = {}    # plan id -> (n_vox, rows)

    def register(self, dims, traj, coil_maps=None, b0_hz=None, times=None, lam=1e-3,
                 lambda_mode=L.LAMBDA_REL_MEAN_DIAG, precision=L.FP64, recon_mode=L.RECON_STORE,
                 voxel_index=None, fov=None, refine_max_iters=None,
                 refine_residual=L.RESIDUAL_AUTO) -> int:
        if refine_max_iters is None:
            refine_max_iters = 1 if precision == L.FP64 else 3
        desc, keep = L.make_desc(dims, traj, coil_maps, b0_hz, times, lam, lambda_mode, precision,
                                 recon_mode, voxel_index, fov, refine_max_iters, 0.0, refine_residual)
        # the server keeps plans lean: only what an apply reads stays resident
        pid = C.c_int()
        L.check(L.load().pinv_serve_register(self._h, C.byref(desc), C.byref(pid)))
        self._shapes[pid.value] = (int(desc.n_vox), int(desc.n_samples) * int(desc.n_coils))
        return pid.value

    def register_inputs(self, p, **kw) -> int:
        """Register a synth.PlanInputs-like object (dims, traj, maps, B0, lambda_rel)."""
        kw.setdefault("lam", p.lambda_rel)
        return self.register(p.dims, p.traj, p.coil_maps, p.b0_hz, p.times, **kw)

    def enqueue(self, plan_id: int, data: torch.Tensor, out: torch.Tensor | None = None,
                sync_inputs: bool = True, callback=None):
        """Queue a request; returns (ticket, out). `data` must be complete when
        the server reads it: with sync_inputs the current stream is synchronised.
        callback(ticket, status), if given, runs on the server's worker thread."""
        n_vox, rows = self._shapes[plan_id]
        data = data.contiguous()
        F = data.shape[0]
        if data.numel() != F * rows:
            raise ValueError(f"data has {data.numel()} values, expected F*C*M_k = {F * rows}")
        if out is None:
            out = torch.empty((F, n_vox), dtype=data.dtype, device=data.device)
        if sync_inputs:
            torch.cuda.current_stream().synchronize()
        dt = L.C128 if data.dtype == torch.complex128 else L.C64
        cb = L.DONE_CB(lambda t, st, _u: callback(int(t), int(st))) if callback else None
        t = C.c_uint64()
        L.check(L.load().pinv_serve_enqueue(self._h, plan_id, data.data_ptr(), out.data_ptr(), F, dt,
                                            cb, None, C.byref(t)))
        self._live[t.value] = (data, out, cb)
        return t.value, out

    def wait(self, ticket: int, timeout: float = 600.0) -> int:
        """Block until the request finished; returns its status (0 = OK)."""
        res = C.c_int()
        L.check(L.load().pinv_serve_wait(self._h, ticket, timeout, C.byref(res)))
        self._live.pop(ticket, None)
        return res.value

    def poll(self, ticket: int):
        done, res = C.c_int(), C.c_int()
        L.check(L.load().pinv_serve_poll(self._h, ticket, C.byref(done), C.byref(res)))
        if done.value:
            self._live.pop(ticket, None)
        return bool(done.value), res.value

    def set_merge(self, max_frames: int):
        """Merge queued requests of the dispatched request's plan (same element type)
        into its apply, up to max_frames frames in all (0: off)."""
        L.check(L.load().pinv_server_set_merge(self._h, int(max_frames)))

    def times(self, ticket: int) -> dict:
        """Times of a finished request in ms after the server's creation: enqueue and
        done (host clock), dev_start and dev_end of its device work (device clock; -1
        when it ran nothing)."""
        t = (C.c_double * 4)()
        L.check(L.load().pinv_serve_times(self._h, ticket, t))
        return {"enqueue": t[0], "done": t[1], "dev_start": t[2], "dev_end": t[3]}

    def stats(self) -> dict:
        s = L.ServerStats()
        L.check(L.load().pinv_server_stats(self._h, C.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().pinv_server_destroy(self._h)
            self._h = C.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
