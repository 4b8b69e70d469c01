"""Python front end of a Pinv-Recon plan: torch tensors in, torch tensors out.

A Plan wraps one pinv_plan of the C library. Building forms
G = E^H E + lambda I (Eq. 6), its Cholesky factor and G^-1, and the explicit
reconstruction matrix Recon = E^+ (Eq. 8); apply() computes
image = Recon x data (Eq. 3). torch supplies device memory and the stream;
all arithmetic runs in libpinv.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _stream_handle(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Plan:
    def __init__(self, dims, traj, coil_maps=None, b0_hz=None, times=None, lam=1e-3,
                 lambda_mode=L.LAMBDA_REL_MEAN_DIAG, precision=L.FP64,
                 recon_mode=L.RECON_STORE, voxel_index=None, fov=None,
                 refine_max_iters=None, refine_tol=0.0, refine_residual=L.RESIDUAL_AUTO,
                 keep_gram=False, lean=False, stream=None):
        lib = L.load()
        if refine_max_iters is None:
            # one FP64 refinement step brings the FP64 explicit-inverse image to
            # the direct-solve accuracy; mixed plans need two or three.
            refine_max_iters = 1 if precision == L.FP64 else 3
        desc, self._keep = L.make_desc(dims, traj, coil_maps, b0_hz, times, lam, lambda_mode,
                                       precision, recon_mode, voxel_index, fov,
                                       refine_max_iters, refine_tol, refine_residual, lean)
        h = C.c_void_p()
        L.check(lib.pinv_plan_create(C.byref(desc), _stream_handle(stream), C.byref(h)))
        self._h = h
        self.n_vox = int(desc.n_vox)
        self.n_samples = int(desc.n_samples)
        self.n_coils = int(desc.n_coils)
        self.n_rows = self.n_samples * self.n_coils
        self.precision = precision
        if keep_gram:
            L.check(lib.pinv_plan_keep_gram(self._h, 1))

    @classmethod
    def from_inputs(cls, p, **kw):
        """Plan from a synth.PlanInputs-like object (dims, traj, maps, B0, lambda_rel)."""
        kw.setdefault("lam", p.lambda_rel)
        kw.setdefault("lambda_mode", L.LAMBDA_REL_MEAN_DIAG)
        return cls(p.dims, p.traj, p.coil_maps, p.b0_hz, p.times, **kw)

    # -- build -------------------------------------------------------------
    def build_async(self, stream=None) -> "Plan":
        L.check(L.load().pinv_build(self._h, _stream_handle(stream)))
        return self

    def sync(self) -> "Plan":
        L.check(L.load().pinv_plan_sync(self._h))
        return self

    def build(self, stream=None) -> "Plan":
        return self.build_async(stream).sync()

    # -- apply -------------------------------------------------------------
    def apply(self, data: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """data [F][C][M_k] (or [F][C*M_k]) complex64/complex128 CUDA -> image [F][N]."""
        if not data.is_cuda:
            raise ValueError("data must be a CUDA tensor")
        if data.dtype not in (torch.complex64, torch.complex128):
            raise ValueError("data must be complex64 or complex128")
        data = data.contiguous()
        F = data.shape[0]
        if data.numel() != F * self.n_rows:
            raise ValueError(f"data has {data.numel()} values, expected F*C*M_k = {F * self.n_rows}")
        if out is None:
            out = torch.empty((F, self.n_vox), dtype=data.dtype, device=data.device)
        elif out.dtype != data.dtype or out.numel() != F * self.n_vox or not out.is_contiguous():
            raise ValueError("out must be a contiguous [F][N] tensor of data's dtype")
        dt = L.C128 if data.dtype == torch.complex128 else L.C64
        L.check(L.load().pinv_apply(self._h, data.data_ptr(), out.data_ptr(), F, dt,
                                    _stream_handle(stream)))
        return out

    # -- introspection -------------------------------------------------------
    def export(self, what: int, stream=None) -> torch.Tensor:
        N = self.n_vox
        if what == L.EXPORT_RECON:
            dt = torch.complex128 if self.precision == L.FP64 else torch.complex64
            t = torch.empty((N, self.n_rows), dtype=dt, device="cuda")
        else:
            t = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
        nbytes = t.numel() * t.element_size()
        L.check(L.load().pinv_plan_export(self._h, what, t.data_ptr(), nbytes, _stream_handle(stream)))
        return t

    def map(self, what: int, psi=None, stream=None) -> torch.Tensor:
        """Per-voxel SRF (L.MAP_SRF) or noise (L.MAP_NOISE) map, float64 [N];
        psi: optional [C][C] coil noise covariance (noise map only)."""
        out = torch.empty(self.n_vox, dtype=torch.float64, device="cuda")
        ptr = None
        if psi is not None:
            self._psi = np.ascontiguousarray(psi, dtype=np.complex128)
            ptr = self._psi.ctypes.data_as(C.POINTER(C.c_double))
        L.check(L.load().pinv_plan_map(self._h, int(what), ptr, out.data_ptr(), _stream_handle(stream)))
        return out

    def eig(self, vectors: bool = True, stream=None):
        """Eigenvalues mu (float64 [N], decreasing) of E^H E and, if asked, the
        eigenvectors P (complex128 [N][N], column i for mu[i]); needs keep_gram.
        Returns (mu, P or None, sweeps)."""
        mu = torch.empty(self.n_vox, dtype=torch.float64, device="cuda")
        P = torch.empty((self.n_vox, self.n_vox), dtype=torch.complex128, device="cuda") if vectors else None
        sweeps = C.c_int(0)
        L.check(L.load().pinv_plan_eig(self._h, mu.data_ptr(), P.data_ptr() if P is not None else None,
                                       C.byref(sweeps), _stream_handle(stream)))
        return mu, P, sweeps.value

    def tsvd_apply(self, mu: torch.Tensor, P: torch.Tensor, data: torch.Tensor, energy: float = 0.95,
                   lam: float = 0.0, stream=None):
        """Truncated eigen reconstruction of data [F][C*M_k] (complex64 or complex128):
        returns (images [F][N] in the data's dtype, rank r, condition number)."""
        data = data.contiguous()
        F = data.shape[0] if data.dim() >= 2 else 1  # [F][C*M_k] or [F][C][M_k]
        dtype = L.C128 if data.dtype == torch.complex128 else L.C64
        out = torch.empty((F, self.n_vox), dtype=data.dtype, device="cuda")
        r, kappa = C.c_int(0), C.c_double(0.0)
        L.check(L.load().pinv_tsvd_apply(self._h, mu.data_ptr(), P.data_ptr(), float(energy), float(lam),
                                         data.data_ptr(), out.data_ptr(), F, dtype, C.byref(r), C.byref(kappa),
                                         _stream_handle(stream)))
        return out, r.value, kappa.value

    def info(self) -> dict:
        inf = L.PlanInfo()
        L.check(L.load().pinv_plan_info(self._h, C.byref(inf)))
        return inf.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().pinv_plan_destroy(self._h)
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
