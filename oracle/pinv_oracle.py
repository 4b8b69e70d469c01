"""FP64 CPU oracle for Pinv-Recon (test infrastructure only).

Plain, slow, obviously-correct numpy implementation of the explicit
Tikhonov-regularised pseudoinverse reconstruction of arXiv 2410.06129. It is
used only by the tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py``; the library's product path never imports it. It shares no
code with the CUDA path: voxel geometry, the encoding phase, lambda scaling,
Cholesky and the triangular solves are all written out again here.

Every function follows the paper's definition directly:
  * Encode[(c, m), n] = s_c(r_n) exp(-i 2 pi (k_m . r_n + df_n t_m))
      Eq. 2 (Fourier term), Section 3.3 (coil factor, B0 factor and the
      composite product of factors). The sign is negative (reading 1).
  * G = Encode^H Encode + lambda I                 Eq. 6 (lambda is the
      paper's lambda^2, i.e. the diagonal load itself; reading 2)
  * G = L L^H, Recon = (L^-1)^H L^-1 Encode^H       Eq. 8
  * image = Recon x data                            Eq. 3
  * image = G^-1 (sum_c Encode_c^H data_c)          Section 3.3, last paragraph
  * SRF = Recon x Encode                            Eq. 9
  * X = Recon Psi Recon^H                           Eq. 10
  * Encode^H Encode = P Lambda P^H, eigenvalues the squared singular values of
      Encode; truncated reconstruction P_r Lambda_r^-1 P_r^H Encode^H data with
      r set by a fraction of the energy                Section 2.1 (SVD, tSVD,
      eigenvalue decomposition)
Parity status: every function here is pinned by tests/test_oracle_pins.py
(SVD brute force, Cartesian closed form, invariants). The B0 factor of encode
is pinned by the linear-map identity (a B0 map g . r equals the trajectory
shifted by g t), a uniform offset and a common time delay; noise_matrix with a
coloured Psi by the closed form for Psi = E E^H (Eq. 9 in Eq. 10) and by a
Monte Carlo covariance of reconstructed coil-correlated noise.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# encoding (Eq. 1-2, Section 3.3)
# --------------------------------------------------------------------------
def voxel_positions(dims, fov=None) -> np.ndarray:
    """Voxel centres r_n = ((i - dims/2) / dims) * fov, x index fastest."""
    dims = [int(d) for d in dims]
    fov = [1.0] * len(dims) if fov is None else [float(f) for f in fov]
    n = int(np.prod(dims))
    r = np.zeros((n, len(dims)))
    for flat in range(n):
        rem = flat
        for d in range(len(dims)):
            i = rem % dims[d]
            rem //= dims[d]
            r[flat, d] = (i - dims[d] / 2.0) / dims[d] * fov[d]
    return r


def encode(traj, vox, coil_maps=None, b0_hz=None, times=None) -> np.ndarray:
    """Explicit encoding matrix E, shape [C * M_k][N], complex128.

    Row c * M_k + m, column n holds s_c(r_n) exp(-i2pi(k_m . r_n + df_n t_m)).
    The phase (in cycles) is reduced to [-1/2, 1/2] in FP64 before exp.
    """
    traj = np.asarray(traj, dtype=np.float64)
    vox = np.asarray(vox, dtype=np.float64)
    cycles = traj @ vox.T                                    # k_m . r_n
    if b0_hz is not None:
        cycles = cycles + np.outer(np.asarray(times, np.float64), np.asarray(b0_hz, np.float64))
    cycles = cycles - np.round(cycles)
    fourier = np.exp(-2j * np.pi * cycles)                   # [M_k][N]
    if coil_maps is None:
        return fourier
    blocks = [fourier * np.asarray(s)[None, :] for s in coil_maps]
    return np.concatenate(blocks, axis=0)                    # coils stacked (Eq. 11)


def lambda_abs(E: np.ndarray, lambda_rel: float) -> float:
    """Diagonal load lambda = lambda_rel * trace(E^H E) / N."""
    return float(lambda_rel * np.real(np.sum(np.conj(E) * E)) / E.shape[1])


# --------------------------------------------------------------------------
# normal equations (Eq. 6) and Cholesky (Eq. 8)
# --------------------------------------------------------------------------
def gram(E: np.ndarray, lam: float) -> np.ndarray:
    """G = E^H E + lambda I."""
    return E.conj().T @ E + lam * np.eye(E.shape[1])


def cholesky(G: np.ndarray) -> np.ndarray:
    """Unblocked column-by-column Cholesky: lower L with G = L L^H.

    Raises ValueError with the failing pivot index if G is not positive
    definite.
    """
    n = G.shape[0]
    L = np.zeros_like(G, dtype=np.complex128)
    for j in range(n):
        d = np.real(G[j, j]) - np.sum(np.abs(L[j, :j]) ** 2)
        if not d > 0.0:
            raise ValueError(f"not positive definite at pivot {j}")
        L[j, j] = np.sqrt(d)
        if j + 1 < n:
            L[j + 1:, j] = (G[j + 1:, j] - L[j + 1:, :j] @ np.conj(L[j, :j])) / L[j, j]
    return L


def forward_substitution(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve L Y = B for lower-triangular L, row by row."""
    B = np.asarray(B, dtype=np.complex128)
    Y = np.zeros_like(B)
    for i in range(L.shape[0]):
        Y[i] = (B[i] - L[i, :i] @ Y[:i]) / L[i, i]
    return Y


def back_substitution_h(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve L^H X = B for lower-triangular L, last row first."""
    B = np.asarray(B, dtype=np.complex128)
    X = np.zeros_like(B)
    n = L.shape[0]
    for i in range(n - 1, -1, -1):
        # (L^H)[i, j] = conj(L[j, i]) for j > i
        X[i] = (B[i] - np.conj(L[i + 1:, i]) @ X[i + 1:]) / np.conj(L[i, i])
    return X


def inverse_lower(L: np.ndarray) -> np.ndarray:
    """L^-1 by forward substitution on the identity."""
    return forward_substitution(L, np.eye(L.shape[0], dtype=np.complex128))


def gram_inverse(L: np.ndarray) -> np.ndarray:
    """G^-1 = (L^-1)^H L^-1 (Eq. 8)."""
    W = inverse_lower(L)
    return W.conj().T @ W


def recon_matrix(E: np.ndarray, lam: float) -> tuple[np.ndarray, np.ndarray]:
    """Recon = (L^-1)^H L^-1 E^H with G = E^H E + lam I = L L^H (Eq. 8).

    Returns (Recon [N][C*M_k], L).
    """
    L = cholesky(gram(E, lam))
    W = inverse_lower(L)
    return W.conj().T @ (W @ E.conj().T), L


def reconstruct(recon: np.ndarray, data_cols: np.ndarray) -> np.ndarray:
    """image = Recon x data (Eq. 3); data_cols is [C*M_k][F]."""
    return recon @ data_cols


def solve(E: np.ndarray, L: np.ndarray, data_cols: np.ndarray) -> np.ndarray:
    """Direct solution without Recon: x = L^-H L^-1 (sum_c E_c^H d_c).

    E^H d over the stacked coil rows equals the per-coil sum of Section 3.3.
    """
    rhs = E.conj().T @ data_cols
    return back_substitution_h(L, forward_substitution(L, rhs))


def srf(recon: np.ndarray, E: np.ndarray) -> np.ndarray:
    """Spatial response function matrix SRF = Recon x Encode (Eq. 9)."""
    return recon @ E


def noise_matrix(recon: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Noise matrix X = Recon Psi Recon^H (Eq. 10); psi is [C*M_k]^2."""
    return recon @ psi @ recon.conj().T


# --------------------------------------------------------------------------
# eigenvalue decomposition and truncated SVD (Section 2.1)
# --------------------------------------------------------------------------
def gram_eig(E: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Encode^H Encode = P diag(mu) P^H, mu in decreasing order (Section 2.1,
    eigenvalue decomposition: the eigenvalues of the Gram matrix are the squared
    singular values of Encode). Column i of P is the eigenvector of mu[i]."""
    mu, vecs = np.linalg.eigh(E.conj().T @ E)
    order = np.argsort(mu)[::-1]
    return mu[order], vecs[:, order]


def tsvd_rank(mu: np.ndarray, energy: float) -> int:
    """Smallest r whose r largest eigenvalues hold the fraction `energy` of their
    sum (Section 2.1: the truncation keeps a set share of the energy, e.g. 95 %)."""
    c = np.cumsum(np.maximum(mu, 0.0))
    r = int(np.searchsorted(c, energy * c[-1], side="left")) + 1
    return min(r, len(mu))


def tsvd_condition(mu: np.ndarray, r: int) -> float:
    """Condition number of the truncated problem: largest over smallest kept
    singular value (Section 2.1)."""
    return float(np.sqrt(mu[0] / mu[r - 1]))


def tsvd_solve(mu: np.ndarray, vecs: np.ndarray, b_cols: np.ndarray, r: int, lam: float = 0.0) -> np.ndarray:
    """image = P_r diag(1 / (mu_r + lam)) P_r^H (Encode^H data), the truncated
    eigen-reconstruction, with Tikhonov loading lam when combined (Section 2.1).
    b_cols holds Encode^H data, one column per frame."""
    pr = vecs[:, :r]
    return pr @ ((pr.conj().T @ b_cols) / (mu[:r] + lam)[:, None])


# --------------------------------------------------------------------------
# convenience wrappers over a plan's inputs
# --------------------------------------------------------------------------
def plan_encode(plan, vox=None) -> np.ndarray:
    """E for a synth.PlanInputs-like object (dims, traj, coil_maps, b0_hz, times)."""
    vox = voxel_positions(plan.dims) if vox is None else vox
    return encode(plan.traj, vox, plan.coil_maps, plan.b0_hz, plan.times)


def data_columns(data: np.ndarray) -> np.ndarray:
    """[F][C][M_k] data -> [C*M_k][F] columns (coil-major rows as in encode)."""
    F = data.shape[0]
    return np.asarray(data, dtype=np.complex128).reshape(F, -1).T


def pinv_recon(plan, frames=None):
    """Full explicit path: (images [F][N], Recon, L, lambda)."""
    E = plan_encode(plan)
    lam = lambda_abs(E, plan.lambda_rel)
    R, L = recon_matrix(E, lam)
    d = plan.data if frames is None else plan.data[frames]
    return reconstruct(R, data_columns(d)).T, R, L, lam


def nrmse(x, ref) -> float:
    """||x - ref||_2 / ||ref||_2 over all entries jointly (reading 8)."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))
