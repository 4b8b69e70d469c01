"""Shared helpers for GPU-vs-oracle parity tests (oracle side only)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle.pinv_oracle as O


@dataclass
class OracleResult:
    E: np.ndarray
    lam: float
    G: np.ndarray
    L: np.ndarray
    Ginv: np.ndarray
    R: np.ndarray
    images: np.ndarray   # [F][N], direct solve L^-H L^-1 E^H d
    images_recon: np.ndarray  # [F][N], Recon x data


def oracle_all(p, vox=None, data=None) -> OracleResult:
    """Every stage of the explicit path from the oracle, for one plan."""
    E = O.plan_encode(p, vox)
    lam = O.lambda_abs(E, p.lambda_rel)
    G = O.gram(E, lam)
    L = O.cholesky(G)
    W = O.inverse_lower(L)
    Ginv = W.conj().T @ W
    R = W.conj().T @ (W @ E.conj().T)
    d = p.data if data is None else data
    cols = O.data_columns(d)
    images = O.solve(E, L, cols).T
    images_recon = O.reconstruct(R, cols).T
    return OracleResult(E, lam, G, L, Ginv, R, images, images_recon)


def rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
