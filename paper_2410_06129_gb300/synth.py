"""Seeded synthetic MRI workloads (inputs only).

This module draws the inputs that both the CUDA path and the FP64 oracle
consume: k-space trajectories, coil sensitivity maps, B0 off-resonance maps,
readout times, ellipse phantoms and k-space data. It holds none of the
reconstruction arithmetic: the k-space data are the *continuous* Fourier
transform of the ellipse phantom (closed form, Bessel J1), not the discrete
encoding model data = Encode x image of Eq. 1, so no input is produced by the
method being tested. The paper's in-vivo datasets (Sections 4.1-4.5) are not
available; these generators stand in for their shape classes: variable-density
spirals (Sections 4.1, 4.2, 3.2), radial spokes (Section 4.4), smooth
sum-of-squares-normalised coil maps (Section 6), a smooth B0 map (Section 3.3,
Supplementary 3) and time-modulated phantoms for dynamic series (Section 4.1).

Conventions shared by both sides (they are input conventions, not method):
  * voxel n of a grid (nx, ny[, nz]) sits at r = ((i - dims/2) / dims) * fov,
    with x fastest: n = (iz * ny + iy) * nx + ix;
  * k is in cycles per unit length (cycles/FOV when fov = 1);
  * complex arrays are numpy complex128; data are laid out [F][C][M_k].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import j1

DWELL_S = 4e-6  # sampling dwell of every readout (seconds)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
def voxel_positions(dims, fov=None) -> np.ndarray:
    """[N][D] voxel centres for a Cartesian grid, x fastest."""
    dims = tuple(int(d) for d in dims)
    fov = (1.0,) * len(dims) if fov is None else tuple(float(f) for f in fov)
    axes = [((np.arange(d) - d / 2.0) / d) * f for d, f in zip(dims, fov)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")  # slowest first
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


def spiral(side: int, n_interleaves: int, samples_per_interleave: int):
    """Variable-density Archimedean spiral (denser centre), |k| <= side/2.

    Returns (k [M_k][2], readout_index [M_k]) where readout_index is the
    sample's position within its interleave (used for readout times).
    """
    kmax = side / 2.0
    J, S = int(n_interleaves), int(samples_per_interleave)
    n_turns = math.ceil(1.5 * kmax / J)
    tau = np.arange(S) / max(S - 1, 1)
    rho = kmax * tau ** 1.5
    ks, idx = [], []
    for j in range(J):
        theta = 2 * np.pi * n_turns * tau + 2 * np.pi * j / J
        ks.append(np.stack([rho * np.cos(theta), rho * np.sin(theta)], axis=1))
        idx.append(np.arange(S))
    return np.concatenate(ks), np.concatenate(idx)


def radial(side: int, n_spokes: int, samples_per_spoke: int):
    """Radial spokes through the k-space centre at angles pi*p/P."""
    kmax = side / 2.0
    P, S = int(n_spokes), int(samples_per_spoke)
    kap = kmax * (2 * np.arange(S) - S) / S
    ks, idx = [], []
    for p in range(P):
        th = np.pi * p / P
        ks.append(np.stack([kap * np.cos(th), kap * np.sin(th)], axis=1))
        idx.append(np.arange(S))
    return np.concatenate(ks), np.concatenate(idx)


def cartesian(side: int):
    """Fully sampled Cartesian grid k in {-side/2 .. side/2-1}^2, x fastest."""
    g = np.arange(side) - side // 2
    ky, kx = np.meshgrid(g, g, indexing="ij")
    k = np.stack([kx.ravel(), ky.ravel()], axis=1).astype(np.float64)
    return k, np.arange(k.shape[0]) % side


# --------------------------------------------------------------------------
# physics maps
# --------------------------------------------------------------------------
def coil_maps(dims, n_coils: int, rng: np.random.Generator) -> np.ndarray:
    """[C][N] smooth complex maps normalised to sum-of-squares 1 per voxel."""
    r = voxel_positions(dims)[:, :2]
    if n_coils == 1:
        return np.ones((1, r.shape[0]), dtype=np.complex128)
    maps = []
    for c in range(n_coils):
        ang = 2 * np.pi * c / n_coils
        centre = 0.6 * np.array([np.cos(ang), np.sin(ang)])
        mag = np.exp(-np.sum((r - centre) ** 2, axis=1) / (2 * 0.5 ** 2))
        phi0 = rng.uniform(0, 2 * np.pi)
        a_len, a_ang = 0.5 * np.sqrt(rng.uniform()), rng.uniform(0, 2 * np.pi)
        a = a_len * np.array([np.cos(a_ang), np.sin(a_ang)])
        maps.append(mag * np.exp(1j * (phi0 + 2 * np.pi * (r @ a))))
    maps = np.array(maps)
    return maps / np.sqrt(np.sum(np.abs(maps) ** 2, axis=0, keepdims=True))


def b0_map(dims, rng: np.random.Generator, max_hz: float = 50.0) -> np.ndarray:
    """[N] smooth off-resonance map in Hz, max |df| = max_hz."""
    r = voxel_positions(dims)[:, :2]
    f = np.zeros(r.shape[0])
    for _ in range(3):
        c = rng.uniform(-0.4, 0.4, size=2)
        w = rng.uniform(0.1, 0.3)
        f += rng.uniform(-1, 1) * np.exp(-np.sum((r - c) ** 2, axis=1) / (2 * w * w))
    return f * (max_hz / np.max(np.abs(f)))


@dataclass
class Ellipses:
    centre: np.ndarray   # [E][2]
    axes: np.ndarray     # [E][2] semi-axes
    angle: np.ndarray    # [E]
    amp: np.ndarray      # [E] complex
    tau: np.ndarray      # [E] decay constants (frames)


def ellipses(rng: np.random.Generator, n: int = 10) -> Ellipses:
    return Ellipses(
        centre=rng.uniform(-0.3, 0.3, size=(n, 2)),
        axes=rng.uniform(0.05, 0.25, size=(n, 2)),
        angle=rng.uniform(0, np.pi, size=n),
        amp=rng.uniform(0.2, 1.0, size=n) * np.exp(1j * rng.uniform(0, 2 * np.pi, size=n)),
        tau=rng.uniform(16, 256, size=n),
    )


def _frame_amps(e: Ellipses, frame: int) -> np.ndarray:
    return e.amp * np.exp(-frame / e.tau)


def phantom_image(e: Ellipses, dims, frame: int = 0) -> np.ndarray:
    """[N] summed ellipse indicators at the voxel centres (ground truth)."""
    r = voxel_positions(dims)[:, :2]
    amps = _frame_amps(e, frame)
    x = np.zeros(r.shape[0], dtype=np.complex128)
    for i in range(len(amps)):
        d = r - e.centre[i]
        ca, sa = np.cos(e.angle[i]), np.sin(e.angle[i])
        u = (d[:, 0] * ca + d[:, 1] * sa) / e.axes[i, 0]
        v = (-d[:, 0] * sa + d[:, 1] * ca) / e.axes[i, 1]
        x += amps[i] * (u * u + v * v <= 1.0)
    return x


def _ellipse_ft(k: np.ndarray, centre, axes, angle) -> np.ndarray:
    """Continuous Fourier transform of an ellipse indicator, exp(-i2pi k.r)."""
    ca, sa = np.cos(angle), np.sin(angle)
    ku = k[:, 0] * ca + k[:, 1] * sa
    kv = -k[:, 0] * sa + k[:, 1] * ca
    rho = np.sqrt((axes[0] * ku) ** 2 + (axes[1] * kv) ** 2)
    safe = np.where(rho > 1e-12, rho, 1.0)
    jinc = np.where(rho > 1e-12, j1(2 * np.pi * safe) / safe, np.pi)
    return axes[0] * axes[1] * jinc * np.exp(-2j * np.pi * (k @ centre))


def kspace_data(e: Ellipses, k: np.ndarray, n_vox: int, n_coils: int, frames: int,
                rng: np.random.Generator, noise_frac: float = 0.01) -> np.ndarray:
    """[F][C][M_k] k-space data: analytic phantom spectrum per coil + noise.

    Each coil sees the phantom spectrum shifted by a small per-coil k offset
    and rotated by a per-coil phase (a plane-wave sensitivity), scaled by the
    voxel count so magnitudes match a discrete sum over n_vox voxels.
    Complex Gaussian noise n = sigma/sqrt(2) (g1 + i g2) with sigma =
    noise_frac * RMS(signal) is added.
    """
    M = k.shape[0]
    shifts = rng.uniform(-0.5, 0.5, size=(n_coils, 2)) if n_coils > 1 else np.zeros((1, 2))
    phases = np.exp(1j * rng.uniform(0, 2 * np.pi, size=n_coils)) if n_coils > 1 else np.ones(1)
    weight = 1.0 / np.sqrt(n_coils)
    basis = np.empty((n_coils, len(e.amp), M), dtype=np.complex128)
    for c in range(n_coils):
        kc = k - shifts[c]
        for i in range(len(e.amp)):
            basis[c, i] = _ellipse_ft(kc, e.centre[i], e.axes[i], e.angle[i])
    data = np.empty((frames, n_coils, M), dtype=np.complex128)
    for f in range(frames):
        a = _frame_amps(e, f)
        data[f] = n_vox * weight * phases[:, None] * np.einsum("e,cem->cm", a, basis)
    sigma = noise_frac * np.sqrt(np.mean(np.abs(data) ** 2))
    noise = rng.standard_normal(data.shape) + 1j * rng.standard_normal(data.shape)
    return data + (sigma / np.sqrt(2.0)) * noise


# --------------------------------------------------------------------------
# plan inputs
# --------------------------------------------------------------------------
@dataclass
class PlanInputs:
    """Everything a reconstruction plan is built from, plus its data."""
    dims: tuple
    traj: np.ndarray                 # [M_k][D] float64
    coil_maps: np.ndarray | None     # [C][N] complex128 or None (single coil, s = 1)
    b0_hz: np.ndarray | None         # [N] float64 or None
    times: np.ndarray | None         # [M_k] float64 seconds or None
    lambda_rel: float                # lambda = lambda_rel * trace(E^H E) / N
    data: np.ndarray                 # [F][C][M_k] complex128
    truth: np.ndarray                # [F][N] complex128 phantom at voxel centres
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_vox(self) -> int:
        return int(np.prod(self.dims))

    @property
    def n_coils(self) -> int:
        return 1 if self.coil_maps is None else self.coil_maps.shape[0]

    @property
    def n_samples(self) -> int:
        return self.traj.shape[0]


def make_plan(side: int, n_coils: int, traj: str, n_frames: int, seed: int,
              lambda_rel: float, samples: int | None = None, interleaves: int | None = None,
              b0: bool = False, spokes: int | None = None, per_spoke: int | None = None,
              noise_frac: float = 0.01, name: str = "") -> PlanInputs:
    """One seeded 2D plan. traj in {"spiral", "radial", "cartesian"}."""
    rng = np.random.default_rng(seed)
    dims = (side, side)
    N = side * side
    if traj == "spiral":
        J = interleaves or max(1, side // 16)
        S = (samples or 2 * N) // J
        k, s_idx = spiral(side, J, S)
    elif traj == "radial":
        S = per_spoke or 2 * side
        P = spokes or max(1, (samples or 2 * N) // S)
        k, s_idx = radial(side, P, S)
    elif traj == "cartesian":
        k, s_idx = cartesian(side)
    else:
        raise ValueError(traj)
    maps = coil_maps(dims, n_coils, rng) if n_coils > 1 else None
    b0map = b0_map(dims, rng) if b0 else None
    times = (s_idx * DWELL_S).astype(np.float64) if b0 else None
    if n_frames == 0:  # geometry only (e.g. serving plans, whose data are drawn per request)
        return PlanInputs(dims=dims, traj=k, coil_maps=maps, b0_hz=b0map, times=times,
                          lambda_rel=lambda_rel, data=None, truth=None, name=name)
    e = ellipses(rng)
    data = kspace_data(e, k, N, n_coils, n_frames, rng, noise_frac)
    truth = np.stack([phantom_image(e, dims, f) for f in range(n_frames)])
    return PlanInputs(dims=dims, traj=k, coil_maps=maps, b0_hz=b0map, times=times,
                      lambda_rel=lambda_rel, data=data, truth=truth, name=name)


def config(i: int, reduced: bool = False, frames: int | None = None) -> PlanInputs | list:
    """The five workload configurations (seed = 1000 * i + index).

    1: 32x32 single coil, one spiral of 2048 samples, lambda_rel 1e-3, 1 frame.
    2: 64x64, 8 coils, 4 interleaved spirals x 2048, lambda_rel 1e-4, 64 frames.
    3: 16 uneven plans (side {24..96}, 1-8 coils, spiral/radial, 1-4 x N samples),
       256 frames each (a list of PlanInputs).
    4: 32 cached plans for the serving loop (side {32..128}, coils {1..16},
       1-2 x N samples), generated lazily by serve_plans().
    5: 192x192, 8 coils, 384 radial spokes x 125 samples, B0 +-50 Hz, 64 frames.
    reduced=True shrinks the image side (and samples proportionally) so the
    oracle finishes in seconds while still spanning several kernel tiles.
    """
    if i == 1:
        side = 24 if reduced else 32
        return make_plan(side, 1, "spiral", 1 if frames is None else frames, 1000, 1e-3,
                         samples=2 * side * side, interleaves=1, name="cfg1")
    if i == 2:
        side = 24 if reduced else 64
        spi = 2048 if not reduced else (2 * side * side) // 4
        return make_plan(side, 8, "spiral", (4 if reduced else 64) if frames is None else frames, 2000, 1e-4,
                         samples=4 * spi, interleaves=4, name="cfg2")
    if i == 3:
        rng = np.random.default_rng(3000)
        plans = []
        for p in range(16):
            side = int(rng.choice([24, 32, 48, 64, 96] if not reduced else [8, 12, 16]))
            C = int(rng.integers(1, 9))
            kind = "spiral" if rng.uniform() < 0.5 else "radial"
            mult = int(rng.integers(1, 5))
            nf = (256 if not reduced else 4) if frames is None else frames
            plans.append(make_plan(side, C, kind, nf, 3000 + p + 1, 1e-3, samples=mult * side * side,
                                   name=f"cfg3.{p}"))
        return plans
    if i == 4:
        return serve_plans(reduced=reduced)
    if i == 5:
        side, P, S = (192, 384, 125) if not reduced else (32, 64, 40)
        nf = (64 if not reduced else 2) if frames is None else frames
        return make_plan(side, 8, "radial", nf, 5000, 1e-4, b0=True, spokes=P, per_spoke=S, name="cfg5")
    raise ValueError(i)


def serve_plans(reduced: bool = False, n: int = 32, side_div: int = 1) -> list:
    """Plan descriptors (no data) of the serving workload, seed 4000.

    side_div > 1 divides every image side (same draws, so the same mix of
    sizes, coil counts and trajectories at a smaller scale)."""
    rng = np.random.default_rng(4000)
    out = []
    for p in range(n):
        side = int(rng.choice([32, 48, 64, 96, 128] if not reduced else [8, 12, 16])) // side_div
        C = int(rng.choice([1, 2, 4, 8, 16] if not reduced else [1, 2, 4]))
        mult = int(rng.integers(1, 3))
        kind = "spiral" if p % 2 == 0 else "radial"
        out.append(dict(side=side, n_coils=C, traj=kind, samples=mult * side * side,
                        seed=4000 + p + 1, lambda_rel=1e-3))
    return out


def serve_plan_inputs(d: dict) -> PlanInputs:
    """Geometry (trajectory, coil maps, lambda) of one serve_plans() entry."""
    return make_plan(d["side"], d["n_coils"], d["traj"], 0, d["seed"], d["lambda_rel"],
                     samples=d["samples"], name=f"serve.{d['seed'] - 4000}")


def serve_trace(rate_hz: float, duration_s: float, n_plans: int, seed: int = 4100,
                max_frames: int = 64):
    """Poisson arrival trace: list of (t_arrival_s, plan_index, n_frames)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return out
        out.append((t, int(rng.integers(0, n_plans)), int(rng.integers(1, max_frames + 1))))
