"""Wider encodings on the same path (Section 2.2, Section 3.3).

* Underdetermined plans (fewer samples than voxels): with lambda > 0 the left form
  the library computes equals the right pseudoinverse (push-through identity,
  pinned in test_oracle_pins.py), so the images must match the oracle's.
* Chemical-shift species: a second species is a copy of the voxel grid whose
  off-resonance term carries the species' frequency offset, i.e. explicit voxel
  indices listed twice with per-copy B0. The encoding is then [E_water | E_fat]
  (Section 3.3's product of encoding factors), and the oracle builds it directly.
Bars: FP64 1e-10 (NRMSE), mixed 1e-4 after refinement.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.pinv_oracle as O  # noqa: E402
from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402
from tests._ref import rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()


def _precisions():
    out = [(L.FP64, 1e-10)]
    if L.load().pinv_tc_available():
        out.append((L.MIXED_BF16X6, 1e-4))
    return out


def _oracle_images(E, lam_rel, d):
    lam = O.lambda_abs(E, lam_rel)
    L_ = O.cholesky(O.gram(E, lam))
    return O.back_substitution_h(L_, O.forward_substitution(L_, E.conj().T @ d)).T


@pytest.mark.parametrize("prec,tol", _precisions())
def test_underdetermined_plan_matches_oracle(prec, tol):
    """12 x 12 grid (N = 144) from one spiral of 96 samples."""
    from paper_2410_06129_gb300.plan import Plan
    side, lam_rel = 12, 1e-2
    k, _ = synth.spiral(side, 1, 96)
    vox = O.voxel_positions((side, side))
    E = O.encode(k, vox)
    rng = np.random.default_rng(41)
    x = rng.standard_normal((2, side * side)) + 1j * rng.standard_normal((2, side * side))
    d = (E @ x.T).T
    pl = Plan((side, side), k, lam=lam_rel, precision=prec, refine_max_iters=None).build()
    img = pl.apply(torch.from_numpy(np.ascontiguousarray(d)).cuda()).cpu().numpy()
    assert rel(img, _oracle_images(E, lam_rel, d.T)) < tol


@pytest.mark.parametrize("prec,tol", _precisions())
def test_chemical_shift_species_as_voxel_copies(prec, tol):
    """Water and fat (-440 Hz) on a 10 x 10 grid, 2 coils, radial readouts with a
    4 us dwell and a smooth B0 map: N = 200 unknowns from 2 x 640 samples."""
    from paper_2410_06129_gb300.plan import Plan
    side, lam_rel = 10, 1e-3
    rng = np.random.default_rng(42)
    k, s_idx = synth.radial(side, 16, 40)
    times = s_idx * synth.DWELL_S
    grid = np.arange(side * side)
    maps = synth.coil_maps((side, side), 2, rng)
    b0 = synth.b0_map((side, side), rng)
    vidx = np.concatenate([grid, grid]).astype(np.int64)
    b0_species = np.concatenate([b0, b0 - 440.0])
    maps_species = np.concatenate([maps, maps], axis=1)
    vox = O.voxel_positions((side, side))[vidx]
    E = O.encode(k, vox, maps_species, b0_species, times)
    x = rng.standard_normal((2, 2 * side * side)) + 1j * rng.standard_normal((2, 2 * side * side))
    d = (E @ x.T).T
    pl = Plan((side, side), k, coil_maps=maps_species, b0_hz=b0_species, times=times, lam=lam_rel,
              precision=prec, voxel_index=vidx).build()
    img = pl.apply(torch.from_numpy(np.ascontiguousarray(d)).cuda()).cpu().numpy()
    assert img.shape == (2, 2 * side * side)
    assert rel(img, _oracle_images(E, lam_rel, d.T)) < tol
