"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks retypes the oracle's own formula: each one compares the
oracle with an independent library routine (numpy SVD, pinv, FFT, eigvalsh),
a closed form, or an identity the paper states. The "planted mistake" tests at
the end show that a plausible slip in the oracle (dropped conjugate, wrong
sign, missing lambda, transposed operand) makes one of these pins fail.
"""
import numpy as np
import pytest

import oracle.pinv_oracle as O
from paper_2410_06129_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rand_complex(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _small_plan(seed=7, side=8, coils=3, b0=True, traj="spiral"):
    return synth.make_plan(side, coils, traj, 3, seed, 1e-3, samples=2 * side * side,
                           interleaves=2, b0=b0)


def _svd_tikhonov(E, lam, d):
    """x = V diag(s / (s^2 + lam)) U^H d  (Eq. 4 spectrum + Eq. 6 load)."""
    U, s, Vh = np.linalg.svd(E, full_matrices=False)
    return Vh.conj().T @ ((s / (s * s + lam))[:, None] * (U.conj().T @ d))


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tikhonov_matches_svd_random_matrix(seed):
    """Eq. 6/8 via Cholesky equals the SVD-filtered solution (Section 3.2)."""
    rng = np.random.default_rng(seed)
    E = _rand_complex(rng, 70, 40)
    d = _rand_complex(rng, 70, 3)
    lam = 0.3
    R, _ = O.recon_matrix(E, lam)
    x = O.reconstruct(R, d)
    ref = _svd_tikhonov(E, lam, d)
    assert O.nrmse(x, ref) < 1e-12


def test_tikhonov_matches_svd_encoding_matrix():
    p = _small_plan()
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    R, _ = O.recon_matrix(E, lam)
    d = O.data_columns(p.data)
    assert O.nrmse(O.reconstruct(R, d), _svd_tikhonov(E, lam, d)) < 1e-12


def test_lambda_zero_is_moore_penrose():
    """With lambda = 0 and full column rank, Recon = E^+ (Section 2.1)."""
    rng = np.random.default_rng(3)
    E = _rand_complex(rng, 60, 25)
    R, _ = O.recon_matrix(E, 0.0)
    assert O.nrmse(R, np.linalg.pinv(E)) < 1e-11


def test_gram_eigenvalues_are_squared_singular_values():
    """Eigenvalues of E^H E + lam I are sigma^2 + lam (Section 2.2)."""
    p = _small_plan(seed=11)
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    G = O.gram(E, lam)
    ev = np.sort(np.linalg.eigvalsh(G))
    sv = np.sort(np.linalg.svd(E, compute_uv=False) ** 2 + lam)
    assert np.max(np.abs(ev - sv)) / sv[-1] < 1e-12


# ---------------------------------------------------------------- closed form
@pytest.mark.parametrize("side", [8, 16])
def test_cartesian_closed_form(side):
    """Fully sampled Cartesian: E^H E = N I and E^H d is an inverse DFT."""
    k, _ = synth.cartesian(side)
    vox = O.voxel_positions((side, side))
    E = O.encode(k, vox)
    N = side * side
    lam = 0.25 * N
    G = O.gram(E, lam)
    assert np.max(np.abs(G - (N + lam) * np.eye(N))) < 1e-10 * N
    rng = np.random.default_rng(side)
    d = _rand_complex(rng, N)
    R, _ = O.recon_matrix(E, lam)
    x = R @ d
    # closed form: x = E^H d / (N + lam) with E^H d = (-1)^(ix+iy) N ifft2(d (-1)^(jx+jy))
    j = np.arange(side)
    sgn = ((-1.0) ** (j[:, None] + j[None, :]))
    dg = d.reshape(side, side)                     # [jy][jx]
    adj = sgn * (N * np.fft.ifft2(dg * sgn))       # [iy][ix] (even side)
    assert O.nrmse(x, adj.ravel() / (N + lam)) < 1e-12


def test_lambda_closed_form_sos_coils():
    """trace(E^H E)/N = M_k exactly for sum-of-squares normalised coils."""
    p = _small_plan(seed=5, coils=4)
    E = O.plan_encode(p)
    assert abs(O.lambda_abs(E, 1.0) - p.n_samples) < 1e-10 * p.n_samples


# ---------------------------------------------------------------- invariants
def test_gram_hermitian_pd_and_cholesky():
    p = _small_plan(seed=3)
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    G = O.gram(E, lam)
    assert np.max(np.abs(G - G.conj().T)) <= 1e-14 * np.max(np.abs(G))
    L = O.cholesky(G)
    assert np.allclose(np.triu(L, 1), 0)
    assert np.max(np.abs(L @ L.conj().T - G)) < 1e-13 * np.max(np.abs(G))
    assert np.all(np.real(np.diag(L)) ** 2 >= lam * (1 - 1e-12))
    ref = np.linalg.cholesky(G)
    assert np.max(np.abs(L - ref)) < 1e-12 * np.max(np.abs(ref))


def test_cholesky_rejects_indefinite():
    G = np.diag([1.0, 2.0, -1.0, 3.0]).astype(np.complex128)
    with pytest.raises(ValueError, match="pivot 2"):
        O.cholesky(G)


def test_normal_equation_residual_and_direct_solve():
    p = _small_plan(seed=4)
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    d = O.data_columns(p.data)
    R, L = O.recon_matrix(E, lam)
    x = O.reconstruct(R, d)
    res = E.conj().T @ (d - E @ x) - lam * x
    assert np.linalg.norm(res) / np.linalg.norm(E.conj().T @ d) < 1e-12
    x2 = O.solve(E, L, d)
    assert O.nrmse(x2, x) < 1e-12


def test_srf_tikhonov_identity():
    """SRF = Recon Encode = I - lam G^-1 exactly under Tikhonov (Eq. 9)."""
    p = _small_plan(seed=6)
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    R, L = O.recon_matrix(E, lam)
    Ginv = O.gram_inverse(L)
    S = O.srf(R, E)
    assert np.max(np.abs(S + lam * Ginv - np.eye(E.shape[1]))) < 1e-11
    assert np.max(np.abs(Ginv @ O.gram(E, lam) - np.eye(E.shape[1]))) < 1e-11


def test_noise_matrix_white_noise_identity():
    """X = Recon Recon^H = G^-1 - lam G^-2 for white noise (Eq. 10)."""
    p = _small_plan(seed=8)
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    R, L = O.recon_matrix(E, lam)
    Ginv = O.gram_inverse(L)
    X = O.noise_matrix(R, np.eye(E.shape[0]))
    assert np.max(np.abs(X - (Ginv - lam * Ginv @ Ginv))) < 1e-11 * np.max(np.abs(Ginv))


def test_noise_matrix_signal_shaped_noise_closed_form():
    """Noise with covariance Psi = E E^H (shaped like the signal) maps to
    X = (Recon E)(Recon E)^H = (I - lam G^-1)(I - lam G^-1)^H by Eq. 9's
    Tikhonov identity (Eq. 10). G^-1 here comes from numpy's inverse, not
    from the oracle, and Psi is complex, so Psi^T != Psi."""
    p = _small_plan(seed=16, coils=3)
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    R, _ = O.recon_matrix(E, lam)
    Ginv = np.linalg.inv(E.conj().T @ E + lam * np.eye(E.shape[1]))
    S = np.eye(E.shape[1]) - lam * Ginv
    X = O.noise_matrix(R, E @ E.conj().T)
    assert np.max(np.abs(X - S @ S.conj().T)) < 1e-10


def _coil_covariance(C, rng):
    """A complex Hermitian positive definite C x C coil covariance with strong
    imaginary off-diagonal terms, and a square root P with P P^H = psi."""
    P = np.tril(rng.standard_normal((C, C)) + 1j * rng.standard_normal((C, C)))
    P[np.diag_indices(C)] = np.abs(P[np.diag_indices(C)]) + 1.0
    return P @ P.conj().T, P


def test_noise_matrix_coil_covariance_monte_carlo():
    """Eq. 10 defines X as the covariance of the reconstructed noise. Draw
    k-space noise with coil covariance psi per sample (n = (P (x) I) g, g white
    complex Gaussian), reconstruct it with Recon and compare the sample
    covariance of the images with the oracle's X for Psi = psi (x) I. Only the
    diagonal-dominant relative error of a 1 / sqrt(K) estimate is asked for."""
    rng = np.random.default_rng(17)
    p = _small_plan(seed=17, side=6, coils=3)
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    R, _ = O.recon_matrix(E, lam)
    C, Mk = p.coil_maps.shape[0], p.n_samples
    psi, P = _coil_covariance(C, rng)
    X = O.noise_matrix(R, np.kron(psi, np.eye(Mk)))
    K = 40000
    g = (rng.standard_normal((C, Mk, K)) + 1j * rng.standard_normal((C, Mk, K))) / np.sqrt(2.0)
    n = np.einsum("ab,bmk->amk", P, g).reshape(C * Mk, K)
    xs = R @ n
    X_mc = xs @ xs.conj().T / K
    assert np.linalg.norm(X_mc - X) / np.linalg.norm(X) < 0.03


def test_planted_transposed_psi_fails_noise_pins(monkeypatch):
    """Using Psi^T (= conj(Psi) for a Hermitian Psi) instead of Psi, a
    plausible slip, fails both coloured-noise pins."""
    monkeypatch.setattr(O, "noise_matrix", lambda R, psi: R @ psi.T @ R.conj().T)
    with pytest.raises(AssertionError):
        test_noise_matrix_signal_shaped_noise_closed_form()
    with pytest.raises(AssertionError):
        test_noise_matrix_coil_covariance_monte_carlo()


def test_coil_procedural_equals_stacked_and_hadamard():
    """Eq. 11: sum_c E_c^H E_c = E^H E, and it equals (A^H A) o (S^H S)."""
    p = _small_plan(seed=9, coils=4)
    vox = O.voxel_positions(p.dims)
    E = O.plan_encode(p)
    G_stacked = E.conj().T @ E
    G_proc = sum(
        (lambda Ec: Ec.conj().T @ Ec)(O.encode(p.traj, vox, [s], p.b0_hz, p.times))
        for s in p.coil_maps)
    A = O.encode(p.traj, vox, None, p.b0_hz, p.times)
    S = p.coil_maps
    G_had = (A.conj().T @ A) * (S.conj().T @ S)
    scale = np.max(np.abs(G_stacked))
    assert np.max(np.abs(G_proc - G_stacked)) < 1e-12 * scale
    assert np.max(np.abs(G_had - G_stacked)) < 1e-12 * scale


def test_large_lambda_is_conjugate_phase():
    """lam -> inf: lam * x -> E^H d (Section 2.2, conjugate phase)."""
    p = _small_plan(seed=10)
    E = O.plan_encode(p)
    d = O.data_columns(p.data)
    lam = 1e8 * O.lambda_abs(E, 1.0)
    R, _ = O.recon_matrix(E, lam)
    assert O.nrmse(lam * (R @ d), E.conj().T @ d) < 1e-6


def test_linear_b0_map_equals_shifted_trajectory():
    """A linear off-resonance map df(r) = g . r adds g t_m to every k_m: the
    B0 factor exp(-i2pi df t) and the Fourier factor exp(-i2pi k . r) combine
    into exp(-i2pi (k + g t) . r) (Section 3.3, composite encoding). So the
    oracle's B0 encoding must equal its B0-free encoding of the trajectory
    k_m + g t_m. This fixes the sign of the B0 term relative to the Fourier
    term and which index (sample m, voxel n) each factor follows."""
    p = _small_plan(seed=12, coils=2)
    vox = O.voxel_positions(p.dims)
    g = np.array([37.0, -21.0])                  # Hz per unit length
    b0 = vox @ g
    t = p.times
    E_b0 = O.encode(p.traj, vox, p.coil_maps, b0, t)
    E_shift = O.encode(p.traj + np.outer(t, g), vox, p.coil_maps)
    assert np.max(np.abs(E_b0 - E_shift)) < 1e-12


def test_uniform_b0_is_a_phase_per_sample():
    """A spatially uniform offset df multiplies sample m of every coil by
    exp(-i2pi df t_m), independent of the voxel (Section 3.3)."""
    p = _small_plan(seed=14, coils=3)
    vox = O.voxel_positions(p.dims)
    df = 23.5
    E0 = O.encode(p.traj, vox, p.coil_maps)
    E1 = O.encode(p.traj, vox, p.coil_maps, np.full(vox.shape[0], df), p.times)
    ph = np.tile(np.exp(-2j * np.pi * df * p.times), p.coil_maps.shape[0])
    assert np.max(np.abs(E1 - ph[:, None] * E0)) < 1e-12


def test_b0_time_shift_is_a_voxel_phase():
    """Adding the same delay T to every sample time multiplies column n by
    exp(-i2pi df_n T): the B0 phase accrues linearly in time (Section 3.3)."""
    p = _small_plan(seed=15, coils=2)
    vox = O.voxel_positions(p.dims)
    T = 1.3e-3
    E0 = O.encode(p.traj, vox, p.coil_maps, p.b0_hz, p.times)
    E1 = O.encode(p.traj, vox, p.coil_maps, p.b0_hz, p.times + T)
    ph = np.exp(-2j * np.pi * p.b0_hz * T)
    assert np.max(np.abs(E1 - E0 * ph[None, :])) < 1e-11


def test_voxel_positions_convention():
    r = O.voxel_positions((4, 2))
    assert r.shape == (8, 2)
    assert np.allclose(r[0], [-0.5, -0.5]) and np.allclose(r[1], [-0.25, -0.5])
    assert np.allclose(r[4], [-0.5, 0.0])
    assert np.allclose(r, synth.voxel_positions((4, 2)))


# ---------------------------------------------------------------- planted mistakes
def _bad_cholesky_no_conj(G):
    n = G.shape[0]
    L = np.zeros_like(G, dtype=np.complex128)
    for j in range(n):
        L[j, j] = np.sqrt(np.real(G[j, j]) - np.sum(np.abs(L[j, :j]) ** 2))
        L[j + 1:, j] = (G[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def _bad_back_sub_transposed(L, B):
    X = np.zeros_like(B, dtype=np.complex128)
    for i in range(L.shape[0] - 1, -1, -1):
        X[i] = (B[i] - L[i + 1:, i] @ X[i + 1:]) / L[i, i]
    return X


@pytest.mark.parametrize("mutation", ["chol_no_conj", "no_lambda", "back_sub_no_conj"])
def test_planted_mistake_fails_svd_pin(monkeypatch, mutation):
    rng = np.random.default_rng(42)
    E = _rand_complex(rng, 50, 20)
    d = _rand_complex(rng, 50, 2)
    lam = 0.5
    if mutation == "chol_no_conj":
        monkeypatch.setattr(O, "cholesky", _bad_cholesky_no_conj)
    elif mutation == "no_lambda":
        monkeypatch.setattr(O, "gram", lambda E, lam: E.conj().T @ E)
    else:
        monkeypatch.setattr(O, "back_substitution_h", _bad_back_sub_transposed)
    L = O.cholesky(O.gram(E, lam))
    x = O.back_substitution_h(L, O.forward_substitution(L, E.conj().T @ d))
    assert O.nrmse(x, _svd_tikhonov(E, lam, d)) > 1e-6


def test_planted_sign_flip_fails_cartesian_pin():
    side = 8
    k, _ = synth.cartesian(side)
    vox = O.voxel_positions((side, side))
    E_bad = np.conj(O.encode(k, vox))          # exp(+i2pi k.r)
    rng = np.random.default_rng(1)
    d = _rand_complex(rng, side * side)
    j = np.arange(side)
    sgn = ((-1.0) ** (j[:, None] + j[None, :]))
    adj = sgn * (side * side * np.fft.ifft2(d.reshape(side, side) * sgn))
    assert O.nrmse(E_bad.conj().T @ d, adj.ravel()) > 1e-3


def test_planted_b0_sign_flip_fails_b0_pins(monkeypatch):
    """exp(+i2pi df t) in the B0 factor (the sign the paper prints for its
    exponentials, reading 1) fails the linear-map and uniform-offset pins."""
    good = O.encode

    def flipped(traj, vox, coil_maps=None, b0_hz=None, times=None):
        E = good(traj, vox, coil_maps, None, None)
        if b0_hz is None:
            return E
        ph = np.exp(2j * np.pi * np.outer(np.asarray(times), np.asarray(b0_hz)))
        C = 1 if coil_maps is None else len(coil_maps)
        return E * np.tile(ph, (C, 1))
    monkeypatch.setattr(O, "encode", flipped)
    with pytest.raises(AssertionError):
        test_linear_b0_map_equals_shifted_trajectory()
    with pytest.raises(AssertionError):
        test_uniform_b0_is_a_phase_per_sample()


def test_planted_b0_index_swap_fails_time_shift_pin(monkeypatch):
    """Pairing each sample's time with the wrong voxel's offset (the B0 factor
    built from a reversed voxel order) fails the time-shift pin."""
    good = O.encode
    monkeypatch.setattr(O, "encode", lambda traj, vox, cm=None, b0=None, t=None:
                        good(traj, vox, cm, None if b0 is None else np.asarray(b0)[::-1], t))
    with pytest.raises(AssertionError):
        test_b0_time_shift_is_a_voxel_phase()


# ---------------------------------------------------------------- eigen / tSVD (Section 2.1)
def test_gram_eig_reconstructs_and_matches_svd():
    """P diag(mu) P^H = E^H E with orthonormal P, and mu (decreasing) are the
    squared singular values of E from an SVD (a different factorisation)."""
    p = _small_plan(seed=13, coils=2)
    E = O.plan_encode(p)
    mu, P = O.gram_eig(E)
    G0 = E.conj().T @ E
    assert np.all(np.diff(mu) <= 1e-9 * mu[0])
    assert np.max(np.abs(P.conj().T @ P - np.eye(len(mu)))) < 1e-12
    assert np.max(np.abs(P @ np.diag(mu) @ P.conj().T - G0)) < 1e-11 * mu[0]
    sv = np.linalg.svd(E, compute_uv=False) ** 2
    assert np.max(np.abs(mu - sv)) < 1e-11 * mu[0]


def test_gram_eig_cartesian_closed_form():
    """Fully sampled Cartesian single coil: E^H E = N I, so every eigenvalue is N."""
    side = 8
    k, _ = synth.cartesian(side)
    E = O.encode(k, O.voxel_positions((side, side)))
    mu, _ = O.gram_eig(E)
    N = side * side
    assert np.max(np.abs(mu - N)) < 1e-10 * N


def test_tsvd_rank_and_condition_hand_example():
    """mu = (4, 3, 2, 1): cumulative energy 4, 7, 9, 10; 70 % -> r = 2, kappa =
    sqrt(4 / 3); 100 % keeps everything."""
    mu = np.array([4.0, 3.0, 2.0, 1.0])
    assert O.tsvd_rank(mu, 0.7) == 2
    assert O.tsvd_rank(mu, 0.71) == 3
    assert O.tsvd_rank(mu, 1.0) == 4
    assert abs(O.tsvd_condition(mu, 2) - np.sqrt(4.0 / 3.0)) < 1e-15


def test_tsvd_full_rank_equals_normal_equation_solution():
    """With every eigenvalue kept and no loading, the truncated reconstruction is
    the least-squares solution, here from the oracle's Cholesky path at lam = 0."""
    rng = np.random.default_rng(21)
    E = _rand_complex(rng, 60, 24)
    d = _rand_complex(rng, 60, 2)
    mu, P = O.gram_eig(E)
    b = E.conj().T @ d
    x = O.tsvd_solve(mu, P, b, len(mu))
    L = O.cholesky(O.gram(E, 0.0))
    ref = O.back_substitution_h(L, O.forward_substitution(L, b))
    assert O.nrmse(x, ref) < 1e-10


def test_tsvd_truncation_on_a_constructed_spectrum():
    """E = U diag(s) V^H with known s: keeping r singular values gives
    V_r diag(1 / s_r) U_r^H d, and with loading lam, V_r diag(s_r / (s_r^2 + lam)) U_r^H d."""
    rng = np.random.default_rng(22)
    U, _ = np.linalg.qr(_rand_complex(rng, 40, 16))
    V, _ = np.linalg.qr(_rand_complex(rng, 16, 16))
    s = np.geomspace(10.0, 0.01, 16)
    E = U @ np.diag(s) @ V.conj().T
    d = _rand_complex(rng, 40, 3)
    mu, P = O.gram_eig(E)
    r = O.tsvd_rank(mu, 0.999)
    b = E.conj().T @ d
    want = V[:, :r] @ ((U[:, :r].conj().T @ d) / s[:r, None])
    assert O.nrmse(O.tsvd_solve(mu, P, b, r), want) < 1e-10
    want_t = V[:, :r] @ ((s[:r] / (s[:r] ** 2 + 0.1))[:, None] * (U[:, :r].conj().T @ d))
    assert O.nrmse(O.tsvd_solve(mu, P, b, r, lam=0.1), want_t) < 1e-10
    assert abs(O.tsvd_condition(mu, r) - s[0] / s[r - 1]) < 1e-9 * s[0] / s[r - 1]


def test_planted_mistake_fails_tsvd_pin():
    """Dropping the conjugate of P_r^H (a plausible slip) fails the constructed pin."""
    rng = np.random.default_rng(23)
    U, _ = np.linalg.qr(_rand_complex(rng, 30, 10))
    V, _ = np.linalg.qr(_rand_complex(rng, 10, 10))
    s = np.geomspace(5.0, 0.1, 10)
    E = U @ np.diag(s) @ V.conj().T
    d = _rand_complex(rng, 30, 1)
    mu, P = O.gram_eig(E)
    b = E.conj().T @ d
    bad = P[:, :6] @ ((P[:, :6].T @ b) / mu[:6, None])
    want = V[:, :6] @ ((U[:, :6].conj().T @ d) / s[:6, None])
    assert O.nrmse(bad, want) > 1e-3


def test_underdetermined_right_form_equals_left_form():
    """Fewer samples than voxels (Section 2.2, underdetermined case): with lambda > 0
    the right pseudoinverse E^H (E E^H + lambda I)^-1 d equals the left form the
    oracle computes (push-through identity), so one path serves both cases."""
    rng = np.random.default_rng(31)
    E = _rand_complex(rng, 30, 80)
    d = _rand_complex(rng, 30, 2)
    lam = 0.05
    right = E.conj().T @ np.linalg.solve(E @ E.conj().T + lam * np.eye(30), d)
    L = O.cholesky(O.gram(E, lam))
    left = O.back_substitution_h(L, O.forward_substitution(L, E.conj().T @ d))
    assert O.nrmse(left, right) < 1e-11
