"""Mixed-precision (split-BF16 tcgen05) path vs the FP64 oracle.

Bars:
  * images after FP64-residual refinement: NRMSE <= 1e-4 (the mixed target);
  * the tensor-core Gram: relative Frobenius error within the split/FP32
    accumulation bound (2 slices ~ 2^-17 per product, 3 slices ~ 2^-24);
  * the tensor-core Recon kernel, isolated: Recon vs G^-1 (the plan's own, in
    FP64) times E^H from the oracle, same bounds.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle.pinv_oracle as O  # noqa: E402
from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402
from tests._ref import oracle_all, rel  # noqa: E402

pytestmark = pytest.mark.gpu
SPLIT_TOL = {L.MIXED_BF16X3: 1e-4, L.MIXED_BF16X6: 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _need_tc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")


def _plan(p, **kw):
    from paper_2410_06129_gb300.plan import Plan
    return Plan.from_inputs(p, **kw)


@pytest.mark.parametrize("prec", [L.MIXED_BF16X6, L.MIXED_BF16X3])
def test_gram_tc_small_ragged(prec):
    """N = 400 (3 row tiles of 128 + tail, 2 column tiles of 256), 2 coils, B0."""
    p = synth.make_plan(20, 2, "spiral", 1, 2101, 1e-3, samples=800, interleaves=2, b0=True)
    ref = oracle_all(p)
    pl = _plan(p, precision=prec, keep_gram=True, refine_max_iters=0).build()
    G = pl.export(L.EXPORT_GRAM).cpu().numpy()
    assert rel(np.tril(G), np.tril(ref.G)) < SPLIT_TOL[prec]


def _gram(p, prec):
    pl = _plan(p, precision=prec, keep_gram=True, refine_max_iters=0).build()
    return np.tril(pl.export(L.EXPORT_GRAM).cpu().numpy())


@pytest.mark.parametrize("prec", [L.MIXED_BF16X6, L.MIXED_BF16X3])
def test_gram_bulk_bit_identical_to_generated(prec, monkeypatch):
    """One sample split: the bulk-fed Gram copies the very slices the generating
    kernel writes and sums them in the same MMA and drain order, so G is the same
    bit for bit. M_k = 808 (a last sample chunk half full), N = 441 (ragged)."""
    p = synth.make_plan(21, 2, "spiral", 1, 2107, 1e-3, samples=808, interleaves=2, b0=True)
    g_bulk = _gram(p, prec)
    monkeypatch.setenv("PINV_GRAM_BULK", "0")
    g_gen = _gram(p, prec)
    assert np.array_equal(g_bulk, g_gen)
    assert rel(g_bulk, np.tril(oracle_all(p).G)) < SPLIT_TOL[prec]


def test_factor_bulk_updates_bit_identical(monkeypatch):
    """The bulk-fed panel trailing updates (HERK of the Cholesky, the inverse's
    row update) copy the slices the generating kernels form and sum them in the
    same order: L and W = L^-1 are the same bit for bit. N = 576 has two
    trailing updates after the 256-wide panels."""
    p = synth.make_plan(24, 2, "spiral", 1, 2115, 1e-3, samples=1152, interleaves=2)

    def factor():
        pl = _plan(p, precision=L.MIXED_BF16X6, keep_gram=True, refine_max_iters=0).build()
        return pl.export(L.EXPORT_CHOL).cpu().numpy(), pl.export(L.EXPORT_LINV).cpu().numpy()

    Lb, Wb = factor()
    monkeypatch.setenv("PINV_CHOL_BULK", "0")
    Lg, Wg = factor()
    assert np.array_equal(np.tril(Lb), np.tril(Lg))
    assert np.array_equal(Wb, Wg)


def test_gram_bulk_split_samples():
    """32x32, 4 coils, 4096 samples: 36 lower tiles are too few for the SMs, so
    the sample range is cut into parts whose FP32 partial sums are added in
    order; G stays within the split bound of the oracle."""
    p = synth.make_plan(32, 4, "spiral", 1, 2111, 1e-4, samples=4096, interleaves=2)
    assert rel(_gram(p, L.MIXED_BF16X6), np.tril(oracle_all(p).G)) < SPLIT_TOL[L.MIXED_BF16X6]


@pytest.mark.parametrize("bulk", ["1", "0"])
@pytest.mark.parametrize("prec", [L.MIXED_BF16X6, L.MIXED_BF16X3])
def test_recon_tc_isolated(prec, bulk, monkeypatch):
    """Recon = W^H (W E^H) with the plan's own W = L^-1: isolates the tensor-core
    kernels, bulk-fed from split tables (bulk = 1) or generating their operands.

    Bound: each of the two products carries a relative error of the split
    arithmetic (SPLIT_TOL, taken per product) on its inputs' magnitudes, so the
    error relative to Recon is at most ~ SPLIT_TOL * ||W|| ||W E^H|| / ||Recon||
    (the cancellation factor, about kappa(L)), computed here from the data.
    """
    monkeypatch.setenv("PINV_RECON_BULK", bulk)
    p = synth.make_plan(16, 3, "radial", 1, 2102, 1e-3, b0=True, spokes=20, per_spoke=33)
    pl = _plan(p, precision=prec, refine_max_iters=0).build()
    W = pl.export(L.EXPORT_LINV).cpu().numpy()
    R = pl.export(L.EXPORT_RECON).cpu().numpy()
    E = O.plan_encode(p)
    T = W @ E.conj().T
    want = W.conj().T @ T
    amp = np.linalg.norm(W) * np.linalg.norm(T) / np.linalg.norm(want)
    assert rel(R, want) < SPLIT_TOL[prec] * max(1.0, amp)
    assert np.allclose(np.triu(W, 1), 0)


@pytest.mark.parametrize("prec", [L.MIXED_BF16X6])
def test_recon_against_oracle_recon(prec):
    """The mixed explicit Recon (Eq. 8 formed from the split-precision factor) against
    the oracle's FP64 Recon = W^H W E^H. The factor's rounding is about the split
    arithmetic's 2^-24 relative, which the inverse amplifies by up to kappa(G), so
    the bar is 20 kappa_est 2^-24 with the plan's own condition estimate; spiral and
    radial-with-B0 plans of N = 256 and 324."""
    for p in (synth.make_plan(16, 3, "radial", 1, 2102, 1e-3, b0=True, spokes=20, per_spoke=33),
              synth.make_plan(18, 4, "spiral", 1, 2111, 1e-3, samples=900, interleaves=2)):
        pl = _plan(p, precision=prec, refine_max_iters=0).build()
        R = pl.export(L.EXPORT_RECON).cpu().numpy()
        kappa = pl.info()["kappa_est"]
        ref = oracle_all(p).R
        err = rel(R, ref)
        assert err < 20.0 * kappa * 2.0 ** -24, (err, kappa)


def test_recon_bulk_chunks_bit_identical(monkeypatch):
    """The bulk Recon over one sample tile per chunk (a 1 MB chunk cap) gives the
    same Recon bit for bit as one chunk: every tile sums the same tables in the
    same order. N = 441, M = 3 x 1000 (24 tiles, the last ragged)."""
    p = synth.make_plan(21, 3, "spiral", 1, 2109, 1e-3, samples=1000, interleaves=2)

    def recon():
        pl = _plan(p, precision=L.MIXED_BF16X6, refine_max_iters=0).build()
        return pl.export(L.EXPORT_RECON).cpu().numpy()

    whole = recon()
    monkeypatch.setenv("PINV_RECON_CHUNK_MB", "1")
    assert np.array_equal(recon(), whole)


@pytest.mark.parametrize("prec,iters", [(L.MIXED_BF16X6, 2), (L.MIXED_BF16X3, 4)])
def test_images_after_refinement_cfg2_reduced(prec, iters):
    """Workload 2 shrunk to 24x24 (kappa(G) ~ 4e5): NRMSE <= 1e-4 after refinement."""
    p = synth.config(2, reduced=True)
    ref = oracle_all(p)
    pl = _plan(p, precision=prec, refine_max_iters=iters, refine_tol=1e-9).build()
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    info = pl.info()
    assert rel(x, ref.images) <= 1e-4, (rel(x, ref.images), info)
    assert info["last_refine_iters"] >= 1


@pytest.mark.parametrize("residual", [L.RESIDUAL_DOUBLE_FLOAT, L.RESIDUAL_FP64])
def test_refinement_residual_arithmetic(residual):
    """Double-float and FP64 residuals both reach the mixed bar, and agree."""
    p = synth.config(2, reduced=True)
    ref = oracle_all(p)
    pl = _plan(p, precision=L.MIXED_BF16X6, refine_max_iters=3, refine_residual=residual).build()
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    assert rel(x, ref.images) <= 1e-4
    if residual == L.RESIDUAL_DOUBLE_FLOAT:
        pl64 = _plan(p, precision=L.MIXED_BF16X6, refine_max_iters=3, refine_residual=L.RESIDUAL_FP64).build()
        x64 = pl64.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
        assert rel(x, x64) <= 1e-6


def test_images_cfg1_full_complex64_io():
    """Workload 1 at full size with complex64 data in and out."""
    p = synth.config(1)
    ref = oracle_all(p)
    pl = _plan(p, precision=L.MIXED_BF16X6, refine_max_iters=2).build()
    d = torch.from_numpy(p.data.astype(np.complex64)).cuda()
    x = pl.apply(d)
    assert x.dtype == torch.complex64
    ref32 = O.solve(ref.E, ref.L, O.data_columns(p.data.astype(np.complex64))).T
    assert rel(x.cpu().numpy(), ref32) <= 1e-4


def test_b0_radial_reduced_cfg5():
    """Workload 5 shrunk to 32x32: 8 coils, radial, B0 +-50 Hz, 4 us dwell."""
    p = synth.config(5, reduced=True)
    ref = oracle_all(p)
    pl = _plan(p, precision=L.MIXED_BF16X6, refine_max_iters=3, refine_tol=1e-9).build()
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    assert rel(x, ref.images) <= 1e-4


@pytest.mark.parametrize("b0", [True, False])
def test_tensor_core_correction_many_frames(b0):
    """20 frames take the tensor-core correction x += W^H (W r) (split-K over k,
    partial sums added in order): a factor-only plan gets its initial image and
    every refinement step from it; the images reach the oracle's within 1e-6.
    N = 324 (ragged row tiles), with and without B0 (double-float and exact
    Gram residuals)."""
    p = synth.make_plan(18, 3, "spiral", 20, 2113, 1e-3, samples=720, interleaves=2, b0=b0)
    ref = oracle_all(p)
    pl = _plan(p, precision=L.MIXED_BF16X6, recon_mode=L.RECON_NONE, refine_max_iters=4,
               refine_tol=0.0).build()
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    assert rel(x, ref.images) <= 1e-6


def test_factor_only_mixed():
    p = synth.make_plan(16, 4, "spiral", 2, 2103, 1e-3, samples=512, interleaves=2, b0=True)
    ref = oracle_all(p)
    pl = _plan(p, precision=L.MIXED_BF16X6, recon_mode=L.RECON_NONE, refine_max_iters=2).build()
    x = pl.apply(torch.from_numpy(p.data).cuda()).cpu().numpy()
    assert rel(x, ref.images) <= 1e-4


@pytest.mark.parametrize("side", [16, 23])
def test_diag_block_cluster_matches_one_cta_sweep(side, monkeypatch):
    """The diagonal Cholesky blocks on a two-CTA cluster (factor on one CTA, block
    inverse on the other, each with a one-column lookahead) against the one-CTA
    column sweep: every entry takes the same double-float operations in the same
    order, so L and W = L^-1 are the same bit for bit; the images reach the oracle
    within the mixed target. 23 x 23 has a ragged last block."""
    p = synth.make_plan(side, 3, "spiral", 2, 2120 + side, 1e-3, samples=3 * side * side, interleaves=2)
    ref = oracle_all(p)
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("PINV_DIAG_CLUSTER", mode)
        with _plan(p, precision=L.MIXED_BF16X6) as pl:
            pl.build()
            x = pl.apply(torch.from_numpy(p.data.astype(np.complex64)).cuda()).cpu().numpy()
            out[mode] = (pl.export(L.EXPORT_CHOL).cpu().numpy(), pl.export(L.EXPORT_LINV).cpu().numpy(), x)
    assert np.array_equal(out["1"][0], out["0"][0])
    assert np.array_equal(out["1"][1], out["0"][1])
    assert np.array_equal(out["1"][2], out["0"][2])
    # the split-precision factor itself is about kappa^(1/2) 2^-24 from the exact one
    assert rel(out["1"][0], np.linalg.cholesky(ref.G)) < 1e-3
    assert rel(out["1"][2], ref.images) < 1e-4


def test_cholesky_lookahead_bit_identical(monkeypatch):
    """The trailing updates beyond the next panel run on a second stream beside the
    next panel's steps, and inside a panel the solves and updates beyond the next
    diagonal block on a third, beside that block (lookahead); every tile, row and
    entry is computed the same way, so L and W = L^-1 are the same bit for bit as
    with all of it on the chain's stream. 32 x 32 (N = 1024): after the first panel
    the trailing matrix has six column tiles."""
    p = synth.make_plan(32, 2, "spiral", 1, 2131, 1e-3, samples=2048, interleaves=2)
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("PINV_CHOL_LOOKAHEAD", mode)
        with _plan(p, precision=L.MIXED_BF16X6) as pl:
            pl.build()
            out[mode] = (pl.export(L.EXPORT_CHOL).cpu(), pl.export(L.EXPORT_LINV).cpu())
    assert torch.equal(out["0"][0], out["1"][0])
    assert torch.equal(out["0"][1], out["1"][1])


def test_b0_exact_products_many_frames(monkeypatch):
    """Plans with B0 refine with exact tensor-core E x and E^H u (digit tables of
    A and conj(A), 48 bytes per entry) for 16 or more frames. Workload 5 shrunk to
    32x32 (8 coils, 64 radial spokes x 40 samples, B0 +-50 Hz), 40 frames (a
    ragged second frame tile): the images reach the oracle's within 1e-6, like the
    double-float residual's (PINV_B0_EXACT=0), and the plan holds the tables."""
    p = synth.config(5, reduced=True, frames=40)
    ref = oracle_all(p)
    d = torch.from_numpy(p.data).cuda()
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("PINV_B0_EXACT", mode)
        with _plan(p, precision=L.MIXED_BF16X6, recon_mode=L.RECON_NONE, refine_max_iters=4,
                   refine_tol=0.0) as pl:
            pl.build()
            out[mode] = (pl.apply(d).cpu().numpy(), pl.info())
    table = 48 * p.n_vox * p.n_samples
    assert out["1"][1]["bytes_device"] - out["0"][1]["bytes_device"] >= table
    assert rel(out["1"][0], ref.images) <= 1e-6
    assert rel(out["0"][0], ref.images) <= 1e-6
    assert rel(out["1"][0], out["0"][0]) <= 1e-6
