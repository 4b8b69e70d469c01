"""Batched build and apply of uneven plans (pinv_batch_*), eager and from CUDA graphs.

A batch must not change any result: every Recon, every W = L^-1 and every
image is compared bit for bit with the same plan built and applied on its own
(pinv_build / pinv_apply), which the other GPU tests hold to the oracle. One
batched image is also checked against the oracle directly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2410_06129_gb300 import _lib as L  # noqa: E402
from paper_2410_06129_gb300 import synth  # noqa: E402
from tests._ref import oracle_all, rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load()


def _inputs():
    """Uneven plans: ragged sides, 1-4 coils, spiral and radial, one with B0
    (double-float residual), one factor-only."""
    return [
        (synth.make_plan(12, 1, "spiral", 3, 2401, 1e-3, samples=300, interleaves=1), {}),
        (synth.make_plan(20, 4, "radial", 2, 2402, 1e-3, samples=1200), {}),
        (synth.make_plan(24, 2, "spiral", 4, 2403, 1e-4, samples=1152, interleaves=2), {}),
        (synth.make_plan(16, 3, "radial", 2, 2404, 1e-3, b0=True, spokes=12, per_spoke=40), {}),
        (synth.make_plan(16, 2, "spiral", 3, 2405, 1e-3, samples=512, interleaves=2),
         dict(recon_mode=L.RECON_NONE)),
    ]


def _plans(cases, precision):
    from paper_2410_06129_gb300.plan import Plan
    return [Plan.from_inputs(p, precision=precision, refine_max_iters=2, **kw) for p, kw in cases]


def _exports(pl, precision):
    out = []
    if pl.info()["has_recon"]:
        out.append(pl.export(L.EXPORT_RECON))
    if precision != L.FP64:
        out.append(pl.export(L.EXPORT_LINV))
    return out


@pytest.mark.parametrize("precision", [L.MIXED_BF16X6, L.FP64])
def test_batch_bit_identical_to_single_plans(precision):
    from paper_2410_06129_gb300.batch import Batch
    if precision != L.FP64 and not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")
    cases = _inputs()
    datas = [torch.from_numpy(p.data).cuda() for p, _ in cases]
    singles = _plans(cases, precision)
    want_x, want_exp = [], []
    for pl, d in zip(singles, datas):
        pl.build()
        want_x.append(pl.apply(d))
        want_exp.append(_exports(pl, precision))
    torch.cuda.synchronize()

    stream = torch.cuda.Stream()
    plans = _plans(cases, precision)
    with Batch(plans, graph=True) as b:
        for rep in range(3):  # eager, captured, replayed
            b.build(stream)
            with torch.cuda.stream(stream):
                xs = b.apply(datas, stream=stream)
            stream.synchronize()
            for i, pl in enumerate(plans):
                assert torch.equal(xs[i], want_x[i]), (rep, i)
                for got, want in zip(_exports(pl, precision), want_exp[i]):
                    assert torch.equal(got, want), (rep, i)
    for pl in singles + plans:
        pl.close()


def test_batch_graph_replay_sees_new_data_and_new_shapes():
    """Replays read the buffers' current contents; a new frame count re-captures."""
    from paper_2410_06129_gb300.batch import Batch
    from paper_2410_06129_gb300.plan import Plan
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")
    cases = _inputs()[:3]
    plans = _plans(cases, L.MIXED_BF16X6)
    stream = torch.cuda.Stream()
    datas = [torch.from_numpy(p.data).cuda().to(torch.complex64) for p, _ in cases]
    outs = [torch.empty((d.shape[0], p.n_vox), dtype=torch.complex64, device="cuda") for d, (p, _) in zip(datas, cases)]
    with Batch(plans, graph=True) as b:
        b.build(stream)
        stream.synchronize()
        b.apply(datas, outs, stream=stream)
        stream.synchronize()
        gen = torch.Generator(device="cuda").manual_seed(3)
        for d in datas:  # new contents, same buffers: the replay must see them
            d.copy_(torch.randn(d.shape, dtype=torch.complex64, device="cuda", generator=gen))
        torch.cuda.synchronize()
        b.apply(datas, outs, stream=stream)
        stream.synchronize()
        for pl, d, o in zip(plans, datas, outs):
            assert torch.equal(o, pl.apply(d))
        short = [d[:1].clone() for d in datas]
        torch.cuda.synchronize()
        xs = b.apply(short, stream=stream)
        stream.synchronize()
        for pl, d, x in zip(plans, short, xs):
            assert torch.equal(x, pl.apply(d))
    for pl in plans:
        pl.close()


def test_batched_image_matches_oracle():
    from paper_2410_06129_gb300.batch import Batch
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")
    cases = _inputs()
    plans = _plans(cases, L.MIXED_BF16X6)
    stream = torch.cuda.Stream()
    with Batch(plans, graph=False) as b:
        b.build(stream)
        with torch.cuda.stream(stream):
            xs = b.apply([torch.from_numpy(p.data).cuda() for p, _ in cases], stream=stream)
        stream.synchronize()
    for i in (1, 3):
        ref = oracle_all(cases[i][0])
        assert rel(xs[i].cpu().numpy(), ref.images) <= 1e-4
    for pl in plans:
        pl.close()


def test_batch_rejects_mixed_precisions_and_repeats():
    from paper_2410_06129_gb300.batch import Batch
    if not L.load().pinv_tc_available():
        pytest.skip("tcgen05 kernels need sm_103a")
    cases = _inputs()[:2]
    a = _plans(cases[:1], L.FP64)[0]
    b = _plans(cases[1:], L.MIXED_BF16X6)[0]
    with pytest.raises(L.PinvError, match="INVALID_ARG"):
        Batch([a, b])
    with pytest.raises(L.PinvError, match="INVALID_ARG"):
        Batch([b, b])
    a.close()
    b.close()
