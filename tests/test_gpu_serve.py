"""Serving loop (pinv_server_*) on the GPU.

A request's image must not depend on what else the server runs: every
result served in a mix of plans, precisions and frame counts is compared
bit for bit with a standalone pinv_apply of the same plan, which the other
GPU tests hold to the oracle. One FP64 result is also checked against the
oracle directly. Failures (budget, non-positive-definite Gram) stay with
their own requests.
"""
import threading

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


def _cases():
    """(inputs, plan keyword arguments): FP64 explicit, FP64 factor-only with
    B0, and (where tcgen05 is present) a mixed split-BF16 plan."""
    cases = [
        (synth.make_plan(16, 2, "spiral", 3, 2101, 1e-3, samples=512, interleaves=1),
         dict(precision=L.FP64)),
        (synth.make_plan(20, 4, "radial", 3, 2102, 1e-3, b0=True, spokes=16, per_spoke=40),
         dict(precision=L.FP64, recon_mode=L.RECON_NONE)),
    ]
    if L.load().pinv_tc_available():
        cases.append((synth.make_plan(24, 4, "spiral", 3, 2103, 1e-4, samples=1152, interleaves=2),
                      dict(precision=L.MIXED_BF16X6)))
    return cases


def _standalone(p, kw, data):
    from paper_2410_06129_gb300.plan import Plan
    pl = Plan.from_inputs(p, **kw).build()
    x = pl.apply(data)
    torch.cuda.synchronize()
    pl.close()
    return x


def _requests(cases):
    """Interleaved requests over all plans: varying frame counts and dtypes."""
    reqs = []
    for r in range(4):
        for i, (p, _) in enumerate(cases):
            F = 1 + (r + i) % 3
            d = torch.from_numpy(p.data[:F]).cuda()
            if (r + i) % 2:
                d = d.to(torch.complex64)
            reqs.append((i, d))
    return reqs


def test_serve_mix_matches_standalone_apply():
    from paper_2410_06129_gb300.serve import Server
    cases = _cases()
    reqs = _requests(cases)
    expect = [_standalone(cases[i][0], cases[i][1], d) for i, d in reqs]
    seen = []
    lock = threading.Lock()

    def cb(t, st):
        with lock:
            seen.append((t, st))

    with Server(budget_bytes=8 << 30, max_slots=3) as sv:
        ids = [sv.register_inputs(p, **kw) for p, kw in cases]
        tickets = [sv.enqueue(ids[i], d, callback=cb) for i, d in reqs]
        for t, _ in tickets:
            assert sv.wait(t) == L.OK
        for t, _ in tickets:
            assert sv.poll(t) == (True, L.OK)
        st = sv.stats()
    for (t, out), x in zip(tickets, expect):
        assert out.dtype == x.dtype
        assert torch.equal(out, x), f"ticket {t} differs from a standalone apply"
    assert sorted(seen) == sorted((t, L.OK) for t, _ in tickets)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["builds"] == len(cases) and st["evictions"] == 0
    assert st["frames"] == sum(d.shape[0] for _, d in reqs)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["resident_plans"] == len(cases) and st["queued"] == 0


def test_serve_fp64_result_matches_oracle():
    from paper_2410_06129_gb300.serve import Server
    p, kw = _cases()[0]
    ref = oracle_all(p)
    with Server(budget_bytes=1 << 30, max_slots=2) as sv:
        pid = sv.register_inputs(p, **kw)
        t, out = sv.enqueue(pid, torch.from_numpy(p.data).cuda())
        assert sv.wait(t) == L.OK
    assert rel(out.cpu().numpy(), ref.images) < 1e-10


def _resident_bytes(p, kw):
    from paper_2410_06129_gb300.serve import Server
    with Server(budget_bytes=8 << 30, max_slots=1) as sv:
        pid = sv.register_inputs(p, **kw)
        t, _ = sv.enqueue(pid, torch.from_numpy(p.data[:1]).cuda())
        assert sv.wait(t) == L.OK
        return sv.stats()["resident_bytes"]


def test_serve_lru_eviction_under_budget():
    """A budget that holds one (factor-only) plan at a time: alternating
    requests rebuild and evict, requests wait for in-flight work instead of
    failing, and results stay identical to standalone applies."""
    from paper_2410_06129_gb300.serve import Server
    cases = [(p, dict(kw, recon_mode=L.RECON_NONE)) for p, kw in _cases()[:2]]
    b = [_resident_bytes(p, kw) for p, kw in cases]
    budget = max(b) + min(b) // 2  # the larger plan fits, both do not
    assert budget < sum(b)
    order = [0, 1, 0, 1, 0]
    datas = [torch.from_numpy(cases[i][0].data[:2]).cuda() for i in order]
    expect = [_standalone(cases[i][0], cases[i][1], d) for i, d in zip(order, datas)]
    with Server(budget_bytes=budget, max_slots=4) as sv:
        ids = [sv.register_inputs(p, **kw) for p, kw in cases]
        tickets = [sv.enqueue(ids[i], d) for i, d in zip(order, datas)]
        assert [sv.wait(t) for t, _ in tickets] == [L.OK] * len(order)
        st = sv.stats()
    for (_, out), x in zip(tickets, expect):
        assert torch.equal(out, x)
    assert st["builds"] == len(order) and st["evictions"] == len(order) - 1
    assert st["resident_plans"] == 1 and st["resident_bytes"] <= budget


def test_serve_drops_recon_before_evicting():
    """A budget with room for both plans' factors but one Recon: the idle
    plan's Recon is dropped, nothing is evicted, and that plan then serves from
    its factors exactly as a standalone factor-only plan does."""
    from paper_2410_06129_gb300.serve import Server
    (p0, _), (p1, _) = _cases()[0], (synth.make_plan(18, 2, "spiral", 2, 2105, 1e-3, samples=648,
                                                     interleaves=1), {})
    full = dict(precision=L.FP64, recon_mode=L.RECON_STORE)
    fac = dict(precision=L.FP64, recon_mode=L.RECON_NONE)
    f0, f1, c0 = _resident_bytes(p0, full), _resident_bytes(p1, full), _resident_bytes(p0, fac)
    budget = c0 + f1 + (f0 - c0) // 2
    d0 = torch.from_numpy(p0.data[:2]).cuda()
    d1 = torch.from_numpy(p1.data[:2]).cuda()
    want0_full = _standalone(p0, full, d0)
    want0_fac = _standalone(p0, fac, d0)
    want1 = _standalone(p1, full, d1)
    with Server(budget_bytes=budget, max_slots=2) as sv:
        i0, i1 = sv.register_inputs(p0, **full), sv.register_inputs(p1, **full)
        outs = []
        for pid, d in ((i0, d0), (i1, d1), (i0, d0)):
            t, o = sv.enqueue(pid, d)
            assert sv.wait(t) == L.OK
            outs.append(o)
        st = sv.stats()
    assert torch.equal(outs[0], want0_full)
    assert torch.equal(outs[1], want1)
    assert torch.equal(outs[2], want0_fac)
    assert st["recon_drops"] == 1 and st["evictions"] == 0 and st["builds"] == 2
    assert st["resident_bytes"] <= budget


def test_serve_budget_too_small_fails_request_only():
    from paper_2410_06129_gb300.serve import Server
    p, kw = _cases()[0]
    with Server(budget_bytes=1 << 20, max_slots=2) as sv:
        pid = sv.register_inputs(p, **kw)
        t, _ = sv.enqueue(pid, torch.from_numpy(p.data[:1]).cuda())
        assert sv.wait(t) == L.ERR_BUDGET
        st = sv.stats()
    assert st["failed"] == 1 and st["completed"] == 0 and st["builds"] == 0


def test_serve_not_pd_plan_fails_its_requests_only():
    """lambda = 0 and a voxel that no coil sees make G singular: the plan's
    requests fail with NOT_PD, requests of a good plan around them succeed."""
    from paper_2410_06129_gb300.serve import Server
    bad = synth.make_plan(12, 2, "spiral", 1, 1901, 0.0, samples=512, interleaves=1)
    maps = bad.coil_maps.copy()
    maps[:, 70] = 0.0
    good, gkw = _cases()[0]
    dg = torch.from_numpy(good.data[:2]).cuda()
    db = torch.from_numpy(bad.data[:1]).cuda()
    expect = _standalone(good, gkw, dg)
    with Server(budget_bytes=4 << 30, max_slots=3) as sv:
        ib = sv.register(bad.dims, bad.traj, maps, lam=0.0, lambda_mode=L.LAMBDA_ABS)
        ig = sv.register_inputs(good, **gkw)
        tickets = [sv.enqueue(ib, db), sv.enqueue(ig, dg), sv.enqueue(ib, db), sv.enqueue(ig, dg)]
        res = [sv.wait(t) for t, _ in tickets]
        late, _ = sv.enqueue(ib, db)
        res.append(sv.wait(late))
        st = sv.stats()
    assert res == [L.ERR_NOT_PD, L.OK, L.ERR_NOT_PD, L.OK, L.ERR_NOT_PD]
    assert torch.equal(tickets[1][1], expect) and torch.equal(tickets[3][1], expect)
    assert st["failed"] == 3 and st["completed"] == 2
    assert st["resident_plans"] == 1  # the singular plan was dropped


def test_serve_zero_frames_and_bad_plan_id():
    from paper_2410_06129_gb300.serve import Server
    p, kw = _cases()[0]
    with Server(budget_bytes=1 << 30, max_slots=1) as sv:
        pid = sv.register_inputs(p, **kw)
        t, out = sv.enqueue(pid, torch.zeros((0, p.data[0].size), dtype=torch.complex128, device="cuda"))
        assert sv.wait(t) == L.OK and out.shape == (0, int(np.prod(p.dims)))
        with pytest.raises(KeyError):
            sv.enqueue(pid + 7, torch.from_numpy(p.data[:1]).cuda())
        with pytest.raises(L.PinvError, match="INVALID_ARG"):
            L.check(L.load().pinv_serve_enqueue(sv._h, pid + 7, None, None, 1, L.C128, None, None,
                                                L.C.byref(L.C.c_uint64())))


def test_host_fault_injection_leaves_other_requests_intact(monkeypatch):
    """PINV_FAULT makes failures on the host while requests are in flight: the
    first admission of plan 0 fails as if its allocation had (OOM), the first
    build of plan 1 fails, ticket 7 is dropped and ticket 8's completion is held
    back 300 ms. Those requests report their statuses (ticket 8 succeeds, late);
    every other request completes with an image identical, bit for bit, to a
    standalone apply, and the failed plans are admitted again by their next
    requests."""
    import time
    from paper_2410_06129_gb300.serve import Server
    cases = _cases()
    reqs = _requests(cases)
    expect = [_standalone(cases[i][0], cases[i][1], d) for i, d in reqs]
    monkeypatch.setenv("PINV_FAULT", "alloc:0,build:1,drop:7,delay:8:300")
    with Server(budget_bytes=8 << 30, max_slots=3) as sv:
        ids = [sv.register_inputs(p, **kw) for p, kw in cases]
        t0 = time.perf_counter()
        tickets = [sv.enqueue(ids[i], d) for i, d in reqs]
        status = {t: sv.wait(t) for t, _ in tickets}
        waited = time.perf_counter() - t0
        st = sv.stats()
    first = {}
    for (t, _), (i, _) in zip(tickets, reqs):
        first.setdefault(i, t)
    want = {t: L.OK for t, _ in tickets}
    want[first[0]] = L.ERR_OOM
    want[first[1]] = L.ERR_INTERNAL
    want[7] = L.ERR_INTERNAL
    assert status == want
    assert waited >= 0.3  # ticket 8 was reported no sooner than its delay
    for (t, out), x in zip(tickets, expect):
        if want[t] == L.OK:
            assert torch.equal(out, x), f"ticket {t} differs from a standalone apply"
    assert st["failed"] == 3 and st["completed"] == len(reqs) - 3
    assert st["builds"] == len(cases)  # the failed admission and build were retried once each


def test_two_slots_run_on_the_device_at_the_same_time():
    """Two requests of two resident FP64 plans, enqueued together on a two-slot
    server: the device intervals of their work (timing events on the slot
    streams, pinv_serve_times) intersect, each request's times are ordered, and
    both images equal standalone applies.
    32x32, 4 coils, 2048 samples per coil, 64 frames: E^H d alone is about 5e8
    complex FP64 products per request, far longer than the dispatch of the other."""
    from paper_2410_06129_gb300.serve import Server
    kw = dict(precision=L.FP64, recon_mode=L.RECON_NONE)
    ps = [synth.make_plan(32, 4, "spiral", 64, 2140, 1e-3, samples=2048, interleaves=2),
          synth.make_plan(32, 4, "radial", 64, 2141, 1e-3, spokes=32, per_spoke=64)]
    data = [torch.from_numpy(p.data).cuda() for p in ps]
    expect = [_standalone(p, kw, d) for p, d in zip(ps, data)]
    with Server(budget_bytes=8 << 30, max_slots=2) as sv:
        ids = [sv.register_inputs(p, **kw) for p in ps]
        for i in range(2):  # build both plans first: the pair then waits on no build
            t, _ = sv.enqueue(ids[i], data[i][:1])
            assert sv.wait(t) == L.OK
        pair = [sv.enqueue(ids[i], data[i]) for i in range(2)]
        for t, _ in pair:
            assert sv.wait(t) == L.OK
        tt = [sv.times(t) for t, _ in pair]
        with pytest.raises(L.PinvError):
            sv.times(10 ** 9)
    for (t, out), x in zip(pair, expect):
        assert torch.equal(out, x)
    a, b = tt
    for q in tt:
        assert 0 <= q["enqueue"] <= q["done"]
        assert 0 <= q["dev_start"] < q["dev_end"]
    assert max(a["dev_start"], b["dev_start"]) < min(a["dev_end"], b["dev_end"]), tt


def test_merged_requests_share_one_apply():
    """With merging on, requests of one plan that queue behind a request in
    flight are reconstructed by one apply: on a one-slot server busy with a long
    request of plan A, four requests of plan B (2, 5, 1 and 3 frames) wait and then
    run together (the same device interval), and each image matches a standalone
    apply of its frames (FP64 plan: to 1e-13; the sums whose split follows the
    frame count may reassociate). A fifth B request that would pass the frame cap
    runs in its own apply."""
    from paper_2410_06129_gb300.serve import Server
    kw = dict(precision=L.FP64, recon_mode=L.RECON_NONE)
    pa = synth.make_plan(32, 4, "spiral", 64, 2150, 1e-3, samples=2048, interleaves=2)
    pb = synth.make_plan(16, 2, "radial", 20, 2151, 1e-3, spokes=16, per_spoke=24)
    da = torch.from_numpy(pa.data).cuda()
    db = torch.from_numpy(pb.data).cuda()
    sizes = [2, 5, 1, 3, 6]
    parts, o = [], 0
    for F in sizes:
        parts.append(db[o:o + F].clone())
        o += F
    expect = [_standalone(pb, kw, d) for d in parts]
    with Server(budget_bytes=8 << 30, max_slots=1) as sv:
        ia, ib = sv.register_inputs(pa, **kw), sv.register_inputs(pb, **kw)
        for i, d in ((ia, da[:1]), (ib, db[:1])):  # both plans resident first
            t, _ = sv.enqueue(i, d)
            assert sv.wait(t) == L.OK
        sv.set_merge(11)
        ta, _ = sv.enqueue(ia, da)
        tb = [sv.enqueue(ib, d) for d in parts]
        assert sv.wait(ta) == L.OK
        for t, _ in tb:
            assert sv.wait(t) == L.OK
        tt = [sv.times(t) for t, _ in tb]
        st = sv.stats()
    for (t, out), x in zip(tb, expect):
        assert rel(out.cpu().numpy(), x.cpu().numpy()) < 1e-13
    starts = [q["dev_start"] for q in tt]
    assert len(set(starts[:4])) == 1, tt  # 2 + 5 + 1 + 3 = 11 frames: one apply
    assert starts[4] != starts[0]          # 11 + 6 > 11: its own apply
    assert st["completed"] == 2 + 1 + len(sizes)
    assert st["frames"] == 1 + 1 + 64 + sum(sizes)
