"""Pinv-Recon benchmark on GB300: pinv build seconds and recon frames/s.

Workload (default): 64x64 image (N = 4096), 8 coils, 4 interleaved spirals x
2048 samples per coil (M = 65536 rows), lambda = 1e-4 * mean diag(E^H E),
64 frames of complex64 k-space, seeded synthetic inputs. One step is one pass
of the whole hot path on the mixed-precision plan: pinv_build (Gram, blocked
Cholesky, W = L^-1, condition estimate) then pinv_apply on the 64 frames
(G^-1 E^H d = W^H W E^H d plus three refinement steps with exact residuals,
Section 3.3). The mixed plan keeps Recon = E^+ implicit: a split-precision
explicit Recon is only a starting guess (its images are far from 1e-4 before
refinement), so it is built and measured beside the step, not inside it.
The FP64 plan forms the explicit Recon of Eq. 8. Inputs are resident in HBM
before the timed region; G, L and W (268 MB each) and the per-step tables are
rewritten every step, and the build's operand tables (0.8 GB) exceed L2, so no
explicit L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference   # the FP64 oracle on the host cores

For N > 1 (torchrun) every rank builds and applies its own replica plan (the
path has no exchange step); value is the whole-job seconds per plan build,
i.e. max-over-ranks step build time / N.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pinv build s and recon frames/s at NRMSE≤1e-4 vs FP64; p50/p99 serve latency"
WORKLOAD = "SENSE spiral 64x64 (N=4096), 8 coils, 4x2048-sample spirals (M=65536), lambda 1e-4 mean diag, 64 frames"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 SIMT peak of GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _footprint(d):
    """Resident bytes of a mixed serving plan: Recon (c64), G/L, W and its FP32 copy."""
    N = d["side"] ** 2
    M = d["samples"] * d["n_coils"]
    return N * M * 8 + N * N * 40 + (64 << 20)


ROW_BLOCKS = 16  # the reference arm's sample: one of 16 blocks of samples per step


def oracle_row_block_step(inp, block):
    """One bounded sample of the workload through the FP64 oracle, as it stands.

    The oracle's pipeline (explicit E, G = E^H E + lambda I, unblocked
    Cholesky, direct solve of the 64 frames) on one of ROW_BLOCKS contiguous
    blocks of the samples of every coil: E, the Gram and E^H d over 1/16 of
    the rows, the Cholesky and the substitutions at full size. Returns the
    times of its parts; the full workload's build is 16 x (encode + Gram)
    + Cholesky, since the first two are sums over rows and the third is not.
    """
    import numpy as np
    import oracle.pinv_oracle as O
    Mk = inp.n_samples
    lo, hi = block * Mk // ROW_BLOCKS, (block + 1) * Mk // ROW_BLOCKS
    vox = O.voxel_positions(inp.dims)
    t0 = time.perf_counter()
    E = O.encode(inp.traj[lo:hi], vox, inp.coil_maps, inp.b0_hz,
                 None if inp.times is None else inp.times[lo:hi])
    lam = O.lambda_abs(E, inp.lambda_rel) * Mk / (hi - lo)  # the whole workload's load (trace is a sum over rows)
    t1 = time.perf_counter()
    G = O.gram(E, lam)
    t2 = time.perf_counter()
    L = O.cholesky(G)
    t3 = time.perf_counter()
    d = np.asarray(inp.data[:, :, lo:hi], dtype=np.complex128)
    X = O.solve(E, L, O.data_columns(d))
    t4 = time.perf_counter()
    assert np.isfinite(X).all()
    return {"encode": t1 - t0, "gram": t2 - t1, "cholesky": t3 - t2, "solve": t4 - t3, "wall": t4 - t0}


def oracle_full(inp, data):
    """The oracle on the whole workload, once: explicit E, G = E^H E + lambda I,
    unblocked Cholesky and the direct solve x = L^-H L^-1 E^H d of every frame
    (Eq. 6, Eq. 8, Section 3.3). data [F][C][M_k] complex128. Returns (images
    [F][N], seconds per part)."""
    import oracle.pinv_oracle as O
    t0 = time.perf_counter()
    E = O.plan_encode(inp)
    lam = O.lambda_abs(E, inp.lambda_rel)
    t1 = time.perf_counter()
    G = O.gram(E, lam)
    t2 = time.perf_counter()
    L = O.cholesky(G)
    t3 = time.perf_counter()
    X = O.solve(E, L, O.data_columns(data)).T
    t4 = time.perf_counter()
    del E, G, L
    return X, {"encode": t1 - t0, "gram": t2 - t1, "cholesky": t3 - t2, "solve": t4 - t3, "total": t4 - t0,
               "build": t3 - t0}


def lapack_cpu(inp, data):
    """The paper's CPU strategy (Section 3.1: multithreaded LAPACK on the host):
    explicit E, G = E^H E + lambda I by zherk, zpotrf, zpotrs for every frame.
    E comes from the oracle's encode; the rest are library calls."""
    import numpy as np
    import scipy.linalg.blas as BL
    import scipy.linalg.lapack as LA
    import oracle.pinv_oracle as O
    t0 = time.perf_counter()
    E = O.plan_encode(inp)
    t1 = time.perf_counter()
    # zherk on E^T (Fortran view [N][M]): E^T conj(E) = conj(E^H E)
    Gc = BL.zherk(1.0, E.T, trans=0, lower=1)
    lam = inp.lambda_rel * float(np.real(np.trace(Gc))) / inp.n_vox
    G = np.conj(Gc)
    G[np.diag_indices_from(G)] += lam
    t2 = time.perf_counter()
    C, info = LA.zpotrf(G, lower=0)  # upper factor of the stored upper triangle of G (= conj of the lower)
    assert info == 0
    t3 = time.perf_counter()
    B = E.conj().T @ O.data_columns(data)
    X, info = LA.zpotrs(C, B, lower=0)
    t4 = time.perf_counter()
    assert info == 0
    del E, G, C
    return X.T, {"encode": t1 - t0, "gram_zherk": t2 - t1, "zpotrf": t3 - t2, "solve": t4 - t3,
                 "build": t3 - t0, "total": t4 - t0}


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.

    Each step is the oracle's pipeline on one row block of workload 2 (see
    oracle_row_block_step); ms_per_step is that sample's wall time, and value
    is the full workload's oracle build (encode + Gram + Cholesky) formed
    from the step's parts, in the bench's unit (seconds per build)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2410_06129_gb300 import synth
    inp = synth.config(2, frames=64)
    for w in range(args.warmup):
        oracle_row_block_step(inp, w % ROW_BLOCKS)
    parts = []
    for k in range(args.steps):
        parts.append(oracle_row_block_step(inp, k % ROW_BLOCKS))
    full = [ROW_BLOCKS * (q["encode"] + q["gram"]) + q["cholesky"] for q in parts]
    v = statistics.mean(full)
    wall = statistics.mean(q["wall"] for q in parts)
    sample = (f"FP64 oracle (explicit E, Gram, unblocked Cholesky, direct solve of 64 frames) on one of "
              f"{ROW_BLOCKS} sample blocks of the full workload per step; full build = {ROW_BLOCKS} x "
              f"(encode + Gram) + Cholesky")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64-oracle"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": _cores(), "kind": "oracle", "sample": sample,
                             "parts_s": {k: statistics.mean(q[k] for q in parts)
                                         for k in ("encode", "gram", "cholesky", "solve")}},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


SERVE_BUDGET_FULL = 120e9  # bytes of resident plans for the full serving workload


def _phase_stats(sv, tickets, frames):
    """Latency and throughput of one phase from the server's per-request times."""
    import numpy as np
    tt = [sv.times(t) for t in tickets]
    lat = np.array([q["done"] - q["enqueue"] for q in tt])
    span_s = (max(q["done"] for q in tt) - min(q["enqueue"] for q in tt)) * 1e-3
    dev = [q for q in tt if q["dev_start"] >= 0]
    dev_s = (max(q["dev_end"] for q in dev) - min(q["dev_start"] for q in dev)) * 1e-3 if dev else None
    return {"requests": len(tickets), "frames": float(frames),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "frames_per_s": frames / span_s if span_s > 0 else None,
            "requests_per_s": len(tickets) / span_s if span_s > 0 else None,
            "device_span_s": dev_s}


def run_serve(prec, refine, side_div, rate_hz, duration_s, budget, max_slots, recon_mode,
              check_plans=0, seed=4100, sweep=(), sweep_s=1.0, p99_bound_ms=100.0):
    """Serving loop on the Poisson trace of the 32-plan serving workload.

    Requests arrive at their trace times (host thread sleeping until each
    arrival), each one of 32 registered plans with 1-64 frames of complex64
    k-space already resident in HBM; plans are built on admission and
    evicted LRU under `budget`. Returns the server's latency statistics at
    the offered rate, then, on the same server with the plans it kept
    resident: the capacity (the trace's requests enqueued at once) and, for
    each rate of `sweep`, a `sweep_s`-second trace's latencies; `max_rate_hz`
    is the highest swept rate whose p99 stays within `p99_bound_ms`.
    """
    import torch

    from paper_2410_06129_gb300 import _lib as L
    from paper_2410_06129_gb300 import synth
    from paper_2410_06129_gb300.plan import Plan
    from paper_2410_06129_gb300.serve import Server

    descs = synth.serve_plans(side_div=side_div)
    geo = [synth.serve_plan_inputs(d) for d in descs]
    trace = synth.serve_trace(rate_hz, duration_s, len(geo), seed=seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    datas = [torch.randn((64, p.n_coils * p.n_samples), generator=gen, device="cuda",
                         dtype=torch.complex64) for p in geo]
    torch.cuda.synchronize()

    def play(sv, ids, tr, paced=True):
        tickets = []
        t0 = time.perf_counter()
        for t_arr, i, F in tr:
            dt = t0 + t_arr - time.perf_counter()
            if paced and dt > 0:
                time.sleep(dt)
            tickets.append(sv.enqueue(ids[i], datas[i][:F], sync_inputs=False))
        status = [sv.wait(t, timeout=3600.0) for t, _ in tickets]
        return tickets, status

    with Server(budget_bytes=int(budget), max_slots=max_slots) as sv:
        ids = [sv.register_inputs(p, precision=prec, refine_max_iters=refine, recon_mode=recon_mode)
               for p in geo]
        t0 = time.perf_counter()
        tickets, status = play(sv, ids, trace)
        wall = time.perf_counter() - t0
        st = sv.stats()
        # accuracy of served images against FP64 plans on the same data
        worst = None
        if check_plans:
            seen = []
            for (t, out), (_, i, F) in zip(tickets, trace):
                if i in seen or len(seen) >= check_plans:
                    continue
                seen.append(i)
                with Plan.from_inputs(geo[i], precision=L.FP64, recon_mode=L.RECON_NONE) as p64:
                    p64.build()
                    x64 = p64.apply(datas[i][:F].to(torch.complex128))
                e = float(torch.linalg.norm(out.to(torch.complex128) - x64) / torch.linalg.norm(x64))
                worst = e if worst is None else max(worst, e)
        # capacity: the same requests at once, plans as the trace left them
        builds0 = sv.stats()["builds"]
        cap_t, cap_s = play(sv, ids, trace, paced=False)
        capacity = _phase_stats(sv, [t for t, _ in cap_t], sum(F for _, _, F in trace))
        capacity["ok"] = int(sum(s == L.OK for s in cap_s))
        capacity["builds"] = int(sv.stats()["builds"] - builds0)
        capacity["what"] = "the trace's requests enqueued at once on the same server (saturated throughput)"
        # the same burst with same-plan requests merged into one apply (up to 64 frames)
        sv.set_merge(64)
        mt, ms_ = play(sv, ids, trace, paced=False)
        merged = _phase_stats(sv, [t for t, _ in mt], sum(F for _, _, F in trace))
        merged["ok"] = int(sum(q == L.OK for q in ms_))
        merged["applies"] = len({round(sv.times(t)["dev_start"], 6) for t, _ in mt})
        merged["what"] = "the same burst with queued requests of one plan merged into one apply (<= 64 frames)"
        capacity["merged"] = merged
        sv.set_merge(0)
        rates = []
        for k, r in enumerate(sweep):
            tr = synth.serve_trace(r, sweep_s, len(geo), seed=seed + 1 + k)
            tk, ss = play(sv, ids, tr)
            ph = _phase_stats(sv, [t for t, _ in tk], sum(F for _, _, F in tr))
            ph.update(rate_hz=r, ok=int(sum(s == L.OK for s in ss)))
            rates.append(ph)
        ok_rates = [q["rate_hz"] for q in rates if q["p99_ms"] <= p99_bound_ms and q["ok"] == q["requests"]]
    frames = float(st["frames"])
    return {
        "requests": len(trace), "ok": int(sum(s == L.OK for s in status)), "failed": int(st["failed"]),
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
        "frames_per_s": frames / st["span_s"] if st["span_s"] > 0 else None,
        "frames_per_s_note": "at the offered rate: bounded by the trace, not by the server (see capacity)",
        "frames": frames, "builds": int(st["builds"]), "evictions": int(st["evictions"]),
        "recon_drops": int(st["recon_drops"]),
        "wall_s": wall, "trace_s": duration_s, "rate_hz": rate_hz, "slots": max_slots,
        "budget_gb": budget / 1e9, "refine_steps": refine,
        "recon": "explicit" if recon_mode == L.RECON_STORE else "factor-only",
        "nrmse_vs_fp64_max": worst, "nrmse_plans_checked": check_plans,
        "capacity": capacity,
        "rate_sweep": {"seconds_each": sweep_s, "p99_bound_ms": p99_bound_ms, "phases": rates,
                       "max_rate_hz": max(ok_rates) if ok_rates else None},
    }


def run_batch(prec, refine, steps, warmup, frames=256, seed=3100):
    """Workload 3: 16 uneven plans (side 24-96, 1-8 coils, spiral / radial,
    1-4 x N samples per coil), 256 complex64 frames each, built and applied
    as one batch replayed from CUDA graphs. Data are seeded normal values
    generated on the device (the cost does not depend on them)."""
    import torch

    from paper_2410_06129_gb300 import _lib as L
    from paper_2410_06129_gb300 import synth
    from paper_2410_06129_gb300.batch import Batch
    from paper_2410_06129_gb300.plan import Plan

    geo = synth.config(3, frames=0)
    plans = [Plan.from_inputs(p, precision=prec, refine_max_iters=refine) for p in geo]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    datas = [torch.randn((frames, p.n_coils * p.n_samples), generator=gen, device="cuda",
                         dtype=torch.complex64) for p in geo]
    outs = [torch.empty((frames, p.n_vox), dtype=torch.complex64, device="cuda") for p in geo]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    lib = L.load()
    with Batch(plans, graph=True) as b:
        def step():
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            b.build_async(stream)
            e1.record(stream)
            b.apply(datas, outs, stream=stream)
            e2.record(stream)
            stream.synchronize()
            b.sync()
            return e0.elapsed_time(e1), e1.elapsed_time(e2)
        for _ in range(max(warmup, 2)):  # the second build is the graph capture
            step()
        l0 = lib.pinv_kernel_launches()
        bs, aps = [], []
        for _ in range(steps):
            t_b, t_a = step()
            bs.append(t_b)
            aps.append(t_a)
        launches = (lib.pinv_kernel_launches() - l0) // max(steps, 1)
    n_frames = frames * len(geo)
    sum_n2m = sum(float(p.n_vox) ** 2 * p.n_samples * p.n_coils for p in geo)
    build_s = statistics.mean(bs) / 1e3
    apply_s = statistics.mean(aps) / 1e3
    for p in plans:
        p.close()
    return {"workload": "16 uneven plans (side 24-96, 1-8 coils, spiral/radial, 1-4 x N samples per coil), "
                        f"{frames} c64 frames each, one batch replayed from CUDA graphs",
            "build_s": build_s, "apply_s": apply_s, "frames": n_frames,
            "frames_per_s": n_frames / apply_s, "refine_steps": refine,
            "recon_useful_tflops_build": 8.0 * sum_n2m / build_s / 1e12,
            "gpu_launches_per_step": int(launches), "steps": steps}


def run_spectrum(side=32, frames=64, energy=0.95, seed=6100):
    """Eigendecomposition of the Gram matrix and the truncated reconstruction
    (Section 2.1) on workload 1's size (side^2 voxels, one spiral of 2 N samples),
    FP64, with the oracle's eigendecomposition timed on the host beside it."""
    import numpy as np
    import torch

    from paper_2410_06129_gb300 import _lib as L
    from paper_2410_06129_gb300 import synth as _sy
    from paper_2410_06129_gb300.plan import Plan
    inp = _sy.make_plan(side, 1, "spiral", frames, seed, 1e-3, samples=2 * side * side, interleaves=1)
    N = inp.n_vox
    with Plan.from_inputs(inp, precision=L.FP64, keep_gram=True) as pl:
        pl.build()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mu, P, sweeps = pl.eig()
        e1.record()
        torch.cuda.synchronize()
        ms_eig = e0.elapsed_time(e1)
        e0.record()
        mu_only, _, _ = pl.eig(vectors=False)
        e1.record()
        torch.cuda.synchronize()
        ms_eigvals = e0.elapsed_time(e1)
        d = torch.from_numpy(inp.data).cuda()
        pl.tsvd_apply(mu, P, d, energy=energy)  # warm
        torch.cuda.synchronize()
        e0.record()
        x, r, kappa = pl.tsvd_apply(mu, P, d, energy=energy)
        e1.record()
        torch.cuda.synchronize()
        ms_tsvd = e0.elapsed_time(e1)
        mu_h = mu.cpu().numpy()
    # FP64 work of the Jacobi rounds: per round the column pass rotates G and V
    # (2 N^2 entries) and the row pass G (N^2), 14 flop per entry (two complex
    # products and a sum); N - 1 rounds per sweep
    rounds = N - 1 if N % 2 == 0 else N
    flops = 42.0 * N * N * rounds * sweeps
    import oracle.pinv_oracle as O
    t0 = time.perf_counter()
    mu_ref, _ = O.gram_eig(O.plan_encode(inp))
    cpu_s = time.perf_counter() - t0
    return {"workload": f"{side}x{side} (N={N}), 1 coil, one spiral of {2 * N} samples, FP64 plan, {frames} frames",
            "eig_s": ms_eig / 1e3, "eigenvalues_only_s": ms_eigvals / 1e3,
            "eigenvalues_only_max_err_vs_oracle": float(np.max(np.abs(mu_only.cpu().numpy() - mu_ref)) / mu_ref[0]),
            "sweeps": sweeps, "fp64_tflops": flops / (ms_eig / 1e3) / 1e12,
            "fp64_peak_tflops": FP64_PEAK_TFLOPS, "tsvd_energy": energy, "tsvd_rank": r, "tsvd_kappa": kappa,
            "tsvd_apply_ms": ms_tsvd, "max_eig_err_vs_oracle": float(np.max(np.abs(mu_h - mu_ref)) / mu_ref[0]),
            "cpu_oracle_eig_s": cpu_s, "cpu_cores": _cores()}


def run_cfg5(prec, refine, frames=64, seed=5100, fp64=False):
    """Workload 5: 192x192 (N = 36864), 8 coils, 384 radial spokes x 125 samples
    (M = 384000), B0 +-50 Hz, lambda_rel 1e-4, 64 complex64 frames; factor-only
    (Recon would be 113 GB). One build, then the apply timed on its second run
    (fixed refinement steps, no host reads). A second plan then applies once with
    the stopping rule on, which reports the residual of the images it returns and
    the certified bound ||x - x*|| / ||x|| <= ||r|| / (lambda ||x||) (every
    eigenvalue of G is at least lambda). With fp64 the FP64 factor-only plan is
    built too (several minutes) and the mixed images are compared with its."""
    import torch

    from paper_2410_06129_gb300 import _lib as L
    from paper_2410_06129_gb300 import synth
    from paper_2410_06129_gb300.plan import Plan

    geo = synth.config(5, frames=0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    data = torch.randn((frames, geo.n_coils * geo.n_samples), generator=gen, device="cuda", dtype=torch.complex64)
    out = torch.empty((frames, geo.n_vox), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    with Plan.from_inputs(geo, precision=prec, recon_mode=L.RECON_NONE, refine_max_iters=refine,
                          refine_tol=0.0) as plan:
        build_ms = _timed_build(plan, stream)
        inf = plan.info()
        apply_ms = _timed_apply(plan, data, out, stream)
    with Plan.from_inputs(geo, precision=prec, recon_mode=L.RECON_NONE, refine_max_iters=refine,
                          refine_tol=1e-300) as plan:
        plan.build()
        plan.apply(data, out)
        torch.cuda.synchronize()
        inf2 = plan.info()
    vs64 = None
    if fp64 and prec != L.FP64:
        x_mixed = out.to(torch.complex128).cpu()
        with Plan.from_inputs(geo, precision=L.FP64, recon_mode=L.RECON_NONE, refine_max_iters=1) as p64:
            b64 = _timed_build(p64, stream)
            i64 = p64.info()
            out64 = torch.empty((frames, geo.n_vox), dtype=torch.complex128, device="cuda")
            d128 = data.to(torch.complex128)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p64.apply(d128, out64, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            x64 = out64.cpu()
        vs64 = {"fp64_build_s": b64 / 1e3, "fp64_apply_s": e0.elapsed_time(e1) / 1e3,
                "fp64_kappa_est": i64["kappa_est"], "nrmse_vs_fp64": _rel(x_mixed, x64),
                "nrmse_vs_fp64_max_frame": _rel_frames(x_mixed, x64),
                "speedup_build_vs_fp64": b64 / build_ms}
    res = {"workload": "192x192 (N=36864), 8 coils, 384 radial spokes x 125 samples (M=384000), B0 +-50 Hz, "
                        f"lambda 1e-4 mean diag, {frames} c64 frames, factor-only",
            "build_s": build_ms / 1e3,
            "stage_ms": {k: inf[k] for k in ("ms_gram", "ms_chol", "ms_inverse", "ms_cond")},
            "apply_s": apply_ms / 1e3, "frames_per_s": frames / (apply_ms / 1e3), "refine_steps": refine,
            "kappa_est": inf["kappa_est"],
            "final_residual_ratio": inf2["last_refine_resid"], "certified_bound": inf2["last_refine_bound"],
            "bytes_device": inf["bytes_device"]}
    if vs64 is not None:
        res["fp64"] = vs64
    return res


def _rel(a, b):
    import torch
    return float(torch.linalg.norm((a - b).flatten()) / torch.linalg.norm(b.flatten()))


def _rel_frames(a, b):
    """largest per-frame NRMSE (reading 8: joint and per-frame maximum)"""
    import torch
    return float(max(torch.linalg.norm(a[f] - b[f]) / torch.linalg.norm(b[f]) for f in range(b.shape[0])))


def _timed_build(plan, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.build_async(stream)
    e1.record(stream)
    plan.sync()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _timed_apply(plan, data, out, stream):
    import torch
    plan.apply(data, out, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.apply(data, out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "mixed", "fp64"])
    ap.add_argument("--frames", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--refine", type=int, default=3, help="refinement steps (mixed)")
    ap.add_argument("--side", type=int, default=64,
                    help="image side; 64 is the benchmark workload, smaller sides are for profiling")
    ap.add_argument("--serve", default="half", choices=["off", "half", "full"],
                    help="serving trace: 'full' = 32 plans of side 32-128 under a 120 GB budget, "
                         "'half' = the same plans at half the side under the same budget fraction")
    ap.add_argument("--serve-duration", type=float, default=3.0, help="seconds of Poisson arrivals")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-sweep", default="100,200,400,800,1600",
                    help="offered rates (req/s) swept for one second each on the same server, after the "
                         "trace and the capacity burst ('' = none)")
    ap.add_argument("--serve-refine", type=int, default=3)
    ap.add_argument("--batch", default="on", choices=["on", "off"],
                    help="workload 3: 16 uneven plans x 256 frames as one graph-replayed batch")
    ap.add_argument("--spectrum", default="on", choices=["on", "off"],
                    help="Gram eigendecomposition and tSVD reconstruction at workload 1's size")
    ap.add_argument("--cfg5", default="on", choices=["on", "off"],
                    help="workload 5 (192x192, B0, factor-only): one build and one timed apply")
    ap.add_argument("--cfg5-fp64", default="off", choices=["on", "off"],
                    help="also build workload 5 in FP64 (about 7 minutes) and compare the images")
    ap.add_argument("--serve-fp64-duration", type=float, default=1.0,
                    help="seconds of the same trace served by FP64 plans (0 = skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2410_06129_gb300 import _lib as L
    from paper_2410_06129_gb300 import synth
    from paper_2410_06129_gb300.plan import Plan

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = L.load()
    tc = bool(lib.pinv_tc_available())
    prec_name = args.precision if args.precision != "auto" else ("mixed" if tc else "fp64")
    prec = L.MIXED_BF16X6 if prec_name == "mixed" else L.FP64

    if args.side == 64:
        inp = synth.config(2, frames=args.frames)
    else:
        spi = (2 * args.side * args.side) // 4
        inp = synth.make_plan(args.side, 8, "spiral", args.frames, 2000, 1e-4, samples=4 * spi,
                              interleaves=4)
    refine = args.refine if prec != L.FP64 else 1
    F = args.frames
    N, M = inp.n_vox, inp.n_samples * inp.n_coils
    stream = torch.cuda.current_stream()
    # mixed plans keep Recon implicit (factor-only); FP64 plans form Recon = E^+ (Eq. 8)
    recon_mode = L.RECON_NONE if prec != L.FP64 else L.RECON_STORE
    plan = Plan.from_inputs(inp, precision=prec, refine_max_iters=refine, refine_tol=0.0, recon_mode=recon_mode)
    data64 = inp.data.astype(np.complex64)  # the workload's complex64 k-space
    data = torch.from_numpy(data64).cuda()
    out = torch.empty((F, N), dtype=torch.complex64, device="cuda")

    def step():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.build_async(stream)
        e1.record(stream)
        plan.apply(data, out, stream)
        e2.record(stream)
        plan.sync()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), plan.info()

    for _ in range(max(args.warmup, 0)):
        step()
    launches0 = lib.pinv_kernel_launches()
    builds, applies, infos = [], [], []
    with ClockSampler(local) as clk:
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        for _ in range(args.steps):
            b, a, inf = step()
            builds.append(b)
            applies.append(a)
            infos.append(inf)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        wall = time.perf_counter() - t_start
    launches = (lib.pinv_kernel_launches() - launches0) // max(args.steps, 1)
    build_s = statistics.mean(builds) / 1e3
    apply_s = statistics.mean(applies) / 1e3
    step_s = build_s + apply_s
    if ws > 1:
        t = torch.tensor([build_s, apply_s, step_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        build_s, apply_s, step_s = t.tolist()
    mean_info = {k: statistics.mean(i[k] for i in infos)
                 for k in ("ms_gram", "ms_gram_kernel", "ms_chol", "ms_inverse", "ms_recon", "ms_cond")}
    kappa = infos[-1]["kappa_est"]
    peaks, peak_src = _peaks()
    roof, gram = _roofline(prec, inp, mean_info, peaks, peak_src)

    acc = {}
    x_mixed = out.to(torch.complex128).cpu()
    x64 = None
    if rank == 0 and not args.no_fp64_check:
        # FP64 GPU plan on the same complex64 data (promoted): explicit Recon (Eq. 8) and one refinement step
        with Plan.from_inputs(inp, precision=L.FP64, refine_max_iters=1) as p64:
            ms64 = _timed_build(p64, stream)
            i64 = p64.info()
            d128 = data.to(torch.complex128)
            out64 = torch.empty((F, N), dtype=torch.complex128, device="cuda")
            ams64 = _timed_apply(p64, d128, out64, stream)
            x64 = out64.cpu()
            R64 = p64.export(L.EXPORT_RECON) if prec != L.FP64 else None
        acc["fp64"] = {"build_s": ms64 / 1e3, "apply_ms": ams64, "kappa_est": i64["kappa_est"],
                       "what": "explicit Recon = (L^-1)^H L^-1 E^H in FP64 (Eq. 8), 1 refinement step"}
        if prec != L.FP64:
            acc["nrmse_vs_fp64"] = _rel(x_mixed, x64)
            acc["nrmse_vs_fp64_max_frame"] = _rel_frames(x_mixed, x64)
            acc["speedup_build_vs_fp64"] = (ms64 / 1e3) / build_s
            # the mixed explicit Recon, measured beside the step: its build, its own accuracy
            # against the FP64 Recon, and the images it gives before and after refinement
            with Plan.from_inputs(inp, precision=prec, refine_max_iters=0, refine_tol=0.0,
                                  recon_mode=L.RECON_STORE) as pr:
                _timed_build(pr, stream)
                ms_r = _timed_build(pr, stream)
                ir = pr.info()
                x0 = pr.apply(data).to(torch.complex128).cpu()
                Rm = pr.export(L.EXPORT_RECON).to(torch.complex128)
                r_err = _rel(Rm, R64)
                del Rm
            del R64
            with Plan.from_inputs(inp, precision=prec, refine_max_iters=refine, refine_tol=0.0,
                                  recon_mode=L.RECON_STORE) as pr3:
                pr3.build()
                o3 = torch.empty((F, N), dtype=torch.complex64, device="cuda")
                ams_r = _timed_apply(pr3, data, o3, stream)
                x3 = o3.to(torch.complex128).cpu()
            acc["explicit_recon"] = {
                "build_ms": ms_r, "ms_recon": ir["ms_recon"], "apply_ms": ams_r,
                "recon_nrmse_vs_fp64_recon": r_err,
                "image_nrmse_vs_fp64_0_steps": _rel(x0, x64),
                f"image_nrmse_vs_fp64_{refine}_steps": _rel(x3, x64),
                "note": "split-precision Recon x data is a starting guess only; the step keeps Recon implicit"}

    # end to end through the public API with host buffers
    e2e = None
    if rank == 0:
        pin_data = torch.from_numpy(data64).pin_memory()
        pin_out = torch.empty((F, N), dtype=torch.complex64).pin_memory()
        reps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            with Plan.from_inputs(inp, precision=prec, refine_max_iters=refine, refine_tol=0.0,
                                  recon_mode=recon_mode) as p2:
                p2.build()
                d_dev = pin_data.to("cuda", non_blocking=True)
                x = p2.apply(d_dev)
                pin_out.copy_(x, non_blocking=True)
                torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / reps
        h2d = pin_data.numel() * 8 + inp.traj.nbytes + inp.coil_maps.nbytes
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(pin_out.numel() * 8),
               "what": "plan_create from host arrays + build + apply of 64 host frames + image D2H"}

    # the oracle on the whole workload (the CPU baseline, and the images every NRMSE is checked against)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        d_or = data64.astype(np.complex128)  # the same complex64 values, promoted
        x_or, t_or = oracle_full(inp, d_or)
        xo = torch.from_numpy(x_or)
        acc["nrmse_vs_oracle"] = _rel(x_mixed, xo)
        acc["nrmse_vs_oracle_max_frame"] = _rel_frames(x_mixed, xo)
        if x64 is not None:
            acc["fp64"]["nrmse_vs_oracle"] = _rel(x64, xo)
            acc["fp64"]["nrmse_vs_oracle_max_frame"] = _rel_frames(x64, xo)
        cpu = {"value": t_or["build"], "unit": "s", "cores": _cores(), "kind": "oracle",
               "sample": "the full workload (64x64, 8 coils, M=65536, 64 frames), run once: no extrapolation; "
                         "value = the oracle's build (explicit E, Gram, unblocked Cholesky)",
               "parts_s": t_or}
        del x_or, xo
        x_lp, t_lp = lapack_cpu(inp, d_or)
        cpu["lapack"] = {"value": t_lp["build"], "unit": "s", "threads": _cores(),
                         "what": "the paper's CPU strategy: numpy/scipy LAPACK zherk + zpotrf + zpotrs "
                                 "(BLAS threads = the host cores)",
                         "parts_s": t_lp, "nrmse_vs_oracle_images": None}
        del x_lp

    serve = None
    if rank == 0 and args.serve != "off":
        full = args.serve == "full"
        div = 1 if full else 2
        from paper_2410_06129_gb300 import synth as _sy
        fp_full = sum(_footprint(d) for d in _sy.serve_plans())
        fp_this = sum(_footprint(d) for d in _sy.serve_plans(side_div=div))
        budget = SERVE_BUDGET_FULL * fp_this / fp_full
        serve = {"workload": ("32 plans, side 32-128" if full else "32 plans, side 16-64 (cfg side / 2)")
                 + ", 1-16 coils, 1-2 x N samples per coil, Poisson arrivals, 1-64 c64 frames",
                 "budget_rule": "120 GB x (this plan set's footprint / the full set's)"}
        sweep = [float(r) for r in args.serve_sweep.split(",") if r] if args.serve_sweep else []
        serve["mixed"] = run_serve(prec, args.serve_refine if prec != L.FP64 else 0, div, args.serve_rate,
                                   args.serve_duration, budget, args.serve_slots,
                                   L.RECON_STORE, check_plans=4, sweep=sweep)
        if prec != L.FP64 and args.serve_fp64_duration > 0:
            serve["fp64"] = run_serve(L.FP64, 0, div, args.serve_rate, args.serve_fp64_duration, budget,
                                      args.serve_slots, L.RECON_NONE)

    spectrum = None
    if rank == 0 and args.spectrum == "on":
        spectrum = run_spectrum()

    cfg5 = None
    if rank == 0 and args.cfg5 == "on":
        cfg5 = run_cfg5(prec, refine if prec != L.FP64 else 1, fp64=args.cfg5_fp64 == "on")

    batch = None
    if rank == 0 and args.batch == "on" and prec != L.FP64:
        batch = run_batch(prec, refine, steps=2, warmup=2)

    if rank == 0:
        line = {
            "metric": METRIC, "value": build_s / ws, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == L.FP64 else "bf16x6+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": prec_name, "frames": F,
                       "recon": "explicit E^+" if recon_mode == L.RECON_STORE else "implicit (W^H W E^H, Section 3.3)",
                       "refine_steps": refine,
                       "l2": "inputs/outputs larger than L2 (G, L, W and operand tables rewritten each step)",
                       "parallelism": f"replicas x{ws}"},
            "recon_frames_per_s": F / apply_s * ws,
            "build_ms": build_s * 1e3, "apply_ms": apply_s * 1e3,
            "kappa_est": kappa,
            "nrmse_vs_oracle": acc.pop("nrmse_vs_oracle", None),
            "nrmse_vs_oracle_max_frame": acc.pop("nrmse_vs_oracle_max_frame", None),
            "stage_ms": {"gram": mean_info["ms_gram"], "chol": mean_info["ms_chol"],
                         "inverse_and_cond": mean_info["ms_inverse"], "cond": mean_info["ms_cond"],
                         "recon": mean_info["ms_recon"]},
            "roofline": roof, "gram_kernel": gram, "gpu_launches": int(launches), "e2e": e2e,
            "cpu_baseline": cpu, "clocks": clk.summary(), "wall_s_timed": wall,
        }
        line.update(acc)
        if cfg5 is not None:
            line["cfg5"] = cfg5
        if batch is not None:
            line["batch"] = batch
        if serve is not None:
            line["serve"] = serve
            line["serve_p50_ms"] = serve["mixed"]["p50_ms"]
            line["serve_p99_ms"] = serve["mixed"]["p99_ms"]
        if spectrum is not None:
            line["spectrum"] = spectrum
        line["autotune_classes"] = L.autotune_report().count("->")
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


# DRAM bytes (read + write) of one Gram launch at the 64x64 SENSE workload: ncu
# dram__bytes_read.sum + dram__bytes_write.sum of the current kernel (one launch captured)
GRAM_TRAFFIC_64 = 2058256384 + 119207168


def _roofline(prec, inp, mi, peaks, peak_src):
    """The roofline object of the step's dominant kernel, and the Gram kernel
    against the tensor-core peak (counted on the MMAs it issues)."""
    from paper_2410_06129_gb300 import _lib as L
    N = inp.n_vox
    gram = None
    pk = peaks.get("bf16_tflops_sustained", 1700.0)
    if prec != L.FP64:
        nt, kcn = -(-N // 128), -(-inp.n_samples // 16)
        pairs = 6 if prec == L.MIXED_BF16X6 else 3
        # per lower tile and 16-sample chunk: pairs x 2 MMAs of M 128, N 256, K 16
        issued = (nt * (nt + 1) // 2) * kcn * pairs * 2 * (2.0 * 128 * 256 * 16)
        useful = 8.0 * N * (N + 1) / 2 * inp.n_samples
        ms = mi["ms_gram_kernel"]
        gram = {"kernel": "gram_tc (split-BF16 tcgen05, bulk-copied operand table)", "ms": ms,
                "issued_tflops": issued / (ms / 1e3) / 1e12, "useful_tflops": useful / (ms / 1e3) / 1e12,
                "peak": pk, "peak_source": f"{peak_src} bf16_tflops_sustained"}
        gram["frac_issued"] = gram["issued_tflops"] / pk
        roof = {"kernel": gram["kernel"], "bound": "tensor", "launches": 1, "unit": "TFLOP/s",
                "achieved": gram["issued_tflops"], "peak": pk, "peak_source": gram["peak_source"],
                "frac": gram["frac_issued"], "useful_tflops": gram["useful_tflops"],
                "counted": "MMAs issued (6 split products per complex MAC of the Hermitian Gram)",
                "traffic": GRAM_TRAFFIC_64 if (N == 4096 and pairs == 6) else None,
                "traffic_unit": "bytes per launch",
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_tc_bulk<GramBulk> "
                                  "at this workload (profiles/ncu_gram_bulk_64x64_8coil.md)",
                "ms_per_launch": ms}
    else:
        ms = mi["ms_gram"]
        flops = 8.0 * N * (N + 1) / 2 * inp.n_samples * inp.n_coils
        roof = {"kernel": "gram (FP64 SIMT)", "bound": "alu", "launches": 1, "unit": "TFLOP/s",
                "achieved": flops / (ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz", "traffic": None,
                "ms_per_launch": ms}
        roof["frac"] = roof["achieved"] / roof["peak"]
    return roof, gram


if __name__ == "__main__":
    sys.exit(main())
