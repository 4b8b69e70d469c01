"""Pinv-Recon benchmark on GB300: pinv build seconds and recon frames/s.

Workload (default): 64x64 image (N = 4096), 8 coils, 4 interleaved spirals x
2048 samples per coil (M = 65536 rows), lambda = 1e-4 * mean diag(E^H E),
64 frames of complex64 k-space, seeded synthetic inputs. One step is one pass
of the whole hot path: pinv_build (Gram, Cholesky, G^-1, Recon = E^+) then
pinv_apply on the 64 frames (Recon x data plus FP64-residual refinement for
mixed-precision plans). Inputs are resident in HBM before the timed region;
Recon alone (2.1 GB c64 / 4.3 GB c128) is larger than L2, and every step
rewrites it, so no explicit L2 flush is needed.

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


def oracle_sample_step(side=32):
    """One bounded sample of the workload through the FP64 oracle.

    The full oracle pipeline (explicit E, Gram, unblocked Cholesky, L^-1,
    Recon, 64-frame apply) on the same workload shrunk to side x side with the
    same coils, spiral structure and lambda. Returns (seconds, scale) where
    scale converts to the full 64x64 workload by the N^2 M (= N^3 here) cost.
    """
    import numpy as np
    import oracle.pinv_oracle as O
    from paper_2410_06129_gb300 import synth
    spi = (2 * side * side) // 4
    p = synth.make_plan(side, 8, "spiral", 64, 2000, 1e-4, samples=4 * spi, interleaves=4)
    t0 = time.perf_counter()
    E = O.plan_encode(p)
    lam = O.lambda_abs(E, p.lambda_rel)
    R, _ = O.recon_matrix(E, lam)
    X = O.reconstruct(R, O.data_columns(p.data))
    t = time.perf_counter() - t0
    assert np.isfinite(X).all()
    N, M = p.n_vox, p.n_samples * 8
    scale = (4096.0 ** 2 * 65536.0) / (float(N) ** 2 * M)
    return t, scale


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample_step()
    ts, scale = [], None
    for _ in range(args.steps):
        t, scale = oracle_sample_step()
        ts.append(t)
    v = statistics.mean(ts) * scale
    sample = "full FP64 oracle pipeline (E, Gram, Cholesky, L^-1, Recon, 64-frame apply) at 32x32 " \
             f"(N=1024, 8 coils, M=16384), x{scale:.0f} by N^2 M cost"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64-oracle"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": _cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


SERVE_BUDGET_FULL = 120e9  # bytes of resident plans for the full serving workload


def run_serve(prec, refine, side_div, rate_hz, duration_s, budget, max_slots, recon_mode,
              check_plans=0, seed=4100):
    """Serving loop on the Poisson trace of the 32-plan serving workload.

    Requests arrive at their trace times (host thread sleeping until each
    arrival), each one of 32 registered plans with 1-64 frames of complex64
    k-space already resident in HBM; plans are built on admission and
    evicted LRU under `budget`. Returns the server's latency statistics.
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
    with Server(budget_bytes=int(budget), max_slots=max_slots) as sv:
        ids = [sv.register_inputs(p, precision=prec, refine_max_iters=refine, recon_mode=recon_mode)
               for p in geo]
        tickets = []
        t0 = time.perf_counter()
        for t_arr, i, F in trace:
            dt = t0 + t_arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(sv.enqueue(ids[i], datas[i][:F], sync_inputs=False))
        status = [sv.wait(t, timeout=3600.0) for t, _ in tickets]
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
    frames = float(st["frames"])
    return {
        "requests": len(trace), "ok": int(sum(s == L.OK for s in status)), "failed": int(st["failed"]),
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
        "frames_per_s": frames / st["span_s"] if st["span_s"] > 0 else None,
        "frames": frames, "builds": int(st["builds"]), "evictions": int(st["evictions"]),
        "recon_drops": int(st["recon_drops"]),
        "wall_s": wall, "trace_s": duration_s, "rate_hz": rate_hz, "slots": max_slots,
        "budget_gb": budget / 1e9, "refine_steps": refine,
        "recon": "explicit" if recon_mode == L.RECON_STORE else "factor-only",
        "nrmse_vs_fp64_max": worst, "nrmse_plans_checked": check_plans,
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


def run_cfg5(prec, refine, frames=64, seed=5100):
    """Workload 5: 192x192 (N = 36864), 8 coils, 384 radial spokes x 125 samples
    (M = 384000), B0 +-50 Hz, lambda_rel 1e-4, 64 complex64 frames; factor-only
    (Recon would be 113 GB). One build, then the apply timed on its second run.
    Without an oracle at this size, accuracy is reported as the refinement's
    final residual ||E^H (d - E x) - lambda x|| / ||E^H d|| (largest over frames)."""
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
                          refine_tol=1e-300) as plan:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.build_async(stream)
        e1.record(stream)
        plan.sync()
        torch.cuda.synchronize()
        build_s = e0.elapsed_time(e1) / 1e3
        inf = plan.info()
        plan.apply(data, out)
        torch.cuda.synchronize()
        e0.record(stream)
        plan.apply(data, out)
        e1.record(stream)
        torch.cuda.synchronize()
        apply_s = e0.elapsed_time(e1) / 1e3
        inf2 = plan.info()
    return {"workload": "192x192 (N=36864), 8 coils, 384 radial spokes x 125 samples (M=384000), B0 +-50 Hz, "
                        f"lambda 1e-4 mean diag, {frames} c64 frames, factor-only",
            "build_s": build_s, "stage_ms": {k: inf[k] for k in ("ms_gram", "ms_chol", "ms_inverse", "ms_recon")},
            "apply_s": apply_s, "frames_per_s": frames / apply_s, "refine_steps": refine,
            "final_residual_ratio": inf2["last_refine_resid"], "bytes_device": inf["bytes_device"]}


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
    ap.add_argument("--refine", type=int, default=3, help="FP64-residual refinement steps (mixed)")
    ap.add_argument("--side", type=int, default=64,
                    help="image side; 64 is the benchmark workload, smaller sides are for profiling")
    ap.add_argument("--serve", default="half", choices=["off", "half", "full"],
                    help="serving trace: 'full' = 32 plans of side 32-128 under a 120 GB budget, "
                         "'half' = the same plans at half the side under the same budget fraction")
    ap.add_argument("--serve-duration", type=float, default=3.0, help="seconds of Poisson arrivals")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-refine", type=int, default=3)
    ap.add_argument("--batch", default="on", choices=["on", "off"],
                    help="workload 3: 16 uneven plans x 256 frames as one graph-replayed batch")
    ap.add_argument("--spectrum", default="on", choices=["on", "off"],
                    help="Gram eigendecomposition and tSVD reconstruction at workload 1's size")
    ap.add_argument("--cfg5", default="off", choices=["on", "off"],
                    help="workload 5 (192x192, B0, factor-only): one build and one timed apply")
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
    tc = bool(getattr(lib, "pinv_tc_available", lambda: 0)()) if hasattr(lib, "pinv_tc_available") else False
    prec_name = args.precision if args.precision != "auto" else ("mixed" if tc else "fp64")
    prec = L.MIXED_BF16X6 if prec_name == "mixed" else L.FP64

    if args.side == 64:
        inp = synth.config(2, frames=args.frames)
    else:
        spi = (2 * args.side * args.side) // 4
        inp = synth.make_plan(args.side, 8, "spiral", args.frames, 2000, 1e-4, samples=4 * spi,
                              interleaves=4)
    refine = args.refine if prec != L.FP64 else 0
    F = args.frames
    stream = torch.cuda.current_stream()
    plan = Plan.from_inputs(inp, precision=prec, refine_max_iters=refine, refine_tol=0.0)
    data = torch.from_numpy(inp.data.astype(np.complex64)).cuda()
    out = torch.empty((F, inp.n_vox), dtype=torch.complex64, device="cuda")

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

    # dominant kernel: Recon formation
    N, M = inp.n_vox, inp.n_samples * inp.n_coils
    ms_gram = statistics.mean(i["ms_gram"] for i in infos)
    ms_recon_stage = statistics.mean(i["ms_recon"] for i in infos)
    peaks, peak_src = _peaks()
    if prec == L.FP64:
        ms_recon = ms_recon_stage
        flops_recon = 8.0 * N * N * M  # one launch
        roof = {"kernel": "recon (FP64 SIMT, generated E^H)", "bound": "alu", "launches": 1,
                "achieved": flops_recon / (ms_recon / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    else:
        # two triangular products, each N^2 M / 2 CMAC, over `chunks` ranges of samples:
        # 2 x chunks launches of equal work; the stage time also holds the operand-table
        # kernels, so the per-launch rate below is a lower bound
        nt, mt = -(-N // 128), -(-M // 128)
        slices = 3 if prec == L.MIXED_BF16X6 else 2
        per_tile = 2 * (nt * 8) * slices * 8192  # ET + TT bytes per 128 samples (4 GiB per chunk)
        cap = max(1, (4 << 30) // per_tile)
        chunks = -(-mt // cap)
        launches_r = 2 * chunks
        ms_recon = ms_recon_stage / launches_r
        flops_recon = 8.0 * N * N * M / launches_r
        pk = peaks.get("bf16_tflops_sustained", 1700.0)
        roof = {"kernel": "recon_tc (split-BF16 tcgen05, bulk-copied operand tables: "
                          "T^T = conj(E) W^T, then Recon^T = T^T conj(W))",
                "bound": "tensor", "launches": launches_r,
                "achieved": flops_recon / (ms_recon / 1e3) / 1e12, "peak": pk, "unit": "TFLOP/s",
                "peak_source": f"{peak_src} bf16_tflops_sustained",
                "issued_tflops": 6 * flops_recon / (ms_recon / 1e3) / 1e12}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["traffic_source"] = "not measured for this workload"
    if prec != L.FP64 and N == 4096 and M == 65536:
        # ncu dram__bytes_read.sum + dram__bytes_write.sum of the four Recon launches of
        # one build of this workload (step 1: 8.95 + 1.58 GB, step 2: 8.49 + 1.05 GB per
        # launch), mean per launch; algorithmic: the operand tables read once and the
        # outputs written once, 3.2 GB per launch (the excess is W-table re-reads)
        roof["traffic"] = (8947746816 + 1579998976 + 8494012672 + 1049467392) / 2
        roof["traffic_source"] = "ncu dram bytes of the Recon launches at this workload, mean per launch"
        roof["algorithmic_bytes"] = (3.4e9 + 2.9e9) / 2
    roof["ms_per_launch"] = ms_recon

    # the tensor-core Gram kernels alone (operand table + Gram launch + split sum)
    gram = None
    if prec != L.FP64:
        ms_gk = statistics.mean(i["ms_gram_kernel"] for i in infos)
        nt, kcn = -(-N // 128), -(-inp.n_samples // 16)
        pairs = 6 if prec == L.MIXED_BF16X6 else 3
        # per lower tile and 16-sample chunk: pairs x 2 MMAs of M 128, N 256, K 16
        issued = (nt * (nt + 1) // 2) * kcn * pairs * 2 * (2.0 * 128 * 256 * 16)
        useful = 8.0 * N * (N + 1) / 2 * inp.n_samples
        pk = peaks.get("bf16_tflops_sustained", 1700.0)
        gram = {"kernel": "gram_tc (split-BF16 tcgen05, bulk-copied operand table)", "ms": ms_gk,
                "issued_tflops": issued / (ms_gk / 1e3) / 1e12, "useful_tflops": useful / (ms_gk / 1e3) / 1e12,
                "peak": pk, "peak_source": f"{peak_src} bf16_tflops_sustained"}
        gram["frac_issued"] = gram["issued_tflops"] / pk

    res = {}
    # accuracy vs the FP64 GPU path (mixed plans)
    if prec != L.FP64 and not args.no_fp64_check and rank == 0:
        x_mixed = plan.apply(data).to(torch.complex128)
        t0 = time.perf_counter()
        with Plan.from_inputs(inp, precision=L.FP64) as p64:
            p64.build()
            i64 = p64.info()
            x64 = p64.apply(data.to(torch.complex128))
        res["fp64_build_s"] = (i64["ms_gram"] + i64["ms_chol"] + i64["ms_inverse"] + i64["ms_recon"]) / 1e3
        res["nrmse_vs_fp64"] = float(torch.linalg.norm(x_mixed - x64) / torch.linalg.norm(x64))
        res["speedup_build_vs_fp64"] = res["fp64_build_s"] / build_s
        res["refine_iters"] = plan.info()["last_refine_iters"]

    # end to end through the public API with host buffers
    e2e = None
    if rank == 0:
        pin_data = torch.from_numpy(inp.data.astype(np.complex64)).pin_memory()
        pin_out = torch.empty((F, N), dtype=torch.complex64).pin_memory()
        reps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            with Plan.from_inputs(inp, precision=prec, refine_max_iters=refine, refine_tol=0.0) as p2:
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

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t, scale = oracle_sample_step()
        cpu = {"value": t * scale, "unit": "s", "cores": _cores(), "kind": "oracle",
               "sample": f"full FP64 oracle pipeline at 32x32 (N=1024, 8 coils, M=16384, 64 frames), "
                         f"{t:.2f} s x{scale:.0f} by N^2 M cost"}

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
        serve["mixed"] = run_serve(prec, args.serve_refine if prec != L.FP64 else 0, div, args.serve_rate,
                                   args.serve_duration, budget, args.serve_slots,
                                   L.RECON_STORE, check_plans=4)
        if prec != L.FP64 and args.serve_fp64_duration > 0:
            serve["fp64"] = run_serve(L.FP64, 0, div, args.serve_rate, args.serve_fp64_duration, budget,
                                      args.serve_slots, L.RECON_NONE)

    spectrum = None
    if rank == 0 and args.spectrum == "on":
        spectrum = run_spectrum()

    cfg5 = None
    if rank == 0 and args.cfg5 == "on":
        cfg5 = run_cfg5(prec, refine if prec != L.FP64 else 1)

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
                       "l2": "inputs/outputs larger than L2 (Recon rewritten each step)",
                       "parallelism": f"replicas x{ws}"},
            "recon_frames_per_s": F / apply_s * ws,
            "build_ms": build_s * 1e3, "apply_ms": apply_s * 1e3,
            "stage_ms": {"gram": ms_gram, "chol": statistics.mean(i["ms_chol"] for i in infos),
                         "inverse": statistics.mean(i["ms_inverse"] for i in infos),
                         "recon": statistics.mean(i["ms_recon"] for i in infos)},
            "refine_steps": refine,
            "gram_kernel": gram,
            "roofline": roof, "gpu_launches": int(launches), "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clk.summary(), "wall_s_timed": wall,
        }
        line.update(res)
        line["autotune"] = L.autotune_report()
        if batch is not None:
            line["batch"] = batch
        if cfg5 is not None:
            line["cfg5"] = cfg5
        if spectrum is not None:
            line["spectrum"] = spectrum
        if serve is not None:
            line["serve"] = serve
            line["serve_p50_ms"] = serve["mixed"]["p50_ms"]
            line["serve_p99_ms"] = serve["mixed"]["p99_ms"]
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
