#!/usr/bin/env python
"""Throughput benchmark of the long-range (history) evaluator.

Workload (one step): the full-size starfish problem — 1e5 boundary nodes (6,250 panels x 16
Gauss-Legendre) on r = 1 + 0.3 cos 5t, ~1e6 cut-cell volume nodes with the manufactured source
f = (13 + alpha^2) sin 2x cos 3y, 1e6 uniform targets in [-1.5, 1.5]^2 — evaluated at
alpha = 1, 10 and 100 in FP64 at relative accuracy 1e-10.  Per alpha the step runs the whole hot
path: bin/sort of sources and targets (yk_set_points) and spread, FFTs with the multiplier, and
interpolation (yk_eval_longrange).  Inputs are synthetic and resident in HBM before timing.

The three evaluations of a step are independent: each alpha's plan has its own CUDA stream, so
their kernels overlap and, end to end, one alpha's host copies overlap another's kernels.

`value` = source+target points of all alphas and ranks per second of device time (CUDA events on
the main stream around the fork to and join from the three streams, max over ranks).  `e2e` = the
same through the C ABI with page-locked host buffers, host<->device copies inside the timed
region.  `roofline` = the stage with the largest device time, against the measured ALU peak
(double-float stages: FP32 FMA rate / DF_COST) or the measured HBM copy bandwidth; its durations
come from the timed region (overlapping streams), `achieved_alone` from the kernels run alone.  `cpu_baseline` = the
FP64 oracle (direct pair sum) on the host cores for a bounded sample of targets, scaled to a full
evaluation.  `--impl reference` times that oracle alone as the reference arm.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "source+target points/s at rel err 1e-10 (FP64) & 1e-6 (FP32); p50/p99 latency"
ALPHAS = (1.0, 10.0, 100.0)
TOL = 1e-10
L2_BYTES = 126 * 1024 * 1024
DF_COST = 10  # FP32 operations per double-float add or multiply (two-sum / two-product)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--alphas", default=",".join(str(a) for a in ALPHAS))
    ap.add_argument("--cpu-targets", type=int, default=1500,
                    help="targets in the bounded CPU-oracle sample (all sources)")
    ap.add_argument("--ref-targets", type=int, default=120,
                    help="targets per alpha in each reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32c", action="store_true", help="skip the FP32C measurement")
    ap.add_argument("--no-dlp", action="store_true", help="skip the double-layer measurement")
    ap.add_argument("--no-local", action="store_true", help="skip the local-part measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-instance batch section")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving section")
    ap.add_argument("--serve-requests", type=int, default=4000,
                    help="requests of the Rothe stream (Poisson, 2000 req/s)")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# algorithmic work per stage (per launch), used for the roofline of the dominant stage
def stage_work(info, ns, nt):
    """(bytes, fp64 flops) each stage must move / compute at minimum for one launch.

    The double-float path computes every point's window values once, in the set-up stages
    (bin_src: sources, bin_trg: targets), by Horner on per-tap polynomials of degree w - 1 (2 flops
    per step); the spread and the interpolation read them (16 bytes per point and tap pair).
    """
    n, M, w = info["n_grid"], info["n_modes"], info["w"]
    G = n * n
    L = n // 2
    entries = ns * (1 + (w - 1) / info["tile"]) ** 2  # windows spread into each tile they touch
    win = 2 * (w - 1)                                 # flops per window value
    fft_row = 5 * L * math.log2(L) + 12 * L   # complex FFT of n/2 points + real post-processing
    fft_col = 5 * n * math.log2(n)
    return {
        "bin_src": (ns * (16 + 16 + 4 * 3 + 16 * w) + entries * 20, ns * (20 + 2 * w * win)),
        "bin_trg": (nt * (16 + 16 + 4 * 3 + 16 * w) + nt * 20, nt * (20 + 2 * w * win)),
        "spread": (entries * (20 + 16 * w) + ns * 16 + G * 8, entries * (2 * w * w + 2 * w)),
        "row_fwd": (G * 8 + (M + 1) * n * 16, n * fft_row),
        "columns": (2 * (M + 1) * n * 16 + (M + 1) * (2 * M + 1) * 8,
                    (M + 1) * (2 * fft_col + 6 * n)),
        "row_inv": ((M + 1) * n * 16 + G * 8, n * fft_row),
        "interp": (G * 8 + nt * (28 + 16 * w), nt * (2 * w * w + 2 * w)),
    }


def workload_config(alphas, works):
    """The workload both arms report (the reference arm samples its targets)."""
    w = works[alphas[0]]
    return {"workload": "starfish 1e5 boundary + ~1e6 volume sources, 1e6 targets, alpha in "
                        + str(alphas) + ", FP64, rel tol 1e-10; set_points + eval per alpha "
                        "per step",
            "alphas": alphas, "n_src": int(w.n_src), "n_trg": int(w.n_trg), "tol": TOL}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


# the sources that define the stage kernels whose DRAM bytes profiles/ncu_traffic.json records
TRAFFIC_SOURCES = ("yk_core.h", "yk_internal.h", "yk_kernels.cu", "yk_stages.cuh")


def load_traffic():
    """ncu DRAM bytes per launch per stage recorded under profiles/, valid for the current source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return {}
    import hashlib
    with open(path) as f:
        d = json.load(f)
    h = hashlib.sha256()
    for fn in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2606_28865_b300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    if d.get("csrc_sha256") != h.hexdigest():
        return {}
    return d.get("bytes_per_launch", {})


# ---------------------------------------------------------------------------------------------
def cpu_baseline(alphas, n_targets):
    """FP64 oracle, all sources x a bounded sample of targets, scaled to full evaluations."""
    import oracle
    total_pts = 0.0
    total_t = 0.0
    for a in alphas:
        work = W.config_large(a)
        rng = np.random.default_rng(1)
        idx = rng.choice(work.n_trg, n_targets, replace=False)
        table = oracle.GHTable(a, _delta(work, a), oracle.pair_rmax(work.xs, work.ys, work.xt,
                                                                      work.yt))
        t0 = time.perf_counter()
        oracle.direct_sum(a, _delta(work, a), work.xs, work.ys, work.q, work.xt[idx],
                          work.yt[idx], table=table)
        dt = time.perf_counter() - t0
        total_t += dt * work.n_trg / n_targets           # time of the full evaluation
        total_pts += work.n_src + work.n_trg
    return {"value": total_pts / total_t, "unit": "points/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": (f"FP64 direct pair sum over all {int(W.config_large(alphas[0]).n_src)} "
                       f"sources for {n_targets} of the 1e6 targets at each alpha in "
                       f"{list(alphas)}; time scaled by 1e6/{n_targets} to a full evaluation")}


def _delta(work, alpha):
    import oracle.params as OP
    return OP.delta_from_mesh(alpha, work.h_vol)


def run_reference(args, rank, world, pg):
    """Reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return 0
    import oracle
    alphas = [float(a) for a in args.alphas.split(",")]
    works = {a: W.config_large(a) for a in alphas}
    tables = {a: oracle.GHTable(a, _delta(works[a], a),
                                oracle.pair_rmax(works[a].xs, works[a].ys, works[a].xt,
                                                 works[a].yt)) for a in alphas}
    rng = np.random.default_rng(2)
    idx = {a: rng.choice(works[a].n_trg, args.ref_targets, replace=False) for a in alphas}

    def step():
        for a in alphas:
            wk = works[a]
            oracle.direct_sum(a, _delta(wk, a), wk.xs, wk.ys, wk.q, wk.xt[idx[a]], wk.yt[idx[a]],
                              table=tables[a])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    scale = works[alphas[0]].n_trg / args.ref_targets
    pts = sum(works[a].n_src + works[a].n_trg for a in alphas)
    value = pts / (dt * scale)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * scale * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(alphas, works),
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"all sources x {args.ref_targets} targets per alpha per "
                                       f"step, scaled to full evaluations"},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
def batch_section(yk, torch, rank):
    """256 uneven instances (points log-uniform in [1e3, 2e5], random starfish, alpha log-uniform
    in [1, 300]): plain per-call evaluation vs one persistent launch replayed from a graph."""
    works = W.batch_instances(256, seed=rank)
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    bufs = [(t(wk.xs), t(wk.ys), t(wk.w), t(wk.xt), t(wk.yt), t(wk.density),
             torch.empty(wk.n_trg, dtype=torch.float64, device=dev)) for wk in works]
    pts = sum(wk.n_src + wk.n_trg for wk in works)
    stream = torch.cuda.current_stream()
    out = {"instances": len(works), "points": pts,
           "workload": "256 random starfish instances, points log-uniform in [1e3, 2e5], "
                       "alpha log-uniform in [1, 300], targets at the volume nodes"}
    for prec, tol, key in ((yk.YK_FP32C, 1e-6, "fp32c"), (yk.YK_FP64, 1e-10, "fp64")):
        # autotune the tile edge on eight instances spread over the size range; plans of the
        # same (window, grid band, density band) then take the tuned edge
        t_tune = time.perf_counter()
        order = np.argsort([wk.n_src for wk in works])
        for k in order[:: max(1, len(works) // 8)]:
            wk, bf = works[k], bufs[k]
            yk.autotune(wk.alpha, bf[0], bf[1], bf[2], bf[5], bf[3], bf[4], tol=tol,
                        precision=prec, h_vol=wk.h_vol, box=wk.box)
        t_tune = time.perf_counter() - t_tune
        plans = []
        for wk, bf in zip(works, bufs):
            p = yk.Plan(wk.alpha, tol=tol, precision=prec, h_vol=wk.h_vol, box=wk.box,
                        use_tuned=True, n_src_hint=wk.n_src)
            p.set_points(*bf[:5])
            plans.append(p)
        torch.cuda.synchronize()

        def per_call():
            for p, bf in zip(plans, bufs):
                p.eval(bf[5], out=bf[6])

        reps = 10
        per_call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            per_call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_call = e0.elapsed_time(e1) / reps
        b = yk.Batch(plans, use_graph=True)
        dens = [bf[5] for bf in bufs]
        outs = [bf[6] for bf in bufs]
        b.run(dens, outs)
        b.sync()
        t0 = time.perf_counter()
        for _ in range(reps):
            b.run(dens, outs)
        b.sync()
        ms_batch = (time.perf_counter() - t0) / reps * 1e3
        out[key] = {"per_call_ms": ms_call, "per_call_points_per_s": pts / (ms_call * 1e-3),
                    "batch_ms": ms_batch, "batch_points_per_s": pts / (ms_batch * 1e-3),
                    "tol": tol, "autotune_s": t_tune}
        b.close()
        for p in plans:
            p.close()
    return out


def serving_section(yk, n_req):
    """Rothe stream: 64 simulations (points log-uniform in [1e3, 1e6], dt log-uniform in
    [1e-4, 1e-1]), Poisson arrivals at 2000 req/s: FP32C continuous batching vs the plain FP64
    per-call form on the same arrivals."""
    from paper_2606_28865_b300.serving import RotheServer
    geoms, reqs = W.rothe_stream(n_req=n_req, rate=2000.0, n_geom=64, seed=0)
    out = {"workload": f"{n_req} requests, Poisson 2000 req/s, 64 resident geometries",
           "points_total": int(sum(geoms[r["geom"]].n_src + geoms[r["geom"]].n_trg
                                   for r in reqs))}
    for key, prec, batch in (("fp32c_batched", yk.YK_FP32C, True),
                             ("fp64_per_call", yk.YK_FP64, False)):
        srv = RotheServer(geoms, precision=prec, max_inflight=64, n_streams=4, batch=batch)
        srv.warm(range(len(geoms)))
        st = srv.serve(reqs)
        st.pop("results", None)
        out[key] = st
        srv.close()
    return out


def main():
    args = parse()
    rank, world, local, pg = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, rank, world, pg)

    import torch
    import paper_2606_28865_b300 as yk

    alphas = [float(a) for a in args.alphas.split(",")]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # one stream per alpha: the three evaluations of a step are independent, so their kernels and
    # (for e2e) their host copies overlap; a timed region forks from `stream` and joins back to it
    lanes = {a: torch.cuda.Stream(device=dev) for a in alphas}

    def fork():
        ev = torch.cuda.Event()
        ev.record(stream)
        for s_ in lanes.values():
            s_.wait_event(ev)

    def join():
        for s_ in lanes.values():
            ev = torch.cuda.Event()
            ev.record(s_)
            stream.wait_event(ev)

    works, plans, dbufs, outs = {}, {}, {}, {}
    for a in alphas:
        wk = W.config_large(a, seed=rank)
        works[a] = wk
        plans[a] = yk.Plan(a, tol=TOL, h_vol=wk.h_vol, box=wk.box, profile=True, stream=lanes[a])
        t = lambda v: torch.as_tensor(v, dtype=torch.float64, device=dev)
        dbufs[a] = [t(wk.xs), t(wk.ys), t(wk.w), t(wk.xt), t(wk.yt), t(wk.density)]
        outs[a] = torch.empty(wk.n_trg, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    def step():
        for a in alphas:
            xs, ys, w, xt, yt, d = dbufs[a]
            plans[a].set_points(xs, ys, w, xt, yt)
            plans[a].eval(d, out=outs[a])

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    for a in alphas:
        plans[a].stage_times()  # restart the per-stage event averages
    barrier(pg)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fork()
    for _ in range(args.steps):
        step()
    join()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(pg)
    ms_step = max_over_ranks(pg, e0.elapsed_time(e1) / args.steps)
    stage_ms = {a: plans[a].stage_times() for a in alphas}
    pts_step = sum(works[a].n_src + works[a].n_trg for a in alphas)
    value = pts_step * world / (ms_step * 1e-3)

    # per-eval latency distribution (device events per call)
    lat = []
    for a in alphas:
        xs, ys, w, xt, yt, d = dbufs[a]
        for _ in range(5):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(lanes[a])
            plans[a].eval(d, out=outs[a])
            s1.record(lanes[a])
            torch.cuda.synchronize()
            lat.append(s0.elapsed_time(s1))

    # cold: plan creation (parameters, multiplier, FFT tables) + set_points + eval, host wall time
    cold_ms = {}
    for a in alphas:
        xs, ys, w, xt, yt, d = dbufs[a]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pc = yk.Plan(a, tol=TOL, h_vol=works[a].h_vol, box=works[a].box, stream=lanes[a])
        pc.set_points(xs, ys, w, xt, yt)
        pc.eval(d, out=outs[a])
        pc.sync()
        cold_ms[str(a)] = (time.perf_counter() - t0) * 1e3
        pc.close()

    # end to end through the C ABI with pinned host buffers
    hbufs = {}
    for a in alphas:
        wk = works[a]
        pin = lambda v: torch.as_tensor(v, dtype=torch.float64).pin_memory()
        hbufs[a] = [pin(wk.xs), pin(wk.ys), pin(wk.w), pin(wk.xt), pin(wk.yt), pin(wk.density),
                    torch.empty(wk.n_trg, dtype=torch.float64).pin_memory()]

    def step_host():
        for a in alphas:
            xs, ys, w, xt, yt, d, u = hbufs[a]
            plans[a].set_points(xs, ys, w, xt, yt)
            plans[a].eval(d, out=u)

    step_host()
    torch.cuda.synchronize()
    barrier(pg)
    k_e2e = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        step_host()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(pg, (time.perf_counter() - t0) / k_e2e)
    h2d = sum((4 * works[a].n_src + 2 * works[a].n_trg) * 8 for a in alphas)
    d2h = sum(works[a].n_trg * 8 for a in alphas)
    for a in alphas:
        plans[a].stage_times()

    # the same step with one alpha at a time (no other stream running): stage durations of the
    # kernels alone, reported beside the timed region's (where the three alphas overlap)
    for a in alphas:
        plans[a].stage_times()
    for _ in range(3):
        for a in alphas:
            xs, ys, w, xt, yt, d = dbufs[a]
            plans[a].set_points(xs, ys, w, xt, yt)
            plans[a].eval(d, out=outs[a])
            torch.cuda.synchronize()
    stage_ms_alone = {a: plans[a].stage_times() for a in alphas}
    # evaluation stages only (a resident layout), summed over the alphas, kernels alone
    eval_only_ms = sum(sum(v for k, v in stage_ms_alone[a].items()
                           if k not in ("bin_src", "bin_trg") and v) for a in alphas)

    # roofline of the dominant stage (largest device time per step)
    hbm_peak, peak_kind = load_peaks()
    fp64_peak = yk.fma_peak_tflops(yk.YK_FP64)
    fp32_peak = yk.fma_peak_tflops(yk.YK_FP32C)

    def stage_totals(sms):
        tot, work_b, work_f = {}, {}, {}
        for a in alphas:
            sw = stage_work(plans[a].info, works[a].n_src, works[a].n_trg)
            for k, v in sms[a].items():
                if v is None:
                    continue
                tot[k] = tot.get(k, 0.0) + v
                work_b[k] = work_b.get(k, 0.0) + sw[k][0]
                work_f[k] = work_f.get(k, 0.0) + sw[k][1]
        return tot, work_b, work_f

    tot, work_b, work_f = stage_totals(stage_ms)
    tot1, _, _ = stage_totals(stage_ms_alone)
    dom = max(tot1, key=tot1.get)  # the costliest stage when each kernel runs alone
    t_dom = tot[dom] * 1e-3
    gbs = work_b[dom] / t_dom / 1e9
    tfl = work_f[dom] / t_dom / 1e12
    t_dom1 = tot1[dom] * 1e-3
    traffic = load_traffic().get(dom)
    # the FP64 path computes spread, FFTs and interpolation in FP32 pairs (double-float)
    # (the set-up stages' arithmetic is the double-float window kernel)
    df_stage = dom in ("bin_src", "bin_trg", "spread", "row_fwd", "columns", "row_inv", "interp")
    alu_peak = fp32_peak / DF_COST if df_stage else fp64_peak
    if tfl / alu_peak >= gbs / hbm_peak:
        roof = {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": tfl / alu_peak, "traffic": traffic}
        peak_note = ("FP32 FMA rate measured by yk_fma_peak / %d FP32 ops per double-float "
                     "flop" % DF_COST) if df_stage else "FP64 FMA rate measured by yk_fma_peak"
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak, "traffic": traffic}
        peak_note = f"HBM copy bandwidth, {peak_kind} (MEASURED_PEAKS.json)"
    roof.update({"kernel": dom, "launches_per_step": len(alphas), "peak_source": peak_note,
                 "hbm_achieved_gbs": gbs, "alu_achieved_tflops": tfl,
                 "fp64_peak_tflops": fp64_peak, "fp32_peak_tflops": fp32_peak,
                 "durations": "CUDA events around the stage on its stream in the timed region, "
                              "where the three alphas' streams overlap (so the durations include "
                              "other streams' kernels)",
                 "achieved_alone": (work_f[dom] / t_dom1 / 1e12 if roof["unit"] == "TFLOP/s"
                                    else work_b[dom] / t_dom1 / 1e9),
                 "frac_alone": ((work_f[dom] / t_dom1 / 1e12 if roof["unit"] == "TFLOP/s"
                                 else work_b[dom] / t_dom1 / 1e9) / roof["peak"]),
                 "alone": "the same stage timed with one alpha at a time, no other stream running"})

    # the FP32C form of the same workload (FP32 spread/FFT/interp, two-sum grid sums, FP64
    # final sums at the targets; relative accuracy 1e-6)
    fp32c = None
    if not args.no_fp32c:
        plans32 = {a: yk.Plan(a, tol=1e-6, precision=yk.YK_FP32C, h_vol=works[a].h_vol,
                              box=works[a].box, profile=True, stream=lanes[a]) for a in alphas}

        def step32():
            for a in alphas:
                xs, ys, w, xt, yt, d = dbufs[a]
                plans32[a].set_points(xs, ys, w, xt, yt)
                plans32[a].eval(d, out=outs[a])

        for _ in range(max(3, args.warmup)):
            step32()
        torch.cuda.synchronize()
        for a in alphas:
            plans32[a].stage_times()
        barrier(pg)
        e0.record(stream)
        fork()
        for _ in range(args.steps):
            step32()
        join()
        e1.record(stream)
        torch.cuda.synchronize()
        ms32 = max_over_ranks(pg, e0.elapsed_time(e1) / args.steps)
        st32 = {str(a): plans32[a].stage_times() for a in alphas}
        lat32 = []
        for a in alphas:
            for _ in range(5):
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(lanes[a])
                plans32[a].eval(dbufs[a][5], out=outs[a])
                s1.record(lanes[a])
                torch.cuda.synchronize()
                lat32.append(s0.elapsed_time(s1))
        fp32c = {"value": pts_step * world / (ms32 * 1e-3), "unit": "points/s",
                 "ms_per_step": ms32, "tol": 1e-6, "dtype": "f32 (two-sum grid, f64 final sums)",
                 "grids": {str(a): plans32[a].info["n_grid"] for a in alphas},
                 "stage_ms": st32,
                 "latency_ms": {"p50": float(np.percentile(lat32, 50)),
                                "p99": float(np.percentile(lat32, 99))}}
        for a in alphas:
            plans32[a].close()

    # the same step with the double layer D_H added: 1e5 boundary dipoles (the boundary nodes with
    # their normals and mu = sin 2t + 0.3 cos t) on top of the charges, one grid for both
    dlp = None
    if not args.no_dlp:
        xd, yd, wd, nx, ny, mu = W.double_layer_nodes(W.Starfish(), 6250)
        t = lambda v: torch.as_tensor(v, dtype=torch.float64, device=dev)
        dl_dev = tuple(t(v) for v in (xd, yd, wd, nx, ny))
        mu_dev = t(mu)
        plans_dl = {a: yk.Plan(a, tol=TOL, h_vol=works[a].h_vol, box=works[a].box, profile=True,
                               stream=lanes[a], dlp=True) for a in alphas}

        def step_dl():
            for a in alphas:
                xs, ys, w, xt, yt, d = dbufs[a]
                plans_dl[a].set_points(xs, ys, w, xt, yt, dipoles=dl_dev)
                plans_dl[a].eval(d, out=outs[a], mu=mu_dev)

        for _ in range(max(3, args.warmup)):
            step_dl()
        torch.cuda.synchronize()
        for a in alphas:
            plans_dl[a].stage_times()
        barrier(pg)
        e0.record(stream)
        fork()
        for _ in range(args.steps):
            step_dl()
        join()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_dl = max_over_ranks(pg, e0.elapsed_time(e1) / args.steps)
        pts_dl = pts_step + len(alphas) * len(mu)
        dlp = {"value": pts_dl * world / (ms_dl * 1e-3), "unit": "points/s",
               "ms_per_step": ms_dl, "n_dip": int(len(mu)), "tol": TOL,
               "what": "S_H + V_H + D_H: set_points_dl + eval_longrange_dl per alpha per step",
               "w": {str(a): plans_dl[a].info["w"] for a in alphas},
               "grids": {str(a): plans_dl[a].info["n_grid"] for a in alphas},
               "stage_ms": {str(a): plans_dl[a].stage_times() for a in alphas}}
        for a in alphas:
            plans_dl[a].close()

    # single-layer local asymptotic part S_{L,A} (closest point + lemma) at the 1e6 targets for
    # the 1e5-node boundary, delta* = delta of the alpha = 10 plan (one call, host wall time: the
    # call bins the panels, evaluates and returns after its stream finished)
    local = None
    if not args.no_local:
        a_loc = 10.0 if 10.0 in alphas else alphas[0]
        xb, yb, _, tb = W.boundary_nodes(W.Starfish(), 6250, 16)
        t = lambda v: torch.as_tensor(v, dtype=torch.float64, device=dev)
        lb = (t(xb), t(yb), t(W.boundary_density(tb)))
        dstar = plans[a_loc].info["delta"]
        xt_l, yt_l = dbufs[a_loc][3], dbufs[a_loc][4]
        ul = torch.empty_like(xt_l)
        for _ in range(2):
            yk.slp_local(a_loc, dstar, *lb, xt_l, yt_l, q=16, out=ul, stream=lanes[a_loc])
        reps = 5
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            yk.slp_local(a_loc, dstar, *lb, xt_l, yt_l, q=16, out=ul, stream=lanes[a_loc])
        ms_loc = (time.perf_counter() - t0) / reps * 1e3
        near = int((ul != 0).sum().item())
        local = {"value": (len(xb) + xt_l.numel()) / (ms_loc * 1e-3), "unit": "points/s",
                 "ms": ms_loc, "alpha": a_loc, "delta_star": dstar, "n_boundary": len(xb),
                 "n_targets": int(xt_l.numel()), "targets_within_locality": near,
                 "what": "yk_slp_local: panel series, cell lists, closest point, lemma terms"}

    # volume local part V_L at the volume nodes strictly inside the curve (the cut-cell nodes by
    # concave chords may lie just outside it), delta* = the plan's delta, same boundary
    vlocal = None
    if not args.no_local:
        wk = works[a_loc]
        vx, vy = wk.xs[wk.n_bdry:], wk.ys[wk.n_bdry:]
        keep = W.inside_starfish(W.Starfish(), vx, vy)
        vx, vy = vx[keep], vy[keep]
        xv, yv = t(vx), t(vy)
        fdv = t(W.manufactured_source_derivs(vx, vy, a_loc))
        uv = torch.empty_like(xv)
        for _ in range(2):
            yk.vp_local(a_loc, dstar, lb[0], lb[1], xv, yv, fdv, q=16, out=uv, stream=lanes[a_loc])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            yk.vp_local(a_loc, dstar, lb[0], lb[1], xv, yv, fdv, q=16, out=uv, stream=lanes[a_loc])
        ms_v = (time.perf_counter() - t0) / reps * 1e3
        rl_v = math.sqrt(dstar) * (12 + 2 * a_loc * math.sqrt(dstar))
        vlocal = {"value": (len(xb) + len(vx)) / (ms_v * 1e-3), "unit": "points/s", "ms": ms_v,
                  "alpha": a_loc, "delta_star": dstar, "n_boundary": len(xb),
                  "n_targets": int(len(vx)), "locality_radius": rl_v,
                  "what": "yk_vp_local at the volume nodes: interior form everywhere, closest point "
                          "+ lemma within the locality radius"}

    # dyadic corrections of the single-layer local part (J = 3 levels below the plan's delta) at
    # the same 1e6 targets and boundary
    dyadic = None
    if not args.no_local:
        J = 3
        ud = torch.empty_like(xt_l)
        for _ in range(2):
            yk.slp_dyadic(a_loc, dstar, J, *lb, xt_l, yt_l, q=16, out=ud, stream=lanes[a_loc])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            yk.slp_dyadic(a_loc, dstar, J, *lb, xt_l, yt_l, q=16, out=ud, stream=lanes[a_loc])
        ms_d = (time.perf_counter() - t0) / reps * 1e3
        udl = torch.empty_like(xt_l)
        for _ in range(2):
            yk.dlp_dyadic(a_loc, dstar, J, *lb, xt_l, yt_l, q=16, out=udl, stream=lanes[a_loc])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            yk.dlp_dyadic(a_loc, dstar, J, *lb, xt_l, yt_l, q=16, out=udl, stream=lanes[a_loc])
        ms_dl = (time.perf_counter() - t0) / reps * 1e3
        dyadic = {"value": (len(xb) + xt_l.numel()) / (ms_d * 1e-3), "unit": "points/s",
                  "double_layer_ms": ms_dl,
                  "ms": ms_d, "alpha": a_loc, "delta": dstar, "levels": J,
                  "n_boundary": len(xb), "n_targets": int(xt_l.numel()),
                  "targets_reached": int((ud != 0).sum().item()),
                  "what": "yk_slp_dyadic: per level resampled panel nodes binned in cells, "
                          "difference kernel from a table, summed over nodes within R_j"}

    batch = None if args.no_batch else batch_section(yk, torch, rank)
    serving = None if args.no_serving else serving_section(yk, args.serve_requests)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(alphas, args.cpu_targets)

    launches_per_eval = 5
    # count, three scan passes, fill for sources and for targets; three for the tile order
    launches_per_set = 13
    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {**workload_config(alphas, works),
                   "grids": {str(a): plans[a].info["n_grid"] for a in alphas},
                   "l2": "inputs and grids larger than L2 (126 MB) per step; no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": pts_step * world / e2e_s, "unit": "points/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * len(alphas) * (launches_per_eval + launches_per_set),
        "gpu_launches_what": "library kernels in the timed FP64 region (5 evaluation + 13 set-up per alpha)",
        "clocks": clk,
        "stage_ms": {str(a): stage_ms[a] for a in alphas},
        "stage_ms_alone": {str(a): stage_ms_alone[a] for a in alphas},
        "cold_ms": cold_ms,
        "eval_only": {"ms_per_step": eval_only_ms,
                      "value": pts_step * world / (eval_only_ms * 1e-3) if eval_only_ms else None},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "what": "one yk_eval_longrange on a resident layout, all alphas"},
        "fp32c": fp32c,
        "double_layer": dlp,
        "slp_local": local,
        "vp_local": vlocal,
        "slp_dyadic": dyadic,
        "batch": batch,
        "serving": serving,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    for a in alphas:
        plans[a].close()
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
