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
region.  `roofline` = the stage with the largest device time (each alpha run alone), its
algorithmic flops (the method's: N_s (2w^2 + 2w) for the spread) against the measured rate of the
arithmetic it is built from (double-float multiply-add chains, yk_fma_peak) and its algorithmic
bytes against the measured HBM copy bandwidth; durations from the timed region (overlapping
streams), `alone` from the kernels run one alpha at a time.  `fp32c.roofline` is the same for the
FP32C step.  `cpu_baseline` = the FP64 oracle (direct pair sum) on the host cores for a bounded
sample of targets, scaled to a full evaluation; `error_vs_oracle` = the timed step's results on
that sample.  `--impl reference` times that oracle alone as the reference arm.
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
    ap.add_argument("--serve-requests", type=int, default=20000,
                    help="requests of the Rothe stream per arrival rate")
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
def stage_work(info, ns, nt, b=8):
    """(bytes, flops) each stage must move / compute for one launch, counting the method's work
    only: b bytes per real (8 FP64, 4 FP32C), G = n^2 grid cells.

    * spread: 3 b N_s in (two coordinates and a strength per source) and b G out; N_s (2w^2 + 2w)
      flops (w^2 taps of one multiply and one add, plus the strength times the w y-windows and
      the w x-windows).
    * interp: b G in, 3 b N_t (two coordinates in, one value out); N_t (2w^2 + 2w) flops.
    * FFT passes: the pruned passes' own reads and writes of the grid and the half spectrum,
      5 L log2 L flops per complex L-point transform.
    * bin_src / bin_trg (set-up): 2 b per point in and the sorted layout (a grid coordinate pair
      and an index) out; the window values per point: 2w values by Horner of degree w - 1.
    What the resident layout adds on top (per-point window records read by the spread and the
    interpolation) is reported apart as `layout_bytes`, not counted as the method's work.
    """
    n, M, w = info["n_grid"], info["n_modes"], info["w"]
    G = n * n
    L = n // 2
    win = 2 * (w - 1)                                 # flops per window value (Horner, deg w-1)
    fft_row = 5 * L * math.log2(L) + 12 * L   # complex FFT of n/2 points + real post-processing
    fft_col = 5 * n * math.log2(n)
    c = 2 * b                                          # bytes of a complex value
    return {
        "bin_src": (ns * (2 * b + 2 * b + 4), ns * 2 * w * win),
        "bin_trg": (nt * (2 * b + 2 * b + 4), nt * 2 * w * win),
        "spread": (3 * b * ns + b * G, ns * (2 * w * w + 2 * w)),
        "row_fwd": (b * G + (M + 1) * n * c, n * fft_row),
        "columns": (2 * (M + 1) * n * c + (M + 1) * (2 * M + 1) * b,
                    (M + 1) * (2 * fft_col + 6 * n)),
        "row_inv": ((M + 1) * n * c + b * G, n * fft_row),
        "interp": (b * G + 3 * b * nt, nt * (2 * w * w + 2 * w)),
    }


def layout_bytes(info, ns, nt):
    """Bytes per launch the FP64 path's resident layout adds: per-point window records (2w
    double-float values of 8 bytes) read by the spread and the interpolation."""
    w = info["w"]
    return {"spread": ns * 16 * w, "interp": nt * 16 * w}


def algorithmic_bytes_eval(info, ns, nt, b):
    """Section 8(d) bytes of one evaluation: points b (3 N_s + 3 N_t) plus ten grid sweeps."""
    G = info["n_grid"] ** 2
    return b * (3 * ns + 3 * nt) + 10 * G * b


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


LAT_SAMPLES = 200  # evaluations per alpha behind each p50/p99


def latency_samples(torch, plans, dbufs, outs, lanes, alphas, n=LAT_SAMPLES):
    """Device time of single yk_eval_longrange calls on a resident layout (events around each
    call on the plan's stream, synchronised per call): n samples per alpha."""
    lat = []
    for a in alphas:
        d = dbufs[a][5]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        for s0, s1 in ev:
            s0.record(lanes[a])
            plans[a].eval(d, out=outs[a])
            s1.record(lanes[a])
            s1.synchronize()
        lat.extend(s0.elapsed_time(s1) for s0, s1 in ev)
    return lat


def roofline(stage_ms, stage_ms_alone, plans, works, alphas, peaks, hbm_peak, peak_kind, b, df):
    """Roofline block of the dominant stage (largest summed device time over the alphas when
    each kernel runs alone): algorithmic flops against the measured rate of the arithmetic the
    stage is built from, and algorithmic bytes against the measured HBM copy bandwidth."""
    def totals(sms):
        tot, wb, wf, lb = {}, {}, {}, {}
        for a in alphas:
            info = plans[a].info
            sw = stage_work(info, works[a].n_src, works[a].n_trg, b)
            lay = layout_bytes(info, works[a].n_src, works[a].n_trg) if df else {}
            for k, v in sms[a].items():
                if v is None:
                    continue
                tot[k] = tot.get(k, 0.0) + v
                wb[k] = wb.get(k, 0.0) + sw[k][0]
                wf[k] = wf.get(k, 0.0) + sw[k][1]
                lb[k] = lb.get(k, 0.0) + lay.get(k, 0)
        return tot, wb, wf, lb

    tot, wb, wf, lb = totals(stage_ms)
    tot1, _, _, _ = totals(stage_ms_alone)
    dom = max(tot1, key=tot1.get)
    if df:
        # the FP64 path's spread accumulates with the unnormalised double-float multiply-add, the
        # other stages with the renormalised one (both measured by yk_fma_peak)
        key = "df_lazy" if dom == "spread" else "df"
        note = ("double-float multiply-add chains measured by yk_fma_peak (%s form), 2 "
                "FP64-equivalent flops each" % ("unnormalised" if key == "df_lazy" else
                                                "renormalised"))
    else:
        key = "fp32"
        note = "FP32 FMA chains measured by yk_fma_peak"
    alu_peak = peaks[key]
    t_in, t_al = tot[dom] * 1e-3, tot1[dom] * 1e-3
    alu_in, alu_al = wf[dom] / t_in / 1e12, wf[dom] / t_al / 1e12
    hbm_in, hbm_al = wb[dom] / t_in / 1e9, wb[dom] / t_al / 1e9
    fa, fh = alu_in / alu_peak, hbm_in / hbm_peak
    alu = fa >= fh
    traffic = load_traffic().get(dom) if df else None
    return {"bound": "alu" if alu else "hbm",
            "achieved": alu_in if alu else hbm_in, "peak": alu_peak if alu else hbm_peak,
            "unit": "TFLOP/s" if alu else "GB/s", "frac": fa if alu else fh,
            "traffic": traffic, "kernel": dom, "launches_per_step": len(alphas),
            "peak_source": note if alu else f"HBM copy bandwidth, {peak_kind} "
                                              "(MEASURED_PEAKS.json)",
            "frac_alu": fa, "frac_hbm": fh, "alu_peak_tflops": alu_peak,
            "hbm_peak_gbs": hbm_peak, "alu_achieved_tflops": alu_in, "hbm_achieved_gbs": hbm_in,
            "algorithmic_flops_per_step": wf[dom], "algorithmic_bytes_per_step": wb[dom],
            "layout_bytes_per_step": lb.get(dom, 0),
            "durations": "CUDA events around the stage on its stream in the timed region, where "
                         "the alphas' streams overlap (so the durations include other streams' "
                         "kernels), summed over the alphas",
            "alone": {"alu_achieved_tflops": alu_al, "hbm_achieved_gbs": hbm_al,
                      "frac_alu": alu_al / alu_peak, "frac_hbm": hbm_al / hbm_peak,
                      "what": "the same stage with each alpha run alone (no other stream "
                              "running)"},
            "measured_peaks_tflops": peaks}


# ---------------------------------------------------------------------------------------------
def cpu_baseline(alphas, n_targets, results=None):
    """FP64 oracle, all sources x a bounded sample of targets, scaled to full evaluations.

    results: {name: {alpha: u at all targets}} from the GPU runs; each gets its relative L-inf
    error against the oracle on the sampled targets, max |u - u_oracle| / max |u_oracle|."""
    import oracle
    total_pts = 0.0
    total_t = 0.0
    errors = {name: {} for name in (results or {})}
    for a in alphas:
        work = W.config_large(a)
        rng = np.random.default_rng(1)
        idx = rng.choice(work.n_trg, n_targets, replace=False)
        table = oracle.GHTable(a, _delta(work, a), oracle.pair_rmax(work.xs, work.ys, work.xt,
                                                                      work.yt))
        t0 = time.perf_counter()
        ref = oracle.direct_sum(a, _delta(work, a), work.xs, work.ys, work.q, work.xt[idx],
                                work.yt[idx], table=table)
        dt = time.perf_counter() - t0
        total_t += dt * work.n_trg / n_targets           # time of the full evaluation
        total_pts += work.n_src + work.n_trg
        for name, res in (results or {}).items():
            if res is not None and a in res:
                errors[name][str(a)] = float(np.max(np.abs(res[a][idx] - ref)) /
                                             np.max(np.abs(ref)))
    out = {"value": total_pts / total_t, "unit": "points/s", "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": (f"FP64 direct pair sum over all {int(W.config_large(alphas[0]).n_src)} "
                      f"sources for {n_targets} of the 1e6 targets at each alpha in "
                      f"{list(alphas)}; time scaled by 1e6/{n_targets} to a full evaluation")}
    return out, errors


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


SERVE_RATES = (2000.0, 8000.0, 32000.0, 128000.0)


def serving_section(yk, n_req):
    """Rothe stream (config 5): 64 simulations (points log-uniform in [1e3, 1e6], dt log-uniform
    in [1e-4, 1e-1]), n_req Poisson arrivals, swept over arrival rates up to saturation: the FP32C
    continuous-batching server against the plain FP64 per-call form (one stream, each call waited
    for) on the same requests and the same GPU.  The same geometries and requests at every rate
    (only the arrival times scale)."""
    from paper_2606_28865_b300.serving import RotheServer
    geoms, _ = W.rothe_stream(n_req=1, rate=SERVE_RATES[0], n_geom=64, seed=0)
    out = {"workload": f"{n_req} requests per rate, Poisson arrivals, 64 resident geometries "
                       f"(points log-uniform in [1e3, 1e6])",
           "rates_req_per_s": list(SERVE_RATES)}
    forms = (("fp32c_batched", yk.YK_FP32C, dict(max_inflight=64, n_streams=4), "serve"),
             ("fp64_plain", yk.YK_FP64, dict(n_streams=1), "serve_plain"))
    for key, prec, kw, how in forms:
        srv = RotheServer(geoms, precision=prec, **kw)
        srv.warm(range(len(geoms)))
        per_rate = []
        for rate in SERVE_RATES:
            _, reqs = W.rothe_stream(n_req=n_req, rate=rate, n_geom=64, seed=0)
            st = getattr(srv, how)(reqs)
            st.pop("results", None)
            st["rate_req_per_s"] = rate
            st["offered_points_per_s"] = (sum(geoms[r["geom"]].n_src + geoms[r["geom"]].n_trg
                                              for r in reqs) / reqs[-1]["t_arrive"])
            per_rate.append(st)
        out[key] = per_rate
        out[key + "_saturated"] = {"points_per_s": per_rate[-1]["points_per_s"],
                                   "p50_ms": per_rate[-1]["latency_ms"]["p50"],
                                   "p99_ms": per_rate[-1]["latency_ms"]["p99"],
                                   "mean_batch": per_rate[-1]["mean_batch"],
                                   "rate_req_per_s": SERVE_RATES[-1]}
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

    # the step's results, kept for the per-alpha error against the oracle sample
    u_fp64 = {a: outs[a].cpu().numpy().copy() for a in alphas}

    # per-eval latency distribution (device events per call, LAT_SAMPLES calls per alpha)
    lat = latency_samples(torch, plans, dbufs, outs, lanes, alphas)

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
    peaks = {"fp64": yk.fma_peak_tflops(yk.YK_FP64), "fp32": yk.fma_peak_tflops(yk.YK_FP32C),
             "df": yk.fma_peak_tflops(yk.YK_PEAK_DF),
             "df_lazy": yk.fma_peak_tflops(yk.YK_PEAK_DF_LAZY)}
    roof = roofline(stage_ms, stage_ms_alone, plans, works, alphas, peaks, hbm_peak, peak_kind,
                    b=8, df=True)

    # the FP32C form of the same workload (FP32 spread/FFT/interp, two-sum grid sums, FP64
    # final sums at the targets; relative accuracy 1e-6)
    fp32c, u_fp32c = None, None
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
        st32 = {a: plans32[a].stage_times() for a in alphas}
        u_fp32c = {a: outs[a].cpu().numpy().copy() for a in alphas}
        lat32 = latency_samples(torch, plans32, dbufs, outs, lanes, alphas)
        # each alpha alone: stage durations without the other streams, and the evaluation
        # stages' Section 8(d) bytes per second against the HBM copy bandwidth
        for _ in range(3):
            for a in alphas:
                xs, ys, w, xt, yt, d = dbufs[a]
                plans32[a].set_points(xs, ys, w, xt, yt)
                plans32[a].eval(d, out=outs[a])
                torch.cuda.synchronize()
        st32_alone = {a: plans32[a].stage_times() for a in alphas}
        eval_hbm = {}
        for a in alphas:
            ms_e = sum(v for k, v in st32_alone[a].items()
                       if k not in ("bin_src", "bin_trg") and v)
            by = algorithmic_bytes_eval(plans32[a].info, works[a].n_src, works[a].n_trg, 4)
            eval_hbm[str(a)] = {"eval_ms": ms_e, "algorithmic_bytes": by,
                                "gbs": by / (ms_e * 1e-3) / 1e9,
                                "frac_hbm": by / (ms_e * 1e-3) / 1e9 / hbm_peak}
        roof32 = roofline(st32, st32_alone, plans32, works, alphas, peaks, hbm_peak, peak_kind,
                          b=4, df=False)
        fp32c = {"value": pts_step * world / (ms32 * 1e-3), "unit": "points/s",
                 "ms_per_step": ms32, "tol": 1e-6, "dtype": "f32 (two-sum grid, f64 final sums)",
                 "grids": {str(a): plans32[a].info["n_grid"] for a in alphas},
                 "stage_ms": {str(a): v for a, v in st32.items()},
                 "stage_ms_alone": {str(a): v for a, v in st32_alone.items()},
                 "roofline": roof32,
                 "eval_only_hbm": eval_hbm,
                 "latency_ms": {"p50": float(np.percentile(lat32, 50)),
                                "p99": float(np.percentile(lat32, 99)),
                                "samples": len(lat32)}}
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

    # double-layer local asymptotic part D_{L,A} at the same targets, boundary and delta*
    dlocal = None
    if not args.no_local:
        udla = torch.empty_like(xt_l)
        for _ in range(2):
            yk.dlp_local(a_loc, dstar, *lb, xt_l, yt_l, q=16, out=udla, stream=lanes[a_loc])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            yk.dlp_local(a_loc, dstar, *lb, xt_l, yt_l, q=16, out=udla, stream=lanes[a_loc])
        ms_dla = (time.perf_counter() - t0) / reps * 1e3
        dlocal = {"value": (len(xb) + xt_l.numel()) / (ms_dla * 1e-3), "unit": "points/s",
                  "ms": ms_dla, "alpha": a_loc, "delta_star": dstar, "n_boundary": len(xb),
                  "n_targets": int(xt_l.numel()),
                  "targets_within_locality": int((udla != 0).sum().item()),
                  "what": "yk_dlp_local: as yk_slp_local, with the curve's and the density's "
                          "first four derivatives at the closest point"}

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

    cpu, errors = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, errors = cpu_baseline(alphas, args.cpu_targets,
                                   {"fp64": u_fp64, "fp32c": u_fp32c})
        errors["what"] = (f"relative L-inf error max|u - u_oracle| / max|u_oracle| on the "
                          f"{args.cpu_targets} sampled targets per alpha of the timed step's "
                          f"results; bars 1e-10 (fp64) and 1e-6 (fp32c)")

    launches_per_eval = 5

    def launches_per_set(info):
        # sources: count, scan, fill, the tile order (one kernel up to 8,192 tiles, else three),
        # the window values; targets: chunk histograms, column offsets, scan, scatter, the window
        # values (or, beyond 16,384 target tiles, count, scan, fill); a scan is one kernel up to
        # 8,192 counts, else three
        n = info["n_grid"]
        ts, tt = (n // info["tile"]) ** 2, (n // info["interp_tile"]) ** 2
        scan = lambda c: 1 if c <= 8192 else 3
        src = 1 + scan(ts) + 1 + (1 if ts <= 8192 else 3) + 1
        trg = (1 + 1 + scan(tt) + 1 if tt <= 16384 else 1 + scan(tt) + 1) + 1
        return src + trg
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
        "gpu_launches": args.steps * sum(launches_per_eval + launches_per_set(plans[a].info)
                                         for a in alphas),
        "gpu_launches_what": "library kernels in the timed FP64 region: 5 evaluation and 10 to 16 "
                             "set-up launches per alpha (scans of up to 8,192 counts and tile "
                             "orders of up to 8,192 tiles in one kernel)",
        "clocks": clk,
        "stage_ms": {str(a): stage_ms[a] for a in alphas},
        "stage_ms_alone": {str(a): stage_ms_alone[a] for a in alphas},
        "cold_ms": cold_ms,
        "eval_only": {"ms_per_step": eval_only_ms,
                      "value": pts_step * world / (eval_only_ms * 1e-3) if eval_only_ms else None},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "samples": len(lat),
                       "what": f"one yk_eval_longrange on a resident layout, {LAT_SAMPLES} calls "
                               f"per alpha"},
        "error_vs_oracle": errors,
        "fp32c": fp32c,
        "double_layer": dlp,
        "slp_local": local,
        "dlp_local": dlocal,
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
