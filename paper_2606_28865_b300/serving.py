"""Continuous-batching server for Rothe time stepping over resident geometries.

Each simulation (geometry) keeps its plan and its sorted point layout on the device; a request is
one time step: new strengths on that geometry, u = S_H[sigma] + V_H[f] at its targets.  The loop:

* admits arrived requests while in-flight slots are free, at most one in flight per plan (the
  plan's grid buffers belong to one evaluation at a time);
* creates plans on demand under a device-memory budget, evicting the least recently used idle
  plans when the budget would be exceeded (memory-based admission: a request whose plan cannot
  be made resident waits in the queue);
* launches every tick's admitted requests as one batch (yk_batch_run) on the next stream of a
  small pool, so batches admitted while others are still on the GPU overlap with them;
* retires requests when their batch's CUDA event completes and records arrival-to-completion
  latency.

Marshalling and scheduling only: every evaluation runs in the library's kernels.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import YK_FP32C, YK_FP64, Batch, Plan, plan_params


class Geometry:
    """Resident device copy of one simulation's points, weights and strength variants."""

    def __init__(self, work, dev, n_variants, strengths_fn):
        import torch
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        self.work = work
        self.alpha = work.alpha
        self.xs, self.ys, self.w = t(work.xs), t(work.ys), t(work.w)
        self.xt, self.yt = t(work.xt), t(work.yt)
        self.dens = [t(strengths_fn(work, work.alpha, seed=v)) for v in range(n_variants)]
        self.out = torch.empty(work.n_trg, dtype=torch.float64, device=dev)
        self.points = work.n_src + work.n_trg
        self.bytes = 8 * (3 * work.n_src + 3 * work.n_trg + n_variants * work.n_src)


class RotheServer:
    def __init__(self, works, precision=YK_FP32C, tol=None, mem_budget=40 << 30,
                 max_inflight=64, n_streams=4, n_variants=4, batch=True, dev="cuda"):
        import torch
        import workloads as W
        self.torch = torch
        self.precision = precision
        self.tol = tol if tol is not None else (1e-6 if precision == YK_FP32C else 1e-10)
        self.mem_budget = int(mem_budget)
        self.max_inflight = int(max_inflight)
        self.batch = batch
        self.dev = torch.device(dev)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_streams)]
        self.batches = [None] * n_streams      # one reusable batch per stream
        self.geoms = [Geometry(wk, self.dev, n_variants, W.strengths_for) for wk in works]
        self.plans = collections.OrderedDict()   # geometry id -> Plan (LRU order)
        self.plan_bytes = {}
        self.busy = set()                        # geometries with a request in flight
        self.resident = sum(g.bytes for g in self.geoms)
        self.n_created = 0
        self.n_evicted = 0
        torch.cuda.synchronize()

    # -- memory-based admission ------------------------------------------------------------
    def _predicted(self, gid):
        g = self.geoms[gid]
        info = plan_params(g.alpha, g.work.n_src, g.work.n_trg, tol=self.tol,
                           precision=self.precision, h_vol=g.work.h_vol, box=g.work.box)
        return int(info["device_bytes"])

    def _ensure_plan(self, gid, pinned=()):
        """Plan of geometry gid, created if needed; idle plans (not busy, not pinned) are evicted
        least recently used first to keep within the memory budget.  None if it cannot fit."""
        if gid in self.plans:
            self.plans.move_to_end(gid)
            return self.plans[gid]
        need = self._predicted(gid)
        while self.resident + need > self.mem_budget:
            victim = next((k for k in self.plans if k not in self.busy and k not in pinned),
                          None)
            if victim is None:
                return None          # nothing idle to evict: the request waits
            self.plans.pop(victim).close()
            self.resident -= self.plan_bytes.pop(victim)
            self.n_evicted += 1
        g = self.geoms[gid]
        st = self.streams[gid % len(self.streams)]
        p = Plan(g.alpha, tol=self.tol, precision=self.precision, h_vol=g.work.h_vol,
                 box=g.work.box, stream=st)
        p.stream_obj = st
        p.set_points(g.xs, g.ys, g.w, g.xt, g.yt)
        p.sync()
        self.plans[gid] = p
        self.plan_bytes[gid] = need
        self.resident += need
        self.n_created += 1
        return p

    def warm(self, gids):
        """Make the plans of the given geometries resident ahead of the stream (as a simulation
        start-up would)."""
        for gid in gids:
            self._ensure_plan(gid)

    # -- the loop ------------------------------------------------------------------------------
    def serve(self, requests, keep_results=()):
        """Run the request stream in real time.  requests: dicts {t_arrive, geom, seed} with
        t_arrive in seconds from the start.  Returns statistics; results of the request indices
        in keep_results are copied to the host."""
        torch = self.torch
        pending = collections.deque(sorted(range(len(requests)),
                                           key=lambda i: requests[i]["t_arrive"]))
        queue = collections.deque()
        inflight = []           # ([events], [request ids], stream index)
        lat = np.full(len(requests), np.nan)
        done_points = 0
        kept = {}
        keep = set(keep_results)
        n_batches = 0
        batch_sizes = []
        s_next = 0
        t0 = time.perf_counter()
        t_first = None
        t_last = None
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            while pending and requests[pending[0]]["t_arrive"] <= now:
                queue.append(pending.popleft())
            # retire finished batches
            still = []
            for evs, rids, _ in inflight:
                if all(ev.query() for ev in evs):
                    tc = time.perf_counter() - t0
                    for r in rids:
                        lat[r] = tc - requests[r]["t_arrive"]
                        g = requests[r]["geom"]
                        self.busy.discard(g)
                        done_points += self.geoms[g].points
                        if r in keep:
                            kept[r] = self.geoms[g].out.cpu().numpy()
                    t_last = tc
                else:
                    still.append((evs, rids, _))
            inflight = still
            # admit
            n_in = sum(len(x[1]) for x in inflight)
            admitted = []
            if queue and n_in < self.max_inflight:
                skipped = collections.deque()
                seen = set()
                while queue and n_in + len(admitted) < self.max_inflight:
                    r = queue.popleft()
                    g = requests[r]["geom"]
                    if g in self.busy or g in seen:
                        skipped.append(r)
                        continue
                    p = self._ensure_plan(g, pinned=seen)
                    if p is None:
                        skipped.append(r)
                        break
                    admitted.append(r)
                    seen.add(g)
                queue.extendleft(reversed(skipped))
            if admitted:
                si = s_next % len(self.streams)
                s_next += 1
                stream = self.streams[si]
                plans = [self.plans[requests[r]["geom"]] for r in admitted]
                dens = [self.geoms[requests[r]["geom"]].dens[requests[r]["seed"] % len(
                    self.geoms[requests[r]["geom"]].dens)] for r in admitted]
                outs = [self.geoms[requests[r]["geom"]].out for r in admitted]
                evs = []
                if self.batch:
                    if self.batches[si] is None:
                        self.batches[si] = Batch(plans, use_graph=False, stream=stream)
                    else:
                        self.batches[si].set_plans(plans)  # waits for this stream's last batch
                    self.batches[si].run(dens, outs)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                    evs.append(ev)
                else:
                    # plain per-call form: each request on its own plan's stream
                    for p, d, o in zip(plans, dens, outs):
                        p.eval(d, out=o)
                        ev = torch.cuda.Event()
                        ev.record(p.stream_obj)
                        evs.append(ev)
                for r in admitted:
                    self.busy.add(requests[r]["geom"])
                inflight.append((evs, admitted, si))
                n_batches += 1
                batch_sizes.append(len(admitted))
                if t_first is None:
                    t_first = now
            elif not inflight and queue:
                # nothing can be admitted and nothing is running: the memory budget is too small
                raise RuntimeError("a request cannot be admitted within the memory budget")
            else:
                time.sleep(0)
        torch.cuda.synchronize()
        wall = (t_last or 0.0) - float(requests[0]["t_arrive"] if requests else 0.0)
        ok = lat[~np.isnan(lat)]
        return {
            "requests": int(len(ok)),
            "points": int(done_points),
            "points_per_s": done_points / wall if wall > 0 else None,
            "wall_s": wall,
            "latency_ms": {"p50": float(np.percentile(ok, 50) * 1e3),
                           "p99": float(np.percentile(ok, 99) * 1e3),
                           "max": float(np.max(ok) * 1e3)},
            "batches": n_batches,
            "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0.0,
            "plans_created": self.n_created,
            "plans_evicted": self.n_evicted,
            "resident_bytes": int(self.resident),
            "results": kept,
        }

    def serve_plain(self, requests, keep_results=()):
        """The plain per-call form, for comparison: no admission loop and no batching;
        requests are taken in arrival order, each evaluated as soon as it has arrived and the
        previous call has returned, and each call waits for its result (a caller that calls the
        evaluator and uses the potential).  Meant for a server built with n_streams=1, so every
        call runs on one stream.  Same statistics as serve()."""
        order = sorted(range(len(requests)), key=lambda i: requests[i]["t_arrive"])
        lat = np.full(len(requests), np.nan)
        kept, keep = {}, set(keep_results)
        done_points = 0
        for g in {requests[r]["geom"] for r in order}:
            self._ensure_plan(g)
        t0 = time.perf_counter()
        t_last = None
        for r in order:
            while time.perf_counter() - t0 < requests[r]["t_arrive"]:
                pass
            g = requests[r]["geom"]
            geo = self.geoms[g]
            p = self.plans[g]
            p.eval(geo.dens[requests[r]["seed"] % len(geo.dens)], out=geo.out)
            p.stream_obj.synchronize()
            tc = time.perf_counter() - t0
            lat[r] = tc - requests[r]["t_arrive"]
            done_points += geo.points
            if r in keep:
                kept[r] = geo.out.cpu().numpy()
            t_last = tc
        wall = (t_last or 0.0) - float(requests[order[0]]["t_arrive"] if requests else 0.0)
        return {
            "requests": int(np.sum(~np.isnan(lat))),
            "points": int(done_points),
            "points_per_s": done_points / wall if wall > 0 else None,
            "wall_s": wall,
            "latency_ms": {"p50": float(np.nanpercentile(lat, 50) * 1e3),
                           "p99": float(np.nanpercentile(lat, 99) * 1e3),
                           "max": float(np.nanmax(lat) * 1e3)},
            "batches": len(order),
            "mean_batch": 1.0,
            "plans_created": self.n_created,
            "plans_evicted": self.n_evicted,
            "resident_bytes": int(self.resident),
            "results": kept,
        }

    def eval_alone(self, req):
        """The same request evaluated alone on an idle GPU (for the mix-invariance check)."""
        g = req["geom"]
        p = self._ensure_plan(g)
        geo = self.geoms[g]
        d = geo.dens[req["seed"] % len(geo.dens)]
        out = self.torch.empty_like(geo.out)
        p.eval(d, out=out)
        p.sync()
        return out.cpu().numpy()

    def close(self):
        for b in self.batches:
            if b is not None:
                b.close()
        self.batches = [None] * len(self.streams)
        for p in self.plans.values():
            p.close()
        self.plans.clear()
