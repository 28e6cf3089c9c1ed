"""Rothe-stepping server: every request completes, results in the mix equal the same request
evaluated alone (within the plan's tolerance), and a small memory budget forces plan eviction
without losing requests."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stream_small():
    return W.rothe_stream(n_req=400, rate=2000.0, n_geom=8, seed=5, n_lo=1e3, n_hi=4e4)


@pytest.mark.parametrize("precision", [1, 0])
def test_results_same_alone_and_in_the_mix(stream_small, precision):
    from paper_2606_28865_b300.serving import RotheServer
    geoms, reqs = stream_small
    srv = RotheServer(geoms, precision=precision, max_inflight=32, n_streams=3)
    srv.warm(range(len(geoms)))
    sample = list(range(0, len(reqs), 37))
    st = srv.serve(reqs, keep_results=sample)
    assert st["requests"] == len(reqs)
    assert st["latency_ms"]["p99"] >= st["latency_ms"]["p50"] > 0.0
    assert st["mean_batch"] >= 1.0
    tol = srv.tol
    for r in sample:
        alone = srv.eval_alone(reqs[r])
        mixed = st["results"][r]
        assert np.max(np.abs(mixed - alone)) <= tol * np.max(np.abs(alone)), r
    srv.close()


def test_memory_budget_evicts_idle_plans(stream_small):
    from paper_2606_28865_b300.serving import RotheServer
    import paper_2606_28865_b300 as yk
    geoms, reqs = stream_small
    sizes = [yk.plan_params(g.alpha, g.n_src, g.n_trg, tol=1e-6, precision=1, h_vol=g.h_vol,
                            box=g.box)["device_bytes"] for g in geoms]
    base = sum(8 * (7 * g.n_src + 3 * g.n_trg) for g in geoms)
    # room for the point data and about three plans at a time
    budget = base + 3 * max(sizes)
    srv = RotheServer(geoms, precision=1, mem_budget=budget, max_inflight=8, n_streams=2)
    st = srv.serve(reqs[:150], keep_results=[0, 75, 149])
    assert st["requests"] == 150
    assert st["plans_evicted"] > 0 and st["resident_bytes"] <= budget
    for r in (0, 75, 149):
        alone = srv.eval_alone(reqs[r])
        assert np.max(np.abs(st["results"][r] - alone)) <= 1e-6 * np.max(np.abs(alone))
    srv.close()


def test_saturated_stream_batches_and_matches_alone():
    """Requests arriving faster than the GPU serves them (all 400 within ~1 ms): the server must
    batch (mean batch > 1) and each result must still equal the request evaluated alone; the plain
    per-call form on one stream gives the same potentials."""
    from paper_2606_28865_b300.serving import RotheServer
    import paper_2606_28865_b300 as yk
    geoms, reqs = W.rothe_stream(n_req=400, rate=4e5, n_geom=8, seed=5, n_lo=1e3, n_hi=4e4)
    sample = list(range(0, len(reqs), 41))
    srv = RotheServer(geoms, precision=yk.YK_FP32C, max_inflight=32, n_streams=3)
    srv.warm(range(len(geoms)))
    st = srv.serve(reqs, keep_results=sample)
    assert st["requests"] == len(reqs)
    assert st["mean_batch"] > 1.0
    for r in sample:
        alone = srv.eval_alone(reqs[r])
        assert np.max(np.abs(st["results"][r] - alone)) <= srv.tol * np.max(np.abs(alone)), r
    srv.close()
    plain = RotheServer(geoms, precision=yk.YK_FP64, n_streams=1)
    sp = plain.serve_plain(reqs, keep_results=sample)
    assert sp["requests"] == len(reqs) and sp["mean_batch"] == 1.0
    for r in sample:
        alone = plain.eval_alone(reqs[r])
        assert np.max(np.abs(sp["results"][r] - alone)) <= 1e-10 * np.max(np.abs(alone)), r
    plain.close()
