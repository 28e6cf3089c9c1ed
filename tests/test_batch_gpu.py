"""Batched persistent launch: results equal to per-plan evaluation, graph replay, rebuild after
new points, trivial instances, and a bounded wait that runs out by design.

The batch kernel runs the same stage bodies as the per-stage kernels, but compiled into another
kernel the compiler may fuse a multiply-add differently, so the two agree to rounding (checked at
1e-13 of the result's size, far below the 1e-10 / 1e-6 tolerances) while replays of one batch are
bitwise identical."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def make_instances(n_inst, seed, lo=1e3, hi=3e4):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        alpha = math.exp(rng.uniform(math.log(1.0), math.log(300.0)))
        out.append(W.random_instance(rng, n, alpha))
    return out


def check_against_oracle(wk, info, u, tol, seed, n=200):
    """Relative L-inf error of u on n sampled targets (the largest |u| among them) <= tol."""
    rng = np.random.default_rng(seed)
    idx = np.unique(np.r_[rng.choice(wk.n_trg, min(n, wk.n_trg) - 1, replace=False),
                          np.argmax(np.abs(u))])
    r = oracle.direct_sum(wk.alpha, info["delta"], wk.xs, wk.ys, wk.q, wk.xt[idx], wk.yt[idx])
    err = np.max(np.abs(u[idx] - r)) / np.max(np.abs(r))
    assert err <= tol, (wk.alpha, wk.n_src, err)
    return err


def plan_for(yk, wk, prec):
    tol = 1e-10 if prec == 0 else 1e-6
    p = yk.Plan(wk.alpha, tol=tol, precision=prec, h_vol=wk.h_vol, box=wk.box)
    p.set_points(dev(wk.xs), dev(wk.ys), dev(wk.w), dev(wk.xt), dev(wk.yt))
    return p


def test_batch_matches_per_plan_bitwise():
    import paper_2606_28865_b300 as yk
    works = make_instances(12, seed=1)
    plans = [plan_for(yk, wk, i % 2) for i, wk in enumerate(works)]   # FP64 and FP32C mixed
    dens = [dev(wk.density) for wk in works]
    ref = [p.eval(d).cpu().numpy() for p, d in zip(plans, dens)]
    outs = [torch.full((wk.n_trg,), np.nan, dtype=torch.float64, device="cuda") for wk in works]
    b = yk.Batch(plans)
    first = None
    for rep in range(3):  # first run captures the graph, later runs replay it
        for o in outs:
            o.fill_(np.nan)
        b.run(dens, outs)
        b.sync()
        got = [o.cpu().numpy() for o in outs]
        for k in range(len(works)):
            scale = np.max(np.abs(ref[k]))
            assert np.max(np.abs(got[k] - ref[k])) <= 1e-13 * scale, (k, rep)
        if first is None:
            first = got
        else:
            assert all(np.array_equal(a, c) for a, c in zip(first, got))
    # every instance against the oracle at its plan's tolerance, on 200 sampled targets that
    # include the largest |u| (the tolerance is relative to max |u|)
    for k, wk in enumerate(works):
        check_against_oracle(wk, plans[k].info, got[k], 1e-10 if k % 2 == 0 else 1e-6, seed=k)
    # new densities with the same graph
    dens2 = [dev(W.strengths_for(wk, wk.alpha, seed=9)) for wk in works]
    b.run(dens2, outs)
    b.sync()
    for k in range(len(works)):
        alone = plans[k].eval(dens2[k]).cpu().numpy()
        assert np.max(np.abs(outs[k].cpu().numpy() - alone)) <= 1e-13 * np.max(np.abs(alone))
    b.close()
    for p in plans:
        p.close()


def test_batch_rebuilds_after_new_points_and_handles_trivial_plans():
    import paper_2606_28865_b300 as yk
    works = make_instances(4, seed=2)
    plans = [plan_for(yk, wk, 0) for wk in works]
    # a plan whose history part is below tolerance (printed k_max rule), and one without targets
    zero = yk.Plan(200.0, tol=1e-6, delta=1.01 * math.log(4e6) / 200.0 ** 2, kmax_rule=1)
    zero.set_points(dev(works[0].xs), dev(works[0].ys), dev(works[0].w), dev(works[0].xt),
                    dev(works[0].yt))
    empty = yk.Plan(10.0, tol=1e-10, delta=0.0167)
    empty.set_points(dev(works[1].xs), dev(works[1].ys), dev(works[1].w), dev([]), dev([]))
    allp = plans + [zero, empty]
    dens = [dev(wk.density) for wk in works] + [dev(works[0].density), dev(works[1].density)]
    outs = [torch.full((p.n_trg,), np.nan, dtype=torch.float64, device="cuda") for p in allp]
    b = yk.Batch(allp)
    b.run(dens, outs)
    b.sync()
    assert torch.all(outs[4] == 0.0)
    # move the targets of plan 2: the batch notices and rebuilds its work list
    wk = works[2]
    plans[2].set_points(dev(wk.xs), dev(wk.ys), dev(wk.w), dev(wk.xt[::-1].copy()),
                        dev(wk.yt[::-1].copy()))
    b.run(dens, outs)
    b.sync()
    alone = plans[2].eval(dens[2]).cpu().numpy()
    assert np.max(np.abs(outs[2].cpu().numpy() - alone)) <= 1e-13 * np.max(np.abs(alone))
    b.close()
    for p in allp:
        p.close()


def test_batch_wait_times_out_without_hanging():
    import paper_2606_28865_b300 as yk
    works = make_instances(3, seed=3, hi=5e3)
    plans = [plan_for(yk, wk, 0) for wk in works]
    dens = [dev(wk.density) for wk in works]
    outs = [torch.empty(wk.n_trg, dtype=torch.float64, device="cuda") for wk in works]
    # one dependency can never be met; each wait gives up after ~20000 polls
    b = yk.Batch(plans, use_graph=False, spin_limit=20000, inject_stall=True)
    b.run(dens, outs)
    with pytest.raises(yk.YkError) as ei:
        b.sync()
    assert ei.value.status == yk.YK_ERR_TIMEOUT
    b.close()
    # the context is still usable
    u = plans[0].eval(dens[0]).cpu().numpy()
    assert np.all(np.isfinite(u))
    for p in plans:
        p.close()
