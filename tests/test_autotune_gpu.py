"""The autotuner times every admissible tile edge on real points and records the fastest."""
import numpy as np
import pytest

import oracle
import oracle.params as OP
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_records_the_fastest_tile():
    import paper_2606_28865_b300 as yk
    yk.tune_cache_clear()
    wk = W.config_large(10.0)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    args = [t(wk.xs), t(wk.ys), t(wk.w), t(wk.density), t(wk.xt), t(wk.yt)]
    res = yk.autotune(10.0, *args, tol=1e-6, precision=yk.YK_FP32C, h_vol=wk.h_vol)
    assert len(res["tried"]) >= 2
    assert res["tried"][res["best_tile"]] == min(res["tried"].values()) > 0
    assert res["best_ms"] > 0   # one evaluation at the best tile and the tuned launch shape
    info = yk.plan_params(10.0, wk.n_src, wk.n_trg, tol=1e-6, precision=yk.YK_FP32C,
                          h_vol=wk.h_vol, use_tuned=True, n_src_hint=wk.n_src)
    assert info["tile"] == res["best_tile"]
    # a tuned plan gives the same potentials (within the tolerance) as the default one
    plan_t = yk.Plan(10.0, tol=1e-6, precision=yk.YK_FP32C, h_vol=wk.h_vol, use_tuned=True,
                     n_src_hint=wk.n_src)
    plan_d = yk.Plan(10.0, tol=1e-6, precision=yk.YK_FP32C, h_vol=wk.h_vol)
    for p in (plan_t, plan_d):
        p.set_points(args[0], args[1], args[2], args[4], args[5])
    ut = plan_t.eval(args[3]).cpu().numpy()
    ud = plan_d.eval(args[3]).cpu().numpy()
    assert np.max(np.abs(ut - ud)) <= 1e-6 * np.max(np.abs(ud))
    yk.tune_cache_clear()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_every_admissible_tile_and_the_tuned_plan_match_the_oracle(prec, tol):
    """Each tile edge a plan may take (the autotuner's candidates), and the plan built from the
    tuned cache, against the FP64 oracle at the stated tolerance (config-1 workload, alpha = 10,
    and a larger grid at alpha = 0.5)."""
    import paper_2606_28865_b300 as yk
    wk = W.config_small()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    args = [t(wk.xs), t(wk.ys), t(wk.w), t(wk.density), t(wk.xt), t(wk.yt)]
    for alpha in (wk.alpha, 0.5):
        ref = oracle.direct_sum(alpha, OP.delta_from_mesh(alpha, wk.h_vol), wk.xs, wk.ys, wk.q,
                                wk.xt, wk.yt)
        scale = np.max(np.abs(ref))
        yk.tune_cache_clear()
        res = yk.autotune(alpha, *args, tol=tol, precision=prec, h_vol=wk.h_vol, box=wk.box)
        assert len(res["tried"]) >= 1
        for tile in sorted(res["tried"]):
            with yk.Plan(alpha, tol=tol, precision=prec, h_vol=wk.h_vol, box=wk.box,
                         tile=int(tile)) as p:
                assert p.info["tile"] == int(tile)
                p.set_points(args[0], args[1], args[2], args[4], args[5])
                u = p.eval(args[3]).cpu().numpy()
            assert np.max(np.abs(u - ref)) <= tol * scale, (alpha, tile)
        # every edge of the targets' tiles (apart from the spread's tile edge)
        n, w = res["n_grid"], yk.plan_params(alpha, tol=tol, precision=prec, h_vol=wk.h_vol)["w"]
        edges = [e for e in range(w, 33) if n % e == 0 and n >= 2 * e]
        assert res["best_interp_tile"] in edges
        for ti in edges:
            with yk.Plan(alpha, tol=tol, precision=prec, h_vol=wk.h_vol, box=wk.box,
                         interp_tile=ti) as p:
                assert p.info["interp_tile"] == ti
                p.set_points(args[0], args[1], args[2], args[4], args[5])
                u = p.eval(args[3]).cpu().numpy()
            assert np.max(np.abs(u - ref)) <= tol * scale, (alpha, ti)
        # the launch shape was searched too, and a tuned plan takes all of it
        assert 1 <= res["best_spread_warps"] <= 4 and res["best_interp_threads"] in (64, 128, 256)
        assert res["best_spread_batch"] in ((4, 8, 16) if prec == 0 else (8, 16, 32))
        with yk.Plan(alpha, tol=tol, precision=prec, h_vol=wk.h_vol, box=wk.box, use_tuned=True,
                     n_src_hint=wk.n_src) as p:
            info = p.info
            assert info["tile"] == res["best_tile"]
            assert (info["spread_warps"], info["spread_batch"], info["interp_threads"],
                    info["interp_tile"]) == (res["best_spread_warps"], res["best_spread_batch"],
                                             res["best_interp_threads"], res["best_interp_tile"])
            p.set_points(args[0], args[1], args[2], args[4], args[5])
            u = p.eval(args[3]).cpu().numpy()
        assert np.max(np.abs(u - ref)) <= tol * scale, alpha
        # every launch shape the tuner may pick gives the same potentials within the tolerance
        for sw, sb, it in ((1, 4 if prec == 0 else 8, 64), (2, 8 if prec == 0 else 16, 128),
                           (3, 16 if prec == 0 else 32, 256)):
            with yk.Plan(alpha, tol=tol, precision=prec, h_vol=wk.h_vol, box=wk.box,
                         spread_warps=sw, spread_batch=sb, interp_threads=it) as p:
                p.set_points(args[0], args[1], args[2], args[4], args[5])
                u = p.eval(args[3]).cpu().numpy()
            assert np.max(np.abs(u - ref)) <= tol * scale, (alpha, sw, sb, it)
    yk.tune_cache_clear()


def test_tune_cache_round_trip_keeps_the_launch_shape(tmp_path):
    import paper_2606_28865_b300 as yk
    yk.tune_cache_clear()
    wk = W.config_small()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    args = [t(wk.xs), t(wk.ys), t(wk.w), t(wk.density), t(wk.xt), t(wk.yt)]
    res = yk.autotune(wk.alpha, *args, tol=1e-10, h_vol=wk.h_vol, box=wk.box)
    path = str(tmp_path / "tune.txt")
    yk.tune_cache_save(path)
    yk.tune_cache_clear()
    yk.tune_cache_load(path)
    info = yk.plan_params(wk.alpha, wk.n_src, wk.n_trg, tol=1e-10, h_vol=wk.h_vol, box=wk.box,
                          use_tuned=True, n_src_hint=wk.n_src)
    assert (info["tile"], info["spread_warps"], info["spread_batch"], info["interp_threads"],
            info["interp_tile"]) == (res["best_tile"], res["best_spread_warps"],
                                     res["best_spread_batch"], res["best_interp_threads"],
                                     res["best_interp_tile"])
    yk.tune_cache_clear()
