"""The autotuner times every admissible tile edge on real points and records the fastest."""
import numpy as np
import pytest

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
    assert res["best_ms"] == min(res["tried"].values()) > 0
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
