"""The allocation-free entry point (yk_eval_longrange_static) against the regular plan path.

Some callers cannot call cudaMalloc (code embedded in an application that owns every device
allocation, or a process whose device footprint is fixed at start-up).  For them the library
runs a whole evaluation out of one static 32 MiB device array.  This file is collected last so
that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_static_entry_matches_plan_path_twice():
    import paper_2606_28865_b300 as yk
    w = W.config_small()
    args = [dev(a) for a in (w.xs, w.ys, w.w, w.density, w.xt, w.yt)]
    with yk.Plan(w.alpha, tol=TOL64, h_vol=w.h_vol, box=w.box) as plan:
        plan.set_points(args[0], args[1], args[2], args[4], args[5])
        ref = plan.eval(args[3]).cpu().numpy()
    scale = np.max(np.abs(ref))
    for _ in range(2):  # the second call reuses the static scratch left by the first
        out = torch.full((w.n_trg,), np.nan, dtype=torch.float64, device="cuda")
        yk.eval_longrange_static(w.alpha, *args, out, tol=TOL64, h_vol=w.h_vol, box=w.box)
        u = out.cpu().numpy()
        assert np.all(np.isfinite(u))
        assert np.max(np.abs(u - ref)) <= TOL64 * scale


def test_static_entry_rejects_what_it_cannot_hold():
    import paper_2606_28865_b300 as yk
    w = W.config_small()
    out = torch.empty(w.n_trg, dtype=torch.float64, device="cuda")
    args = [dev(a) for a in (w.xs, w.ys, w.w, w.density, w.xt, w.yt)]
    # alpha = 0.5 needs a 960^2 grid plus ~1e7 bytes of spectrum: fits; alpha = 1 with a tiny
    # delta needs a grid far beyond 32 MiB
    with pytest.raises(yk.YkError) as ei:
        yk.eval_longrange_static(1.0, *args, out, tol=TOL64, delta=4e-5, box=w.box)
    assert ei.value.status == yk.YK_ERR_UNSUPPORTED and "static scratch" in str(ei.value)
    # host arrays would need staging copies: refused
    with pytest.raises(yk.YkError) as ei:
        yk.eval_longrange_static(w.alpha, w.xs, w.ys, w.w, w.density, w.xt, w.yt,
                                 np.empty(w.n_trg), tol=TOL64, h_vol=w.h_vol, box=w.box)
    assert ei.value.status == yk.YK_ERR_ARG
