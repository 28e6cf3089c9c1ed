"""The allocation-free entry point (yk_eval_longrange_static) against the oracle and the plan path.

Some callers cannot call cudaMalloc: code embedded in an application that owns every device
allocation (a plug-in handed fixed buffers), or a process whose device footprint is fixed at
start-up.  For them the library runs a whole evaluation out of one static 32 MiB device array.
This file is collected last so that a failure here leaves every other test already run; it also
passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def oracle_u(w, alpha):
    import oracle
    import oracle.params as OP
    delta = OP.delta_from_mesh(alpha, w.h_vol)
    return oracle.direct_sum(alpha, delta, w.xs, w.ys, w.q, w.xt, w.yt)


def plan_u(w, alpha, args):
    import paper_2606_28865_b300 as yk
    # the static entry point builds the plain (untruncated) multiplier: compare like with like
    with yk.Plan(alpha, tol=TOL64, h_vol=w.h_vol, box=w.box, truncate=1) as plan:
        plan.set_points(args[0], args[1], args[2], args[4], args[5])
        return plan.eval(args[3]).cpu().numpy()


def test_static_entry_two_calls_match_oracle_and_plan_path():
    """A larger grid first (alpha = 0.5: 960^2 cells), then the 144^2 grid at alpha = 10: the second
    call must not see the first call's leftovers in the shared array.  Each call is checked against
    the FP64 oracle at the stated tolerance and against the plan path; no call allocates."""
    import paper_2606_28865_b300 as yk
    w = W.config_small()
    args = [dev(a) for a in (w.xs, w.ys, w.w, w.density, w.xt, w.yt)]
    cases = [(0.5, oracle_u(w, 0.5), plan_u(w, 0.5, args)),
             (w.alpha, oracle_u(w, w.alpha), plan_u(w, w.alpha, args))]
    outs = [torch.full((w.n_trg,), np.nan, dtype=torch.float64, device="cuda")
            for _ in range(len(cases) + 1)]
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    for (alpha, ref, via_plan), out in zip(cases, outs):
        yk.eval_longrange_static(alpha, *args, out, tol=TOL64, h_vol=w.h_vol, box=w.box)
        assert torch.cuda.memory_allocated() == before
        u = out.cpu().numpy()
        assert np.all(np.isfinite(u))
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(u - ref)) <= TOL64 * scale, alpha
        assert np.max(np.abs(u - via_plan)) <= TOL64 * scale, alpha
    # and once more in the first order, after the small grid
    out = outs[-1]
    yk.eval_longrange_static(0.5, *args, out, tol=TOL64, h_vol=w.h_vol, box=w.box)
    assert torch.cuda.memory_allocated() == before
    ref = cases[0][1]
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= TOL64 * np.max(np.abs(ref))


def test_static_entry_rejects_what_it_cannot_hold():
    import paper_2606_28865_b300 as yk
    w = W.config_small()
    out = torch.empty(w.n_trg, dtype=torch.float64, device="cuda")
    args = [dev(a) for a in (w.xs, w.ys, w.w, w.density, w.xt, w.yt)]
    # alpha = 1 with a tiny delta needs a grid far beyond 32 MiB
    with pytest.raises(yk.YkError) as ei:
        yk.eval_longrange_static(1.0, *args, out, tol=TOL64, delta=4e-5, box=w.box)
    assert ei.value.status == yk.YK_ERR_UNSUPPORTED and "static scratch" in str(ei.value)
    # host arrays would need staging copies, a strided output a temporary copy: both refused
    with pytest.raises(TypeError):
        yk.eval_longrange_static(w.alpha, w.xs, w.ys, w.w, w.density, w.xt, w.yt,
                                 np.empty(w.n_trg), tol=TOL64, h_vol=w.h_vol, box=w.box)
    strided = torch.empty(2 * w.n_trg, dtype=torch.float64, device="cuda")[::2]
    with pytest.raises(TypeError):
        yk.eval_longrange_static(w.alpha, *args, strided, tol=TOL64, h_vol=w.h_vol, box=w.box)
