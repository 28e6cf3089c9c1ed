"""Allocator failures through the plan's allocator callback (yk_opts.alloc returning NULL).

The failure is made on the host: a callback that refuses the k-th request.  Every refusal must
surface as YK_ERR_OOM from the call that needed the memory, leak nothing (every buffer the
callback handed out comes back through the free callback once the plan is destroyed), and leave
the plan usable where it exists: set_points can be repeated and the results are the same."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class CountingAllocator:
    """Device buffers from torch's caching allocator; refuses request number `fail_at`."""

    def __init__(self, fail_at=None):
        self.calls = 0
        self.fail_at = fail_at
        self.live = {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.calls == self.fail_at:
            return 0
        t = torch.empty(max(1, nbytes), dtype=torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr, stream):
        del self.live[ptr]


def run(yk, w, args, allocator):
    """plan + set_points + eval with the given allocator; returns (u or None, plan or None, err)."""
    try:
        plan = yk.Plan(w.alpha, tol=1e-10, h_vol=w.h_vol, box=w.box, allocator=allocator)
    except yk.YkError as e:
        return None, None, e
    try:
        plan.set_points(args[0], args[1], args[2], args[4], args[5])
        u = plan.eval(args[3])
        return u.cpu().numpy(), plan, None
    except yk.YkError as e:
        return None, plan, e


def test_refused_allocations_give_oom_leak_nothing_and_leave_the_plan_usable():
    import paper_2606_28865_b300 as yk
    w = W.config_small()
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    args = [dev(a) for a in (w.xs, w.ys, w.w, w.density, w.xt, w.yt)]
    full = CountingAllocator()
    ref, plan, err = run(yk, w, args, full)
    assert err is None and full.calls >= 3
    plan.close()
    assert not full.live
    n_calls = full.calls
    for k in sorted({1, 2, n_calls // 2, n_calls - 1, n_calls}):
        a = CountingAllocator(fail_at=k)
        u, plan, err = run(yk, w, args, a)
        assert err is not None and err.status == yk.YK_ERR_OOM, k
        if plan is not None:
            # the refusal came after the plan existed: the same calls again succeed
            plan.set_points(args[0], args[1], args[2], args[4], args[5])
            u = plan.eval(args[3]).cpu().numpy()
            # a new binning may order a tile's sources differently: rounding-level agreement
            assert np.max(np.abs(u - ref)) <= 1e-13 * np.max(np.abs(ref)), k
            plan.close()
        assert not a.live, (k, len(a.live))
