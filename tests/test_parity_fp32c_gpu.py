"""GPU parity of the FP32C path (FP32 spread/FFT/interpolation with two-sum grid accumulation and
FP64 final sums at the targets) against the FP64 CPU oracle, relative L-infinity <= 1e-6."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-6


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def run32(work, alpha, **opts):
    import paper_2606_28865_b300 as yk
    opts.setdefault("h_vol", work.h_vol)
    plan = yk.Plan(alpha, tol=TOL32, precision=yk.YK_FP32C, box=work.box, **opts)
    plan.set_points(dev(work.xs), dev(work.ys), dev(work.w), dev(work.xt), dev(work.yt))
    u = plan.eval(dev(work.density)).cpu().numpy()
    info = plan.info
    plan.close()
    return u, info


@pytest.fixture(scope="module")
def small():
    return W.config_small()


@pytest.mark.parametrize("alpha", [0.5, 10.0, 200.0])
def test_fp32c_config_small(small, alpha):
    u, info = run32(small, alpha)
    assert info["precision"] == 1 and info["w"] == 8
    ref = oracle.direct_sum(alpha, info["delta"], small.xs, small.ys, small.q, small.xt, small.yt)
    err = float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))
    print(f"FP32C alpha={alpha}: relative Linf error vs FP64 oracle = {err:.3e}")
    assert err <= TOL32, f"alpha={alpha} err={err:.3e} info={info}"


def test_fp32c_rothe_reuse_and_edges(small):
    import paper_2606_28865_b300 as yk
    plan = yk.Plan(10.0, tol=TOL32, precision=yk.YK_FP32C, h_vol=small.h_vol, box=small.box)
    plan.set_points(dev(small.xs), dev(small.ys), dev(small.w), dev(small.xt), dev(small.yt))
    u1 = plan.eval(dev(small.density)).cpu().numpy()
    d2 = W.strengths_for(small, 10.0, seed=5)
    u2 = plan.eval(dev(d2)).cpu().numpy()
    ref2 = oracle.direct_sum(10.0, plan.info["delta"], small.xs, small.ys, small.w * d2,
                             small.xt, small.yt)
    assert np.max(np.abs(u2 - ref2)) <= TOL32 * np.max(np.abs(ref2))
    u3 = plan.eval(dev(small.density)).cpu().numpy()
    assert np.max(np.abs(u3 - u1)) <= 1e-12 * np.max(np.abs(u1))
    # no sources -> zeros
    plan.set_points(dev([]), dev([]), dev([]), dev(small.xt[:7]), dev(small.yt[:7]))
    assert np.all(plan.eval(dev([])).cpu().numpy() == 0.0)
    plan.close()


@pytest.mark.parametrize("alpha", [10.0, 100.0, 1.0])
def test_fp32c_config_large_sampled(alpha):
    work = W.config_large(alpha)
    u, info = run32(work, alpha)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(work.n_trg, 1000, replace=False))
    ref = oracle.direct_sum(alpha, info["delta"], work.xs, work.ys, work.q, work.xt[idx],
                            work.yt[idx])
    err = float(np.max(np.abs(u[idx] - ref)) / np.max(np.abs(ref)))
    print(f"FP32C large alpha={alpha}: relative Linf error = {err:.3e}")
    assert err <= TOL32, f"alpha={alpha} err={err:.3e} info={info}"
