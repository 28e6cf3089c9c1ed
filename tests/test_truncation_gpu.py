"""GPU parity of the truncated-kernel (small-alpha) path.

Every source-target distance is at most the box diagonal D, so the plan may evaluate
G_T = G_H chi (chi = 1 on r <= D, a smooth step to 0 on [D, D + 12 s]) instead of G_H, with a
period of span + D + 12 s instead of span + decay length, which at small alpha shrinks the grid
several-fold (the paper defers alpha -> 0 to the truncated-kernel method of Vico et al., Section
5.2).  The result must still be the untruncated potential: the same FP64 oracle and tolerances as
the plain path (relative L-infinity 1e-10 FP64, 1e-6 FP32C).
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-10, 1e-6


def _yk():
    import paper_2606_28865_b300 as yk
    return yk


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel_err(u, ref):
    return float(np.max(np.abs(u - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def small():
    return W.config_small()


def run(work, alpha, tol=TOL64, dipoles=None, mu=None, **opts):
    yk = _yk()
    opts.setdefault("h_vol", work.h_vol)
    plan = yk.Plan(alpha, tol=tol, box=work.box, **opts)
    plan.set_points(dev(work.xs), dev(work.ys), dev(work.w), dev(work.xt), dev(work.yt),
                    dipoles=None if dipoles is None else tuple(dev(a) for a in dipoles))
    u = plan.eval(dev(work.density), mu=None if mu is None else dev(mu))
    plan.sync()
    info = plan.info
    out = u.cpu().numpy()
    plan.close()
    return out, info


def ref_u(work, alpha, delta):
    return oracle.direct_sum(alpha, delta, work.xs, work.ys, work.q, work.xt, work.yt)


@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.2])
def test_truncated_small_alpha_fp64(small, alpha):
    u, info = run(small, alpha)
    assert info["truncated"] == 1
    err = rel_err(u, ref_u(small, alpha, info["delta"]))
    assert err <= TOL64, f"alpha={alpha} err={err:.3e} info={info}"


@pytest.mark.parametrize("alpha,delta", [(3.0, 1e-3), (1.0, 3.45e-5)])
def test_truncated_fine_delta(small, alpha, delta):
    # a small delta (fine volume mesh) makes k_max large and the transition narrow
    u, info = run(small, alpha, delta=delta)
    assert info["truncated"] == 1
    assert rel_err(u, ref_u(small, alpha, delta)) <= TOL64


@pytest.mark.parametrize("alpha", [10.0, 200.0])
def test_truncation_forced_at_large_alpha(small, alpha):
    u, info = run(small, alpha, truncate=2)
    assert info["truncated"] == 1
    assert rel_err(u, ref_u(small, alpha, info["delta"])) <= TOL64


def test_truncated_fixed_point_path(small):
    u, info = run(small, 1.0, fft_fp64=True)
    assert info["truncated"] == 1
    assert rel_err(u, ref_u(small, 1.0, info["delta"])) <= TOL64


@pytest.mark.parametrize("alpha,delta", [(1.0, 3.45e-5), (0.5, 1e-3), (0.2, None)])
def test_truncated_fp32c(small, alpha, delta):
    yk = _yk()
    kw = {} if delta is None else {"delta": delta}
    u, info = run(small, alpha, tol=TOL32, precision=yk.YK_FP32C, **kw)
    assert info["truncated"] == 1
    assert rel_err(u, ref_u(small, alpha, info["delta"])) <= TOL32


def test_truncated_and_plain_agree(small):
    # alpha = 3: both forms fit the grid limit; each meets the tolerance, so they agree within it
    ut, it = run(small, 3.0, delta=1e-3)
    up, ip = run(small, 3.0, delta=1e-3, truncate=1)
    assert it["truncated"] == 1 and ip["truncated"] == 0
    assert it["n_grid"] < ip["n_grid"]
    assert np.max(np.abs(ut - up)) <= 2 * TOL64 * np.max(np.abs(up))


def test_truncated_double_layer(small):
    xd, yd, wd, nx, ny, mu = W.double_layer_nodes(W.Starfish(), 32)
    u, info = run(small, 1.0, dipoles=(xd, yd, wd, nx, ny), mu=mu, dlp=True)
    assert info["truncated"] == 1
    ref = ref_u(small, 1.0, info["delta"]) + oracle.direct_sum_dl(
        1.0, info["delta"], xd, yd, mu * wd * nx, mu * wd * ny, small.xt, small.yt)
    assert rel_err(u, ref) <= TOL64


def test_truncated_corner_to_corner():
    # the farthest pair the box allows (opposite corners: distance exactly D, where chi is still 1)
    yk = _yk()
    alpha = 1.0
    xs, ys, w = np.array([-1.5]), np.array([-1.5]), np.array([1.0])
    xt, yt = np.array([1.5, 1.5, -1.5]), np.array([1.5, -1.5, -1.5])
    plan = yk.Plan(alpha, tol=TOL64, delta=1e-3, box=(-1.5, 1.5, -1.5, 1.5))
    plan.set_points(xs, ys, w, xt, yt)
    u = plan.eval(np.array([1.0]))
    info = plan.info
    plan.close()
    assert info["truncated"] == 1
    ref = oracle.direct_sum(alpha, 1e-3, xs, ys, w, xt, yt)
    assert np.max(np.abs(u - ref)) <= TOL64 * np.max(np.abs(ref))


def test_truncated_batch(small):
    # plans with the truncated multiplier run unchanged in the persistent batch kernel
    yk = _yk()
    plans, dens, outs, refs = [], [], [], []
    for alpha in (1.0, 0.5):
        p = yk.Plan(alpha, tol=TOL64, h_vol=small.h_vol, box=small.box)
        p.set_points(dev(small.xs), dev(small.ys), dev(small.w), dev(small.xt), dev(small.yt))
        plans.append(p)
        dens.append(dev(small.density))
        outs.append(torch.empty(small.n_trg, dtype=torch.float64, device="cuda"))
        refs.append(ref_u(small, alpha, p.info["delta"]))
    b = yk.Batch(plans, use_graph=True)
    b.run(dens, outs)
    b.sync()
    for o, r in zip(outs, refs):
        assert rel_err(o.cpu().numpy(), r) <= TOL64
    b.close()
    for p in plans:
        p.close()
