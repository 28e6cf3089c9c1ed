"""GPU parity of the double-layer history part D_H (Section 2, eq. dlp; Section 5.1, D_H formula).

The CUDA path spreads each dipole with the gradient of the window onto the charges' grid; the
oracle sums F_D(r) (x - y) . (mu w nu) directly (FP64, Hankel-tabulated F_D).  Tolerance: relative
L-infinity error max_i |u - u_oracle| / max_i |u_oracle| <= tol (1e-10 FP64, 1e-6 FP32C).
"""
import numpy as np
import pytest

import oracle
import oracle.params as OP
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
    w = W.config_small()
    xd, yd, wd, nx, ny, mu = W.double_layer_nodes(W.Starfish(), 32)
    return w, (xd, yd, wd, nx, ny), mu


def run(work, dl, mu, alpha, tol=TOL64, charges=True, **opts):
    yk = _yk()
    opts.setdefault("h_vol", work.h_vol)
    plan = yk.Plan(alpha, tol=tol, box=work.box, dlp=True, **opts)
    e = np.zeros(0)
    xs, ys, w, dens = ((work.xs, work.ys, work.w, work.density) if charges else (e, e, e, e))
    plan.set_points(dev(xs), dev(ys), dev(w), dev(work.xt), dev(work.yt),
                    dipoles=tuple(dev(a) for a in dl))
    u = plan.eval(dev(dens), mu=dev(mu))
    plan.sync()
    info = plan.info
    out = u.cpu().numpy()
    plan.close()
    return out, info


def oracle_u(work, dl, mu, alpha, delta, charges=True):
    xd, yd, wd, nx, ny = dl
    u = oracle.direct_sum_dl(alpha, delta, xd, yd, mu * wd * nx, mu * wd * ny, work.xt, work.yt)
    if charges:
        u = u + oracle.direct_sum(alpha, delta, work.xs, work.ys, work.q, work.xt, work.yt)
    return u


@pytest.mark.parametrize("alpha", [10.0, 0.5, 200.0])
def test_double_layer_plus_charges_fp64(small, alpha):
    work, dl, mu = small
    u, info = run(work, dl, mu, alpha)
    ref = oracle_u(work, dl, mu, alpha, info["delta"])
    err = rel_err(u, ref)
    assert err <= TOL64, f"alpha={alpha} err={err:.3e}"


@pytest.mark.parametrize("alpha", [10.0, 0.5, 200.0])
def test_double_layer_alone_fp64(small, alpha):
    work, dl, mu = small
    u, info = run(work, dl, mu, alpha, charges=False)
    ref = oracle_u(work, dl, mu, alpha, info["delta"], charges=False)
    err = rel_err(u, ref)
    assert err <= TOL64, f"alpha={alpha} err={err:.3e}"


def test_double_layer_fixed_point_path(small):
    work, dl, mu = small
    u, info = run(work, dl, mu, 10.0, fft_fp64=True)
    ref = oracle_u(work, dl, mu, 10.0, info["delta"])
    assert rel_err(u, ref) <= TOL64


@pytest.mark.parametrize("alpha", [10.0, 0.5, 200.0])
def test_double_layer_fp32c(small, alpha):
    yk = _yk()
    work, dl, mu = small
    u, info = run(work, dl, mu, alpha, tol=TOL32, precision=yk.YK_FP32C)
    ref = oracle_u(work, dl, mu, alpha, info["delta"])
    err = rel_err(u, ref)
    assert err <= TOL32, f"alpha={alpha} err={err:.3e}"
    ref_d = oracle_u(work, dl, mu, alpha, info["delta"], charges=False)
    u_d, _ = run(work, dl, mu, alpha, tol=TOL32, precision=yk.YK_FP32C, charges=False)
    assert rel_err(u_d, ref_d) <= TOL32


def test_double_layer_discrete_formula(small):
    # explicit k_max and period: the GPU result reproduces the discrete Fourier formula with the
    # -i k . s dipole coefficient to the NUFFT accuracy
    work, dl, mu = small
    alpha = 10.0
    delta = OP.delta_from_mesh(alpha, work.h_vol)
    eps = TOL64 / 4
    kmax = max(OP.kmax_relative(alpha, delta, eps), OP.kmax_dlp_relative(alpha, delta, eps))
    period = 3.0 + OP.r_tol(alpha, delta, eps)
    M = OP.modes(kmax, period)
    u, info = run(work, dl, mu, alpha, delta=delta, kmax=kmax, period=period)
    assert info["n_modes"] == M
    xd, yd, wd, nx, ny = dl
    ref = oracle.discrete_sum(alpha, delta, period, M, (0.0, 0.0), work.xs, work.ys, work.q,
                              work.xt, work.yt, dipoles=(xd, yd, mu * wd * nx, mu * wd * ny))
    assert rel_err(u, ref) <= TOL64 / 4


def test_double_layer_linear_and_host_arrays(small):
    yk = _yk()
    work, dl, mu = small
    plan = yk.Plan(10.0, tol=TOL64, h_vol=work.h_vol, box=work.box, dlp=True)
    plan.set_points(work.xs, work.ys, work.w, work.xt, work.yt, dipoles=dl)   # host arrays
    u1 = plan.eval(work.density, mu=mu)
    u2 = plan.eval(work.density, mu=2 * mu)
    u0 = plan.eval(work.density, mu=np.zeros_like(mu))
    # D_H is linear in mu; with mu = 0 the plan gives the charges' potential (a plain plan's, up to
    # the tolerance: the double-layer plan uses one more digit of window)
    scale = np.max(np.abs(u1))
    assert np.max(np.abs((u2 - u0) - 2 * (u1 - u0))) <= 1e-13 * scale
    plain = yk.Plan(10.0, tol=TOL64, h_vol=work.h_vol, box=work.box)
    plain.set_points(work.xs, work.ys, work.w, work.xt, work.yt)
    u_plain = plain.eval(work.density)
    assert np.max(np.abs(u_plain - u0)) <= TOL64 * np.max(np.abs(u_plain))
    # device and host inputs give the same answer
    u_dev, _ = run(work, dl, mu, 10.0)
    assert np.max(np.abs(u_dev - u1)) <= 1e-13 * scale
    plan.close()
    plain.close()


def test_double_layer_permutation_invariance(small):
    work, dl, mu = small
    u, _ = run(work, dl, mu, 10.0)
    perm = np.random.default_rng(4).permutation(len(mu))
    dlp = tuple(a[perm] for a in dl)
    up, _ = run(work, dlp, mu[perm], 10.0)
    assert np.max(np.abs(u - up)) <= 1e-13 * np.max(np.abs(u))


def test_double_layer_argument_errors(small):
    yk = _yk()
    work, dl, mu = small
    plan = yk.Plan(10.0, tol=TOL64, h_vol=work.h_vol, box=work.box)   # no dlp
    with pytest.raises(yk.YkError) as ei:
        plan.set_points(work.xs, work.ys, work.w, work.xt, work.yt, dipoles=dl)
    assert ei.value.status == yk.YK_ERR_ARG
    plan.close()
    plan = yk.Plan(10.0, tol=TOL64, h_vol=work.h_vol, box=work.box, dlp=True)
    plan.set_points(dev(work.xs), dev(work.ys), dev(work.w), dev(work.xt), dev(work.yt),
                    dipoles=tuple(dev(a) for a in dl))
    with pytest.raises(yk.YkError) as ei:
        plan.eval(dev(work.density))                  # mu missing
    assert ei.value.status == yk.YK_ERR_ARG
    with pytest.raises(yk.YkError) as ei:
        yk.Batch([plan], use_graph=False)
    assert ei.value.status == yk.YK_ERR_UNSUPPORTED
    # a dipole outside the box is reported like any other point
    bad = tuple(np.array(a, copy=True) for a in dl)
    bad[0][3] = 5.0
    with pytest.raises(yk.YkError) as ei:
        plan.set_points(work.xs, work.ys, work.w, work.xt, work.yt, dipoles=bad)
    assert ei.value.status == yk.YK_ERR_ARG
    plan.close()


@pytest.mark.slow
def test_double_layer_large_sampled():
    # 1e5 boundary dipoles + 1.1e6 charges, 1e6 targets; oracle at 200 sampled targets
    alpha = 10.0
    work = W.config_large(alpha)
    dl_all = W.double_layer_nodes(W.Starfish(), 6250)
    dl, mu = dl_all[:5], dl_all[5]
    yk = _yk()
    plan = yk.Plan(alpha, tol=TOL64, h_vol=work.h_vol, box=work.box, dlp=True)
    plan.set_points(dev(work.xs), dev(work.ys), dev(work.w), dev(work.xt), dev(work.yt),
                    dipoles=tuple(dev(a) for a in dl))
    u = plan.eval(dev(work.density), mu=dev(mu)).cpu().numpy()
    delta = plan.info["delta"]
    plan.close()
    idx = np.random.default_rng(9).choice(work.n_trg, 200, replace=False)
    xd, yd, wd, nx, ny = dl
    ref = (oracle.direct_sum(alpha, delta, work.xs, work.ys, work.q, work.xt[idx], work.yt[idx])
           + oracle.direct_sum_dl(alpha, delta, xd, yd, mu * wd * nx, mu * wd * ny,
                                  work.xt[idx], work.yt[idx]))
    assert rel_err(u[idx], ref) <= TOL64
