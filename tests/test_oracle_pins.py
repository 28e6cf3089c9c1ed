"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Every check here is independent of the oracle's own arithmetic: closed forms, identities
evaluated with separate library routines (scipy), brute force by a different quadrature, and the
worked example printed in Section 6.4.  A dropped factor, a wrong sign or a transposed operand
in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle as O
import oracle.params as OP
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

CASES = [(10.0, 0.0167), (10.0, 3.93e-5), (1.0, 3.93e-5), (100.0, 3.82e-5), (0.5, 0.019),
         (200.0, 3.4e-4)]


def g_r_tquad(alpha, delta, r):
    """int_0^delta H(t, r) dt by scipy quad with t = delta e^{-s} (Section 2.1, eq. equiv_split)."""
    f = lambda s: math.exp(-r * r / (4 * delta * math.exp(-s)) - alpha ** 2 * delta * math.exp(-s)) / (4 * math.pi)
    return si.quad(f, 0.0, 60.0, epsabs=0.0, epsrel=1e-13, limit=500)[0]


def g_h_tquad(alpha, delta, r):
    """int_delta^inf H(t, r) dt by scipy quad with t = delta e^{s} (Section 2.1, eq. sl_sh)."""
    f = lambda s: math.exp(-r * r / (4 * delta * math.exp(s)) - alpha ** 2 * delta * math.exp(s)) / (4 * math.pi)
    return si.quad(f, 0.0, 80.0, epsabs=0.0, epsrel=1e-13, limit=500)[0]


@pytest.mark.parametrize("alpha,delta", CASES)
def test_p1_origin_closed_form(alpha, delta):
    # G_H(0) = int_delta^inf e^{-alpha^2 t}/(4 pi t) dt = E1(alpha^2 delta) / (4 pi)
    g0 = sp.exp1(alpha * alpha * delta) / (4 * math.pi)
    T = O.GHTable(alpha, delta, 4.3)
    assert abs(T(0.0)[0] - g0) <= 1e-14 * g0
    assert abs(O.gh_hankel(alpha, delta, [0.0])[0] - g0) <= 1e-14 * g0


@pytest.mark.parametrize("alpha,delta", CASES)
def test_p2_split_identity(alpha, delta):
    # G_H + G^R = K0(alpha r)/(2 pi)  (Section 1 eq. Greens, Section 2.1 eqs. ker_greens, equiv_split)
    T = O.GHTable(alpha, delta, 4.3)
    g0 = T.g0
    for r in [1e-3, 0.01, 0.05, 0.1, 0.3, 1.0, 2.0]:
        k0 = sp.k0(alpha * r) / (2 * math.pi)
        gr = g_r_tquad(alpha, delta, r)
        resid = abs(T(r)[0] + gr - k0)
        # K0 and G^R are each accurate to ~1e-16 of themselves; they can be much larger than G_H
        assert resid <= 1e-13 * max(g0, k0, gr), (r, resid)


@pytest.mark.parametrize("alpha,delta", CASES[:4])
def test_p3_heat_kernel_at_delta(alpha, delta):
    # d G_H / d delta = -H(delta, r)  and  (-Lap + alpha^2) G_H = H(delta, r)
    # (Section 2.1 eq. H_ker; Section 5.1: the symbol e^{-delta(alpha^2+k^2)}/(alpha^2+k^2))
    s = math.sqrt(delta)
    for r in [0.3 * s, 1.0 * s, 2.0 * s, 4.0 * s]:
        H = math.exp(-r * r / (4 * delta) - alpha * alpha * delta) / (4 * math.pi * delta)
        # Richardson-extrapolated centred difference in delta
        def d_delta(e):
            return (O.gh_hankel(alpha, delta * (1 + e), [r])[0]
                    - O.gh_hankel(alpha, delta * (1 - e), [r])[0]) / (2 * e * delta)
        dd = (4 * d_delta(1e-3) - d_delta(2e-3)) / 3
        assert abs(dd + H) <= 1e-6 * H, (r, dd, H)
        # radial Laplacian G'' + G'/r by centred differences of the table, step h = s/50
        T = O.GHTable(alpha, delta, r + s)
        h = s / 50
        g = T(np.array([r - 2 * h, r - h, r, r + h, r + 2 * h]))
        d1 = (g[0] - 8 * g[1] + 8 * g[3] - g[4]) / (12 * h)
        d2 = (-g[0] + 16 * g[1] - 30 * g[2] + 16 * g[3] - g[4]) / (12 * h * h)
        lhs = -(d2 + d1 / r) + alpha * alpha * g[2]
        assert abs(lhs - H) <= 2e-6 * H, (r, lhs, H)


@pytest.mark.parametrize("alpha,delta", CASES)
def test_table_matches_direct_quadrature(alpha, delta):
    rng = np.random.default_rng(1)
    r = np.sort(rng.uniform(0, 4.3, 200))
    T = O.GHTable(alpha, delta, 4.3)
    assert np.max(np.abs(T(r) - O.gh_hankel(alpha, delta, r))) <= 1e-14 * T.g0


def test_table_against_time_integral():
    # an independent definition of the same kernel: the t-integral (Section 2.1, eq. sl_sh)
    for alpha, delta in CASES:
        T = O.GHTable(alpha, delta, 4.3)
        for r in [0.0, 0.5 * math.sqrt(delta), 3 * math.sqrt(delta), 0.2, 1.0]:
            ref = g_h_tquad(alpha, delta, r)
            assert abs(T(r)[0] - ref) <= 1e-13 * T.g0, (alpha, delta, r)


def test_p7_brute_force_tiny():
    # direct sum vs per-pair t-quadrature (scipy), tiny inputs
    rng = np.random.default_rng(7)
    alpha, delta = 10.0, 0.0167
    xs, ys = rng.uniform(-1, 1, 12), rng.uniform(-1, 1, 12)
    q = rng.normal(size=12)
    xt, yt = rng.uniform(-1.5, 1.5, 9), rng.uniform(-1.5, 1.5, 9)
    u = O.direct_sum(alpha, delta, xs, ys, q, xt, yt)
    ref = np.array([sum(q[j] * g_h_tquad(alpha, delta, math.hypot(xt[i] - xs[j], yt[i] - ys[j]))
                        for j in range(12)) for i in range(9)])
    scale = np.abs(q).sum() * sp.exp1(alpha ** 2 * delta) / (4 * math.pi)
    assert np.max(np.abs(u - ref)) <= 1e-13 * scale


def test_direct_sum_conditioning_output_and_linearity():
    rng = np.random.default_rng(3)
    alpha, delta = 10.0, 0.0167
    xs, ys = rng.uniform(-1, 1, 50), rng.uniform(-1, 1, 50)
    q1, q2 = rng.normal(size=50), rng.normal(size=50)
    xt, yt = rng.uniform(-1.5, 1.5, 20), rng.uniform(-1.5, 1.5, 20)
    u1, a1 = O.direct_sum(alpha, delta, xs, ys, q1, xt, yt, return_abs=True)
    u2 = O.direct_sum(alpha, delta, xs, ys, q2, xt, yt)
    u12 = O.direct_sum(alpha, delta, xs, ys, 2 * q1 - 3 * q2, xt, yt)
    assert np.allclose(u12, 2 * u1 - 3 * u2, rtol=0, atol=1e-14 * np.abs(a1).max() * 10)
    ua = O.direct_sum(alpha, delta, xs, ys, np.abs(q1), xt, yt)
    assert np.allclose(a1, ua, rtol=1e-14, atol=0)
    # swapping the roles of a single source and target leaves G_H unchanged (symmetry in r)
    v = O.direct_sum(alpha, delta, xt[:1], yt[:1], [1.0], xs[:1], ys[:1])
    w = O.direct_sum(alpha, delta, xs[:1], ys[:1], [1.0], xt[:1], yt[:1])
    assert abs(v[0] - w[0]) <= 1e-15 * abs(v[0]) + 1e-300


@pytest.mark.parametrize("alpha,delta", [(10.0, 0.0167), (30.0, 0.002)])
def test_p4_gaussian_source(alpha, delta):
    # f = exp(-|x|^2/a): heat kernel convolved with f is e^{-alpha^2 t} a/(a+4t) e^{-|x|^2/(a+4t)},
    # so V_H[f](x) = int_delta^inf e^{-alpha^2 t} a/(a+4t) e^{-|x|^2/(a+4t)} dt, and at x = 0
    # V_H[f](0) = (a/4) e^{alpha^2 a/4} E1(alpha^2 (a + 4 delta)/4).
    a = 0.1
    xi, wi = np.polynomial.legendre.leggauss(160)
    xi, wi = 2.0 * xi, 2.0 * wi           # [-2, 2]; f < e^{-40} outside
    X, Y = np.meshgrid(xi, xi)
    WW = np.outer(wi, wi)
    q = (np.exp(-(X ** 2 + Y ** 2) / a) * WW).ravel()
    xt = np.array([0.0, 0.05, 0.2, 0.37, 0.8])
    yt = np.array([0.0, -0.1, 0.1, 0.4, -0.3])
    u = O.direct_sum(alpha, delta, X.ravel(), Y.ravel(), q, xt, yt)
    ref = []
    for x, y in zip(xt, yt):
        r2 = x * x + y * y
        f = lambda s: math.exp(-alpha ** 2 * delta * math.exp(s)) * a / (a + 4 * delta * math.exp(s)) \
            * math.exp(-r2 / (a + 4 * delta * math.exp(s))) * delta * math.exp(s)
        ref.append(si.quad(f, 0.0, 60.0, epsabs=0, epsrel=1e-13, limit=500)[0])
    ref = np.array(ref)
    closed0 = a / 4 * math.exp(alpha ** 2 * a / 4) * sp.exp1(alpha ** 2 * (a + 4 * delta) / 4)
    assert abs(ref[0] - closed0) <= 1e-12 * closed0
    assert np.max(np.abs(u - ref)) <= 1e-11 * closed0, np.abs(u - ref)


def _ring_hankel(alpha, delta, n, R, r):
    """R int_0^inf e^{-delta(alpha^2+k^2)}/(alpha^2+k^2) J_n(kR) J_n(kr) k dk (GL panels, numpy)."""
    kc = math.sqrt(45.0 / delta)
    L = min(math.pi / max(R, r, 1e-3), 1.0 / math.sqrt(delta), alpha)
    npan = int(math.ceil(kc / L))
    xg, wg = np.polynomial.legendre.leggauss(30)
    a = np.arange(npan) * L
    k = (a[:, None] + 0.5 * L * (xg[None, :] + 1)).ravel()
    w = (0.5 * L * np.broadcast_to(wg, (npan, 30))).ravel()
    s = alpha ** 2 + k ** 2
    return R * np.sum(w * np.exp(-delta * s) / s * sp.jv(n, k * R) * sp.jv(n, k * r) * k)


@pytest.mark.parametrize("nmode", [0, 3])
def test_p5_circle_single_layer(nmode):
    # ring of radius R, density cos(n theta): S_H = R cos(n theta) int Ghat J_n(kR) J_n(kr) k dk
    alpha, delta, R = 10.0, 0.0167, 1.0
    N = 512
    th = 2 * math.pi * np.arange(N) / N
    xs, ys = R * np.cos(th), R * np.sin(th)
    q = np.cos(nmode * th) * (2 * math.pi * R / N)
    rt = np.array([0.0, 0.4, 0.9, 1.1, 1.6])
    tt = np.array([0.3, 1.0, 2.0, 4.0, 5.5])
    u = O.direct_sum(alpha, delta, xs, ys, q, rt * np.cos(tt), rt * np.sin(tt))
    ref = np.array([math.cos(nmode * t) * _ring_hankel(alpha, delta, nmode, R, r) for r, t in zip(rt, tt)])
    scale = np.abs(q).sum() * sp.exp1(alpha ** 2 * delta) / (4 * math.pi)
    assert np.max(np.abs(u - ref)) <= 1e-12 * scale, np.abs(u - ref)


def test_p8_discrete_sum_is_periodic_image_sum():
    # Poisson summation: (1/P^2) sum_{m in Z^2} Ghat(2 pi m / P) e^{i k_m . r} = sum_n G_H(r + n P).
    # With M large enough the paper's discrete formula equals the periodised kernel.
    alpha, delta, P = 10.0, 0.0167, 1.0
    M = 14
    rng = np.random.default_rng(5)
    xs, ys, q = rng.uniform(-0.4, 0.4, 5), rng.uniform(-0.4, 0.4, 5), rng.normal(size=5)
    xt, yt = rng.uniform(-0.5, 0.5, 7), rng.uniform(-0.5, 0.5, 7)
    u = O.discrete_sum(alpha, delta, P, M, (0.1, -0.2), xs, ys, q, xt, yt)
    T = O.GHTable(alpha, delta, 6.0)
    ref = np.zeros(7)
    for nx in range(-3, 4):
        for ny in range(-3, 4):
            ref += O.direct_sum(alpha, delta, xs + nx * P, ys + ny * P, q, xt, yt, table=T)
    scale = np.abs(q).sum() * T.g0
    assert np.max(np.abs(u - ref)) <= 1e-12 * scale, np.abs(u - ref).max() / scale
    # the images matter at this period: dropping them changes the answer well above tolerance
    direct = O.direct_sum(alpha, delta, xs, ys, q, xt, yt, table=T)
    assert np.max(np.abs(direct - ref)) > 1e-7 * scale


def test_p8_discrete_sum_shift_invariance():
    alpha, delta, P, M = 10.0, 0.0167, 5.7, 33
    rng = np.random.default_rng(11)
    xs, ys, q = rng.uniform(-1, 1, 30), rng.uniform(-1, 1, 30), rng.normal(size=30)
    xt, yt = rng.uniform(-1.5, 1.5, 10), rng.uniform(-1.5, 1.5, 10)
    u1 = O.discrete_sum(alpha, delta, P, M, (0.0, 0.0), xs, ys, q, xt, yt)
    u2 = O.discrete_sum(alpha, delta, P, M, (0.7, -0.3), xs, ys, q, xt, yt)
    assert np.max(np.abs(u1 - u2)) <= 1e-12 * np.abs(q).sum()


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_p9_parameter_worked_example():
    g = _golden("section6_4_parameters.txt")
    # eq. kmax solved for delta with k_max = 1141 reproduces the printed delta and delta*
    dx = 0.9 * math.pi / g["kmax"]
    delta = OP.delta_from_mesh(g["alpha"], dx, g["eps"])
    assert float(f"{delta:.3g}") == g["delta"]
    assert float(f"{delta / 4 ** g['J']:.3g}") == g["delta_star"]
    # and eq. kmax at the printed (rounded) delta gives back k_max within the rounding of delta
    k = OP.kmax_paper(g["alpha"], g["delta"], g["eps"])
    assert abs(k - g["kmax"]) <= 0.005 * g["kmax"]


def test_p9_kmax_zero_regime():
    # delta alpha^2 >= ln(1/eps) -> k_max = 0 and the history part is already below eps
    alpha, eps = 200.0, 1e-6
    delta = math.log(1 / eps) / alpha ** 2 * 1.01
    assert OP.kmax_paper(alpha, delta, eps) == 0.0
    g0 = O.gh_hankel(alpha, delta, [0.0])[0]
    assert g0 * 4 * math.pi <= eps   # E1(x) < e^{-x} for x > 1


def test_kmax_relative_tail():
    # the radial Fourier tail beyond k_max equals eps * G_H(0) (independent scipy quadrature)
    for alpha, delta in CASES[:4]:
        eps = 2.5e-11
        k = OP.kmax_relative(alpha, delta, eps)
        tail = si.quad(lambda kk: math.exp(-delta * (alpha ** 2 + kk * kk)) / (alpha ** 2 + kk * kk) * kk / (2 * math.pi),
                       k, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
        g0 = sp.exp1(alpha ** 2 * delta) / (4 * math.pi)
        assert abs(tail - eps * g0) <= 1e-6 * eps * g0


def test_r_tol():
    alpha, delta, eps = 10.0, 0.0167, 2.5e-11
    r = OP.r_tol(alpha, delta, eps)
    g = O.gh_hankel(alpha, delta, [0.0, r * (1 - 1e-6), r, 1.2 * r])
    # quadrature noise is ~1e-17 G_H(0), i.e. ~1e-6 of eps G_H(0) at this radius
    assert g[1] >= eps * g[0] * (1 - 1e-4) and g[2] <= eps * g[0] * (1 + 1e-4)
    assert g[3] < g[2]


def test_workload_generators():
    w = W.config_small()
    assert w.n_bdry == 512 and w.n_trg == 2048
    assert 2048 <= w.n_src - w.n_bdry <= 2200
    c = W.Starfish()
    # boundary weights integrate arc length, volume weights integrate area
    assert abs(w.w[:512].sum() - W._perimeter(c, 1 << 16)) <= 1e-10
    # straight chords in cut cells drop the curved caps: O(perimeter dx^2) of area
    assert abs(w.w[512:].sum() - c.area()) <= 1e-2
    assert np.all(np.abs(w.xt) <= 1.5) and np.all(np.abs(w.yt) <= 1.5)
    w2 = W.config_small()
    assert np.array_equal(w.xt, w2.xt) and np.array_equal(w.density, w2.density)
