"""Pins of the oracle's double-layer history part (no GPU needed).

D_H[mu](x) = sum_d mu_d w_d nu_d . grad_y G_H(x - y_d) (Section 2, eq. dlp, with the split of
Section 2.1; Section 5.1, the D_H formula).  The oracle writes it as F_D(r) (x - y) . s with
F_D = -G_H'/r from a J1 Hankel quadrature.  Each check is independent of that arithmetic:
closed forms (E2 at r = 0, the Bessel K1 far field of Section 3's matrix entries), the
t-integral definition by scipy, a centred difference of the single-layer kernel in the source
point (fixes the sign and orientation), and Poisson summation against the discrete Fourier formula
(fixes the sign of the i k factor).
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle as O
import oracle.params as OP
import workloads as W

CASES = [(10.0, 0.0167), (10.0, 3.93e-5), (1.0, 3.93e-5), (100.0, 3.82e-5), (0.5, 0.019),
         (200.0, 3.4e-4)]


def fd_tquad(alpha, delta, r):
    """int_delta^inf exp(-r^2/(4t) - alpha^2 t) / (8 pi t^2) dt by scipy with t = delta e^s."""
    f = lambda s: (math.exp(-r * r / (4 * delta * math.exp(s)) - alpha ** 2 * delta * math.exp(s))
                   / (8 * math.pi * delta * math.exp(s)))
    return si.quad(f, 0.0, 80.0, epsabs=0.0, epsrel=1e-13, limit=500)[0]


def gh_tquad(alpha, delta, r):
    f = lambda s: math.exp(-r * r / (4 * delta * math.exp(s)) - alpha ** 2 * delta * math.exp(s)) / (4 * math.pi)
    return si.quad(f, 0.0, 80.0, epsabs=0.0, epsrel=1e-13, limit=500)[0]


@pytest.mark.parametrize("alpha,delta", CASES)
def test_dl_origin_closed_form(alpha, delta):
    # F_D(0) = int_delta^inf e^{-alpha^2 t} / (8 pi t^2) dt = E2(alpha^2 delta) / (8 pi delta)
    f0 = sp.expn(2, alpha * alpha * delta) / (8 * math.pi * delta)
    T = O.FDTable(alpha, delta, 4.3)
    assert abs(T(0.0)[0] - f0) <= 1e-13 * f0
    assert abs(O.fd_hankel(alpha, delta, [0.0])[0] - f0) <= 1e-13 * f0


@pytest.mark.parametrize("alpha,delta", CASES)
def test_dl_far_field_bessel(alpha, delta):
    # beyond r = 12 sqrt(delta) the local part int_0^delta is below e^{-36} of it, so F_D equals
    # the full kernel's alpha K1(alpha r) / (2 pi r) (Section 3, the double-layer matrix entries)
    T = O.FDTable(alpha, delta, 4.3)
    for r in [12 * math.sqrt(delta), 0.3, 1.0, 2.5]:
        if r < 12 * math.sqrt(delta) or alpha * r > 600:
            continue
        ref = alpha * sp.k1(alpha * r) / (2 * math.pi * r)
        assert abs(T(r)[0] - ref) <= 1e-12 * ref + 1e-14 * T.g0, (r, T(r)[0], ref)


def test_dl_table_against_time_integral():
    for alpha, delta in CASES:
        T = O.FDTable(alpha, delta, 4.3)
        for r in [0.0, 0.5 * math.sqrt(delta), 3 * math.sqrt(delta), 0.2, 1.0]:
            ref = fd_tquad(alpha, delta, r)
            assert abs(T(r)[0] - ref) <= 1e-13 * T.g0, (alpha, delta, r)


@pytest.mark.parametrize("alpha,delta", CASES[:4])
def test_dl_is_minus_radial_derivative_over_r(alpha, delta):
    # F_D(r) r = -G_H'(r): 5-point centred difference of the single-layer table
    s = math.sqrt(delta)
    G = O.GHTable(alpha, delta, 4.3)
    F = O.FDTable(alpha, delta, 4.3)
    for r in [0.5 * s, 2 * s, 5 * s]:
        h = s / 50
        g = G(np.array([r - 2 * h, r - h, r + h, r + 2 * h]))
        d1 = (g[0] - 8 * g[1] + 8 * g[2] - g[3]) / (12 * h)
        assert abs(F(r)[0] * r + d1) <= 1e-7 * F.g0 * s, (r, F(r)[0] * r, -d1)


def test_dl_brute_force_tiny_sign_and_orientation():
    # nu . grad_y G_H(x - y) by a centred difference of the t-quadrature kernel in the source point
    rng = np.random.default_rng(17)
    alpha, delta = 10.0, 0.0167
    n, m = 8, 6
    xd, yd = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    th = rng.uniform(0, 2 * math.pi, n)
    nx, ny = np.cos(th), np.sin(th)
    mw = rng.normal(size=n)
    xt, yt = rng.uniform(-1.5, 1.5, m), rng.uniform(-1.5, 1.5, m)
    u = O.direct_sum_dl(alpha, delta, xd, yd, mw * nx, mw * ny, xt, yt)
    h = 1e-4
    ref = np.zeros(m)
    for i in range(m):
        for j in range(n):
            gp = gh_tquad(alpha, delta, math.hypot(xt[i] - xd[j] - h * nx[j], yt[i] - yd[j] - h * ny[j]))
            gm = gh_tquad(alpha, delta, math.hypot(xt[i] - xd[j] + h * nx[j], yt[i] - yd[j] + h * ny[j]))
            ref[i] += mw[j] * (gp - gm) / (2 * h)
    scale = np.abs(mw).sum() * O.FDTable(alpha, delta, 4.3).g0 * 0.1
    assert np.max(np.abs(u - ref)) <= 1e-7 * scale, (u, ref)


def test_dl_discrete_sum_is_periodic_image_sum():
    # Poisson summation for dipoles: the discrete formula with the -i k . s factor equals the
    # periodised double-layer kernel; a flipped sign of k fails by O(1)
    alpha, delta, P, M = 10.0, 0.0167, 1.0, 15
    rng = np.random.default_rng(19)
    n = 5
    xd, yd = rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n)
    sx, sy = rng.normal(size=n), rng.normal(size=n)
    xt, yt = rng.uniform(-0.5, 0.5, 7), rng.uniform(-0.5, 0.5, 7)
    z = np.zeros(0)
    u = O.discrete_sum(alpha, delta, P, M, (0.1, -0.2), z, z, z, xt, yt, dipoles=(xd, yd, sx, sy))
    T = O.FDTable(alpha, delta, 6.0)
    ref = np.zeros(7)
    for kx in range(-3, 4):
        for ky in range(-3, 4):
            ref += O.direct_sum_dl(alpha, delta, xd + kx * P, yd + ky * P, sx, sy, xt, yt, table=T)
    scale = np.hypot(sx, sy).sum() * T.g0 * math.sqrt(delta)
    assert np.max(np.abs(u - ref)) <= 1e-11 * scale, np.abs(u - ref).max() / scale
    flipped = O.discrete_sum(alpha, delta, P, M, (0.1, -0.2), z, z, z, xt, yt,
                             dipoles=(xd, yd, -sx, -sy))
    assert np.max(np.abs(flipped + u)) <= 1e-12 * scale


def test_dl_linear_and_charges_add():
    rng = np.random.default_rng(23)
    alpha, delta, P, M = 10.0, 0.0167, 5.7, 33
    xs, ys, q = rng.uniform(-1, 1, 10), rng.uniform(-1, 1, 10), rng.normal(size=10)
    xd, yd = rng.uniform(-1, 1, 6), rng.uniform(-1, 1, 6)
    sx, sy = rng.normal(size=6), rng.normal(size=6)
    xt, yt = rng.uniform(-1.5, 1.5, 9), rng.uniform(-1.5, 1.5, 9)
    both = O.discrete_sum(alpha, delta, P, M, (0, 0), xs, ys, q, xt, yt, dipoles=(xd, yd, sx, sy))
    z = np.zeros(0)
    only_q = O.discrete_sum(alpha, delta, P, M, (0, 0), xs, ys, q, xt, yt)
    only_d = O.discrete_sum(alpha, delta, P, M, (0, 0), z, z, z, xt, yt, dipoles=(xd, yd, sx, sy))
    assert np.max(np.abs(both - only_q - only_d)) <= 1e-13 * (np.abs(only_q).max() + np.abs(only_d).max())


def test_kmax_dlp_rules():
    for alpha, delta in CASES[:4]:
        eps = 2.5e-11
        k = OP.kmax_dlp_paper(alpha, delta, eps)
        # eq. kmax_dlp holds with equality at k and is stricter than eq. kmax
        assert abs(k * math.exp(-delta * (alpha ** 2 + k * k)) - eps) <= 1e-9 * eps
        assert k >= OP.kmax_paper(alpha, delta, eps)
        kr = OP.kmax_dlp_relative(alpha, delta, eps)
        assert kr >= OP.kmax_relative(alpha, delta, eps)
        # the relative tail by an independent closed form: int_k^inf e^{-d s^2} ds minus alpha^2
        # times int_k^inf e^{-d s^2} / (alpha^2 + s^2) ds (the latter by a separate quadrature)
        g1 = lambda kk: 0.5 * math.sqrt(math.pi / delta) * sp.erfc(math.sqrt(delta) * kk)
        g2 = lambda kk: si.quad(lambda s: math.exp(-delta * s * s) / (alpha ** 2 + s * s), kk,
                                kk + 40 / math.sqrt(delta), epsabs=0, epsrel=1e-13, limit=400)[0]
        tail = lambda kk: g1(kk) - alpha ** 2 * g2(kk)
        assert abs(tail(kr) - eps * tail(0.0)) <= 1e-5 * eps * tail(0.0)
    # the regime where eq. kmax_dlp needs no modes at all
    alpha = 200.0
    delta = math.log(1 / 1e-6) / alpha ** 2 * 2
    assert OP.kmax_dlp_paper(alpha, delta, 1e-6) == 0.0


def test_double_layer_nodes_geometry():
    c = W.Starfish()
    x, y, w, nx, ny, mu = W.double_layer_nodes(c, 32)
    assert np.allclose(np.hypot(nx, ny), 1.0, atol=1e-15)
    # divergence theorem: int nu . x ds = 2 area; int nu ds = 0
    assert abs(np.sum(w * (nx * x + ny * y)) - 2 * c.area()) <= 1e-11
    assert abs(np.sum(w * nx)) <= 1e-12 and abs(np.sum(w * ny)) <= 1e-12
    # outward: a step along nu leaves the domain
    assert not np.any(c.inside(x + 1e-3 * nx, y + 1e-3 * ny))
    assert np.all(c.inside(x - 1e-3 * nx, y - 1e-3 * ny))
