"""Pins of the oracle's double-layer local asymptotic part D_{L,A} (Section 4.1, the double-layer
lemma, eq. dlp_local1, and its corollary, eq. dlp_local2; definition eq. dla).  Independent of the
oracle's arithmetic: the exact values for a straight boundary with a quartic density (the integral
over the boundary in closed form, then 1-D scipy quadrature in t, for which the lemma through
delta*^2 is exact), the exact values for a circle and for the starfish by 2-D Gauss-Legendre
quadrature of eq. dla (the lemma converges at its order, delta*^{5/2}: this fixes the overall sign
and the gamma'''' term's factor, see oracle/local.py), the double layer's jump
across the boundary, the corollary for boundary targets and the locality remark.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si

import oracle.local as OL

_GU = np.polynomial.legendre.leggauss(300)   # outer rule, in u = log t
_GS = np.polynomial.legendre.leggauss(96)    # inner rule, along the boundary


def dla_quadrature(alpha, ds, x, y, curve, s0):
    """eq. dla with the normal derivative in the source point,
    int_0^ds int mu(s) nu(s).(x - gamma(s)) e^{-alpha^2 t - |x - gamma(s)|^2/(4t)} / (8 pi t^2)
    |gamma'(s)| ds dt, by Gauss-Legendre in u = log t on [log ds - 30, log ds] (targets at least
    0.5 sqrt(ds) from the boundary, so smaller t contribute below e^{-1e11}) and, for each t, in the
    curve parameter over s0 +- 16 sqrt(t) / |gamma'(s0)| (the kernel's Gaussian factor is e^{-64}
    at the ends).  curve(s) -> (gx, gy, dgx, dgy, mu) with the outward normal (dgy, -dgx)/|dg|."""
    xu, wu = _GU
    xs, ws = _GS
    lo, hi = math.log(ds) - 30.0, math.log(ds)
    u = 0.5 * (hi - lo) * xu + 0.5 * (hi + lo)
    t = np.exp(u)
    wt = 0.5 * (hi - lo) * wu * t                       # dt = t du
    _, _, d0x, d0y, _ = curve(np.array([s0]))
    L = 16.0 * np.sqrt(t) / math.hypot(d0x[0], d0y[0])
    s = s0 + L[:, None] * xs[None, :]
    gx, gy, dx, dy, mu = curve(s)
    ex, ey = x - gx, y - gy
    nrm = np.hypot(dx, dy)
    kern = (mu * (dy * ex - dx * ey) * np.exp(-alpha * alpha * t[:, None]
                                               - (ex * ex + ey * ey) / (4 * t[:, None]))
            / (8 * math.pi * t[:, None] ** 2))          # nu |gamma'| = (dy, -dx)
    inner = (kern * ws[None, :]).sum(axis=1) * L
    return float((inner * wt).sum())


def test_straight_boundary_quartic_density_is_exact():
    # boundary y = 0 (outward normal +y), target (0, rho r), mu = a + b xi + c xi^2/2 + d xi^3/6
    # + e xi^4/24: int mu e^{-xi^2/4t} dxi = sqrt(4 pi t)(a + c t + e t^2/2), so
    # D = int_0^ds rho r e^{-alpha^2 t - r^2/4t} (a + c t + e t^2/2) / (4 sqrt(pi) t^{3/2}) dt, and
    # the lemma through delta*^2 holds exactly
    for alpha, ds in [(10.0, 1e-4), (1.0, 3e-3), (100.0, 1e-5)]:
        for a, b, c, d, e in [(1.0, 0.0, 0.0, 0.0, 0.0), (0.3, 2.0, -40.0, 7.0, 0.0),
                              (-0.5, 1.0, 3.0, 0.0, 5e4)]:
            for c1 in [0.3, 1.0, 4.0, 9.0]:
                r = c1 * math.sqrt(ds)
                f = lambda t: (r * math.exp(-alpha * alpha * t - r * r / (4 * t))
                               * (a + c * t + e * t * t / 2) / (4 * math.sqrt(math.pi) * t ** 1.5))
                ref = si.quad(f, 0.0, ds, epsabs=0.0, epsrel=1e-13, limit=300)[0]
                # the size of the terms (the density's terms may cancel)
                fa = lambda t: (r * math.exp(-alpha * alpha * t - r * r / (4 * t))
                                * (abs(a) + abs(c) * t + abs(e) * t * t / 2)
                                / (4 * math.sqrt(math.pi) * t ** 1.5))
                size = si.quad(fa, 0.0, ds, epsabs=0.0, epsrel=1e-13, limit=300)[0]
                for rho in (1.0, -1.0):
                    v = float(OL.dla_lemma_terms(alpha, ds, r, rho, 0.0, a, b, c, e, 0.0, 0.0))
                    # relative to the terms, or to the layer's O(1) scale mu0 / 2 in the far tail
                    tol = 1e-12 * size + 1e-15 * (abs(a) + abs(c) * ds + abs(e) * ds * ds)
                    assert abs(v - rho * ref) <= tol, (alpha, ds, c1, v, ref)


def _circle(R=1.0):
    # mu = 1 + 0.5 cos 2 theta = 1.5 - xi^2/R^2 in the tangent-line parameter xi = R sin theta at
    # theta = 0; the graph R cos theta - R = -xi^2/(2R) - xi^4/(8R^3): kappa0 = -1/R, gamma''' = 0,
    # gamma'''' = -3/R^3
    def curve(s):
        return (R * np.cos(s), R * np.sin(s), -R * np.sin(s), R * np.cos(s),
                1.0 + 0.5 * np.cos(2 * s))
    return curve, dict(kappa0=-1.0 / R, mu0=1.5, mu1=0.0, mu2=-2.0 / R ** 2, mu4=0.0, g3=0.0,
                       g4=-3.0 / R ** 3)


@pytest.mark.parametrize("alpha", [10.0, 1.0])
def test_circle_converges_at_the_lemma_order(alpha):
    # relative error O(delta*^2) through the delta*^{3/2} term would fall 100-fold from
    # delta* = 1e-4 to 1e-5, through the delta*^2 term (the lemma as printed) 316-fold
    curve, p = _circle()
    errs = {}
    for ds in (1e-4, 1e-5):
        worst = 0.0
        for c1 in (0.5, 2.0):
            for rho in (1.0, -1.0):
                X = 1.0 + rho * c1 * math.sqrt(ds)
                ref = dla_quadrature(alpha, ds, X, 0.0, curve, 0.0)
                v = float(OL.dla_lemma_terms(alpha, ds, abs(X - 1.0), rho, **p))
                worst = max(worst, abs(v - ref) / abs(ref))
        errs[ds] = worst
    assert errs[1e-5] > 0 and errs[1e-5] <= 1e-10, errs
    assert errs[1e-4] / errs[1e-5] >= 150.0, errs
    # the curvature's sign, and the overall sign of the printed lemma, are wrong at first order
    X = 1.0 + 0.5 * math.sqrt(1e-5)
    ref = dla_quadrature(alpha, 1e-5, X, 0.0, curve, 0.0)
    bad = dict(p, kappa0=1.0, g4=3.0)
    assert abs(float(OL.dla_lemma_terms(alpha, 1e-5, X - 1.0, 1.0, **bad)) - ref) > 1e-4 * abs(ref)
    printed = -float(OL.dla_lemma_terms(alpha, 1e-5, X - 1.0, 1.0, **p))
    assert abs(printed - ref) > abs(ref)


def _starfish_curve():
    g = OL.StarfishGeom()

    def curve(s):
        p, p1, _ = g.derivs(s)
        return p[0], p[1], p1[0], p1[1], OL.starfish_density4(s)[0]
    return g, curve


def test_starfish_converges_at_the_lemma_order():
    # the general case: gamma''' and mu' nonzero, the tangent-line derivatives from the curve
    # parameter's; moderate curvature so that the expansion's constants stay small
    g, curve = _starfish_curve()
    alpha = 10.0
    errs = {}
    for ds in (1e-4, 1e-5):
        worst = 0.0
        for t0 in (0.33, 2.9, 4.0, 5.3):   # |kappa0| below ~3, away from tips and valleys
            p, p1, _ = g.derivs(np.array([t0]))
            nrm = math.hypot(p1[0][0], p1[1][0])
            nx, ny = p1[1][0] / nrm, -p1[0][0] / nrm
            for c1 in (0.5, 2.0):
                for rho in (1.0, -1.0):
                    d = rho * c1 * math.sqrt(ds)
                    x, y = p[0][0] + d * nx, p[1][0] + d * ny
                    ref = dla_quadrature(alpha, ds, x, y, curve, t0)
                    v = float(OL.dla_local_starfish(alpha, ds, g, OL.starfish_density4,
                                                    np.array([x]), np.array([y]))[0])
                    worst = max(worst, abs(v - ref) / abs(ref))
        errs[ds] = worst
    assert errs[1e-5] > 0 and errs[1e-5] <= 2e-9, errs
    assert errs[1e-4] / errs[1e-5] >= 150.0, errs


def test_tangent_line_derivatives_against_finite_differences():
    # F(xi) = f(t(xi)) with t(xi) the inverse of xi(t) = (gamma(t) - x0) . tangent, by a root
    # solve and centred differences of F (step 2e-3, fourth-order stencils)
    g = OL.StarfishGeom()
    t0 = 1.1
    p = g.derivs4(np.array([t0]))
    sp_ = math.hypot(p[1][0][0], p[1][1][0])
    tx, ty = p[1][0][0] / sp_, p[1][1][0] / sp_
    x0 = np.array([p[0][0][0], p[0][1][0]])

    def t_of(xi):
        t = t0 + xi / sp_
        for _ in range(50):
            q, q1, _ = g.derivs(np.array([t]))
            t -= ((q[0][0] - x0[0]) * tx + (q[1][0] - x0[1]) * ty - xi) / (q1[0][0] * tx + q1[1][0] * ty)
        return t

    def F(xi):
        t = t_of(xi)
        q, _, _ = g.derivs(np.array([t]))
        eta = (q[0][0] - x0[0]) * ty - (q[1][0] - x0[1]) * tx
        return eta, OL.starfish_density4(np.array([t]))[0][0]

    h = 2e-3
    vals = np.array([F(k * h) for k in range(-3, 4)])
    d2 = (-vals[5] + 16 * vals[4] - 30 * vals[3] + 16 * vals[2] - vals[1]) / (12 * h * h)
    d1 = (-vals[5] + 8 * vals[4] - 8 * vals[2] + vals[1]) / (12 * h)
    d3 = (-vals[6] + 8 * vals[5] - 13 * vals[4] + 13 * vals[2] - 8 * vals[1] + vals[0]) / (8 * h ** 3)
    d4 = (-vals[6] + 12 * vals[5] - 39 * vals[4] + 56 * vals[3] - 39 * vals[2] + 12 * vals[1]
          - vals[0]) / (6 * h ** 4)
    xi = [p[k][0][0] * tx + p[k][1][0] * ty for k in range(1, 5)]
    eta = [p[k][0][0] * ty - p[k][1][0] * tx for k in range(1, 5)]
    G = OL.tangent_line_derivs(xi, eta)
    M = OL.tangent_line_derivs(xi, [v[0] for v in OL.starfish_density4(np.array([t0]))[1:]])
    for k, (fd, an) in enumerate(zip((d1, d2, d3, d4), zip(G, M))):
        for j in range(2):
            assert abs(fd[j] - an[j]) <= (1e-7 if k < 2 else 1e-3) * max(1.0, abs(an[j])), (k, j)
    # the graph's second derivative is the single-layer lemma's kappa0
    kappa = -(p[1][0][0] * p[2][1][0] - p[1][1][0] * p[2][0][0]) / sp_ ** 3
    assert abs(G[1] - kappa) <= 1e-13 * abs(kappa)


def test_jump_and_on_boundary_corollary():
    # r = 0, rho = 0: eq. dlp_local2 with the sign of the source-point derivative; the limits from
    # either side differ from it by +-mu0/2 (the double layer's jump, outside minus inside = mu0)
    for alpha, ds, k, m0, m1, m2, g3, g4 in [(10.0, 1e-4, -1.3, 0.7, 0.4, 2.0, 3.0, -5.0),
                                             (1.0, 1e-3, 0.4, -1.1, -2.0, -5.0, -1.0, 8.0)]:
        c2 = alpha * math.sqrt(ds)
        kq = 2 * math.erf(c2) - 4 * c2 / math.sqrt(math.pi) * math.exp(-c2 * c2)
        printed = (-math.sqrt(ds) * k * m0 / (4 * c2) * math.erf(c2)
                   + ds ** 1.5 / c2 ** 3 * (15 * k ** 3 * m0 / 64 - 3 * m0 * g4 / 32
                                            - 3 * k * m2 / 16 - m1 * g3 / 4) * kq)
        v = float(OL.dla_lemma_terms(alpha, ds, 0.0, 0.0, k, m0, m1, m2, 9.0, g3, g4))
        assert abs(v + printed) <= 1e-12 * abs(printed)
        for rho in (1.0, -1.0):
            w = float(OL.dla_lemma_terms(alpha, ds, 1e-12 * math.sqrt(ds), rho, k, m0, m1, m2, 9.0,
                                         g3, g4))
            assert abs(w - v - rho * m0 / 2) <= 1e-10 * abs(m0)


def test_locality_and_far_targets():
    alpha, ds = 10.0, 1e-4
    rl = OL.locality_radius(alpha, ds)
    args = (-1.0, 1.0, 0.5, 2.0, 3.0, 0.7, -1.2)
    far = float(OL.dla_lemma_terms(alpha, ds, 1.0001 * rl, 1.0, *args))
    near = float(OL.dla_lemma_terms(alpha, ds, 1e-12 * math.sqrt(ds), 1.0, *args))
    assert abs(far) <= 1e-15 * abs(near)
    u = OL.dla_local_starfish(alpha, ds, OL.StarfishGeom(), OL.starfish_density4,
                              np.array([3.0]), np.array([0.0]))
    assert u[0] == 0.0
