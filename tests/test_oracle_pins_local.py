"""Pins of the oracle's single-layer local asymptotic part S_{L,A} (Section 4.1, Lemma, eq.
slp_local1 through its delta*^2 term; definition eq. sla).  Independent of the oracle's
arithmetic: the exact value for a straight boundary with constant density (1-D scipy quadrature),
the exact value for a circle with a two-mode density (the boundary integral reduces to modified
Bessel functions, then 1-D quadrature) and the starfish (2-D Gauss-Legendre quadrature of eq. sla),
both converging at the lemma's order, the corollary for targets on the boundary (eq. slp_local2),
the small-c2 limits of the remark on P_m and Q_m, the locality remark, and the closest point's
orthogonality.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle.local as OL


def circle_exact(alpha, ds, X, R=1.0):
    """S_{L,A} at (X, 0) for the circle of radius R and sigma = 1 + 0.5 cos 2 theta:
    int_0^ds (R / (4 pi t)) e^{-alpha^2 t} int_0^2pi e^{-|x - gamma|^2/(4t)} sigma dtheta dt with
    int e^{b cos theta} cos(n theta) dtheta = 2 pi I_n(b), b = X R / (2t)."""
    def f(v):  # t = v^2 removes the t^{-1/2} behaviour at t = 0
        t = v * v
        if t < 1e-200:
            return 0.0
        e = math.exp(-alpha * alpha * t - (X - R) ** 2 / (4 * t))
        if e == 0.0:
            return 0.0
        b = X * R / (2 * t)
        # scaled Bessel I_n e^{-b}; for b > 1e6 its two-term asymptotic form (error < 1e-13)
        ive = (lambda n: sp.ive(n, b)) if b < 1e6 else \
            (lambda n: (1 - (4 * n * n - 1) / (8 * b)) / math.sqrt(2 * math.pi * b))
        return (2 * v * R / (4 * math.pi * t)) * e * 2 * math.pi * (ive(0) + 0.5 * ive(2))
    return si.quad(f, 0.0, math.sqrt(ds), epsabs=0.0, epsrel=1e-13, limit=500)[0]


def test_flat_boundary_constant_density_is_exact():
    # straight boundary, sigma = 1: every term beyond the first vanishes and the lemma is exact:
    # S = int_0^ds e^{-alpha^2 t - d^2/(4t)} / (2 sqrt(pi t)) dt
    for alpha, ds in [(10.0, 1e-4), (1.0, 3e-3), (100.0, 1e-5)]:
        for c1 in [0.0, 0.3, 1.0, 4.0, 9.0]:
            d = c1 * math.sqrt(ds)
            ref = si.quad(lambda t: math.exp(-alpha * alpha * t - d * d / (4 * t)) / (2 * math.sqrt(math.pi * t)),
                          0.0, ds, epsabs=0.0, epsrel=1e-13, limit=300)[0]
            for rho in (1.0, -1.0):
                v = float(OL.lemma_terms(alpha, ds, d, rho, 0.0, 1.0, 0.0))
                assert abs(v - ref) <= 1e-12 * ref + 1e-300, (alpha, ds, c1, v, ref)


@pytest.mark.parametrize("alpha", [10.0, 1.0])
def test_circle_converges_at_the_lemma_order(alpha):
    # curved boundary, varying density: through the delta*^2 term the relative error is
    # O(delta*^2) (O(delta*^{3/2}) without it); it fixes the sign of kappa0 (curvature of the
    # graph in the outward-normal frame: -1/R here), Z's c2 and the delta*^2 term's kappa0^3 and
    # gamma0^(4) parts (the circle's graph -xi^2/(2R) - xi^4/(8R^3): gamma0^(4) = -3/R^3)
    errs = {}
    for ds in (1e-4, 1e-5):
        worst = 0.0
        for c1 in (0.0, 0.5, 2.0):
            for rho in (1.0, -1.0):
                X = 1.0 + rho * c1 * math.sqrt(ds)
                ref = circle_exact(alpha, ds, X)
                v = float(OL.lemma_terms(alpha, ds, abs(X - 1.0), rho, -1.0, 1.5, -2.0, 0.0,
                                         0.0, -3.0))
                worst = max(worst, abs(v - ref) / abs(ref))
        errs[ds] = worst
    assert all(np.isfinite(v) for v in errs.values()) and errs[1e-5] > 0, errs
    assert errs[1e-5] <= 2e-10, errs
    assert errs[1e-4] / errs[1e-5] >= 60.0, errs     # order 2 gives 100, order 3/2 31.6
    # the opposite curvature sign is wrong at first order
    X = 1.0 + 0.5 * math.sqrt(1e-5)
    bad = float(OL.lemma_terms(alpha, 1e-5, X - 1.0, 1.0, +1.0, 1.5, -2.0, 0.0, 0.0, 3.0))
    assert abs(bad - circle_exact(alpha, 1e-5, X)) / circle_exact(alpha, 1e-5, X) > 1e-4


_GU = np.polynomial.legendre.leggauss(300)   # outer rule, in u = log t
_GS = np.polynomial.legendre.leggauss(96)    # inner rule, along the boundary


def sla_quadrature(alpha, ds, x, y, geom, s0, sigma):
    """eq. sla at (x, y): int_0^ds int e^{-alpha^2 t - |x - gamma(s)|^2/(4t)} / (4 pi t) sigma(s)
    |gamma'(s)| ds dt by Gauss-Legendre in u = log t on [log ds - 30, log ds] (targets at least
    0.5 sqrt(ds) from the boundary) and, per t, over s0 +- 16 sqrt(t) / |gamma'(s0)|."""
    xu, wu = _GU
    xs, ws = _GS
    lo, hi = math.log(ds) - 30.0, math.log(ds)
    t = np.exp(0.5 * (hi - lo) * xu + 0.5 * (hi + lo))
    wt = 0.5 * (hi - lo) * wu * t
    _, d0, _ = geom.derivs(np.array([s0]))
    L = 16.0 * np.sqrt(t) / math.hypot(d0[0][0], d0[1][0])
    sv = s0 + L[:, None] * xs[None, :]
    g, g1, _ = geom.derivs(sv)
    ex, ey = x - g[0], y - g[1]
    kern = (np.exp(-alpha * alpha * t[:, None] - (ex * ex + ey * ey) / (4 * t[:, None]))
            / (4 * math.pi * t[:, None]) * sigma(sv)[0] * np.hypot(g1[0], g1[1]))
    return float(((kern * ws[None, :]).sum(axis=1) * L * wt).sum())


def test_starfish_converges_at_the_lemma_order():
    # the general case: sigma0' and gamma0^(3) nonzero, so the delta*^2 term's sigma0' gamma0^(3)
    # part is exercised too; moderate curvature (|kappa0| below ~3)
    g = OL.StarfishGeom()
    alpha = 10.0
    errs = {}
    for ds in (1e-4, 1e-5):
        worst = 0.0
        for t0 in (0.33, 2.9, 4.0, 5.3):
            p, p1, _ = g.derivs(np.array([t0]))
            nrm = math.hypot(p1[0][0], p1[1][0])
            nx, ny = p1[1][0] / nrm, -p1[0][0] / nrm
            for c1 in (0.5, 2.0):
                for rho in (1.0, -1.0):
                    d = rho * c1 * math.sqrt(ds)
                    x, y = p[0][0] + d * nx, p[1][0] + d * ny
                    ref = sla_quadrature(alpha, ds, x, y, g, t0, OL.starfish_density)
                    v = float(OL.slp_local_starfish(alpha, ds, g, OL.starfish_density,
                                                    np.array([x]), np.array([y]))[0])
                    worst = max(worst, abs(v - ref) / abs(ref))
        errs[ds] = worst
    assert errs[1e-5] > 0 and errs[1e-5] <= 1e-8, errs
    assert errs[1e-4] / errs[1e-5] >= 60.0, errs     # order 2 gives 100 (without the delta*^2
    #                                                   term ~32)


def test_on_boundary_corollary():
    # r = 0: eq. slp_local2
    for alpha, ds, kappa0, s0, s0pp in [(10.0, 1e-4, -1.3, 0.7, 2.0), (1.0, 1e-3, 0.4, -1.1, -5.0)]:
        c2 = alpha * math.sqrt(ds)
        ref = (math.sqrt(ds) * s0 / (2 * c2) * math.erf(c2)
               + ds ** 1.5 / c2 ** 3 * (kappa0 ** 2 * s0 / 32 + s0pp / 8)
               * (2 * math.erf(c2) - 4 * c2 / math.sqrt(math.pi) * math.exp(-c2 * c2)))
        v = float(OL.lemma_terms(alpha, ds, 0.0, 1.0, kappa0, s0, s0pp))
        assert abs(v - ref) <= 1e-12 * abs(ref)


def test_small_c2_limits_of_P_and_Q():
    # remark on P_m, Q_m: P0 -> 2(G - c1 E), Q0 -> (2/3)((2 - c1^2) G + c1^3 E) as c2 -> 0
    ds, alpha = 1e-4, 1e-2           # c2 = 1e-4
    for c1 in (0.0, 0.7, 2.5, 6.0):
        G = 2 / math.sqrt(math.pi) * math.exp(-c1 * c1 / 4)
        E = math.erfc(c1 / 2)
        P0 = 2 * (G - c1 * E)
        Q0 = 2.0 / 3.0 * ((2 - c1 * c1) * G + c1 ** 3 * E)
        r = c1 * math.sqrt(ds)
        # isolate the terms: sigma0 = 1, kappa0 = 0, sigma0'' = 0 gives sqrt(ds)/4 P0;
        # sigma0 = 0, sigma0'' = 8 gives ds^{3/2} Q0
        p = float(OL.lemma_terms(alpha, ds, r, 1.0, 0.0, 1.0, 0.0)) / (math.sqrt(ds) / 4)
        q = float(OL.lemma_terms(alpha, ds, r, 1.0, 0.0, 0.0, 8.0)) / ds ** 1.5
        assert abs(p - P0) <= 1e-6 * max(1.0, abs(P0))
        assert abs(q - Q0) <= 1e-3 * max(1.0, abs(Q0))   # Q0 loses digits to cancellation at c2 = 1e-4


def test_locality_and_closest_point():
    g = OL.StarfishGeom()
    alpha, ds = 10.0, 1e-4
    rl = OL.locality_radius(alpha, ds)
    rng = np.random.default_rng(3)
    t_true = rng.uniform(0, 2 * np.pi, 40)
    gg, g1, _ = g.derivs(t_true)
    nrm = np.hypot(g1[0], g1[1])
    off = rng.uniform(-0.8, 0.8, 40) * rl
    xt, yt = gg[0] + off * g1[1] / nrm, gg[1] - off * g1[0] / nrm
    t = g.closest(xt, yt)
    gc, gc1, _ = g.derivs(t)
    # orthogonality of x - x0 to the tangent, and the smallest distance over a fine scan
    assert np.max(np.abs((xt - gc[0]) * gc1[0] + (yt - gc[1]) * gc1[1])) <= 1e-13
    ts = np.linspace(0, 2 * np.pi, 200001)
    gs, _, _ = g.derivs(ts)
    dmin = np.min(np.hypot(gs[0][None, :] - xt[:, None], gs[1][None, :] - yt[:, None]), axis=1)
    assert np.all(np.hypot(xt - gc[0], yt - gc[1]) <= dmin + 1e-12)
    # beyond the locality radius the lemma's value is below 1e-15 of the on-boundary value
    far = float(OL.lemma_terms(alpha, ds, 1.0001 * rl, 1.0, -1.0, 1.0, 1.0))
    near = float(OL.lemma_terms(alpha, ds, 0.0, 1.0, -1.0, 1.0, 1.0))
    assert abs(far) <= 1e-15 * abs(near)
    u = OL.slp_local_starfish(alpha, ds, g, OL.starfish_density, np.array([3.0]), np.array([0.0]))
    assert u[0] == 0.0
