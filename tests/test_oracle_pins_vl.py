"""Pins of the oracle's volume local part V_L (Section 4.1, Lemma for V_L, eq. vp_local1;
definition eq. vl).  Independent of the oracle's arithmetic: eq. vl by scipy quadrature for a
half-plane with a quadratic f (where the expansion is exact), for a disk (convergence at the
lemma's order, which fixes the sign of kappa0), and the free-space heat semigroup of an
eigenfunction of the Laplacian far from the boundary (eq. vp_local3).
"""
import math

import mpmath as mp
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle.local as OL


def tail_moments(t, r):
    """M_k = int_{-r}^inf b^k e^{-b^2/4t} / sqrt(4 pi t) db, k = 0, 1, 2 (Gaussian tail moments)."""
    e = mp.exp(-r * r / (4 * t))
    m0 = mp.erfc(-r / (2 * mp.sqrt(t))) / 2
    m1 = mp.sqrt(t / mp.pi) * e
    return m0, m1, 2 * t * m0 - r * m1


def halfplane_exact(alpha, ds, r, f0, f_eta, f_xi, f_xixi, f_xieta, f_etaeta):
    """eq. vl for the half-plane {eta >= -r} (target at the origin, eta the inward normal) and
    f = f0 + f_xi a + f_eta b + f_xixi a^2/2 + f_xieta a b + f_etaeta b^2/2 at (a, b): the a-integral
    of the Gaussian gives the moments 1, 0, 2t, the b-integral the tail moments, and the t-integral
    is a 30-digit quadrature (t = ds v^2)."""
    mp.mp.dps = 30

    def inner(t):
        m0, m1, m2 = tail_moments(t, mp.mpf(r))
        return f0 * m0 + f_eta * m1 + 0.5 * f_xixi * 2 * t * m0 + 0.5 * f_etaeta * m2
    return float(mp.quad(lambda v: 2 * ds * v * mp.exp(-alpha ** 2 * ds * v * v) * inner(ds * v * v),
                         [0, 0.25, 1]))


def test_tail_moments_by_quadrature():
    mp.mp.dps = 30
    for t in [1e-6, 1e-4]:
        for r in [0.0, 1e-3, 2e-2]:
            got = tail_moments(mp.mpf(t), mp.mpf(r))
            for k in range(3):
                ref = mp.quad(lambda b: b ** k * mp.exp(-b * b / (4 * t)) / mp.sqrt(4 * mp.pi * t),
                              [-r, 0, mp.inf])
                assert abs(got[k] - ref) <= mp.mpf(10) ** -25 * max(abs(ref), mp.mpf(t))


@pytest.mark.parametrize("alpha", [1.0, 10.0, 100.0])
def test_halfplane_quadratic_f_is_exact(alpha):
    ds = 1e-4
    sd = math.sqrt(ds)
    coef = dict(f0=1.3, f_eta=0.7, f_xi=-0.4, f_xixi=2.1, f_xieta=0.9, f_etaeta=-1.6)
    for r in [0.0, 0.3 * sd, sd, 3 * sd, 8 * sd]:
        ex = halfplane_exact(alpha, ds, r, **coef)
        v = OL.vl_lemma_terms(alpha, ds, r, 0.0, coef["f0"], coef["f_eta"], coef["f_etaeta"],
                              coef["f_xixi"])
        # exact up to the rounding of the lemma's terms (cancellation ~ 1e-16 / c2^2)
        assert abs(v - ex) <= 1e-11 * abs(ex), (r, v, ex)


def disk_exact(alpha, ds, d, R, fpow):
    """eq. vl for the disk of radius R centred at 0, f = |y|^fpow (0 or 2), target at distance d
    from the centre: the angular integral gives I0, rho = d + 2 sqrt(t) s."""
    def inner(t):
        st = math.sqrt(t)

        def g(s):
            rho = d + 2 * st * s
            if rho <= 0.0:
                return 0.0
            z = d * rho / (2 * t)
            return rho * rho ** fpow * math.exp(-s * s) * sp.ive(0, z) / st / 1.0
        lo, hi = -d / (2 * st), (R - d) / (2 * st)
        return si.quad(g, max(lo, -40.0), hi, epsabs=0, epsrel=1e-13, limit=400)[0]
    return si.quad(lambda t: math.exp(-alpha * alpha * t) * inner(t), 0, ds, epsabs=0,
                   epsrel=1e-12, limit=200)[0]


def disk_lemma(alpha, ds, d, R, fpow, kappa_sign=1.0):
    r = R - d
    kappa0 = kappa_sign / R
    if fpow == 0:
        f, f_eta, f_etaeta, f_xixi = 1.0, 0.0, 0.0, 0.0
    else:  # f = |y|^2: grad = 2y, Hessian 2I; eta points to the centre
        f, f_eta, f_etaeta, f_xixi = d * d, -2 * d, 2.0, 2.0
    return OL.vl_lemma_terms(alpha, ds, r, kappa0, f, f_eta, f_etaeta, f_xixi)


@pytest.mark.parametrize("fpow", [0, 2])
def test_disk_converges_at_lemma_order_and_fixes_kappa_sign(fpow):
    alpha, R = 10.0, 1.0
    # relative errors: the expansion through delta*^2 leaves O(delta*^{5/2}) of an O(delta*)
    # value, so they fall by 4^{3/2} = 8 per factor 4 in delta*; with the opposite sign of kappa0
    # the delta*^{3/2} term is wrong and they fall by 4^{1/2} = 2
    ratios, ratios_wrong = [], []
    for c in [0.0, 0.5, 2.0]:
        errs, errs_wrong = [], []
        for ds in [4e-4, 1e-4]:
            d = R - c * math.sqrt(ds)
            ex = disk_exact(alpha, ds, d, R, fpow)
            errs.append(abs(disk_lemma(alpha, ds, d, R, fpow) - ex) / abs(ex))
            errs_wrong.append(abs(disk_lemma(alpha, ds, d, R, fpow, -1.0) - ex) / abs(ex))
        ratios.append(errs[0] / errs[1])
        ratios_wrong.append(errs_wrong[0] / errs_wrong[1])
        assert errs[1] < 2e-6
    assert min(ratios) > 6.5, ratios
    assert max(ratios_wrong) < 3, ratios_wrong


def test_interior_eigenfunction():
    # far from the boundary V_L = int_0^delta e^{-alpha^2 t} (e^{t Lap} f) dt; for f = sin 2x cos 3y,
    # e^{t Lap} f = e^{-13 t} f, so V_L = f (1 - e^{-(13 + alpha^2) delta}) / (13 + alpha^2);
    # eq. vp_local3 is its expansion to O(delta^3)
    fd = OL.sincos_field()
    x, y = 0.31, -0.27
    f, _, _, fxx, _, fyy = fd(np.array([x]), np.array([y]))
    # the remainder is f int_0^delta e^{-alpha^2 t} (e^{-13 t} - 1 + 13 t) dt, at most
    # (13^2 / 6) delta^3 |f|, and of that size while alpha^2 delta is small
    for alpha in [1.0, 10.0, 100.0]:
        errs = []
        for ds in [1e-3, 5e-4]:
            lam = 13 + alpha ** 2
            ex = f[0] * (1 - math.exp(-lam * ds)) / lam
            v = OL.vl_interior(alpha, ds, f[0], fxx[0] + fyy[0])
            errs.append(abs(v - ex))
            assert abs(v - ex) <= 169 / 6 * ds ** 3 * abs(f[0]) * (1 + 1e-6)
        if alpha <= 10:
            assert errs[0] / errs[1] > 7.5   # O(delta^3)


def test_boundary_and_far_limits_of_the_lemma():
    # the lemma at c1 = 0 is the printed corollary for boundary targets (eq. vp_local2), and at
    # the locality radius the printed interior form (eq. vp_local3)
    for alpha, ds in [(10.0, 1e-4), (100.0, 1e-5), (3.0, 1e-3)]:
        args = (0.7, 1.3, 0.4, -2.0, 0.5)
        v1 = OL.vl_lemma_terms(alpha, ds, 0.0, *args)
        v2 = OL.vl_boundary(alpha, ds, *args)
        assert abs(v1 - v2) <= 1e-13 * abs(v2)
        rl = OL.locality_radius(alpha, ds)
        v3 = OL.vl_lemma_terms(alpha, ds, rl, *args)
        v4 = OL.vl_interior(alpha, ds, 1.3, -1.5)
        assert abs(v3 - v4) <= 1e-13 * abs(v4)


def test_starfish_targets_inside_and_outside():
    g = OL.StarfishGeom()
    fd = OL.sincos_field()
    ds = 1e-5
    # inside (centre and near the boundary) are finite; outside is flagged
    t = np.array([0.3, 1.9])
    p, d1, _ = g.derivs(t)
    nrm = np.hypot(d1[0], d1[1])
    xin = p[0] - 0.002 * d1[1] / nrm     # inward normal = (-y', x') / |gamma'|
    yin = p[1] + 0.002 * d1[0] / nrm
    xout = p[0] + 0.002 * d1[1] / nrm
    yout = p[1] - 0.002 * d1[0] / nrm
    u = OL.vp_local_starfish(10.0, ds, g, fd, np.r_[0.0, xin, xout], np.r_[0.0, yin, yout])
    assert np.all(np.isfinite(u[:3])) and np.all(np.isnan(u[3:]))


def test_high_precision_lemma_agrees_with_fp64_where_conditioned():
    # where c2 is not small the FP64 and the 40-digit evaluations of the printed lemma agree; at
    # c2 = 3e-3 the FP64 form is off by ~1e-16 / c2^2 relative
    rng = np.random.default_rng(1)
    for alpha, ds in [(10.0, 1e-4), (100.0, 1e-5), (30.0, 1e-3)]:
        sd = math.sqrt(ds)
        r = rng.uniform(0, 10 * sd, 20)
        args = (r, 0.8, 1.1, -0.3, 0.7, 2.0)
        a = OL.vl_lemma_terms(alpha, ds, *args)
        b = OL.vl_lemma_terms_mp(alpha, ds, *args)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    ds = 1e-5
    ex = halfplane_exact(1.0, ds, 0.3 * math.sqrt(ds), 1.3, 0.7, -0.4, 2.1, 0.9, -1.6)
    v = OL.vl_lemma_terms_mp(1.0, ds, 0.3 * math.sqrt(ds), 0.0, 1.3, 0.7, -1.6, 2.1)
    assert abs(v - ex) <= 1e-14 * abs(ex)
