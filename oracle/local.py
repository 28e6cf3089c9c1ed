"""Oracle for the local asymptotic parts S_{L,A}, D_{L,A} and V_L and the dyadic corrections —
TEST INFRASTRUCTURE ONLY.

S_{L,A}[sigma](x) = int_0^{delta*} int_{boundary} H(t, x - x') sigma(x') ds dt, H the heat kernel of
(-Lap + alpha^2) (Section 2.1, eq. sla), evaluated by the asymptotic expansion of Section 4.1
(Lemma, eq. slp_local1) through its delta*^2 term, at the closest boundary point x0 found by
Newton on d/dt |x - gamma(t)|^2 = 0 (Section 3.2, closest point), here on the analytic starfish.

Readings (where the printed lemma is garbled or silent):
* Z = 4 c2 exp(-c1^2/4 - c2^2) / sqrt(pi): the printed Z lacks the factor c2, with which Q_m would
  blow up like c2^-3 instead of being O(1) as the remark on P_m, Q_m states, and the corollary for
  targets on the boundary (eq. slp_local2) would not follow.
* kappa0 is the curvature of the boundary graph xi -> gamma(xi) in the frame (tangent, outward
  normal nu0) of the lemma's local coordinates: for a convex domain the boundary bends away from
  nu0, so kappa0 = -(x'y'' - y'x'') / |gamma'|^3 for a counter-clockwise parametrisation.
* rho = sign((x - x0) . nu0) (the lemma's (x - x0).nu0 / |x - x0| at the closest point).
* sigma0'' is the second derivative along the tangent-line parameter, which at x0 equals the
  second arclength derivative.
The pins of tests/test_oracle_pins_local.py fix all four against the definition (eq. sla).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sp


def locality_radius(alpha: float, dstar: float) -> float:
    """Beyond r = sqrt(d*)(12 + 2 alpha sqrt(d*)) S_{L,A} is below machine precision (remark on
    locality, Section 4.1)."""
    s = math.sqrt(dstar)
    return s * (12.0 + 2.0 * alpha * s)


def lemma_terms(alpha, dstar, r, rho, kappa0, s0, s0pp, s0p=0.0, g3=0.0, g4=0.0):
    """The expansion of the lemma (eq. slp_local1) through its delta*^2 term, vectorised; s0p,
    g3, g4 are sigma0', gamma0^(3) and gamma0^(4) in the tangent-line parameter (the delta*^2
    term's only new inputs; 0 for a straight boundary, and a circle has gamma0^(3) = 0)."""
    r, rho, kappa0, s0, s0pp, s0p, g3, g4 = map(np.asarray, (r, rho, kappa0, s0, s0pp, s0p, g3, g4))
    sd = math.sqrt(dstar)
    c1 = r / sd
    c2 = alpha * sd
    em = np.exp(-c1 * c2) * sp.erfc(c1 / 2 - c2)
    ep = np.exp(c1 * c2) * sp.erfc(c1 / 2 + c2)
    phi_m, phi_p = em - ep, em + ep
    Z = 4.0 * c2 * np.exp(-c1 * c1 / 4 - c2 * c2) / math.sqrt(math.pi)
    P0 = phi_m / c2
    P1 = c1 * P0
    P2 = c1 * P1
    Q0 = (phi_m - Z) / c2 ** 3 + c1 * phi_p / c2 ** 2
    P3, Q1 = c1 * P2, c1 * Q0
    k = kappa0
    return (sd * s0 / 4 * P0 + dstar * rho * k * s0 / 8 * P1
            + dstar * sd * (k ** 2 * s0 / 32 * (Q0 + 3 * P2) + s0pp / 8 * Q0)
            + dstar ** 2 * rho * (k ** 3 * s0 / 64 * (-3 * Q1 + 5 * P3)
                                  + (3 * k * s0pp / 16 + s0p * g3 / 8 + s0 * g4 / 32) * Q1))


class StarfishGeom:
    """Analytic starfish r(t) = r0 + a cos(m t + phase), gamma(t) = r(t)(cos t, sin t)."""

    def __init__(self, r0=1.0, a=0.3, arms=5, phase=0.0):
        self.r0, self.a, self.m, self.ph = r0, a, arms, phase

    def derivs(self, t):
        """gamma, gamma', gamma'' at parameter t (arrays of shape (2,) + t.shape)."""
        a, m, ph = self.a, self.m, self.ph
        r = self.r0 + a * np.cos(m * t + ph)
        r1 = -a * m * np.sin(m * t + ph)
        r2 = -a * m * m * np.cos(m * t + ph)
        c, s = np.cos(t), np.sin(t)
        g = np.array([r * c, r * s])
        g1 = np.array([r1 * c - r * s, r1 * s + r * c])
        g2 = np.array([r2 * c - 2 * r1 * s - r * c, r2 * s + 2 * r1 * c - r * s])
        return g, g1, g2

    def derivs4(self, t):
        """gamma and its first four derivatives at parameter t (Leibniz on r(t) e(t), e = (cos t,
        sin t), whose derivatives cycle e, e_perp, -e, -e_perp)."""
        a, m, ph = self.a, self.m, self.ph
        ph_t = m * t + ph
        rk = [self.r0 + a * np.cos(ph_t), -a * m * np.sin(ph_t), -a * m ** 2 * np.cos(ph_t),
              a * m ** 3 * np.sin(ph_t), a * m ** 4 * np.cos(ph_t)]
        c, s = np.cos(t), np.sin(t)
        ek = [np.array([c, s]), np.array([-s, c]), np.array([-c, -s]), np.array([s, -c]),
              np.array([c, s])]
        return [sum(math.comb(k, j) * rk[j] * ek[k - j] for j in range(k + 1)) for k in range(5)]

    def closest(self, x, y, n_scan=4096, iters=60):
        """Parameter of the closest boundary point: best of a dense scan, then Newton on
        f(t) = (gamma(t) - x) . gamma'(t) = 0 with f' = |gamma'|^2 + (gamma - x) . gamma''."""
        x, y = np.atleast_1d(x).astype(float), np.atleast_1d(y).astype(float)
        ts = np.linspace(0.0, 2 * np.pi, n_scan, endpoint=False)
        g, _, _ = self.derivs(ts)
        d2 = (g[0][None, :] - x[:, None]) ** 2 + (g[1][None, :] - y[:, None]) ** 2
        t = ts[np.argmin(d2, axis=1)]
        for _ in range(iters):
            g, g1, g2 = self.derivs(t)
            ex, ey = g[0] - x, g[1] - y
            f = ex * g1[0] + ey * g1[1]
            fp = g1[0] ** 2 + g1[1] ** 2 + ex * g2[0] + ey * g2[1]
            t = t - f / fp
        return t


def slp_local_starfish(alpha, dstar, geom: StarfishGeom, sigma, xt, yt):
    """S_{L,A}[sigma] at the targets for the analytic starfish; sigma(t) -> (sigma, sigma_t,
    sigma_tt) in the curve parameter.  Targets beyond the locality radius get 0."""
    xt, yt = np.atleast_1d(xt).astype(float), np.atleast_1d(yt).astype(float)
    t = geom.closest(xt, yt)
    g = geom.derivs4(t)
    g1, g2 = g[1], g[2]
    sp_ = np.hypot(g1[0], g1[1])                      # ds/dt
    nux, nuy = g1[1] / sp_, -g1[0] / sp_              # outward normal (counter-clockwise)
    dx, dy = xt - g[0][0], yt - g[0][1]
    r = np.hypot(dx, dy)
    rho = np.where(dx * nux + dy * nuy >= 0.0, 1.0, -1.0)
    kappa0 = -(g1[0] * g2[1] - g1[1] * g2[0]) / sp_ ** 3
    s0, s1, s2 = sigma(t)
    spp = (g1[0] * g2[0] + g1[1] * g2[1]) / sp_        # d2s/dt2
    s0pp = (s2 - s1 * spp / sp_) / sp_ ** 2             # second arclength derivative
    # gamma0^(3), gamma0^(4) of the boundary graph and sigma0' in the tangent-line parameter
    tx, ty = g1[0] / sp_, g1[1] / sp_
    xi = [g[k][0] * tx + g[k][1] * ty for k in range(1, 5)]
    eta = [g[k][0] * nux + g[k][1] * nuy for k in range(1, 5)]
    G = tangent_line_derivs(xi, eta)
    s0p = s1 / xi[0]
    u = lemma_terms(alpha, dstar, r, rho, kappa0, s0, s0pp, s0p, G[2], G[3])
    return np.where(r < locality_radius(alpha, dstar), u, 0.0)


def starfish_density(t):
    """sigma = cos 3t + 0.5 sin t (the workloads' boundary density) and its t-derivatives."""
    return (np.cos(3 * t) + 0.5 * np.sin(t), -3 * np.sin(3 * t) + 0.5 * np.cos(t),
            -9 * np.cos(3 * t) - 0.5 * np.sin(t))


def starfish_density4(t):
    """the same density and its first four t-derivatives"""
    return (np.cos(3 * t) + 0.5 * np.sin(t), -3 * np.sin(3 * t) + 0.5 * np.cos(t),
            -9 * np.cos(3 * t) - 0.5 * np.sin(t), 27 * np.sin(3 * t) - 0.5 * np.cos(t),
            81 * np.cos(3 * t) + 0.5 * np.sin(t))


# ------------------------------------------------------------------------------------------------
# Double-layer local part D_{L,A}[mu](x) = int_0^{delta*} int_boundary dH_t(x - x')/dnu' mu(x')
# ds dt (Section 2.1, eq. dla), by the expansion of the double-layer lemma (Section 4.1,
# eq. dlp_local1) through its delta*^2 term, at the closest boundary point x0.
#
# Readings:
# * the normal derivative is taken in the source point, as for the history part D_H:
#   dH_t(x - x')/dnu' = nu' . (x - x') H_t(x - x') / (2t), positive along nu'.  The printed
#   expansion has the opposite overall sign: its leading term -rho mu0 U0 / 4 is, for a straight
#   boundary and constant mu, the value of a derivative in the target.  Every term is taken with
#   its sign reversed.
# * P_m, Q_m, Z (with its factor c2), rho and kappa0 as in the single-layer lemma; U_m = c1^m Phi_+.
# * the delta*^{3/2} bracket prints (5 kappa0^3 mu0/64 - mu0 gamma0''''/32)(3 Q0 - U_3).  Expanding
#   eq. dla as the lemma's proof describes (z = sqrt(4t), xi = u z, Gaussian moments in u) gives
#   every printed term but this one: the kappa0^3 part multiplies (3 Q0 - U_3), the gamma0''''
#   part (3 Q0 + P_2).  The two agree at c1 = 0, so the corollary (eq. dlp_local2) is unchanged;
#   the circle and starfish pins converge at the lemma's order only with (3 Q0 + P_2).
# * mu0', mu0'', mu0^(4) and gamma0^(3), gamma0^(4) are derivatives in the tangent-line parameter
#   xi at x0, gamma the boundary graph in the frame (tangent, outward normal nu0); they follow
#   from the curve-parameter derivatives through the inverse of xi(t) = (gamma(t) - x0) . tangent.
# * a target within 1e-10 sqrt(delta*) of the boundary is on it: rho = 0, and the value is the
#   corollary's (eq. dlp_local2), the integral at the boundary point itself; any other target
#   carries the layer's jump through the U_0 term (+-mu0/2 as r -> 0).
# tests/test_oracle_pins_dla.py fixes these against eq. dla (straight boundary, circle, starfish).
# ------------------------------------------------------------------------------------------------

def dla_lemma_terms(alpha, dstar, r, rho, kappa0, mu0, mu1, mu2, mu4, g3, g4):
    """The expansion of the double-layer lemma (eq. dlp_local1) through the delta*^2 term, with
    the overall sign of the source-point normal derivative, vectorised."""
    r, rho, kappa0, mu0, mu1, mu2, mu4, g3, g4 = map(
        np.asarray, (r, rho, kappa0, mu0, mu1, mu2, mu4, g3, g4))
    sd = math.sqrt(dstar)
    c1 = r / sd
    c2 = alpha * sd
    em = np.exp(-c1 * c2) * sp.erfc(c1 / 2 - c2)
    ep = np.exp(c1 * c2) * sp.erfc(c1 / 2 + c2)
    phi_m, phi_p = em - ep, em + ep
    Z = 4.0 * c2 * np.exp(-c1 * c1 / 4 - c2 * c2) / math.sqrt(math.pi)
    P = [phi_m / c2]
    for _ in range(3):
        P.append(c1 * P[-1])
    Q0 = (phi_m - Z) / c2 ** 3 + c1 * phi_p / c2 ** 2
    Q1 = c1 * Q0
    U = [phi_p]
    for _ in range(4):
        U.append(c1 * U[-1])
    k = kappa0
    printed = (-rho * mu0 / 4 * U[0]
               - sd * k * mu0 / 8 * (P[0] + U[1])
               - dstar * (rho * mu2 / 8 * P[1] + 3 * rho * k ** 2 * mu0 / 32 * (P[1] + U[2]))
               + dstar * sd * (5 * k ** 3 * mu0 / 64 * (3 * Q0 - U[3])
                               - mu0 * g4 / 32 * (3 * Q0 + P[2])
                               + 3 * k * mu2 / 16 * (-Q0 - P[2])
                               + mu1 * g3 / 8 * (-2 * Q0 - P[2]))
               + dstar ** 2 * (35 * rho * k ** 4 * mu0 / 512 * (9 * Q1 + 2 * P[3] - U[4])
                               - rho * mu4 / 32 * Q1
                               - 15 * rho * k ** 2 * mu2 / 64 * (Q1 + P[3]))
               - dstar ** 2 * (5 * rho * k * mu1 * g3 / 16 * (2 * Q1 + P[3])
                               + (5 * rho * k * mu0 * g4 / 64 + 5 * rho * mu0 * g3 ** 2 / 96)
                               * (3 * Q1 + P[3])))
    return -printed


def tangent_line_derivs(xi, f):
    """Derivatives of F(xi) = f(t(xi)) at x0 from xi_k = d^k xi / dt^k (k = 1..4) and f_k = d^k f
    / dt^k (k = 1..4), xi(t) = (gamma(t) - x0) . tangent (chain rule with the inverse function
    t(xi): t' = 1/xi1, t'' = -xi2/xi1^3, ...).  Returns [F', F'', F''', F'''']."""
    x1, x2, x3, x4 = xi
    f1, f2, f3, f4 = f
    t1 = 1.0 / x1
    t2 = -x2 / x1 ** 3
    t3 = (3 * x2 ** 2 - x1 * x3) / x1 ** 5
    t4 = (-15 * x2 ** 3 + 10 * x1 * x2 * x3 - x1 ** 2 * x4) / x1 ** 7
    return [f1 * t1,
            f2 * t1 ** 2 + f1 * t2,
            f3 * t1 ** 3 + 3 * f2 * t1 * t2 + f1 * t3,
            f4 * t1 ** 4 + 6 * f3 * t1 ** 2 * t2 + f2 * (3 * t2 ** 2 + 4 * t1 * t3) + f1 * t4]


def dla_local_starfish(alpha, dstar, geom: StarfishGeom, mu4, xt, yt):
    """D_{L,A}[mu] at the targets for the analytic starfish; mu4(t) -> mu and its first four
    t-derivatives.  Targets beyond the locality radius get 0."""
    xt, yt = np.atleast_1d(xt).astype(float), np.atleast_1d(yt).astype(float)
    t = geom.closest(xt, yt)
    g = geom.derivs4(t)
    sp_ = np.hypot(g[1][0], g[1][1])
    tx, ty = g[1][0] / sp_, g[1][1] / sp_              # tangent
    nux, nuy = ty, -tx                                  # outward normal (counter-clockwise)
    xi = [g[k][0] * tx + g[k][1] * ty for k in range(1, 5)]
    eta = [g[k][0] * nux + g[k][1] * nuy for k in range(1, 5)]
    G = tangent_line_derivs(xi, eta)                    # G[0] = 0 at x0
    kappa0, g3, g4 = G[1], G[2], G[3]
    m = mu4(t)
    M = tangent_line_derivs(xi, m[1:])
    dx, dy = xt - g[0][0], yt - g[0][1]
    r = np.hypot(dx, dy)
    side = dx * nux + dy * nuy
    rho = np.where(r <= 1e-10 * math.sqrt(dstar), 0.0, np.where(side >= 0.0, 1.0, -1.0))
    u = dla_lemma_terms(alpha, dstar, r, rho, kappa0, m[0], M[0], M[1], M[3], g3, g4)
    return np.where(r < locality_radius(alpha, dstar), u, 0.0)


# ------------------------------------------------------------------------------------------------
# Volume local part V_L[f](x) = int_0^{delta*} int_Omega H_t(x - x') f(x') dx' dt (Section 2.1,
# eq. vl), by the expansion of the Lemma for V_L (Section 4.1, eq. vp_local1) through its
# delta*^2 term, for targets in Omega.
#
# Readings:
# * Q0, Q1 as in the single-layer lemma, with Z = 4 c2 exp(-c1^2/4 - c2^2)/sqrt(pi) (the printed
#   corollary for boundary targets, eq. vp_local2, has exactly that factor).
# * kappa0 is the second derivative of the boundary graph in the lemma's local frame, here
#   (tangent, inward normal eta) with the target at the origin: positive where the domain is
#   convex, kappa0 = (x'y'' - y'x'') / |gamma'|^3 for a counter-clockwise boundary.
# * f^(0,1) = grad f . eta, f^(0,2) = eta^T (Hess f) eta, f^(2,0) = xi^T (Hess f) xi at the target,
#   eta the inward normal at the closest boundary point and xi the tangent there.
# tests/test_oracle_pins_vl.py fixes these against eq. vl (half-plane, disk, interior).
# ------------------------------------------------------------------------------------------------

def vl_lemma_terms(alpha, dstar, r, kappa0, f, f_eta, f_etaeta, f_xixi):
    """The expansion of the lemma (eq. vp_local1) through the delta*^2 term, vectorised."""
    r, kappa0, f, f_eta, f_etaeta, f_xixi = map(np.asarray, (r, kappa0, f, f_eta, f_etaeta,
                                                             f_xixi))
    sd = math.sqrt(dstar)
    c1 = r / sd
    c2 = alpha * sd
    em = np.exp(-c1 * c2) * sp.erfc(c1 / 2 - c2)
    ep = np.exp(c1 * c2) * sp.erfc(c1 / 2 + c2)
    phi_m, phi_p = em - ep, em + ep
    Z = 4.0 * c2 * np.exp(-c1 * c1 / 4 - c2 * c2) / math.sqrt(math.pi)
    P1 = c1 * phi_m / c2
    Q0 = (phi_m - Z) / c2 ** 3 + c1 * phi_p / c2 ** 2
    Q1 = c1 * Q0
    e2 = math.exp(-c2 * c2)
    lam = e2 * sp.erfc(c1 / 2)
    W0 = (4.0 - 4.0 * e2 + 2.0 * lam - phi_p) / c2 ** 2
    W1 = (2.0 * W0 - P1 + 4.0 * (lam - 2.0 * e2)) / c2 ** 2
    return (dstar * f / 4 * W0 + dstar * sd * (2 * f_eta - f * kappa0) / 8 * Q0
            + dstar ** 2 * ((f_eta * kappa0 / 8 - 3 * f * kappa0 ** 2 / 32 - f_etaeta / 8) * Q1
                            + (f_etaeta + f_xixi) / 8 * W1))


def vl_lemma_terms_mp(alpha, dstar, r, kappa0, f, f_eta, f_etaeta, f_xixi, dps=40):
    """eq. vp_local1 as printed, evaluated in 40-digit arithmetic (mpmath), elementwise.  W0's
    numerator 4 - 4 e^{-c2^2} + 2 lambda - Phi_+ is O(c2^2) while its terms are O(1), so in FP64
    the printed form loses ~1e-16 / c2^2 (3e-11 of W0 at c2 = 3e-3); 40 digits keep the oracle
    exact to FP64 for any c2 the tests use."""
    import mpmath as mp
    mp.mp.dps = dps
    sd = mp.sqrt(mp.mpf(dstar))
    c2 = mp.mpf(alpha) * sd

    def one(r_, k_, f_, fe, fee, fxx):
        c1 = mp.mpf(r_) / sd
        em = mp.exp(-c1 * c2) * mp.erfc(c1 / 2 - c2)
        ep = mp.exp(c1 * c2) * mp.erfc(c1 / 2 + c2)
        phi_m, phi_p = em - ep, em + ep
        Z = 4 * c2 * mp.exp(-c1 * c1 / 4 - c2 * c2) / mp.sqrt(mp.pi)
        P1 = c1 * phi_m / c2
        Q0 = (phi_m - Z) / c2 ** 3 + c1 * phi_p / c2 ** 2
        Q1 = c1 * Q0
        e2 = mp.exp(-c2 * c2)
        lam = e2 * mp.erfc(c1 / 2)
        W0 = (4 - 4 * e2 + 2 * lam - phi_p) / c2 ** 2
        W1 = (2 * W0 - P1 + 4 * (lam - 2 * e2)) / c2 ** 2
        k_, f_, fe, fee, fxx = (mp.mpf(float(v)) for v in (k_, f_, fe, fee, fxx))
        ds = sd * sd
        v = (ds * f_ / 4 * W0 + ds * sd * (2 * fe - f_ * k_) / 8 * Q0
             + ds ** 2 * ((fe * k_ / 8 - 3 * f_ * k_ ** 2 / 32 - fee / 8) * Q1
                          + (fee + fxx) / 8 * W1))
        return float(v)
    args = np.broadcast_arrays(*(np.asarray(a, dtype=float) for a in
                                 (r, kappa0, f, f_eta, f_etaeta, f_xixi)))
    out = np.array([one(*vals) for vals in zip(*(a.ravel() for a in args))])
    return out.reshape(args[0].shape)


def vl_interior(alpha, dstar, f, lap_f):
    """Targets at least the locality radius from the boundary (corollary, eq. vp_local3).  Its
    two coefficients (1 - e^{-c})/c and (1 - (1 + c) e^{-c})/c^2, c = alpha^2 delta*, are taken in
    40-digit arithmetic: in FP64 the second loses ~1e-16 / c^2 of itself for small c."""
    import mpmath as mp
    mp.mp.dps = 40
    c = mp.mpf(alpha) ** 2 * mp.mpf(dstar)
    a1 = float((1 - mp.exp(-c)) / c)
    a2 = float((1 - (1 + c) * mp.exp(-c)) / c ** 2)
    return dstar * np.asarray(f) * a1 + dstar ** 2 * np.asarray(lap_f) * a2


def vl_boundary(alpha, dstar, kappa0, f, f_eta, f_etaeta, f_xixi):
    """Targets on the boundary (corollary, eq. vp_local2)."""
    c2 = alpha * math.sqrt(dstar)
    e2 = math.exp(-c2 * c2)
    q = (2.0 * math.erf(c2) - 4.0 * c2 / math.sqrt(math.pi) * e2) / c2 ** 3
    return (dstar * f / (2 * c2 * c2) * (1 - e2)
            + dstar ** 1.5 * (2 * f_eta - f * kappa0) / 8 * q
            + dstar ** 2 * (f_etaeta + f_xixi) / (2 * c2 ** 4) * (1 - (1 + c2 * c2) * e2))


def vp_local_starfish(alpha, dstar, geom: StarfishGeom, fderiv, xt, yt):
    """V_L[f] at targets in the starfish domain; fderiv(x, y) -> (f, f_x, f_y, f_xx, f_xy, f_yy)
    at the targets.  Within the locality radius the lemma (40-digit evaluation) at the closest
    boundary point of the analytic curve, beyond it eq. vp_local3; targets outside the domain get
    NaN."""
    xt, yt = np.atleast_1d(xt).astype(float), np.atleast_1d(yt).astype(float)
    f, fx, fy, fxx, fxy, fyy = (np.asarray(a, dtype=float) for a in fderiv(xt, yt))
    t = geom.closest(xt, yt)
    g, g1, g2 = geom.derivs(t)
    sp_ = np.hypot(g1[0], g1[1])
    tx, ty = g1[0] / sp_, g1[1] / sp_                 # tangent xi
    ex, ey = -ty, tx                                   # inward normal eta (counter-clockwise)
    dx, dy = xt - g[0], yt - g[1]
    r = np.hypot(dx, dy)
    outside = (dx * ex + dy * ey < 0.0) & (r > 1e-8 * math.sqrt(dstar))
    kappa0 = (g1[0] * g2[1] - g1[1] * g2[0]) / sp_ ** 3
    f_eta = fx * ex + fy * ey
    f_etaeta = fxx * ex * ex + 2 * fxy * ex * ey + fyy * ey * ey
    f_xixi = fxx * tx * tx + 2 * fxy * tx * ty + fyy * ty * ty
    rl = locality_radius(alpha, dstar)
    u = vl_interior(alpha, dstar, f, fxx + fyy)
    m = r < rl
    if np.any(m):
        u = np.array(u, dtype=float)
        u[m] = vl_lemma_terms_mp(alpha, dstar, r[m], kappa0[m], f[m], f_eta[m], f_etaeta[m],
                                 f_xixi[m])
    return np.where(outside, np.nan, u)


def sincos_field(kx=2.0, ky=3.0):
    """f = sin(kx x) cos(ky y) and its derivatives (the workloads' manufactured volume field)."""
    def fd(x, y):
        s, c = np.sin(kx * x), np.cos(kx * x)
        sy, cy = np.sin(ky * y), np.cos(ky * y)
        return (s * cy, kx * c * cy, -ky * s * sy, -kx * kx * s * cy, -kx * ky * c * sy,
                -ky * ky * s * cy)
    return fd


# ------------------------------------------------------------------------------------------------
# Dyadic corrections of the single-layer local part (Section 2.1, eqs. slp_dyad, sld; difference
# kernel eq. diffker_s through the identity eq. equiv_split): with delta_j = delta / 4^j,
#   S_{L,D}^{(j)}[sigma](x) = int_boundary K_j(|x - x'|) sigma(x') ds,
#   K_j(r) = int_{delta_j}^{delta_{j-1}} e^{-r^2/4t - alpha^2 t} / (4 pi t) dt
#          = G^R(r, delta_{j-1}) - G^R(r, delta_j).
# The oracle takes K_j from its t-integral (composite Gauss-Legendre in log t), not from
# incomplete Bessel functions.
# ------------------------------------------------------------------------------------------------

_GL32 = np.polynomial.legendre.leggauss(32)


def dyadic_kernel(alpha, delta, j, r):
    """K_j(r) by 4 panels x 32 Gauss-Legendre nodes in u = log t over [log delta_j,
    log delta_{j-1}] (the integrand is smooth in u)."""
    r = np.asarray(r, dtype=float)
    lo, hi = math.log(delta / 4.0 ** j), math.log(delta / 4.0 ** (j - 1))
    x, w = _GL32
    acc = np.zeros_like(r)
    npan = 4
    for p in range(npan):
        a = lo + (hi - lo) * p / npan
        b = lo + (hi - lo) * (p + 1) / npan
        u = 0.5 * (b - a) * x + 0.5 * (a + b)
        t = np.exp(u)
        ww = 0.5 * (b - a) * w
        acc = acc + np.sum(ww * np.exp(-(r[..., None] ** 2) / (4 * t) - alpha * alpha * t), axis=-1)
    return acc / (4 * math.pi)


def slp_dyadic_starfish(alpha, delta, J, geom: StarfishGeom, sigma, xt, yt, n_scan=8192):
    """sum_{j=1}^J S_{L,D}^{(j)}[sigma] at the targets, on the analytic curve: composite
    16-point Gauss-Legendre over the scan intervals of the curve parameter that come within the
    level-1 locality radius sqrt(delta)(12 + 2 alpha sqrt(delta)) of the target (beyond it every
    K_j is below 1e-16 of its peak)."""
    xt, yt = np.atleast_1d(xt).astype(float), np.atleast_1d(yt).astype(float)
    R = locality_radius(alpha, delta)
    ts = np.linspace(0.0, 2 * math.pi, n_scan + 1)
    g, g1, _ = geom.derivs(ts)
    seg = np.hypot(np.diff(g[0]), np.diff(g[1]))        # chord of each scan interval
    xg, wg = np.polynomial.legendre.leggauss(16)
    out = np.zeros(len(xt))
    for i in range(len(xt)):
        d = np.hypot(g[0] - xt[i], g[1] - yt[i])
        near = np.nonzero(np.minimum(d[:-1], d[1:]) < R + seg)[0]
        if len(near) == 0:
            continue
        a, b = ts[near], ts[near + 1]
        t = (0.5 * (b - a))[:, None] * xg[None, :] + (0.5 * (a + b))[:, None]
        w = (0.5 * (b - a))[:, None] * wg[None, :]
        p, p1, _ = geom.derivs(t)
        s0, _, _ = sigma(t)
        r = np.hypot(p[0] - xt[i], p[1] - yt[i])
        q = s0 * np.hypot(p1[0], p1[1]) * w
        for j in range(1, J + 1):
            out[i] += np.sum(q * dyadic_kernel(alpha, delta, j, r))
    return out


# Double layer (Section 2.1, eqs. dld, diffker_dlp): the normal derivative in the source point of
# the heat kernel is nu' . (x - x') H / (2t), so
#   D_{L,D}^{(j)}[mu](x) = int_boundary nu(x') . (x - x') K^D_j(|x - x'|) mu(x') ds,
#   K^D_j(r) = int_{delta_j}^{delta_{j-1}} e^{-r^2/4t - alpha^2 t} / (8 pi t^2) dt
# (eq. diffker_dlp with K_nu(x, y) = int_1^inf s^{nu-1} e^{-x s - y/s} ds).

def dyadic_kernel_dl(alpha, delta, j, r):
    """K^D_j(r) by 4 panels x 32 Gauss-Legendre nodes in u = log t (dt / t^2 = du / t)."""
    r = np.asarray(r, dtype=float)
    lo, hi = math.log(delta / 4.0 ** j), math.log(delta / 4.0 ** (j - 1))
    x, w = _GL32
    acc = np.zeros_like(r)
    for p in range(4):
        a = lo + (hi - lo) * p / 4
        b = lo + (hi - lo) * (p + 1) / 4
        t = np.exp(0.5 * (b - a) * x + 0.5 * (a + b))
        ww = 0.5 * (b - a) * w
        acc = acc + np.sum(ww * np.exp(-(r[..., None] ** 2) / (4 * t) - alpha * alpha * t) / t,
                           axis=-1)
    return acc / (8 * math.pi)


def dlp_dyadic_starfish(alpha, delta, J, geom: StarfishGeom, mu, xt, yt, n_scan=8192):
    """sum_{j=1}^J D_{L,D}^{(j)}[mu] at the targets on the analytic curve (outward normal of the
    counter-clockwise parametrisation), quadrature as slp_dyadic_starfish."""
    xt, yt = np.atleast_1d(xt).astype(float), np.atleast_1d(yt).astype(float)
    R = locality_radius(alpha, delta)
    ts = np.linspace(0.0, 2 * math.pi, n_scan + 1)
    g, _, _ = geom.derivs(ts)
    seg = np.hypot(np.diff(g[0]), np.diff(g[1]))
    xg, wg = np.polynomial.legendre.leggauss(16)
    out = np.zeros(len(xt))
    for i in range(len(xt)):
        d = np.hypot(g[0] - xt[i], g[1] - yt[i])
        near = np.nonzero(np.minimum(d[:-1], d[1:]) < R + seg)[0]
        if len(near) == 0:
            continue
        a, b = ts[near], ts[near + 1]
        t = (0.5 * (b - a))[:, None] * xg[None, :] + (0.5 * (a + b))[:, None]
        w = (0.5 * (b - a))[:, None] * wg[None, :]
        p, p1, _ = geom.derivs(t)
        sp_ = np.hypot(p1[0], p1[1])
        nux, nuy = p1[1] / sp_, -p1[0] / sp_
        m0, _, _ = mu(t)
        dx, dy = xt[i] - p[0], yt[i] - p[1]
        r = np.hypot(dx, dy)
        q = m0 * sp_ * w * (nux * dx + nuy * dy)
        for j in range(1, J + 1):
            out[i] += np.sum(q * dyadic_kernel_dl(alpha, delta, j, r))
    return out
