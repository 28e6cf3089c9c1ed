"""Oracle for the single-layer local asymptotic part S_{L,A} — TEST INFRASTRUCTURE ONLY.

S_{L,A}[sigma](x) = int_0^{delta*} int_{boundary} H(t, x - x') sigma(x') ds dt, H the heat kernel of
(-Lap + alpha^2) (Section 2.1, eq. sla), evaluated by the asymptotic expansion of Section 4.1
(Lemma, eq. slp_local1) through its delta*^{3/2} term, at the closest boundary point x0 found by
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


def lemma_terms(alpha, dstar, r, rho, kappa0, s0, s0pp):
    """The expansion of the lemma (eq. slp_local1) through the delta*^{3/2} term, vectorised."""
    r, rho, kappa0, s0, s0pp = map(np.asarray, (r, rho, kappa0, s0, s0pp))
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
    return (sd * s0 / 4 * P0 + dstar * rho * kappa0 * s0 / 8 * P1
            + dstar * sd * (kappa0 ** 2 * s0 / 32 * (Q0 + 3 * P2) + s0pp / 8 * Q0))


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
    g, g1, g2 = geom.derivs(t)
    sp_ = np.hypot(g1[0], g1[1])                      # ds/dt
    nux, nuy = g1[1] / sp_, -g1[0] / sp_              # outward normal (counter-clockwise)
    dx, dy = xt - g[0], yt - g[1]
    r = np.hypot(dx, dy)
    rho = np.where(dx * nux + dy * nuy >= 0.0, 1.0, -1.0)
    kappa0 = -(g1[0] * g2[1] - g1[1] * g2[0]) / sp_ ** 3
    s0, s1, s2 = sigma(t)
    spp = (g1[0] * g2[0] + g1[1] * g2[1]) / sp_        # d2s/dt2
    s0pp = (s2 - s1 * spp / sp_) / sp_ ** 2             # second arclength derivative
    u = lemma_terms(alpha, dstar, r, rho, kappa0, s0, s0pp)
    return np.where(r < locality_radius(alpha, dstar), u, 0.0)


def starfish_density(t):
    """sigma = cos 3t + 0.5 sin t (the workloads' boundary density) and its t-derivatives."""
    return (np.cos(3 * t) + 0.5 * np.sin(t), -3 * np.sin(3 * t) + 0.5 * np.cos(t),
            -9 * np.cos(3 * t) - 0.5 * np.sin(t))
