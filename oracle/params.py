"""Parameter rules of the long-range evaluation, written from the paper — TEST INFRASTRUCTURE.

These are the oracle's own statements of the rules; the CUDA library's plan implements its
rules separately in C++, and the tests compare the two.

* ``delta_from_mesh``  — Section 6.4's worked example: k_max = 0.9 k_Nyq with k_Nyq = pi/dx
                          (eq. k_nyq), then eq. kmax solved for delta at the history tolerance.
* ``kmax_paper``       — eq. kmax: exp(-delta (alpha^2 + k_max^2)) <= eps, k_max = 0 when
                          delta alpha^2 >= ln(1/eps).
* ``kmax_relative``    — reading of eq. kmax relative to G_H(0): the neglected tail of the radial
                          Fourier integral, E1(delta (alpha^2 + k^2)) / (4 pi), is at most eps times
                          G_H(0) = E1(delta alpha^2) / (4 pi).
* ``r_tol``            — smallest r beyond which G_H <= eps G_H(0) (G_H decreases in r), the
                          reading of the Nyquist/periodicity condition of eq. nf used for the period.
* ``modes``            — largest mode index M = ceil(k_max P / (2 pi)) for Delta k = 2 pi / P
                          (eq. delta_k with the symmetric mode set |m| <= M).
* ``kmax_dlp_paper``   — eq. kmax_dlp as printed: k_max exp(-delta (alpha^2 + k_max^2)) <= eps (the
                          extra factor of k from the normal derivative), 0 when it holds at every k.
* ``kmax_dlp_relative``— the same reading relative to the kernel's size: the tail
                          int_k^inf exp(-delta(alpha^2+s^2)) s^2/(alpha^2+s^2) ds is at most eps times
                          the whole integral (from 0), the bound on |G_H'| of the radial form.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.optimize as so
import scipy.special as sp

from . import gh_hankel


def delta_from_mesh(alpha: float, dx: float, eps_hist: float = 1e-6) -> float:
    kmax = 0.9 * math.pi / dx
    return math.log(1.0 / eps_hist) / (kmax * kmax + alpha * alpha)


def kmax_paper(alpha: float, delta: float, eps: float) -> float:
    return math.sqrt(max(0.0, (math.log(1.0 / eps) - delta * alpha * alpha) / delta))


def kmax_relative(alpha: float, delta: float, eps: float) -> float:
    x0 = delta * alpha * alpha
    target = eps * sp.exp1(x0)
    if sp.exp1(x0) <= target:
        return 0.0
    hi = x0 + 1.0
    while sp.exp1(hi) > target:
        hi = x0 + 2.0 * (hi - x0)
    x = so.brentq(lambda s: sp.exp1(s) - target, x0, hi, xtol=1e-15, rtol=1e-15)
    return math.sqrt(max(0.0, x / delta - alpha * alpha))


def r_tol(alpha: float, delta: float, eps: float) -> float:
    g0 = float(gh_hankel(alpha, delta, [0.0])[0])
    lo, hi = 0.0, max(1.0 / alpha, math.sqrt(delta))
    while float(gh_hankel(alpha, delta, [hi])[0]) > eps * g0:
        lo, hi = hi, 2.0 * hi
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if float(gh_hankel(alpha, delta, [mid])[0]) > eps * g0:
            lo = mid
        else:
            hi = mid
    return hi


def modes(kmax: float, period: float) -> int:
    return int(math.ceil(kmax * period / (2.0 * math.pi)))


def kmax_dlp_paper(alpha: float, delta: float, eps: float) -> float:
    f = lambda k: k * math.exp(-delta * (alpha * alpha + k * k))
    kpk = 1.0 / math.sqrt(2.0 * delta)          # maximiser of k exp(-delta k^2)
    if f(kpk) <= eps:
        return 0.0
    lo, hi = kpk, 2.0 * kpk
    while f(hi) > eps:
        lo, hi = hi, 2.0 * hi
    return so.brentq(lambda k: f(k) - eps, lo, hi, xtol=1e-13, rtol=1e-15)


def _dlp_tail(alpha, delta, k):
    import scipy.integrate as si
    g = lambda s: math.exp(-delta * (alpha * alpha + s * s)) * s * s / (alpha * alpha + s * s)
    return si.quad(g, k, np.inf, epsabs=0.0, epsrel=1e-13, limit=400)[0]


def kmax_dlp_relative(alpha: float, delta: float, eps: float) -> float:
    target = eps * _dlp_tail(alpha, delta, 0.0)
    lo, hi = 0.0, 1.0 / math.sqrt(delta)
    while _dlp_tail(alpha, delta, hi) > target:
        lo, hi = hi, 2.0 * hi
    return so.brentq(lambda k: _dlp_tail(alpha, delta, k) - target, lo, hi, xtol=1e-12,
                     rtol=1e-14)
