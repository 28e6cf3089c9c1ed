"""Pins of the oracle's dyadic corrections (Section 2.1, eqs. slp_dyad, sld, diffker_s,
equiv_split).  Independent of the oracle's arithmetic: the difference kernel at r = 0 in closed
form (E1), the telescoped sum over levels against the history kernel G_H of two deltas from the
oracle's Hankel-transform tables, and a circle with sigma = 1 + 0.5 cos 2 theta, where the boundary
integral reduces to modified Bessel functions and one t-integral.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle
import oracle.local as OL


@pytest.mark.parametrize("alpha,delta", [(10.0, 1e-4), (1.0, 3e-5), (100.0, 1e-5)])
def test_kernel_at_zero_is_e1_difference(alpha, delta):
    for j in (1, 2, 3):
        dj, dj1 = delta / 4.0 ** j, delta / 4.0 ** (j - 1)
        ex = (sp.exp1(alpha ** 2 * dj) - sp.exp1(alpha ** 2 * dj1)) / (4 * math.pi)
        assert abs(OL.dyadic_kernel(alpha, delta, j, 0.0) - ex) <= 1e-14 * ex


@pytest.mark.parametrize("alpha,delta", [(10.0, 1e-4), (3.0, 4e-4)])
def test_levels_telescope_to_history_kernels(alpha, delta):
    # sum_{j=1}^J K_j = G^R(delta) - G^R(delta / 4^J) = G_H(delta / 4^J) - G_H(delta)
    J = 3
    r = np.array([0.0, 0.3, 1.0, 2.5, 5.0]) * math.sqrt(delta)
    tab_hi = oracle.GHTable(alpha, delta, 0.2)
    tab_lo = oracle.GHTable(alpha, delta / 4.0 ** J, 0.2)
    s = sum(OL.dyadic_kernel(alpha, delta, j, r) for j in range(1, J + 1))
    ref = tab_lo(r) - tab_hi(r)
    assert np.max(np.abs(s - ref)) <= 1e-12 * np.max(np.abs(ref))


def circle_level_exact(alpha, delta, j, d, R=1.0):
    """S_{L,D}^{(j)} at (d, 0) for the circle of radius R and sigma = 1 + 0.5 cos 2 theta:
    int_{delta_j}^{delta_{j-1}} (R / (4 pi t)) e^{-alpha^2 t} int e^{-|x - y|^2/4t} sigma dtheta dt,
    the angular integral 2 pi e^{-(d - R)^2/4t} [ive(0, b) + 0.5 ive(2, b)], b = d R / (2t)."""
    def f(t):
        b = d * R / (2 * t)
        return (R / (4 * math.pi * t)) * math.exp(-alpha ** 2 * t - (d - R) ** 2 / (4 * t)) * \
            2 * math.pi * (sp.ive(0, b) + 0.5 * sp.ive(2, b))
    return si.quad(f, delta / 4.0 ** j, delta / 4.0 ** (j - 1), epsabs=0, epsrel=1e-13,
                   limit=200)[0]


def test_circle_levels():
    alpha, delta, J = 10.0, 1e-4, 3
    geom = OL.StarfishGeom(r0=1.0, a=0.0)
    sig = lambda t: (1 + 0.5 * np.cos(2 * t), -np.sin(2 * t), -2 * np.cos(2 * t))
    sd = math.sqrt(delta)
    d = np.array([1.0, 1.0 - 0.5 * sd, 1.0 + 2 * sd, 1.0 - 6 * sd])
    u = OL.slp_dyadic_starfish(alpha, delta, J, geom, sig, d, np.zeros_like(d))
    ref = np.array([sum(circle_level_exact(alpha, delta, j, di) for j in range(1, J + 1))
                    for di in d])
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_far_targets_get_nothing():
    alpha, delta = 10.0, 1e-4
    u = OL.slp_dyadic_starfish(alpha, delta, 3, OL.StarfishGeom(), OL.starfish_density,
                               np.array([0.0, 2.0]), np.array([0.0, 0.0]))
    assert np.all(u == 0.0)


# double layer (eqs. dld, diffker_dlp)

@pytest.mark.parametrize("alpha,delta", [(10.0, 1e-4), (1.0, 3e-5), (100.0, 1e-5)])
def test_dl_kernel_at_zero_is_e2_difference(alpha, delta):
    # int_{t1}^{t2} e^{-a t} t^-2 dt = E2(a t1)/t1 - E2(a t2)/t2
    for j in (1, 2, 3):
        t1, t2 = delta / 4.0 ** j, delta / 4.0 ** (j - 1)
        a = alpha ** 2
        ex = (sp.expn(2, a * t1) / t1 - sp.expn(2, a * t2) / t2) / (8 * math.pi)
        assert abs(OL.dyadic_kernel_dl(alpha, delta, j, 0.0) - ex) <= 1e-14 * ex


@pytest.mark.parametrize("alpha,delta", [(10.0, 1e-4), (3.0, 4e-4)])
def test_dl_levels_telescope_to_history_factor(alpha, delta):
    # sum_j K^D_j = F_D(delta / 4^J) - F_D(delta), F_D = -G_H'(r)/r of the history kernel (the
    # oracle's Hankel-transform tables)
    J = 3
    r = np.array([0.0, 0.3, 1.0, 2.5, 5.0]) * math.sqrt(delta)
    hi = oracle.FDTable(alpha, delta, 0.2)
    lo = oracle.FDTable(alpha, delta / 4.0 ** J, 0.2)
    s = sum(OL.dyadic_kernel_dl(alpha, delta, j, r) for j in range(1, J + 1))
    ref = lo(r) - hi(r)
    assert np.max(np.abs(s - ref)) <= 1e-11 * np.max(np.abs(ref))


def circle_dl_level_exact(alpha, delta, j, d, R=1.0):
    """D_{L,D}^{(j)} at (d, 0) for the circle of radius R, mu = 1 + 0.5 cos 2 theta, outward normal:
    nu . (x - y) = d cos theta - R, and int (d cos th - R) e^{b cos th} (1 + 0.5 cos 2 th) dth
    = 2 pi e^{b} [d (I1 + 0.25 (I1 + I3)) - R (I0 + 0.5 I2)] (scaled), b = d R / (2t)."""
    def f(t):
        b = d * R / (2 * t)
        i0, i1, i2, i3 = (sp.ive(n, b) for n in range(4))
        ang = 2 * math.pi * (d * (i1 + 0.25 * (i1 + i3)) - R * (i0 + 0.5 * i2))
        return (R / (8 * math.pi * t * t)) * math.exp(-alpha ** 2 * t - (d - R) ** 2 / (4 * t)) * ang
    return si.quad(f, delta / 4.0 ** j, delta / 4.0 ** (j - 1), epsabs=0, epsrel=1e-13,
                   limit=200)[0]


def test_circle_dl_levels():
    alpha, delta, J = 10.0, 1e-4, 3
    geom = OL.StarfishGeom(r0=1.0, a=0.0)
    mu = lambda t: (1 + 0.5 * np.cos(2 * t), -np.sin(2 * t), -2 * np.cos(2 * t))
    sd = math.sqrt(delta)
    d = np.array([1.0, 1.0 - 0.5 * sd, 1.0 + 2 * sd, 1.0 - 6 * sd])
    u = OL.dlp_dyadic_starfish(alpha, delta, J, geom, mu, d, np.zeros_like(d))
    ref = np.array([sum(circle_dl_level_exact(alpha, delta, j, di) for j in range(1, J + 1))
                    for di in d])
    assert np.max(np.abs(u - ref)) <= 1e-11 * np.max(np.abs(ref))
