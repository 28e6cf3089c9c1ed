"""FP64 CPU oracle for the long-range (history) potential — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The library's product path never calls it and shares no code with it.

* ``GHTable``       — G_H(r) from its Fourier (Hankel) definition (Section 5.1, eq. sh, in radial
                       form), by Gauss-Legendre quadrature, tabulated as piecewise Chebyshev series.
* ``direct_sum``    — u_H(x_i) = sum_j q_j G_H(|x_i - y_j|) (Section 2.1, eq. sl_sh, summed over
                       the quadrature nodes of eqs. bdry_quad and vol_quad), Neumaier-compensated.
* ``discrete_sum``  — the paper's discrete Fourier formula (Section 5.2, eq. sh_fourier) with the
                       plain type-1 sum of eq. disrete_sigma_hat, as double loops.
* ``gh_hankel``     — G_H at given radii straight from the quadrature (no table).
* ``FDTable``, ``fd_hankel`` — the double-layer radial factor F_D(r) = -G_H'(r)/r (Section 5.1,
                       the D_H formula: one more factor of k, J1 in place of J0), tabulated / direct.
* ``direct_sum_dl`` — D_H[mu](x_i) = sum_d F_D(|x_i - y_d|) (x_i - y_d) . (mu_d w_d nu_d)
                       (Section 2, eq. dlp, history part), Neumaier-compensated.
* ``discrete_sum`` also takes dipoles: coefficient -i (k . s) exp(-i k . y) per dipole.

The C source is ``oracle/oracle.c``; it is compiled by ``oracle/build.py``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        d, i64, vp = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
        P = ctypes.POINTER(ctypes.c_double)
        lib.or_gh_hankel.argtypes = [d, d, i64, P, P]
        lib.or_gh_hankel.restype = ctypes.c_int
        lib.or_kernel_hankel.argtypes = [d, d, ctypes.c_int, i64, P, P]
        lib.or_kernel_hankel.restype = ctypes.c_int
        lib.or_table_create_kind.argtypes = [d, d, d, d, ctypes.c_int]
        lib.or_table_create_kind.restype = vp
        lib.or_direct_sum_dl.argtypes = [vp, i64, P, P, P, P, i64, P, P, P, P]
        lib.or_direct_sum_dl.restype = ctypes.c_int
        lib.or_discrete_sum_dl.argtypes = [d, d, d, i64, d, d, i64, P, P, P, i64, P, P, P, P,
                                           i64, P, P, P]
        lib.or_discrete_sum_dl.restype = ctypes.c_int
        lib.or_table_create.argtypes = [d, d, d, d]
        lib.or_table_create.restype = vp
        lib.or_table_free.argtypes = [vp]
        lib.or_table_npanels.argtypes = [vp]
        lib.or_table_npanels.restype = ctypes.c_int
        lib.or_table_g0.argtypes = [vp]
        lib.or_table_g0.restype = d
        lib.or_table_eval.argtypes = [vp, i64, P, P]
        lib.or_table_eval.restype = ctypes.c_int
        lib.or_direct_sum.argtypes = [vp, i64, P, P, P, i64, P, P, P, P]
        lib.or_direct_sum.restype = ctypes.c_int
        lib.or_discrete_sum.argtypes = [d, d, d, i64, d, d, i64, P, P, P, i64, P, P, P]
        lib.or_discrete_sum.restype = ctypes.c_int
        lib.or_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_lib().or_num_threads())


def gh_hankel(alpha: float, delta: float, r) -> np.ndarray:
    """G_H(r) by direct Hankel quadrature (no table)."""
    r = _f64(np.atleast_1d(r))
    out = np.empty_like(r)
    if _lib().or_gh_hankel(alpha, delta, r.size, _p(r), _p(out)):
        raise MemoryError("or_gh_hankel failed")
    return out


def fd_hankel(alpha: float, delta: float, r) -> np.ndarray:
    """F_D(r) = -G_H'(r)/r by direct Hankel quadrature (no table)."""
    r = _f64(np.atleast_1d(r))
    out = np.empty_like(r)
    if _lib().or_kernel_hankel(alpha, delta, 1, r.size, _p(r), _p(out)):
        raise MemoryError("or_kernel_hankel failed")
    return out


class GHTable:
    """Piecewise Chebyshev table of G_H on [0, rmax] (degree 24, adaptive bisection)."""

    KIND = 0

    def __init__(self, alpha: float, delta: float, rmax: float, tol_rel: float = 1e-14):
        self.alpha, self.delta, self.rmax = float(alpha), float(delta), float(rmax)
        self._h = _lib().or_table_create_kind(self.alpha, self.delta, self.rmax, tol_rel,
                                              self.KIND)
        if not self._h:
            raise ValueError("or_table_create failed (alpha, delta, rmax must be > 0)")

    def __del__(self):
        if getattr(self, "_h", None):
            _lib().or_table_free(self._h)
            self._h = None

    @property
    def npanels(self) -> int:
        return int(_lib().or_table_npanels(self._h))

    @property
    def g0(self) -> float:
        return float(_lib().or_table_g0(self._h))

    def __call__(self, r) -> np.ndarray:
        r = _f64(np.atleast_1d(r))
        out = np.empty_like(r)
        if _lib().or_table_eval(self._h, r.size, _p(r), _p(out)):
            raise ValueError("radius outside [0, rmax]")
        return out


class FDTable(GHTable):
    """Piecewise Chebyshev table of F_D(r) = -G_H'(r)/r on [0, rmax]; g0 is F_D(0)."""

    KIND = 1


def pair_rmax(xs, ys, xt, yt) -> float:
    """Largest source-target distance (bounding-box diagonal bound), with a small margin."""
    dx = max(np.max(xt), np.max(xs)) - min(np.min(xt), np.min(xs))
    dy = max(np.max(yt), np.max(ys)) - min(np.min(yt), np.min(ys))
    return float(np.hypot(dx, dy) * (1.0 + 1e-9) + 1e-12)


def direct_sum(alpha, delta, xs, ys, q, xt, yt, table: GHTable | None = None,
               return_abs: bool = False):
    """u_H at the targets by the plain FP64 pair sum; optionally also sum_j |q_j| G_H."""
    xs, ys, q, xt, yt = map(_f64, (xs, ys, q, xt, yt))
    if table is None:
        table = GHTable(alpha, delta, pair_rmax(xs, ys, xt, yt))
    u = np.empty(xt.shape[0])
    sa = np.empty(xt.shape[0])
    rc = _lib().or_direct_sum(table._h, xs.size, _p(xs), _p(ys), _p(q), xt.size, _p(xt), _p(yt),
                              _p(u), _p(sa))
    if rc:
        raise ValueError("a source-target distance exceeds the table range")
    return (u, sa) if return_abs else u


def direct_sum_dl(alpha, delta, xd, yd, sx, sy, xt, yt, table: FDTable | None = None,
                  return_abs: bool = False):
    """D_H at the targets for dipoles of vector strength (sx, sy) = mu w nu at (xd, yd), by the
    plain FP64 pair sum; optionally also sum_d F_D(r) r |s_d|."""
    xd, yd, sx, sy, xt, yt = map(_f64, (xd, yd, sx, sy, xt, yt))
    if table is None:
        table = FDTable(alpha, delta, pair_rmax(xd, yd, xt, yt))
    u = np.empty(xt.shape[0])
    sa = np.empty(xt.shape[0])
    rc = _lib().or_direct_sum_dl(table._h, xd.size, _p(xd), _p(yd), _p(sx), _p(sy), xt.size,
                                 _p(xt), _p(yt), _p(u), _p(sa))
    if rc:
        raise ValueError("a source-target distance exceeds the table range")
    return (u, sa) if return_abs else u


def discrete_sum(alpha, delta, period, M, center, xs, ys, q, xt, yt, dipoles=None) -> np.ndarray:
    """Paper's discrete formula on modes |m_x|,|m_y| <= M with Delta k = 2 pi / period;
    dipoles = (xd, yd, sx, sy) adds double-layer sources."""
    xs, ys, q, xt, yt = map(_f64, (xs, ys, q, xt, yt))
    if dipoles is None:
        z = np.zeros(0)
        dipoles = (z, z, z, z)
    xd, yd, sx, sy = map(_f64, dipoles)
    u = np.empty(xt.shape[0])
    rc = _lib().or_discrete_sum_dl(float(alpha), float(delta), float(period), int(M),
                                   float(center[0]), float(center[1]), xs.size, _p(xs), _p(ys),
                                   _p(q), xd.size, _p(xd), _p(yd), _p(sx), _p(sy), xt.size,
                                   _p(xt), _p(yt), _p(u))
    if rc:
        raise MemoryError("or_discrete_sum failed")
    return u
