"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *generates inputs*: quadrature nodes and weights on a boundary curve and on a
cut-cell volume mesh, strengths (densities and source values) and target points.  It holds none
of the long-range method's arithmetic, so both the CUDA path and the CPU oracle can consume its
output without sharing any computation.

Geometry follows Section 6 (eq. bound_curve): the starfish r(t) = r0 + a cos(l1 t + phase),
gamma(t) = r(t) (cos t, sin t), with l3 = 0 so the curve parameter is the polar angle.
Boundary quadrature follows Section 3.2 (eq. bdry_quad): M_B uniform parameter panels with an
n_B-point Gauss-Legendre rule each.  The volume quadrature follows Section 3.1 (eq. vol_quad)
with a textbook 3-point triangle rule on a uniform background mesh whose cut cells are clipped
by straight chords (the paper's 6-node rule and isoparametric cells matter only to the PDE's
accuracy, not to the potential evaluated from given nodes and weights).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


# ----------------------------------------------------------------------------------------------
# curve
@dataclasses.dataclass(frozen=True)
class Starfish:
    r0: float = 1.0
    a: float = 0.3
    arms: int = 5
    phase: float = 0.0

    def radius(self, t):
        return self.r0 + self.a * np.cos(self.arms * t + self.phase)

    def dradius(self, t):
        return -self.a * self.arms * np.sin(self.arms * t + self.phase)

    def point(self, t):
        r = self.radius(t)
        return r * np.cos(t), r * np.sin(t)

    def speed(self, t):
        return np.hypot(self.radius(t), self.dradius(t))

    def normal(self, t):
        """Outward unit normal (the parametrisation runs counter-clockwise)."""
        r, dr = self.radius(t), self.dradius(t)
        tx, ty = dr * np.cos(t) - r * np.sin(t), dr * np.sin(t) + r * np.cos(t)
        s = np.hypot(tx, ty)
        return ty / s, -tx / s

    def inside(self, x, y):
        rho = np.hypot(x, y)
        return rho < self.radius(np.arctan2(y, x))

    def rmax(self):
        return self.r0 + abs(self.a)

    def area(self):
        return math.pi * (self.r0 ** 2 + 0.5 * self.a ** 2)


# ----------------------------------------------------------------------------------------------
# boundary quadrature (Section 3.2)
def boundary_nodes(curve: Starfish, n_panels: int, n_gl: int = 16):
    """Composite Gauss-Legendre nodes on uniform parameter panels of [0, 2pi).

    Returns (x, y, w, t): node coordinates, weights |gamma'(t)| * (pi/M_B) * omega_q and the
    parameter value of each node.
    """
    xi, om = np.polynomial.legendre.leggauss(n_gl)
    half = math.pi / n_panels
    centers = (2.0 * np.arange(n_panels) + 1.0) * half
    t = (centers[:, None] + half * xi[None, :]).ravel()
    x, y = curve.point(t)
    w = (curve.speed(t).reshape(n_panels, n_gl) * half * om[None, :]).ravel()
    return x, y, w, t


def double_layer_nodes(curve: Starfish, n_panels: int, n_gl: int = 16):
    """Boundary nodes for a double layer: (x, y, w, nx, ny, mu) with the outward unit normal and
    the smooth density mu(t) = sin(2t) + 0.3 cos(t)."""
    x, y, w, t = boundary_nodes(curve, n_panels, n_gl)
    nx, ny = curve.normal(t)
    return x, y, w, nx, ny, np.sin(2.0 * t) + 0.3 * np.cos(t)


def boundary_density(t):
    """Smooth layer density of the configs: cos(3t) + 0.5 sin(t)."""
    return np.cos(3.0 * t) + 0.5 * np.sin(t)


# ----------------------------------------------------------------------------------------------
# volume quadrature (Section 3.1)
_BARY = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])


def _crossing(curve, ax, ay, bx, by, iters=60):
    """Point on segment a->b where the curve is crossed; a inside, b outside (bisection)."""
    lo = np.zeros_like(ax)
    hi = np.ones_like(ax)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        inside = curve.inside(ax + mid * (bx - ax), ay + mid * (by - ay))
        lo = np.where(inside, mid, lo)
        hi = np.where(inside, hi, mid)
    s = 0.5 * (lo + hi)
    return ax + s * (bx - ax), ay + s * (by - ay)


def _tri_rule(px, py):
    """3-point rule on triangles given as (n,3) vertex arrays -> nodes and weights."""
    area = 0.5 * np.abs((px[:, 1] - px[:, 0]) * (py[:, 2] - py[:, 0])
                        - (px[:, 2] - px[:, 0]) * (py[:, 1] - py[:, 0]))
    nx = px @ _BARY.T
    ny = py @ _BARY.T
    w = np.repeat(area[:, None] / 3.0, 3, axis=1)
    return nx.ravel(), ny.ravel(), w.ravel()


def cut_cell_mesh(curve: Starfish, dx: float):
    """Triangles of a uniform right-triangle background mesh clipped to the curve's interior.

    Each background square of side dx is split along its diagonal.  Triangles with all vertices
    inside are kept, all outside are dropped, cut triangles are clipped by the straight chord
    between their two edge crossings (a triangle or a quadrilateral, fanned into triangles).
    Returns vertex arrays px, py of shape (n_tri, 3).
    """
    R = curve.rmax() + dx
    n = int(math.ceil(2 * R / dx)) + 1
    g = -R + dx * np.arange(n + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    IN = curve.inside(X, Y)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    i = i.ravel()
    j = j.ravel()
    # two triangles per square: (00,10,11) and (00,11,01), counter-clockwise
    tv = [((j, i), (j, i + 1), (j + 1, i + 1)), ((j, i), (j + 1, i + 1), (j + 1, i))]
    tris_x, tris_y = [], []
    for tri in tv:
        vx = np.stack([X[a, b] for a, b in tri], axis=1)
        vy = np.stack([Y[a, b] for a, b in tri], axis=1)
        vin = np.stack([IN[a, b] for a, b in tri], axis=1)
        cnt = vin.sum(axis=1)
        full = cnt == 3
        tris_x.append(vx[full])
        tris_y.append(vy[full])
        for k_in in (1, 2):
            sel = cnt == k_in
            if not np.any(sel):
                continue
            sx, sy, sin_ = vx[sel], vy[sel], vin[sel]
            # rotate vertex order so that vertex 0 is the lone inside (k_in=1) or lone outside
            # (k_in=2) vertex; orientation is preserved by a cyclic shift
            lone = np.argmax(sin_ if k_in == 1 else ~sin_, axis=1)
            idx = (lone[:, None] + np.arange(3)[None, :]) % 3
            sx = np.take_along_axis(sx, idx, axis=1)
            sy = np.take_along_axis(sy, idx, axis=1)
            if k_in == 1:
                c1 = _crossing(curve, sx[:, 0], sy[:, 0], sx[:, 1], sy[:, 1])
                c2 = _crossing(curve, sx[:, 0], sy[:, 0], sx[:, 2], sy[:, 2])
                tris_x.append(np.stack([sx[:, 0], c1[0], c2[0]], axis=1))
                tris_y.append(np.stack([sy[:, 0], c1[1], c2[1]], axis=1))
            else:
                c1 = _crossing(curve, sx[:, 1], sy[:, 1], sx[:, 0], sy[:, 0])
                c2 = _crossing(curve, sx[:, 2], sy[:, 2], sx[:, 0], sy[:, 0])
                # quadrilateral c1, v1, v2, c2 fanned from c1
                tris_x.append(np.stack([c1[0], sx[:, 1], sx[:, 2]], axis=1))
                tris_y.append(np.stack([c1[1], sy[:, 1], sy[:, 2]], axis=1))
                tris_x.append(np.stack([c1[0], sx[:, 2], c2[0]], axis=1))
                tris_y.append(np.stack([c1[1], sy[:, 2], c2[1]], axis=1))
    return np.concatenate(tris_x), np.concatenate(tris_y)


def _perimeter(curve: Starfish, n=4096):
    t = (np.arange(n) + 0.5) * (2 * math.pi / n)
    return float(curve.speed(t).sum() * (2 * math.pi / n))


def volume_nodes(curve: Starfish, n_target: int, search: bool = True):
    """3-point-rule nodes on a cut-cell mesh, about n_target of them.

    With search=True the mesh size is scanned so that the node count is the smallest achievable
    value >= n_target among the candidates tried.  Returns (x, y, w, dx).
    """
    # node count ~ 6 A / dx^2 (three nodes per half square) + ~6.4 P / dx (cut cells split in
    # two); solve for dx and scan around it
    A, P = curve.area(), _perimeter(curve)
    dx0 = (6.4 * P + math.sqrt((6.4 * P) ** 2 + 24.0 * A * n_target)) / (2.0 * n_target)

    def count(dx):
        px, _ = cut_cell_mesh(curve, dx)
        return 3 * px.shape[0]

    if search:
        best = None
        for s in np.linspace(0.94, 1.06, 121 if n_target < 50000 else 13):
            c = count(dx0 * s)
            if c >= n_target and (best is None or c < best[0]):
                best = (c, dx0 * s)
        dx = best[1] if best is not None else dx0 * 0.95
    else:
        dx = dx0
    px, py = cut_cell_mesh(curve, dx)
    x, y, w = _tri_rule(px, py)
    return x, y, w, dx


# ----------------------------------------------------------------------------------------------
# workloads
@dataclasses.dataclass
class Workload:
    """One long-range evaluation problem: sources (boundary then volume), strengths, targets."""
    name: str
    alpha: float
    xs: np.ndarray
    ys: np.ndarray
    w: np.ndarray          # quadrature weights
    density: np.ndarray    # sigma at boundary nodes, then f at volume nodes
    xt: np.ndarray
    yt: np.ndarray
    n_bdry: int
    h_vol: float           # volume mesh size (drives the delta rule)
    box: tuple = (-1.5, 1.5, -1.5, 1.5)

    @property
    def n_src(self):
        return self.xs.shape[0]

    @property
    def n_trg(self):
        return self.xt.shape[0]

    @property
    def q(self):
        return self.w * self.density


def uniform_targets(n, rng, box=(-1.5, 1.5, -1.5, 1.5)):
    x = rng.uniform(box[0], box[1], n)
    y = rng.uniform(box[2], box[3], n)
    return x, y


def gaussian_source(x, y, a=0.1):
    return np.exp(-(x * x + y * y) / a)


def manufactured_source(x, y, alpha):
    """f = (-Lap + alpha^2) u for u = sin(2x) cos(3y)."""
    return (13.0 + alpha * alpha) * np.sin(2.0 * x) * np.cos(3.0 * y)


def manufactured_source_derivs(x, y, alpha):
    """The six planes f, f_x, f_y, f_xx, f_xy, f_yy of manufactured_source (input data for the
    volume local part at the volume nodes)."""
    c = 13.0 + alpha * alpha
    s2, c2 = np.sin(2.0 * x), np.cos(2.0 * x)
    s3, c3 = np.sin(3.0 * y), np.cos(3.0 * y)
    return np.stack([c * s2 * c3, 2 * c * c2 * c3, -3 * c * s2 * s3, -4 * c * s2 * c3,
                     -6 * c * c2 * s3, -9 * c * s2 * c3])


def inside_starfish(curve, x, y):
    """Points strictly inside the star-shaped curve (polar test |x| < r(theta))."""
    return np.hypot(x, y) < curve.radius(np.arctan2(y, x))


def config_small(alpha=10.0, seed=0, n_panels=32, n_vol=2048, n_trg=2048):
    """512 boundary nodes (32 panels x 16 GL) on r = 1 + 0.3 cos 5t, ~2048 volume nodes with
    f = exp(-|x|^2/0.1), 2048 uniform targets in [-1.5, 1.5]^2."""
    rng = np.random.default_rng(seed)
    curve = Starfish()
    bx, by, bw, bt = boundary_nodes(curve, n_panels, 16)
    vx, vy, vw, dx = volume_nodes(curve, n_vol, search=True)
    xt, yt = uniform_targets(n_trg, rng)
    dens = np.concatenate([boundary_density(bt), gaussian_source(vx, vy)])
    return Workload("starfish-2.6k-src-2k-trg", alpha, np.concatenate([bx, vx]),
                    np.concatenate([by, vy]), np.concatenate([bw, vw]), dens, xt, yt,
                    bx.shape[0], dx)


_MESH_CACHE = {}


def config_large(alpha=10.0, seed=0, n_panels=6250, n_vol=1_000_000, n_trg=1_000_000):
    """1e5 boundary nodes on the same starfish, ~1e6 volume nodes with the manufactured source
    f = (13 + alpha^2) sin 2x cos 3y, 1e6 uniform targets in [-1.5, 1.5]^2."""
    rng = np.random.default_rng(seed)
    curve = Starfish()
    key = (n_panels, n_vol)
    if key not in _MESH_CACHE:
        bx, by, bw, bt = boundary_nodes(curve, n_panels, 16)
        vx, vy, vw, dx = volume_nodes(curve, n_vol, search=False)
        _MESH_CACHE[key] = (bx, by, bw, bt, vx, vy, vw, dx)
    bx, by, bw, bt, vx, vy, vw, dx = _MESH_CACHE[key]
    xt, yt = uniform_targets(n_trg, rng)
    dens = np.concatenate([boundary_density(bt), manufactured_source(vx, vy, alpha)])
    return Workload(f"starfish-1.1M-src-1M-trg-alpha{alpha:g}", alpha,
                    np.concatenate([bx, vx]), np.concatenate([by, vy]),
                    np.concatenate([bw, vw]), dens, xt, yt, bx.shape[0], dx)


def random_instance(rng, n_points, alpha):
    """One batch/serving instance: random starfish (3-9 arms, amplitude 0.1-0.4), n_points =
    sources + targets, boundary:volume sources 1:10, targets at the volume nodes."""
    curve = Starfish(1.0, float(rng.uniform(0.1, 0.4)), int(rng.integers(3, 10)),
                     float(rng.uniform(0.0, 2 * math.pi)))
    n_vol = max(30, int(round(n_points * 10 / 21)))
    n_bdry = max(16, int(round(n_points / 21)))
    n_panels = max(1, n_bdry // 16)
    bx, by, bw, bt = boundary_nodes(curve, n_panels, 16)
    vx, vy, vw, dx = volume_nodes(curve, n_vol, search=False)
    dens = np.concatenate([boundary_density(bt), manufactured_source(vx, vy, alpha)])
    return Workload(f"random-starfish-{n_points}", alpha, np.concatenate([bx, vx]),
                    np.concatenate([by, vy]), np.concatenate([bw, vw]), dens,
                    vx.copy(), vy.copy(), bx.shape[0], dx)


def batch_instances(n_inst=256, seed=0, n_lo=1e3, n_hi=2e5, a_lo=1.0, a_hi=300.0):
    """Uneven batch: point counts log-uniform in [n_lo, n_hi], alpha log-uniform in [a_lo, a_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        alpha = math.exp(rng.uniform(math.log(a_lo), math.log(a_hi)))
        out.append(random_instance(rng, n, alpha))
    return out


def rothe_stream(n_req=20000, rate=2000.0, n_geom=64, seed=0, n_lo=1e3, n_hi=1e6,
                 dt_lo=1e-4, dt_hi=1e-1):
    """Request stream for Rothe time stepping.

    n_geom simulations, each a random starfish geometry with a point count log-uniform in
    [n_lo, n_hi] and its own time step dt log-uniform in [dt_lo, dt_hi] (alpha = dt^{-1/2},
    fixed for the simulation).  Requests arrive as a Poisson process of the given rate; each is
    one time step of one simulation (new strengths on that resident geometry).

    Returns (geometries, requests): geometries[g].alpha is its alpha; requests are dicts
    {t_arrive, geom, seed}.
    """
    rng = np.random.default_rng(seed)
    geoms = []
    for g in range(n_geom):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        dt = math.exp(rng.uniform(math.log(dt_lo), math.log(dt_hi)))
        geoms.append(random_instance(rng, n, 1.0 / math.sqrt(dt)))
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    reqs = []
    for i in range(n_req):
        reqs.append(dict(t_arrive=float(t[i]), geom=int(rng.integers(0, n_geom)),
                         seed=int(rng.integers(0, 2 ** 31))))
    return geoms, reqs


def strengths_for(work: Workload, alpha: float, seed: int):
    """New per-step strengths on a resident geometry: the manufactured source at this alpha on
    the volume nodes, plus a seeded smooth random density on the boundary."""
    rng = np.random.default_rng(seed)
    nb = work.n_bdry
    t = np.arctan2(work.ys[:nb], work.xs[:nb])
    c = rng.normal(size=4)
    sig = c[0] * np.cos(3 * t) + c[1] * np.sin(t) + c[2] * np.cos(2 * t) + c[3]
    f = manufactured_source(work.xs[nb:], work.ys[nb:], alpha)
    return np.concatenate([sig, f])
