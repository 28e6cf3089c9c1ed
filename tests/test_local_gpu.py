"""GPU parity of the single-layer local asymptotic part S_{L,A} (Section 4.1, Lemma, eq.
slp_local1; Section 3.2, closest point) against the oracle (oracle/local.py), which evaluates the
same expansion at the closest point of the analytic curve with the analytic density, while the
GPU works from the panels' Gauss-Legendre nodes only.  Tolerance: max_i |u - u_oracle| <= 1e-10
max_i |u_oracle| (relative L-infinity, as for the history part).
"""
import math

import numpy as np
import pytest

import oracle.local as OL
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _yk():
    import paper_2606_28865_b300 as yk
    return yk


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def near_targets(n, offset_max, seed):
    """points at random curve parameters, moved along the normal by up to +-offset_max, plus
    points on the boundary and points just beyond a given distance"""
    g = OL.StarfishGeom()
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, 2 * np.pi, n)
    p, d1, _ = g.derivs(t)
    nrm = np.hypot(d1[0], d1[1])
    off = rng.uniform(-offset_max, offset_max, n)
    off[: n // 10] = 0.0                                   # on the boundary
    return p[0] + off * d1[1] / nrm, p[1] - off * d1[0] / nrm


def run(n_panels, alpha, dstar, xt, yt):
    yk = _yk()
    curve = W.Starfish()
    xb, yb, _, tb = W.boundary_nodes(curve, n_panels, 16)
    sig = W.boundary_density(tb)
    u = yk.slp_local(alpha, dstar, dev(xb), dev(yb), dev(sig), dev(xt), dev(yt), q=16)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("n_panels,alpha,dstar,off", [(32, 10.0, 1e-4, 0.03), (32, 1.0, 1e-5, 0.03),
                                                      (32, 100.0, 1e-5, 0.02), (128, 10.0, 1e-5, 0.03)])
def test_slp_local_matches_oracle(n_panels, alpha, dstar, off):
    rl = OL.locality_radius(alpha, dstar)
    xt, yt = near_targets(3000, min(off, 0.95 * rl), seed=5)
    u = run(n_panels, alpha, dstar, xt, yt)
    ref = OL.slp_local_starfish(alpha, dstar, OL.StarfishGeom(), OL.starfish_density, xt, yt)
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    assert err <= TOL, f"err={err:.3e}"


# At the concave stretches (curvature 13.9, its peak ~0.03 wide in the curve parameter) the
# 128-panel interpolant's third and fourth derivatives carry the node rounding amplified by the
# differentiation (~2e-8 and ~1e-5 absolute in the curve parameter, reproduced in numpy from the
# rounded nodes alone): the lemma from those derivatives differs from the analytic curve's by
# ~1.2e-11, 1.5e-9 of the largest |D| of targets at 0.3 .. 0.97 of the locality radius (<= 8e-3);
# S_{L,A}, whose delta*^2 term takes gamma0^(3) and gamma0^(4) too, differs by 1.1e-9 of the
# largest |S| of those targets (<= 1.5e-5), also reproduced in numpy from the nodes alone.
TOL_CONCAVE = 3e-9


def test_slp_local_outside_concave_tips_at_the_locality_radius():
    """Targets outside the starfish opposite its concave stretches (radius of curvature ~0.072),
    at 0.3 .. 0.97 of a locality radius of ~0.071: there f' of the closest-point Newton,
    |gamma'|^2 (1 - d kappa), nearly vanishes and its quadratic constant is large, so the
    stopping rule must not leave t short of the root (Section 3.2, closest point; Section 4.1,
    Lemma)."""
    alpha, dstar = 10.0, 3.45e-5
    rl = OL.locality_radius(alpha, dstar)
    g = OL.StarfishGeom()
    rng = np.random.default_rng(17)
    n = 2000
    t = np.pi / 5 + 2 * np.pi * rng.integers(0, 5, n) / 5 + rng.uniform(-0.02, 0.02, n)
    p, d1, _ = g.derivs(t)
    nrm = np.hypot(d1[0], d1[1])
    d = rng.uniform(0.3, 0.97, n) * rl
    xt, yt = p[0] + d * d1[1] / nrm, p[1] - d * d1[0] / nrm      # outward
    # the stretch is concave (the lemma's kappa0 > 0: the boundary bends towards the outward
    # normal), its centre of curvature outside, within 10% of the locality radius
    _, d1v, d2v = g.derivs(np.array([np.pi / 5]))
    kappa = -(d1v[0] * d2v[1] - d1v[1] * d2v[0]) / np.hypot(d1v[0], d1v[1]) ** 3
    assert kappa[0] > 0 and 0.9 * rl < 1 / kappa[0] < 1.1 * rl
    u = run(128, alpha, dstar, xt, yt)
    ref = OL.slp_local_starfish(alpha, dstar, g, OL.starfish_density, xt, yt)
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    assert err <= TOL_CONCAVE, f"err={err:.3e}"


def test_slp_local_far_targets_are_zero():
    alpha, dstar = 10.0, 1e-5
    rl = OL.locality_radius(alpha, dstar)
    g = OL.StarfishGeom()
    rng = np.random.default_rng(8)
    t = rng.uniform(0, 2 * np.pi, 500)
    p, d1, _ = g.derivs(t)
    nrm = np.hypot(d1[0], d1[1])
    s = rng.choice([-1.0, 1.0], 500) * 1.05 * rl
    xt = np.concatenate([p[0] + s * d1[1] / nrm, [2.5, -3.0, 0.0]])
    yt = np.concatenate([p[1] - s * d1[0] / nrm, [0.0, 1.0, 0.0]])
    u = run(32, alpha, dstar, xt, yt)
    assert np.all(u == 0.0)


# On very short panels (the 6,250-panel boundary: 1e-3 of arc length) a panel's own series carries
# the node rounding (1e-16 of |x| ~ 1) amplified by differentiation (~1e-6 of the curvature, the
# fourth derivative lost); the kernels take the derivatives of order >= 2 there from a
# least-squares fit over the neighbouring panels' nodes (a window of 0.006 of the boundary's
# extent), which keeps them to ~1e-11 (curvature) and ~1e-4 (fourth derivatives): the bar is the
# same as for coarse panels.
TOL_SHORT_PANELS = TOL


@pytest.mark.slow
def test_slp_local_config_two_boundary():
    # the bench's boundary: 6,250 panels x 16 nodes, delta* from the volume mesh rule at alpha = 10
    alpha = 10.0
    import oracle.params as OP
    dstar = OP.delta_from_mesh(alpha, 0.004467)
    rl = OL.locality_radius(alpha, dstar)
    xt, yt = near_targets(20000, 0.5 * rl, seed=9)
    u = run(6250, alpha, dstar, xt, yt)
    ref = OL.slp_local_starfish(alpha, dstar, OL.StarfishGeom(), OL.starfish_density, xt, yt)
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    print(f"slp 6250 panels err={err:.3e}")
    assert err <= TOL_SHORT_PANELS


def test_slp_local_arguments():
    yk = _yk()
    x = dev(np.zeros(32))
    with pytest.raises(yk.YkError) as ei:
        yk.slp_local(-1.0, 1e-4, x, x, x, dev(np.zeros(3)), dev(np.zeros(3)), q=16)
    assert ei.value.status == yk.YK_ERR_ARG
    with pytest.raises(ValueError):
        yk.slp_local(1.0, 1e-4, x, x, x, dev(np.zeros(3)), dev(np.zeros(3)), q=5)


# ------------------------------------------------------------------------------------------------
# double-layer local part D_{L,A} (the double-layer lemma, eq. dlp_local1, through delta*^2; the
# oracle's readings: source-point normal derivative, the gamma^(4) factor 3 Q0 + P2)

def run_dla(n_panels, alpha, dstar, xt, yt):
    yk = _yk()
    curve = W.Starfish()
    xb, yb, _, tb = W.boundary_nodes(curve, n_panels, 16)
    mu = W.boundary_density(tb)
    u = yk.dlp_local(alpha, dstar, dev(xb), dev(yb), dev(mu), dev(xt), dev(yt), q=16)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("n_panels,alpha,dstar,off", [(32, 10.0, 1e-4, 0.03), (32, 1.0, 1e-5, 0.03),
                                                      (32, 100.0, 1e-5, 0.02), (128, 10.0, 1e-5, 0.03)])
def test_dla_local_matches_oracle(n_panels, alpha, dstar, off):
    rl = OL.locality_radius(alpha, dstar)
    xt, yt = near_targets(3000, min(off, 0.95 * rl), seed=5)
    u = run_dla(n_panels, alpha, dstar, xt, yt)
    ref = OL.dla_local_starfish(alpha, dstar, OL.StarfishGeom(), OL.starfish_density4, xt, yt)
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    assert err <= TOL, f"err={err:.3e}"




def test_dla_local_concave_tips_and_far_targets():
    """Outside the concave stretches up to 0.97 of the locality radius (as for S_{L,A}), and
    targets just beyond the radius or far away (zero)."""
    alpha, dstar = 10.0, 3.45e-5
    rl = OL.locality_radius(alpha, dstar)
    g = OL.StarfishGeom()
    rng = np.random.default_rng(23)
    n = 2000
    t = np.pi / 5 + 2 * np.pi * rng.integers(0, 5, n) / 5 + rng.uniform(-0.02, 0.02, n)
    p, d1, _ = g.derivs(t)
    nrm = np.hypot(d1[0], d1[1])
    d = rng.uniform(0.3, 0.97, n) * rl
    xt, yt = p[0] + d * d1[1] / nrm, p[1] - d * d1[0] / nrm
    u = run_dla(128, alpha, dstar, xt, yt)
    ref = OL.dla_local_starfish(alpha, dstar, g, OL.starfish_density4, xt, yt)
    assert np.max(np.abs(u - ref)) / np.max(np.abs(ref)) <= TOL_CONCAVE
    s = rng.choice([-1.0, 1.0], 500) * 1.05 * rl
    tf = rng.uniform(0, 2 * np.pi, 500)
    p, d1, _ = g.derivs(tf)
    nrm = np.hypot(d1[0], d1[1])
    xf = np.concatenate([p[0] + s * d1[1] / nrm, [2.5, -3.0, 0.0]])
    yf = np.concatenate([p[1] - s * d1[0] / nrm, [0.0, 1.0, 0.0]])
    assert np.all(run_dla(32, alpha, dstar, xf, yf) == 0.0)


def test_dla_local_jump_across_the_boundary():
    """The double layer's jump (the lemma's U_0 term): just outside minus just inside is mu0, and
    a target on the boundary takes the mean of the two (the corollary's value)."""
    alpha, dstar = 10.0, 1e-4
    g = OL.StarfishGeom()
    t = np.linspace(0.05, 2 * np.pi - 0.05, 400)
    p, d1, _ = g.derivs(t)
    nrm = np.hypot(d1[0], d1[1])
    eps = 1e-8 * math.sqrt(dstar)
    xo, yo = p[0] + eps * d1[1] / nrm, p[1] - eps * d1[0] / nrm
    xi, yi = p[0] - eps * d1[1] / nrm, p[1] + eps * d1[0] / nrm
    uo, ui, ub = (run_dla(128, alpha, dstar, x, y) for x, y in ((xo, yo), (xi, yi), (p[0], p[1])))
    mu0 = W.boundary_density(t)
    assert np.max(np.abs(uo - ui - mu0)) <= 1e-7 * np.max(np.abs(mu0))   # O(eps / sqrt(ds))
    assert np.max(np.abs(ub - 0.5 * (uo + ui))) <= 1e-7 * np.max(np.abs(mu0))


@pytest.mark.slow
def test_dla_local_config_two_boundary():
    # the bench's boundary: 6,250 panels x 16 nodes (derivatives from the window fits)
    alpha = 10.0
    import oracle.params as OP
    dstar = OP.delta_from_mesh(alpha, 0.004467)
    rl = OL.locality_radius(alpha, dstar)
    xt, yt = near_targets(20000, 0.5 * rl, seed=9)
    u = run_dla(6250, alpha, dstar, xt, yt)
    ref = OL.dla_local_starfish(alpha, dstar, OL.StarfishGeom(), OL.starfish_density4, xt, yt)
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    print(f"dla 6250 panels err={err:.3e}")
    assert err <= TOL_SHORT_PANELS


def test_dla_local_arguments():
    yk = _yk()
    x = dev(np.zeros(32))
    with pytest.raises(yk.YkError) as ei:
        yk.dlp_local(1.0, -1e-4, x, x, x, dev(np.zeros(3)), dev(np.zeros(3)), q=16)
    assert ei.value.status == yk.YK_ERR_ARG
    with pytest.raises(ValueError):
        yk.dlp_local(1.0, 1e-4, x, x, x, dev(np.zeros(3)), dev(np.zeros(3)), q=5)


# ------------------------------------------------------------------------------------------------
# volume local part V_L (Lemma for V_L, eq. vp_local1; eq. vp_local3 away from the boundary)

def inside_targets(n, rl, seed):
    """near targets moved inward by up to 0.95 r_loc (a tenth on the boundary) and interior
    targets (polar radius < 0.5, the starfish radius is >= 0.7)"""
    g = OL.StarfishGeom()
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, 2 * np.pi, n)
    p, d1, _ = g.derivs(t)
    nrm = np.hypot(d1[0], d1[1])
    off = rng.uniform(0, 0.95 * rl, n)
    off[: n // 10] = 0.0
    xn, yn = p[0] - off * d1[1] / nrm, p[1] + off * d1[0] / nrm      # inward normal
    rad, th = 0.5 * np.sqrt(rng.uniform(0, 1, n // 3)), rng.uniform(0, 2 * np.pi, n // 3)
    return np.r_[xn, rad * np.cos(th)], np.r_[yn, rad * np.sin(th)]


def run_vp(n_panels, alpha, dstar, xt, yt, fd=None):
    yk = _yk()
    xb, yb, _, _ = W.boundary_nodes(W.Starfish(), n_panels, 16)
    fd = fd or OL.sincos_field()
    planes = np.stack(fd(xt, yt))
    u = yk.vp_local(alpha, dstar, dev(xb), dev(yb), dev(xt), dev(yt), dev(planes), q=16)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("n_panels,alpha,dstar", [(32, 10.0, 1e-4), (32, 1.0, 1e-5),
                                                  (32, 0.1, 1e-5), (32, 100.0, 1e-5),
                                                  (128, 10.0, 1e-5)])
def test_vp_local_matches_oracle(n_panels, alpha, dstar):
    rl = OL.locality_radius(alpha, dstar)
    xt, yt = inside_targets(3000, min(rl, 0.03), seed=6)
    u = run_vp(n_panels, alpha, dstar, xt, yt)
    ref = OL.vp_local_starfish(alpha, dstar, OL.StarfishGeom(), OL.sincos_field(), xt, yt)
    assert np.all(np.isfinite(ref))
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    assert err <= TOL, f"err={err:.3e}"


def test_vp_local_interior_is_the_semigroup_expansion():
    # away from the boundary every target takes eq. vp_local3, here against the oracle's form
    alpha, dstar = 10.0, 1e-5
    rng = np.random.default_rng(2)
    rad, th = 0.5 * np.sqrt(rng.uniform(0, 1, 1000)), rng.uniform(0, 2 * np.pi, 1000)
    xt, yt = rad * np.cos(th), rad * np.sin(th)
    u = run_vp(32, alpha, dstar, xt, yt)
    f, _, _, fxx, _, fyy = OL.sincos_field()(xt, yt)
    ref = OL.vl_interior(alpha, dstar, f, fxx + fyy)
    assert np.max(np.abs(u - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_vp_local_outside_targets_are_reported():
    yk = _yk()
    alpha, dstar = 10.0, 1e-5
    rl = OL.locality_radius(alpha, dstar)
    g = OL.StarfishGeom()
    t = np.array([0.4, 2.2, 4.0])
    p, d1, _ = g.derivs(t)
    nrm = np.hypot(d1[0], d1[1])
    xo, yo = p[0] + 0.5 * rl * d1[1] / nrm, p[1] - 0.5 * rl * d1[0] / nrm   # outward
    xt, yt = np.r_[0.1, xo, 0.0], np.r_[0.2, yo, -0.3]
    xb, yb, _, _ = W.boundary_nodes(W.Starfish(), 32, 16)
    planes = np.stack(OL.sincos_field()(xt, yt))
    out = dev(np.zeros(len(xt)))
    with pytest.raises(yk.YkError) as ei:
        yk.vp_local(alpha, dstar, dev(xb), dev(yb), dev(xt), dev(yt), dev(planes), q=16, out=out)
    assert ei.value.status == yk.YK_ERR_ARG
    u = out.cpu().numpy()
    assert np.all(np.isnan(u[1:4])) and np.isfinite(u[0]) and np.isfinite(u[4])


@pytest.mark.slow
def test_vp_local_config_two_boundary():
    alpha = 10.0
    import oracle.params as OP
    dstar = OP.delta_from_mesh(alpha, 0.004467)
    rl = OL.locality_radius(alpha, dstar)
    xt, yt = inside_targets(20000, rl, seed=10)
    u = run_vp(6250, alpha, dstar, xt, yt)
    ref = OL.vp_local_starfish(alpha, dstar, OL.StarfishGeom(), OL.sincos_field(), xt, yt)
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    print(f"vp 6250 panels err={err:.3e}")
    assert err <= TOL_SHORT_PANELS


def test_vp_local_arguments():
    yk = _yk()
    x = dev(np.zeros(32))
    t3 = dev(np.zeros(3))
    with pytest.raises(yk.YkError) as ei:
        yk.vp_local(0.0, 1e-4, x, x, t3, t3, dev(np.zeros(18)), q=16)
    assert ei.value.status == yk.YK_ERR_ARG
    with pytest.raises(ValueError):
        yk.vp_local(1.0, 1e-4, x, x, t3, t3, dev(np.zeros(12)), q=16)
    # no targets: nothing to do
    e = dev(np.zeros(0))
    assert yk.vp_local(1.0, 1e-4, x, x, e, e, dev(np.zeros(0)), q=16).numel() == 0


# ------------------------------------------------------------------------------------------------
# dyadic corrections of the single-layer local part (eqs. slp_dyad, sld, diffker_s)

def run_dy(n_panels, alpha, delta, J, xt, yt):
    yk = _yk()
    xb, yb, _, tb = W.boundary_nodes(W.Starfish(), n_panels, 16)
    sig = W.boundary_density(tb)
    u = yk.slp_dyadic(alpha, delta, J, dev(xb), dev(yb), dev(sig), dev(xt), dev(yt), q=16)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("n_panels,alpha,delta,J", [(32, 10.0, 1e-4, 3), (32, 1.0, 3e-5, 2),
                                                    (128, 100.0, 1e-4, 3), (32, 10.0, 4e-4, 1)])
def test_slp_dyadic_matches_oracle(n_panels, alpha, delta, J):
    R1 = OL.locality_radius(alpha, delta)
    xt, yt = near_targets(300, min(0.9 * R1, 0.05), seed=12)
    u = run_dy(n_panels, alpha, delta, J, xt, yt)
    ref = OL.slp_dyadic_starfish(alpha, delta, J, OL.StarfishGeom(), OL.starfish_density, xt, yt)
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    assert err <= TOL, f"err={err:.3e}"


def test_slp_dyadic_far_targets_and_arguments():
    yk = _yk()
    u = run_dy(32, 10.0, 1e-4, 3, np.array([0.0, 2.5, -3.0]), np.array([0.0, 0.0, 1.0]))
    assert np.all(u == 0.0)
    x = dev(np.zeros(32))
    with pytest.raises(yk.YkError) as ei:
        yk.slp_dyadic(10.0, 1e-4, 0, x, x, x, dev(np.zeros(3)), dev(np.zeros(3)), q=16)
    assert ei.value.status == yk.YK_ERR_ARG


@pytest.mark.slow
def test_slp_dyadic_config_two_boundary():
    alpha, J = 10.0, 3
    import oracle.params as OP
    delta = OP.delta_from_mesh(alpha, 0.004467)
    R1 = OL.locality_radius(alpha, delta)
    xt, yt = near_targets(200, 0.9 * R1, seed=13)
    u = run_dy(6250, alpha, delta, J, xt, yt)
    ref = OL.slp_dyadic_starfish(alpha, delta, J, OL.StarfishGeom(), OL.starfish_density, xt, yt)
    assert np.max(np.abs(u - ref)) / np.max(np.abs(ref)) <= TOL


def run_dl_dy(n_panels, alpha, delta, J, xt, yt):
    yk = _yk()
    xb, yb, _, tb = W.boundary_nodes(W.Starfish(), n_panels, 16)
    mu = W.boundary_density(tb)
    u = yk.dlp_dyadic(alpha, delta, J, dev(xb), dev(yb), dev(mu), dev(xt), dev(yt), q=16)
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("n_panels,alpha,delta,J", [(32, 10.0, 1e-4, 3), (32, 1.0, 3e-5, 2),
                                                    (128, 100.0, 1e-4, 3)])
def test_dlp_dyadic_matches_oracle(n_panels, alpha, delta, J):
    R1 = OL.locality_radius(alpha, delta)
    xt, yt = near_targets(300, min(0.9 * R1, 0.05), seed=14)
    u = run_dl_dy(n_panels, alpha, delta, J, xt, yt)
    ref = OL.dlp_dyadic_starfish(alpha, delta, J, OL.StarfishGeom(), OL.starfish_density, xt, yt)
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    assert err <= TOL, f"err={err:.3e}"


@pytest.mark.slow
def test_dlp_dyadic_config_two_boundary():
    alpha, J = 10.0, 3
    import oracle.params as OP
    delta = OP.delta_from_mesh(alpha, 0.004467)
    R1 = OL.locality_radius(alpha, delta)
    xt, yt = near_targets(200, 0.9 * R1, seed=15)
    u = run_dl_dy(6250, alpha, delta, J, xt, yt)
    ref = OL.dlp_dyadic_starfish(alpha, delta, J, OL.StarfishGeom(), OL.starfish_density, xt, yt)
    assert np.max(np.abs(u - ref)) / np.max(np.abs(ref)) <= TOL


# ------------------------------------------------------------------------------------------------
# edge cases: the closed-form branch of V_L (c2 >= 0.5), another panel order, targets at panel
# junctions (Newton moves across panel ends), no targets

def test_vp_local_closed_form_branch():
    # alpha sqrt(delta*) = 0.95: the lemma's printed closed forms, not the small-c2 series
    alpha, dstar = 300.0, 1e-5
    rl = OL.locality_radius(alpha, dstar)
    xt, yt = inside_targets(2000, rl, seed=21)
    u = run_vp(32, alpha, dstar, xt, yt)
    ref = OL.vp_local_starfish(alpha, dstar, OL.StarfishGeom(), OL.sincos_field(), xt, yt)
    assert np.max(np.abs(u - ref)) <= TOL * np.max(np.abs(ref))


def test_slp_local_ten_point_panels_and_junctions():
    yk = _yk()
    alpha, dstar, n_panels, q = 10.0, 1e-5, 128, 10
    rl = OL.locality_radius(alpha, dstar)
    xb, yb, _, tb = W.boundary_nodes(W.Starfish(), n_panels, q)
    sig = W.boundary_density(tb)
    # targets off the panel junctions (parameters 2 pi p / n_panels) and at random parameters
    g = OL.StarfishGeom()
    tj = 2 * np.pi * np.arange(n_panels) / n_panels
    p, d1, _ = g.derivs(tj)
    nrm = np.hypot(d1[0], d1[1])
    off = np.linspace(-0.9, 0.9, n_panels) * rl
    xj, yj = p[0] + off * d1[1] / nrm, p[1] - off * d1[0] / nrm
    xr, yr = near_targets(1000, 0.9 * rl, seed=22)
    xt, yt = np.r_[xj, xr], np.r_[yj, yr]
    u = yk.slp_local(alpha, dstar, dev(xb), dev(yb), dev(sig), dev(xt), dev(yt), q=q)
    torch.cuda.synchronize()
    ref = OL.slp_local_starfish(alpha, dstar, g, OL.starfish_density, xt, yt)
    assert np.max(np.abs(u.cpu().numpy() - ref)) <= TOL * np.max(np.abs(ref))


def test_local_parts_without_targets():
    yk = _yk()
    xb, yb, _, tb = W.boundary_nodes(W.Starfish(), 32, 16)
    b = (dev(xb), dev(yb), dev(W.boundary_density(tb)))
    e = dev(np.zeros(0))
    assert yk.slp_local(10.0, 1e-5, *b, e, e, q=16).numel() == 0
    assert yk.slp_dyadic(10.0, 1e-4, 2, *b, e, e, q=16).numel() == 0
    assert yk.dlp_dyadic(10.0, 1e-4, 2, *b, e, e, q=16).numel() == 0
    assert yk.vp_local(10.0, 1e-5, b[0], b[1], e, e, dev(np.zeros(0)), q=16).numel() == 0
