"""CPU-side checks of the C ABI: the library loads, exports every declared symbol, validates its
arguments, and chooses the parameters the paper's rules give (compared with the oracle's own
statement of those rules).  No CUDA call is made here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle.params as OP
import paper_2606_28865_b300 as yk
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"YK_API\s+[\w\s\*]+?\b(yk_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert "yk_plan" in names and "yk_eval_longrange" in names and len(names) >= 10
    lib = ctypes.CDLL(yk.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("alpha", [10.0, 0.5, 200.0])
def test_plan_parameters_follow_the_rules(alpha):
    w = W.config_small()
    # the untruncated kernel's rules (the truncated kernel has its own test)
    info = yk.plan_params(alpha, w.n_src, w.n_trg, h_vol=w.h_vol, tol=1e-10, truncate=1)
    eps = 1e-10 / 4
    delta = OP.delta_from_mesh(alpha, w.h_vol)
    assert info["delta"] == pytest.approx(delta, rel=1e-14)
    assert info["kmax"] == pytest.approx(OP.kmax_relative(alpha, delta, eps), rel=1e-10)
    assert info["period"] == pytest.approx(3.0 + OP.r_tol(alpha, delta, eps), rel=1e-5)
    M = OP.modes(info["kmax"], info["period"])
    assert info["n_modes"] == M
    n = info["n_grid"]
    assert n >= 2 * (2 * M + 1) and n % 2 == 0 and n % info["tile"] == 0
    assert info["tile"] >= info["w"] and n >= 2 * info["tile"]
    assert info["w"] == math.ceil(math.log10(1 / eps)) + 1
    assert info["h"] == pytest.approx(info["period"] / n, rel=1e-15)


def test_explicit_parameters_are_used():
    info = yk.plan_params(10.0, delta=0.0167, kmax=30.0, period=6.0, tile=32)
    assert info["delta"] == 0.0167 and info["kmax"] == 30.0 and info["period"] == 6.0
    assert info["n_modes"] == math.ceil(30.0 * 6.0 / (2 * math.pi)) and info["tile"] == 32


def test_paper_kmax_rule_and_zero_case():
    alpha, tol = 200.0, 1e-6
    eps = tol / 4
    delta = 1.01 * math.log(1 / eps) / alpha ** 2
    info = yk.plan_params(alpha, delta=delta, tol=tol, kmax_rule=1)
    assert info["kmax"] == 0.0 and info["n_grid"] == 0
    info = yk.plan_params(10.0, delta=0.0167, tol=tol, kmax_rule=1)
    assert info["kmax"] == pytest.approx(OP.kmax_paper(10.0, 0.0167, eps), rel=1e-14)


@pytest.mark.parametrize("alpha,delta", [(10.0, 0.0167), (10.0, 3.93e-5), (1.0, 3.93e-5),
                                         (100.0, 3.82e-5)])
def test_double_layer_cutoff_rules(alpha, delta):
    # opts.dlp: k_max also meets eq. kmax_dlp (relative reading, or as printed with kmax_rule=1)
    eps = 1e-10 / 4
    info = yk.plan_params(alpha, delta=delta, tol=1e-10, dlp=True)
    ref = max(OP.kmax_relative(alpha, delta, eps), OP.kmax_dlp_relative(alpha, delta, eps))
    assert info["kmax"] == pytest.approx(ref, rel=1e-8)
    info = yk.plan_params(alpha, delta=delta, tol=1e-10, dlp=True, kmax_rule=1)
    ref = max(OP.kmax_paper(alpha, delta, eps), OP.kmax_dlp_paper(alpha, delta, eps))
    assert info["kmax"] == pytest.approx(ref, rel=1e-12)
    plain = yk.plan_params(alpha, delta=delta, tol=1e-10)
    assert info["kmax"] >= plain["kmax"]
    assert info["w"] == plain["w"] + 1   # one more digit of window for the gradient spread


def test_truncated_kernel_parameters():
    # small alpha: the kernel is cut at the box diagonal D with a smooth step of width 12 s,
    # s = 20 / k_max, and the period only exceeds the span by D + 12 s
    eps = 1e-10 / 4
    for alpha in (1.0, 0.5, 3.0):
        delta = 3.45e-5
        info = yk.plan_params(alpha, delta=delta, tol=1e-10)
        kmax = OP.kmax_relative(alpha, delta, eps)
        r1 = math.hypot(3.0, 3.0) + 12 * 20 / kmax
        assert info["truncated"] == 1
        assert info["r_support"] == pytest.approx(r1, rel=1e-12)
        assert info["period"] == pytest.approx(3.0 + r1, rel=1e-12)
        # automatic mode truncates because the decay length is the longer margin
        assert 3.0 + OP.r_tol(alpha, delta, eps) > info["period"]
    plain = yk.plan_params(3.0, delta=3.45e-5, tol=1e-10, truncate=1)
    trunc = yk.plan_params(3.0, delta=3.45e-5, tol=1e-10)
    assert plain["truncated"] == 0 and plain["period"] > trunc["period"]
    assert plain["kmax"] == trunc["kmax"]
    # large alpha: the decay length is shorter, so automatic mode keeps the plain kernel
    info = yk.plan_params(10.0, delta=3.45e-5, tol=1e-10)
    assert info["truncated"] == 0
    forced = yk.plan_params(10.0, delta=3.45e-5, tol=1e-10, truncate=2)
    assert forced["truncated"] == 1 and forced["period"] > info["period"]
    # an explicit period keeps the plain kernel unless truncation is forced
    assert yk.plan_params(1.0, delta=3.45e-5, tol=1e-10, period=30.0)["truncated"] == 0
    with pytest.raises(yk.YkError) as ei:
        yk.plan_params(1.0, delta=3.45e-5, tol=1e-10, period=5.0, truncate=2)
    assert ei.value.status == yk.YK_ERR_ARG
    with pytest.raises(yk.YkError) as ei:
        yk.plan_params(1.0, delta=3.45e-5, tol=1e-10, truncate=3)
    assert ei.value.status == yk.YK_ERR_ARG


@pytest.mark.parametrize("kw,status", [
    (dict(alpha=0.0, delta=0.01), yk.YK_ERR_ARG),
    (dict(alpha=-1.0, delta=0.01), yk.YK_ERR_ARG),
    (dict(alpha=10.0, delta=0.01, tol=0.0), yk.YK_ERR_ARG),
    (dict(alpha=10.0, delta=0.01, tol=1.5), yk.YK_ERR_ARG),
    (dict(alpha=10.0), yk.YK_ERR_ARG),                      # neither delta nor h_vol
    (dict(alpha=10.0, delta=0.01, box=(1, 0, 0, 1)), yk.YK_ERR_ARG),
    (dict(alpha=10.0, delta=0.01, period=2.0), yk.YK_ERR_ARG),  # period below the span
    (dict(alpha=10.0, delta=0.01, kmax_rule=3), yk.YK_ERR_ARG),
    (dict(alpha=0.01, delta=1e-6), yk.YK_ERR_UNSUPPORTED),  # grid beyond the supported size
])
def test_argument_validation(kw, status):
    alpha = kw.pop("alpha")
    with pytest.raises(yk.YkError) as ei:
        yk.plan_params(alpha, **kw)
    assert ei.value.status == status
    assert len(str(ei.value)) > 20


def test_predicted_memory_grows_with_points():
    a = yk.plan_params(10.0, 1000, 1000, delta=0.0167)["device_bytes"]
    b = yk.plan_params(10.0, 2000, 1000, delta=0.0167)["device_bytes"]
    c = yk.plan_params(10.0, 1000, 2000, delta=0.0167)["device_bytes"]
    assert b > a and c > a


def test_fp32c_parameters():
    w = W.config_small()
    info = yk.plan_params(10.0, w.n_src, w.n_trg, h_vol=w.h_vol, tol=1e-6,
                          precision=yk.YK_FP32C)
    eps = 1e-6 / 4
    assert info["precision"] == yk.YK_FP32C and info["w"] == math.ceil(math.log10(1 / eps)) + 1
    f64 = yk.plan_params(10.0, w.n_src, w.n_trg, h_vol=w.h_vol, tol=1e-6)
    assert f64["n_grid"] == info["n_grid"] and f64["device_bytes"] > info["device_bytes"]
    with pytest.raises(yk.YkError):
        yk.plan_params(10.0, delta=0.01, precision=7)


def test_tuned_tile_cache_roundtrip(tmp_path):
    # a cached tile steers the plan's choice to the admissible divisor nearest to it
    yk.tune_cache_clear()
    base = yk.plan_params(10.0, 100000, 100000, delta=3.9e-5, tol=1e-10)
    n, w = base["n_grid"], base["w"]
    # FP64 plans with double-float arithmetic take tiles of at most 32 cells, by default the
    # largest admissible one up to 24
    divisors = [t for t in range(w, 33) if n % t == 0 and n >= 2 * t]
    default = max(t for t in divisors if t <= 24)
    assert base["tile"] == default
    want = max(divisors) if max(divisors) != default else min(divisors)
    import math as _m
    dens = 100000 / (n * n)
    band = lambda v: int(_m.floor(2 * _m.log2(v) + 0.5))
    f = tmp_path / "tune.txt"
    f.write_text(f"# precision w n_band density_band tile\n0 {w} {band(n)} {band(dens)} {want}\n")
    yk.tune_cache_load(str(f))
    tuned = yk.plan_params(10.0, 100000, 100000, delta=3.9e-5, tol=1e-10, use_tuned=True,
                           n_src_hint=100000)
    assert tuned["tile"] == want and tuned["n_grid"] == n
    untuned = yk.plan_params(10.0, 100000, 100000, delta=3.9e-5, tol=1e-10)
    assert untuned["tile"] == default
    g = tmp_path / "saved.txt"
    yk.tune_cache_save(str(g))
    assert f"{want}" in g.read_text().split("\n")[1]
    yk.tune_cache_clear()
    assert yk.plan_params(10.0, 100000, 100000, delta=3.9e-5, tol=1e-10, use_tuned=True,
                          n_src_hint=100000)["tile"] == default


def test_launch_shape_options_are_checked_and_reported():
    """The spread's warps per CTA and sources per batch and the interpolation's threads per CTA:
    defaults, explicit values reported back, and out-of-range values refused."""
    import paper_2606_28865_b300 as yk
    d = yk.plan_params(10.0, delta=0.0167)
    assert (d["spread_warps"], d["spread_batch"], d["interp_threads"]) == (4, 16, 256)
    f = yk.plan_params(10.0, delta=0.0167, tol=1e-6, precision=yk.YK_FP32C)
    assert (f["spread_warps"], f["spread_batch"], f["interp_threads"]) == (4, 32, 256)
    e = yk.plan_params(10.0, delta=0.0167, spread_warps=2, spread_batch=8, interp_threads=128)
    assert (e["spread_warps"], e["spread_batch"], e["interp_threads"]) == (2, 8, 128)
    for bad in (dict(spread_warps=5), dict(spread_batch=32), dict(interp_threads=512),
                dict(spread_warps=-1), dict(tile=64)):
        with pytest.raises(yk.YkError) as ei:
            yk.plan_params(10.0, delta=0.0167, **bad)
        assert ei.value.status == yk.YK_ERR_ARG, bad
    with pytest.raises(yk.YkError):
        yk.plan_params(10.0, delta=0.0167, tol=1e-6, precision=yk.YK_FP32C, spread_batch=4)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6)])
def test_targets_tile_edge_apart_from_the_spread_tile(prec, tol):
    """The targets' tiles (binning and interpolation) take their own edge: by default the
    largest admissible divisor of n up to 32, else the caller's; the all-FP64 path keeps one edge."""
    import paper_2606_28865_b300 as yk
    d = yk.plan_params(10.0, 100000, 100000, delta=3.9e-5, tol=tol, precision=prec)
    n, w = d["n_grid"], d["w"]
    edges = [t for t in range(w, 33) if n % t == 0 and n >= 2 * t]
    assert d["interp_tile"] == max(edges)
    for ti in edges:
        e = yk.plan_params(10.0, delta=3.9e-5, tol=tol, precision=prec, interp_tile=ti)
        assert e["interp_tile"] == ti and e["tile"] == d["tile"]
    # the targets' tile counters are part of the predicted footprint
    small = yk.plan_params(10.0, 0, 0, delta=3.9e-5, tol=tol, precision=prec,
                           interp_tile=min(edges))["device_bytes"]
    large = yk.plan_params(10.0, 0, 0, delta=3.9e-5, tol=tol, precision=prec,
                           interp_tile=max(edges))["device_bytes"]
    assert small > large or len(edges) == 1
    bad = [t for t in range(w, 33) if n % t] + [33, -1]
    for ti in bad[:3] + bad[-2:]:
        with pytest.raises(yk.YkError) as ei:
            yk.plan_params(10.0, delta=3.9e-5, tol=tol, precision=prec, interp_tile=ti)
        assert ei.value.status == yk.YK_ERR_ARG, ti
    f = yk.plan_params(10.0, delta=3.9e-5, tol=tol, fft_fp64=True)
    assert f["interp_tile"] == f["tile"]
    with pytest.raises(yk.YkError):
        yk.plan_params(10.0, delta=3.9e-5, tol=tol, fft_fp64=True, interp_tile=edges[0])
