"""B300-native long-range (history) evaluator for the 2D modified Helmholtz equation.

Thin Python binding over the C ABI of ``include/yk.h`` (``libyk.so``, built in-tree by
``paper_2606_28865_b300/build.py``).  It only marshals arguments: every step of the evaluation
runs in the library's CUDA kernels.  Arrays may be torch tensors (CUDA or CPU, float64,
contiguous) or numpy float64 arrays.  If the library is missing, importing this package fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libyk.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2606_28865_b300/build.py`"
                      " (or __graft_entry__.build()); there is no fallback implementation")

_lib = ctypes.CDLL(LIB_PATH)

YK_OK, YK_ERR_ARG, YK_ERR_OOM, YK_ERR_CUDA, YK_ERR_TIMEOUT, YK_ERR_STATE, YK_ERR_INTERNAL, \
    YK_ERR_UNSUPPORTED = range(8)
YK_FP64, YK_FP32C = 0, 1
YK_PEAK_DF, YK_PEAK_DF_LAZY = 2, 3  # yk_fma_peak: double-float multiply-add chains
_STATUS = {0: "YK_OK", 1: "YK_ERR_ARG", 2: "YK_ERR_OOM", 3: "YK_ERR_CUDA", 4: "YK_ERR_TIMEOUT",
           5: "YK_ERR_STATE", 6: "YK_ERR_INTERNAL", 7: "YK_ERR_UNSUPPORTED"}


class YkError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str | None = None):
        self.status = status
        if msg is None:
            msg = _lib.yk_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")


_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("delta", ctypes.c_double), ("h_vol", ctypes.c_double),
                ("eps_hist", ctypes.c_double), ("box", ctypes.c_double * 4),
                ("kmax", ctypes.c_double), ("kmax_rule", ctypes.c_int),
                ("period", ctypes.c_double), ("tile", ctypes.c_int),
                ("profile", ctypes.c_int), ("stream", ctypes.c_void_p), ("alloc", _ALLOC),
                ("free", _FREE), ("alloc_ctx", ctypes.c_void_p), ("use_tuned", ctypes.c_int),
                ("n_src_hint", ctypes.c_int64), ("fft_fp64", ctypes.c_int), ("dlp", ctypes.c_int),
                ("truncate", ctypes.c_int), ("spread_warps", ctypes.c_int),
                ("spread_batch", ctypes.c_int), ("interp_threads", ctypes.c_int),
                ("interp_tile", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("delta", ctypes.c_double), ("tol", ctypes.c_double),
                ("eps", ctypes.c_double), ("kmax", ctypes.c_double), ("period", ctypes.c_double),
                ("origin", ctypes.c_double * 2), ("h", ctypes.c_double),
                ("n_modes", ctypes.c_int64), ("n_grid", ctypes.c_int64), ("w", ctypes.c_int),
                ("beta", ctypes.c_double), ("tile", ctypes.c_int), ("precision", ctypes.c_int),
                ("device_bytes", ctypes.c_int64), ("truncated", ctypes.c_int),
                ("r_support", ctypes.c_double), ("spread_warps", ctypes.c_int),
                ("spread_batch", ctypes.c_int), ("interp_threads", ctypes.c_int),
                ("interp_tile", ctypes.c_int)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["origin"] = tuple(self.origin)
        return d


_d, _i64, _vp = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p
_lib.yk_opts_default.argtypes = [ctypes.POINTER(Opts)]
_lib.yk_opts_default.restype = None
_lib.yk_last_error.restype = ctypes.c_char_p
_lib.yk_plan.argtypes = [_d, ctypes.POINTER(Opts), ctypes.POINTER(_vp)]
_lib.yk_plan_params.argtypes = [_d, ctypes.POINTER(Opts), _i64, _i64, ctypes.POINTER(Info)]
_lib.yk_set_points.argtypes = [_vp, _i64, _vp, _vp, _vp, _i64, _vp, _vp]
_lib.yk_eval_longrange.argtypes = [_vp, _vp, _vp]
_lib.yk_set_points_dl.argtypes = [_vp, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _i64,
                                  _vp, _vp]
_lib.yk_eval_longrange_dl.argtypes = [_vp, _vp, _vp, _vp]
_lib.yk_sync.argtypes = [_vp]
_lib.yk_stage_times.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
_lib.yk_plan_info.argtypes = [_vp, ctypes.POINTER(Info)]
_lib.yk_destroy.argtypes = [_vp]
_lib.yk_batch_eval.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                               ctypes.c_int]
for _f in ("yk_plan", "yk_plan_params", "yk_set_points", "yk_eval_longrange", "yk_sync",
           "yk_set_points_dl", "yk_eval_longrange_dl",
           "yk_stage_times",
           "yk_plan_info", "yk_destroy", "yk_batch_eval"):
    getattr(_lib, _f).restype = ctypes.c_int


def _check(status: int, where: str):
    if status != YK_OK:
        raise YkError(status, where)


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # numpy-only use
        return None


def _ptr(a, keep: list):
    """Device or host pointer of a float64 contiguous torch tensor or numpy array."""
    if a is None:
        return None
    torch = _torch()
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.float64:
            raise TypeError("tensors must be float64")
        if not a.is_contiguous():
            a = a.contiguous()
        keep.append(a)
        return a.data_ptr() if a.numel() else None
    a = np.ascontiguousarray(a, dtype=np.float64)
    keep.append(a)
    return a.ctypes.data if a.size else None


def _out_ptr(a, keep: list):
    """Pointer of an output array, which the library writes in place: a copy would leave the
    caller's array unchanged, so a non-contiguous or non-float64 output is refused, not copied."""
    if a is None:
        return None
    torch = _torch()
    if torch is not None and isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("outputs must be contiguous float64 tensors (written in place)")
        keep.append(a)
        return a.data_ptr() if a.numel() else None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
            and a.flags.writeable):
        raise TypeError("outputs must be writable C-contiguous float64 numpy arrays")
    keep.append(a)
    return a.ctypes.data if a.size else None


def _dev_ptr(a, keep: list):
    """Pointer of a contiguous float64 tensor on the current CUDA device, with no conversion or
    copy (a copy would be a device allocation, and for an output a silent wrong result)."""
    torch = _torch()
    if torch is None or not isinstance(a, torch.Tensor) or not a.is_cuda:
        raise TypeError("every array must be a CUDA tensor")
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise TypeError("every array must be a contiguous float64 tensor")
    if a.device.index != torch.cuda.current_device():
        raise TypeError(f"tensor on {a.device}, but the current device is "
                        f"cuda:{torch.cuda.current_device()}")
    keep.append(a)
    return a.data_ptr() if a.numel() else None


def _len(a) -> int:
    if a is None:
        return 0
    return int(a.numel()) if hasattr(a, "numel") else int(np.asarray(a).size)


def make_opts(tol=1e-10, precision=YK_FP64, delta=0.0, h_vol=0.0, eps_hist=1e-6,
              box=(-1.5, 1.5, -1.5, 1.5), kmax=0.0, kmax_rule=0, period=0.0, tile=0,
              profile=False, stream=None, use_tuned=False, n_src_hint=0,
              fft_fp64=False, dlp=False, truncate=0, allocator=None, spread_warps=0,
              spread_batch=0, interp_threads=0, interp_tile=0) -> Opts:
    """Plan options.  allocator (optional): an object with alloc(nbytes, stream) -> device
    address (0 when it cannot allocate: the library then returns YK_ERR_OOM) and
    free(address, stream), used for every device buffer of the plan instead of cudaMalloc."""
    o = Opts()
    _lib.yk_opts_default(ctypes.byref(o))
    o.precision = int(precision)
    o.tol = float(tol)
    o.delta = float(delta)
    o.h_vol = float(h_vol)
    o.eps_hist = float(eps_hist)
    for i in range(4):
        o.box[i] = float(box[i])
    o.kmax = float(kmax)
    o.kmax_rule = int(kmax_rule)
    o.period = float(period)
    o.tile = int(tile)
    o.profile = 1 if profile else 0
    o.stream = stream
    o.use_tuned = 1 if use_tuned else 0
    o.n_src_hint = int(n_src_hint)
    o.fft_fp64 = 1 if fft_fp64 else 0
    o.dlp = 1 if dlp else 0
    o.truncate = int(truncate)
    o.spread_warps = int(spread_warps)
    o.spread_batch = int(spread_batch)
    o.interp_threads = int(interp_threads)
    o.interp_tile = int(interp_tile)
    if allocator is not None:
        a_cb = _ALLOC(lambda nbytes, stream, ctx: allocator.alloc(int(nbytes), stream) or None)
        f_cb = _FREE(lambda ptr, stream, ctx: allocator.free(int(ptr), stream))
        o.alloc, o.free = a_cb, f_cb
        o._callbacks = (a_cb, f_cb)  # the plan holds its options: the callbacks stay alive
    return o


def plan_params(alpha: float, n_src: int = 0, n_trg: int = 0, **opts) -> dict:
    """Parameters (and predicted device bytes) of a plan, without touching the GPU."""
    o = make_opts(**opts)
    info = Info()
    _check(_lib.yk_plan_params(float(alpha), ctypes.byref(o), int(n_src), int(n_trg),
                               ctypes.byref(info)), "yk_plan_params")
    return info.as_dict()


def _current_stream():
    torch = _torch()
    if torch is not None and torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None


class Plan:
    """One (alpha, box, tolerance) evaluation plan with resident device buffers."""

    def __init__(self, alpha: float, stream=None, **opts):
        if stream is None:
            stream = _current_stream()
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._opts = make_opts(stream=stream, **opts)
        h = _vp()
        _check(_lib.yk_plan(float(alpha), ctypes.byref(self._opts), ctypes.byref(h)), "yk_plan")
        self._h = h
        self.n_src = 0
        self.n_dip = 0
        self.n_trg = 0

    @property
    def handle(self):
        return self._h

    @property
    def info(self) -> dict:
        info = Info()
        _check(_lib.yk_plan_info(self._h, ctypes.byref(info)), "yk_plan_info")
        return info.as_dict()

    def set_points(self, xs, ys, w, xt, yt, dipoles=None):
        """Charges (xs, ys, w), targets (xt, yt) and optionally double-layer nodes
        dipoles = (xd, yd, wd, nx, ny) (plan created with dlp=True)."""
        keep = []
        ns, nt = _len(xs), _len(xt)
        if _len(ys) != ns or _len(w) != ns or _len(yt) != nt:
            raise ValueError("coordinate/weight lengths differ")
        if dipoles is None:
            _check(_lib.yk_set_points(self._h, ns, _ptr(xs, keep), _ptr(ys, keep), _ptr(w, keep),
                                      nt, _ptr(xt, keep), _ptr(yt, keep)), "yk_set_points")
            nd = 0
        else:
            xd, yd, wd, nx, ny = dipoles
            nd = _len(xd)
            if any(_len(a) != nd for a in (yd, wd, nx, ny)):
                raise ValueError("dipole array lengths differ")
            _check(_lib.yk_set_points_dl(self._h, ns, _ptr(xs, keep), _ptr(ys, keep),
                                         _ptr(w, keep), nd, _ptr(xd, keep), _ptr(yd, keep),
                                         _ptr(wd, keep), _ptr(nx, keep), _ptr(ny, keep), nt,
                                         _ptr(xt, keep), _ptr(yt, keep)), "yk_set_points_dl")
        self._keep_points = keep
        self.n_src, self.n_dip, self.n_trg = ns, nd, nt

    def eval(self, density, out=None, mu=None):
        """u at the targets; `out` (same kind of array as `density` by default) is written.
        mu: double-layer density at the dipole nodes (required when the points include them).
        Device and page-locked (pinned) host arrays are used asynchronously: `out` is valid after
        sync(); pageable host arrays (numpy) are complete on return."""
        if _len(density) != self.n_src:
            raise ValueError("density length differs from the number of sources")
        if mu is not None and _len(mu) != self.n_dip:
            raise ValueError("mu length differs from the number of dipoles")
        torch = _torch()
        ref = density if self.n_src or mu is None else mu
        if out is None:
            if torch is not None and isinstance(ref, torch.Tensor):
                out = torch.empty(self.n_trg, dtype=torch.float64, device=ref.device)
            else:
                out = np.empty(self.n_trg, dtype=np.float64)
        keep = []
        if mu is None:
            _check(_lib.yk_eval_longrange(self._h, _ptr(density, keep), _out_ptr(out, keep)),
                   "yk_eval_longrange")
        else:
            _check(_lib.yk_eval_longrange_dl(self._h, _ptr(density, keep), _ptr(mu, keep),
                                             _out_ptr(out, keep)), "yk_eval_longrange_dl")
        self._keep_eval = keep
        return out

    def sync(self):
        _check(_lib.yk_sync(self._h), "yk_sync")

    STAGES = ("bin_src", "bin_trg", "spread", "row_fwd", "columns", "row_inv", "interp")

    def stage_times(self) -> dict:
        """Device ms of each stage's latest run (plan created with profile=True)."""
        ms = (ctypes.c_double * len(self.STAGES))()
        _check(_lib.yk_stage_times(self._h, ms), "yk_stage_times")
        return {k: (v if v >= 0 else None) for k, v in zip(self.STAGES, ms)}

    def close(self):
        if getattr(self, "_h", None):
            _lib.yk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchOpts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("use_graph", ctypes.c_int),
                ("spin_limit", ctypes.c_int64), ("inject_stall", ctypes.c_int)]


_lib.yk_batch_opts_default.argtypes = [ctypes.POINTER(BatchOpts)]
_lib.yk_batch_opts_default.restype = None
_lib.yk_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(BatchOpts),
                                 ctypes.POINTER(_vp)]
_lib.yk_batch_run.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]
_lib.yk_batch_set_plans.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int]
_lib.yk_batch_sync.argtypes = [_vp]
_lib.yk_batch_destroy.argtypes = [_vp]
for _f in ("yk_batch_create", "yk_batch_set_plans", "yk_batch_run", "yk_batch_sync",
           "yk_batch_destroy"):
    getattr(_lib, _f).restype = ctypes.c_int


class Batch:
    """Many plans evaluated in one persistent launch (captured once in a CUDA graph)."""

    def __init__(self, plans, use_graph=True, spin_limit=0, inject_stall=False, stream=None):
        o = BatchOpts()
        _lib.yk_batch_opts_default(ctypes.byref(o))
        if stream is None:
            stream = _current_stream()
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        o.stream = stream
        o.use_graph = 1 if use_graph else 0
        o.spin_limit = int(spin_limit)
        o.inject_stall = 1 if inject_stall else 0
        self.plans = list(plans)
        hp = (_vp * len(self.plans))(*[p.handle for p in self.plans])
        h = _vp()
        _check(_lib.yk_batch_create(hp, len(self.plans), ctypes.byref(o), ctypes.byref(h)),
               "yk_batch_create")
        self._h = h

    def set_plans(self, plans):
        """Re-target the batch at other plans (its device buffers are reused)."""
        self.plans = list(plans)
        hp = (_vp * len(self.plans))(*[p.handle for p in self.plans])
        _check(_lib.yk_batch_set_plans(self._h, hp, len(self.plans)), "yk_batch_set_plans")

    def run(self, densities, outs):
        n = len(self.plans)
        keep = []
        dp = (_vp * n)(*[_ptr(d, keep) for d in densities])
        up = (_vp * n)(*[_out_ptr(u, keep) for u in outs])
        _check(_lib.yk_batch_run(self._h, dp, up), "yk_batch_run")
        self._keep = keep
        return outs

    def sync(self):
        _check(_lib.yk_batch_sync(self._h), "yk_batch_sync")

    def close(self):
        if getattr(self, "_h", None):
            _lib.yk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_eval(plans, densities, outs):
    """Evaluate several plans in one submission (each plan's points already set)."""
    n = len(plans)
    keep = []
    hp = (_vp * n)(*[p.handle for p in plans])
    dp = (_vp * n)(*[_ptr(d, keep) for d in densities])
    up = (_vp * n)(*[_out_ptr(u, keep) for u in outs])
    _check(_lib.yk_batch_eval(hp, dp, up, n), "yk_batch_eval")
    return outs


_lib.yk_slp_local.argtypes = [_d, _d, _i64, ctypes.c_int, _vp, _vp, _vp, _i64, _vp, _vp, _vp,
                              _vp]
_lib.yk_slp_local.restype = ctypes.c_int


def slp_local(alpha, delta_star, xb, yb, sigma, xt, yt, q=16, out=None, stream=None):
    """Single-layer local asymptotic part at the targets (device float64 tensors); the boundary
    as panels of q Gauss-Legendre nodes, counter-clockwise (see yk_slp_local)."""
    torch = _torch()
    nb, nt = _len(xb), _len(xt)
    if nb % q or _len(yb) != nb or _len(sigma) != nb or _len(yt) != nt:
        raise ValueError("boundary arrays must hold n_panels * q values; target lengths differ")
    if out is None:
        out = torch.empty(nt, dtype=torch.float64, device=xt.device)
    if stream is None:
        stream = _current_stream()
    keep = []
    _check(_lib.yk_slp_local(float(alpha), float(delta_star), nb // q, int(q), _ptr(xb, keep),
                             _ptr(yb, keep), _ptr(sigma, keep), nt, _ptr(xt, keep),
                             _ptr(yt, keep), _out_ptr(out, keep), stream), "yk_slp_local")
    return out


_lib.yk_dlp_local.argtypes = list(_lib.yk_slp_local.argtypes)
_lib.yk_dlp_local.restype = ctypes.c_int


def dlp_local(alpha, delta_star, xb, yb, mu, xt, yt, q=16, out=None, stream=None):
    """Double-layer local asymptotic part at the targets (device float64 tensors); the boundary
    as panels of q Gauss-Legendre nodes, counter-clockwise (see yk_dlp_local)."""
    torch = _torch()
    nb, nt = _len(xb), _len(xt)
    if nb % q or _len(yb) != nb or _len(mu) != nb or _len(yt) != nt:
        raise ValueError("boundary arrays must hold n_panels * q values; target lengths differ")
    if out is None:
        out = torch.empty(nt, dtype=torch.float64, device=xt.device)
    if stream is None:
        stream = _current_stream()
    keep = []
    _check(_lib.yk_dlp_local(float(alpha), float(delta_star), nb // q, int(q), _ptr(xb, keep),
                             _ptr(yb, keep), _ptr(mu, keep), nt, _ptr(xt, keep),
                             _ptr(yt, keep), _out_ptr(out, keep), stream), "yk_dlp_local")
    return out


_lib.yk_slp_dyadic.argtypes = [_d, _d, ctypes.c_int, _i64, ctypes.c_int, _vp, _vp, _vp, _i64,
                               _vp, _vp, _vp, _vp]
_lib.yk_slp_dyadic.restype = ctypes.c_int


def slp_dyadic(alpha, delta, J, xb, yb, sigma, xt, yt, q=16, out=None, stream=None):
    """Sum of the J dyadic corrections of the single-layer local part at the targets (device
    float64 tensors; see yk_slp_dyadic)."""
    torch = _torch()
    nb, nt = _len(xb), _len(xt)
    if nb % q or _len(yb) != nb or _len(sigma) != nb or _len(yt) != nt:
        raise ValueError("boundary arrays must hold n_panels * q values; target lengths differ")
    if out is None:
        out = torch.empty(nt, dtype=torch.float64, device=xt.device)
    if stream is None:
        stream = _current_stream()
    keep = []
    _check(_lib.yk_slp_dyadic(float(alpha), float(delta), int(J), nb // q, int(q),
                              _ptr(xb, keep), _ptr(yb, keep), _ptr(sigma, keep), nt,
                              _ptr(xt, keep), _ptr(yt, keep), _out_ptr(out, keep), stream),
           "yk_slp_dyadic")
    return out


_lib.yk_dlp_dyadic.argtypes = list(_lib.yk_slp_dyadic.argtypes)
_lib.yk_dlp_dyadic.restype = ctypes.c_int


def dlp_dyadic(alpha, delta, J, xb, yb, mu, xt, yt, q=16, out=None, stream=None):
    """Sum of the J dyadic corrections of the double-layer local part at the targets (device
    float64 tensors; see yk_dlp_dyadic)."""
    torch = _torch()
    nb, nt = _len(xb), _len(xt)
    if nb % q or _len(yb) != nb or _len(mu) != nb or _len(yt) != nt:
        raise ValueError("boundary arrays must hold n_panels * q values; target lengths differ")
    if out is None:
        out = torch.empty(nt, dtype=torch.float64, device=xt.device)
    if stream is None:
        stream = _current_stream()
    keep = []
    _check(_lib.yk_dlp_dyadic(float(alpha), float(delta), int(J), nb // q, int(q),
                              _ptr(xb, keep), _ptr(yb, keep), _ptr(mu, keep), nt,
                              _ptr(xt, keep), _ptr(yt, keep), _out_ptr(out, keep), stream),
           "yk_dlp_dyadic")
    return out


_lib.yk_vp_local.argtypes = [_d, _d, _i64, ctypes.c_int, _vp, _vp, _i64, _vp, _vp, _vp, _vp,
                             _vp]
_lib.yk_vp_local.restype = ctypes.c_int


def vp_local(alpha, delta_star, xb, yb, xt, yt, fd, q=16, out=None, stream=None):
    """Volume local part at targets in the domain (device float64 tensors).  fd: the six planes
    f, f_x, f_y, f_xx, f_xy, f_yy at the targets, as a (6, n_trg) tensor or a sequence of six
    (see yk_vp_local)."""
    torch = _torch()
    nb, nt = _len(xb), _len(xt)
    if not isinstance(fd, torch.Tensor):
        fd = torch.stack([torch.as_tensor(a, dtype=torch.float64, device=xt.device) for a in fd])
    fd = fd.contiguous()
    if nb % q or _len(yb) != nb or _len(yt) != nt or fd.numel() != 6 * nt:
        raise ValueError("boundary arrays must hold n_panels * q values; fd must hold 6 * n_trg")
    if out is None:
        out = torch.empty(nt, dtype=torch.float64, device=xt.device)
    if stream is None:
        stream = _current_stream()
    keep = []
    _check(_lib.yk_vp_local(float(alpha), float(delta_star), nb // q, int(q), _ptr(xb, keep),
                            _ptr(yb, keep), nt, _ptr(xt, keep), _ptr(yt, keep), _ptr(fd, keep),
                            _out_ptr(out, keep), stream), "yk_vp_local")
    return out


_lib.yk_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
_lib.yk_fma_peak.restype = ctypes.c_int


def fma_peak_tflops(precision=YK_FP64) -> float:
    """Measured FMA throughput of the current CUDA device (TFLOP/s): YK_FP64, YK_FP32C (FP32),
    YK_PEAK_DF / YK_PEAK_DF_LAZY (double-float multiply-add, 2 FP64-equivalent flops each)."""
    v = ctypes.c_double()
    _check(_lib.yk_fma_peak(int(precision), ctypes.byref(v)), "yk_fma_peak")
    return v.value


_lib.yk_eval_longrange_static.argtypes = [_d, ctypes.POINTER(Opts), _i64, _vp, _vp, _vp, _vp,
                                          _i64, _vp, _vp, _vp, ctypes.c_char_p, ctypes.c_size_t]
_lib.yk_eval_longrange_static.restype = ctypes.c_int


def eval_longrange_static(alpha, xs, ys, w, density, xt, yt, out, stream=None, **opts):
    """One evaluation with no device allocation: all scratch is the library's static 32 MiB
    device array.  Every array (including `out`) must be a contiguous float64 CUDA tensor on the
    current device: anything else raises TypeError (converting it would allocate)."""
    if stream is None:
        stream = _current_stream()
    o = make_opts(stream=stream, **opts)
    keep = []
    ptrs = [_dev_ptr(a, keep) for a in (xs, ys, w, density, xt, yt, out)]
    msg = ctypes.create_string_buffer(512)
    st = _lib.yk_eval_longrange_static(float(alpha), ctypes.byref(o), _len(xs), ptrs[0], ptrs[1],
                                       ptrs[2], ptrs[3], _len(xt), ptrs[4], ptrs[5], ptrs[6],
                                       msg, len(msg))
    if st != YK_OK:
        raise YkError(st, "yk_eval_longrange_static", msg.value.decode(errors="replace"))
    return out


class TuneResult(ctypes.Structure):
    _fields_ = [("n_tried", ctypes.c_int), ("tile", ctypes.c_int * 16),
                ("ms", ctypes.c_double * 16), ("best_tile", ctypes.c_int),
                ("best_ms", ctypes.c_double), ("n_grid", ctypes.c_int64),
                ("best_spread_warps", ctypes.c_int), ("best_spread_batch", ctypes.c_int),
                ("best_interp_threads", ctypes.c_int), ("spread_ms", ctypes.c_double),
                ("interp_ms", ctypes.c_double), ("best_interp_tile", ctypes.c_int)]


_lib.yk_autotune.argtypes = [_d, ctypes.POINTER(Opts), _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp,
                             ctypes.POINTER(TuneResult)]
_lib.yk_autotune.restype = ctypes.c_int
_lib.yk_tune_cache_save.argtypes = [ctypes.c_char_p]
_lib.yk_tune_cache_save.restype = ctypes.c_int
_lib.yk_tune_cache_load.argtypes = [ctypes.c_char_p]
_lib.yk_tune_cache_load.restype = ctypes.c_int
_lib.yk_tune_cache_clear.restype = None


def autotune(alpha, xs, ys, w, density, xt, yt, **opts) -> dict:
    """Time every admissible tile edge on these points; the winner is cached for plans created
    with use_tuned=True.  Arrays must be device tensors."""
    o = make_opts(stream=_current_stream(), **opts)
    keep = []
    r = TuneResult()
    _check(_lib.yk_autotune(float(alpha), ctypes.byref(o), _len(xs), _ptr(xs, keep),
                            _ptr(ys, keep), _ptr(w, keep), _ptr(density, keep), _len(xt),
                            _ptr(xt, keep), _ptr(yt, keep), ctypes.byref(r)), "yk_autotune")
    return {"best_tile": r.best_tile, "best_ms": r.best_ms, "n_grid": r.n_grid,
            "tried": {r.tile[k]: r.ms[k] for k in range(r.n_tried)},
            "best_spread_warps": r.best_spread_warps, "best_spread_batch": r.best_spread_batch,
            "best_interp_threads": r.best_interp_threads, "spread_ms": r.spread_ms,
            "interp_ms": r.interp_ms, "best_interp_tile": r.best_interp_tile}


def tune_cache_save(path: str):
    _check(_lib.yk_tune_cache_save(path.encode()), "yk_tune_cache_save")


def tune_cache_load(path: str):
    _check(_lib.yk_tune_cache_load(path.encode()), "yk_tune_cache_load")


def tune_cache_clear():
    _lib.yk_tune_cache_clear()


def loaded_library_path() -> str:
    return LIB_PATH
