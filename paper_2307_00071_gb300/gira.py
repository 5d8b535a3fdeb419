"""Thin Python binding of libgira (the C ABI in ``include/gira.h``).

Argument marshalling only: every step of the method runs in the CUDA kernels
behind the C ABI.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays;
CUDA tensors are passed as device pointers on torch's current stream, host
arrays as host pointers (the library stages them).  Outputs are allocated on
the same side as ``points``.  There is no CPU fallback: importing this module
raises if the library cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_lib

OK = 0
ERR_INVALID_ARG, ERR_NONFINITE_INPUT, ERR_NOT_PD, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NUMERIC = 1, 2, 3, 4, 5, 6, 7
ERR_BOUNDS = 8   # libraries built with GIRA_DEBUG: a device-side index outside its buffer
INIT_KMEANS, INIT_PARAMS = 0, 1
MAX_K, MAX_K_BATCHED, MAX_K4 = 8192, 1024, 8192


class GiraError(RuntimeError):
    def __init__(self, status: int, message: str, component: int = -1):
        self.status = status
        self.component = component
        super().__init__(f"gira error {status}: {message}")


class FitOpts(C.Structure):
    _fields_ = [("iters", C.c_int), ("tol", C.c_double), ("reg_covar", C.c_double), ("seed", C.c_uint64),
                ("lloyd_iters", C.c_int), ("init_mode", C.c_int)]


class Profile(C.Structure):
    _fields_ = [("calls", C.c_longlong), ("kernel_launches", C.c_longlong), ("estep_launches", C.c_longlong),
                ("estep_ms", C.c_double), ("em_iters", C.c_longlong), ("init_ms", C.c_double), ("em_ms", C.c_double),
                ("total_ms", C.c_double), ("estep_kernel", C.c_char * 128), ("estep_pair_slots", C.c_longlong),
                ("estep_pairs_near", C.c_longlong), ("estep_pairs_live", C.c_longlong)]


def _load():
    # GIRA_DEBUG=1 loads the build with device-side index checks (libgira_debug.so)
    debug = os.environ.get("GIRA_DEBUG", "") not in ("", "0")
    path = build_lib.lib_path(debug)
    if not os.path.exists(path) or build_lib.is_stale(debug):
        path = build_lib.build(debug=debug)   # raises if nvcc fails: no fallback
    lib = C.CDLL(path)
    vp, i64, dp, ip = C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int)
    lib.gira_fit_opts_default.argtypes = [C.POINTER(FitOpts)]
    lib.gira_fit_opts_default.restype = None
    lib.gira_kmeans_init.argtypes = [vp, i64, C.c_int, C.c_uint64, C.c_int, vp, vp, ip, vp]
    lib.gira_gmm_fit.argtypes = [vp, i64, C.c_int, C.POINTER(FitOpts), vp, vp, vp, dp, ip, dp, vp]
    lib.gira_gmm_loglik.argtypes = [vp, i64, C.c_int, vp, vp, vp, dp, vp, vp]
    lib.gira_gmm_loglik_noalloc.argtypes = [vp, i64, C.c_int, vp, vp, vp, dp, vp, vp]
    lib.gira_gmm_loglik_noalloc.restype = C.c_int
    lib.gira_gmm_loglik_grad.argtypes = [vp, i64, C.c_int, vp, vp, vp, vp, dp, vp, vp, vp, vp, vp, vp, vp]
    lib.gira_gmm_fit_batched.argtypes = [vp, vp, C.c_int, vp, C.POINTER(FitOpts), vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gira_gmm_fit_batched.restype = C.c_int
    lib.gira_gmm_loglik_grad_batched.argtypes = [vp, vp, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                                 vp]
    lib.gira_gmm_loglik_grad_batched.restype = C.c_int
    lib.gira_gmm_loglik_grad.restype = C.c_int
    lib.gira_gmm_fit4.argtypes = [vp, i64, C.c_int, C.POINTER(FitOpts), vp, vp, vp, dp, ip, dp, vp]
    lib.gira_gmm_loglik4.argtypes = [vp, i64, C.c_int, vp, vp, vp, dp, vp, vp]
    lib.gira_gmm_conditional4.argtypes = [vp, i64, C.c_int, vp, vp, vp, vp, vp, vp]
    lib.gira_gmm_sample.argtypes = [i64, C.c_int, C.c_int, vp, vp, vp, C.c_uint64, vp, vp, vp]
    lib.gira_gbms.argtypes = [vp, i64, C.c_int, C.c_double, C.c_int, ip, vp, vp, vp]
    lib.gira_test_fail_next_allocations.argtypes = [C.c_int]
    lib.gira_test_fail_next_allocations.restype = None
    lib.gira_test_bounded_wait.argtypes = [C.c_int, C.c_longlong, vp]
    lib.gira_test_bounded_wait.restype = C.c_int
    lib.gira_test_point_order.argtypes = [vp, i64, C.c_int, vp, vp, vp]
    lib.gira_test_point_order.restype = C.c_int
    for f in ("gira_gmm_fit4", "gira_gmm_loglik4", "gira_gmm_conditional4", "gira_gmm_sample", "gira_gbms"):
        getattr(lib, f).restype = C.c_int
    for f in ("gira_kmeans_init", "gira_gmm_fit", "gira_gmm_loglik", "gira_release_workspace"):
        getattr(lib, f).restype = C.c_int
    lib.gira_release_workspace.argtypes = []
    lib.gira_profile_enable.argtypes = [C.c_int]
    lib.gira_profile_enable.restype = None
    lib.gira_profile_read.argtypes = [C.POINTER(Profile), C.c_int]
    lib.gira_profile_read.restype = C.c_int
    lib.gira_last_error_message.restype = C.c_char_p
    lib.gira_last_error_component.restype = C.c_int
    lib.gira_version.restype = C.c_char_p
    return lib


_lib = _load()
LIB_PATH = _lib._name   # the library this process loaded


def _check(status: int):
    if status != OK:
        msg = _lib.gira_last_error_message().decode(errors="replace")
        raise GiraError(status, msg, _lib.gira_last_error_component())


# ----------------------------------------------------------------------------- marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, keepalive, stream) for a torch tensor or numpy array (contiguous float32/int32)."""
    if x is None:
        return None, None, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        stream = None
        if x.is_cuda:
            import torch
            stream = torch.cuda.current_stream(x.device).cuda_stream
        return x.data_ptr(), x, stream
    a = np.ascontiguousarray(x)
    return a.ctypes.data, a, None


def _new(like, shape, dtype):
    if _is_torch(like):
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=tdt, device=like.device)
    return np.empty(shape, dtype=dtype)


def _check_points(points, d: int = 3):
    if points.ndim != 2 or points.shape[1] != d:
        raise ValueError(f"points must be N x {d}")
    dt = points.dtype
    if (_is_torch(points) and str(dt) != "torch.float32") or (not _is_torch(points) and dt != np.float32):
        raise ValueError("points must be float32")
    return int(points.shape[0])


def default_opts() -> FitOpts:
    o = FitOpts()
    _lib.gira_fit_opts_default(C.byref(o))
    return o


def version() -> str:
    return _lib.gira_version().decode()


def gira_profile_enable(on: bool = True, launches: bool = True):
    """Record CUDA events around each call's phases, and with ``launches`` around
    every E-step launch too (process-wide).  Without ``launches`` the EM loop keeps
    its dependent launches (the E-step and the finalize overlap at their edges)."""
    _lib.gira_profile_enable(0 if not on else 1 if launches else 2)


def gira_profile_read(reset: bool = False) -> dict:
    p = Profile()
    _check(_lib.gira_profile_read(C.byref(p), 1 if reset else 0))
    out = {name: getattr(p, name) for name, _ in Profile._fields_}
    out["estep_kernel"] = out["estep_kernel"].decode()
    return out


def gira_release_workspace():
    _check(_lib.gira_release_workspace())


# ----------------------------------------------------------------------------- entry points
def gira_kmeans_init(points, k: int, seed: int = 0, lloyd_iters: int = 10, centers=None, labels=None,
                     want_labels: bool = True):
    """k-means++ + Lloyd (Sec. V KInit).  Returns (centers K x 3, labels N or None, lloyd iterations done)."""
    n = _check_points(points)
    centers = _new(points, (k, 3), np.float32) if centers is None else centers
    if labels is None and want_labels:
        labels = _new(points, (n,), np.int32)
    pp, kp, s = _ptr(points)
    cp, kc, _ = _ptr(centers)
    lp, kl, _ = _ptr(labels)
    done = C.c_int(0)
    _check(_lib.gira_kmeans_init(pp, n, k, seed, lloyd_iters, cp, lp, C.byref(done), s))
    return centers, labels, done.value


def gira_gmm_fit(points, k: int, iters: int = 100, tol: float = 1e-3, reg_covar: float = 1e-6, seed: int = 0,
                 lloyd_iters: int = 10, init=None, weights=None, means=None, covs=None, trace: bool = True,
                 final_loglik: bool = True):
    """EM fit (Sec. V).  ``init`` = (weights, means, covs) starts from given parameters.

    Returns a dict: weights (K), means (K x 3), covs (K x 3 x 3), trace (iters_done,),
    iters_done, final_loglik.
    """
    n = _check_points(points)
    o = default_opts()
    o.iters, o.tol, o.reg_covar, o.seed, o.lloyd_iters = iters, tol, reg_covar, seed, lloyd_iters
    o.init_mode = INIT_KMEANS
    if weights is None:
        weights = _new(points, (k,), np.float32)
    if means is None:
        means = _new(points, (k, 3), np.float32)
    if covs is None:
        covs = _new(points, (k, 3, 3), np.float32)
    if init is not None:
        o.init_mode = INIT_PARAMS
        for dst, src in zip((weights, means, covs), init):
            if _is_torch(dst):
                import torch
                dst.copy_(torch.as_tensor(np.asarray(src, dtype=np.float32) if not _is_torch(src) else src))
            else:
                dst[...] = np.asarray(src, dtype=np.float32)
    tr = np.full(max(iters, 1), np.nan) if trace else None
    pp, kp, s = _ptr(points)
    wp, kw, _ = _ptr(weights)
    mp, km, _ = _ptr(means)
    cp, kc, _ = _ptr(covs)
    done, fll = C.c_int(0), C.c_double(np.nan)
    _check(_lib.gira_gmm_fit(pp, n, k, C.byref(o), wp, mp, cp,
                             tr.ctypes.data_as(C.POINTER(C.c_double)) if tr is not None else None,
                             C.byref(done), C.byref(fll) if final_loglik else None, s))
    return dict(weights=weights, means=means, covs=covs, trace=None if tr is None else tr[:done.value],
                iters_done=done.value, final_loglik=fll.value if final_loglik else None)


def gira_gmm_loglik(points, weights, means, covs, per_point: bool = False, out=None):
    """Mean (and optionally per-point) log-likelihood ln sum_b pi_b N(x|b) (Eq. logestep)."""
    n = _check_points(points)
    k = int(weights.shape[0])
    if per_point and out is None:
        out = _new(points, (n,), np.float32)
    pp, kp, s = _ptr(points)
    wp, kw, _ = _ptr(weights)
    mp, km, _ = _ptr(means)
    cp, kc, _ = _ptr(covs)
    op, ko, _ = _ptr(out if per_point else None)
    mean = C.c_double(np.nan)
    _check(_lib.gira_gmm_loglik(pp, n, k, wp, mp, cp, C.byref(mean), op, s))
    return (mean.value, out) if per_point else mean.value


def gira_gmm_loglik_noalloc(points, weights, means, covs, per_point: bool = False, out=None):
    """gira_gmm_loglik for callers that cannot allocate device memory (CUDA tensors only).

    The library keeps this call's scratch in a static device array instead of
    allocating it (real-time loops that forbid allocation after start-up, hosts
    whose device memory belongs to a pool).  The call copies its status through
    host memory and synchronises its stream.
    """
    n = _check_points(points)
    k = int(weights.shape[0])
    if per_point and out is None:
        out = _new(points, (n,), np.float32)
    pp, kp, s = _ptr(points)
    wp, kw, _ = _ptr(weights)
    mp, km, _ = _ptr(means)
    cp, kc, _ = _ptr(covs)
    op, ko, _ = _ptr(out if per_point else None)
    mean = C.c_double(np.nan)
    _check(_lib.gira_gmm_loglik_noalloc(pp, n, k, wp, mp, cp, C.byref(mean), op, s))
    return (mean.value, out) if per_point else mean.value


# short aliases
kmeans_init = gira_kmeans_init
gmm_fit = gira_gmm_fit
gmm_loglik = gira_gmm_loglik


GRADS = ("points", "pose", "twist", "logits", "means", "chol")


def _f32_like(x, like):
    """x as a contiguous float32 array/tensor on the same side (host/device) as `like`."""
    if x is None:
        return None
    if _is_torch(like):
        import torch
        return torch.as_tensor(x, dtype=torch.float32, device=like.device).contiguous()
    return np.ascontiguousarray(x, dtype=np.float32)


def gira_gmm_loglik_grad(points, logits, means, chol, pose=None, want=GRADS):
    """L = sum_n ln sum_b softmax(logits)_b N(R x_n + t | mu_b, L_b L_b^T) and its gradient.

    pose: 12 values, R (row-major) then t, or None (identity).  chol: K x 3 x 3,
    lower triangle read.  want: any of GRADS.  Returns a dict with "loglik"
    (float) and "grad_<name>" for every requested gradient: points (N,3) f32,
    pose (12,) f64 = dL/dR row-major then dL/dt, twist (6,) f64 = (omega, v),
    logits (K,) f32, means (K,3) f32, chol (K,3,3) f32.  Arrays follow the
    points (torch on the same device, or numpy)."""
    n = _check_points(points)
    k = int(logits.shape[0])
    bad = set(want) - set(GRADS)
    if bad:
        raise ValueError(f"unknown gradient names {sorted(bad)}")
    lg, mu, ch = _f32_like(logits, points), _f32_like(means, points), _f32_like(chol, points)
    po = _f32_like(pose, points)
    if po is not None and po.reshape(-1).shape[0] != 12:
        raise ValueError("pose must hold 12 values: R row-major, then t")
    shapes = {"points": ((n, 3), np.float32), "pose": ((12,), np.float64), "twist": ((6,), np.float64),
              "logits": ((k,), np.float32), "means": ((k, 3), np.float32), "chol": ((k, 3, 3), np.float32)}
    outs = {g: _new(points, *shapes[g]) for g in want}
    pp, kp, s = _ptr(points)
    keep = [kp]
    ptrs = []
    for x in (po, lg, mu, ch):
        p_, k_, _ = _ptr(x)
        ptrs.append(p_)
        keep.append(k_)
    optr = [(_ptr(outs[g])[0] if g in outs else None) for g in GRADS]
    ll = C.c_double(np.nan)
    _check(_lib.gira_gmm_loglik_grad(pp, n, k, ptrs[0], ptrs[1], ptrs[2], ptrs[3], C.byref(ll), *optr, s))
    r = {"loglik": ll.value}
    for g in want:
        r["grad_" + g] = outs[g]
    return r


def gira_gmm_fit_batched(points, offsets, ks, iters: int = 100, tol: float = 1e-3, reg_covar: float = 1e-6,
                         seed: int = 0, lloyd_iters: int = 10, init=None, final_loglik: bool = True,
                         raise_on_error: bool = True):
    """Fit one GMM per instance: instance i = points[offsets[i]:offsets[i+1]] with ks[i] components.

    init: None (k-means++ / Lloyd per instance) or (weights, means, covs) stacked over
    instances (sum K, (sum K,3), (sum K,3,3)).  Returns a dict: weights, means, covs
    (stacked, like the points: torch on their device, or numpy), and per instance
    iters_done, final_loglik, trace (batch x iters, NaN after stopping), status."""
    total = _check_points(points)
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    kk = np.ascontiguousarray(ks, dtype=np.int32)
    B = len(kk)
    if offs.shape != (B + 1,) or offs[-1] != total:
        raise ValueError("offsets must hold batch + 1 entries ending at the number of points")
    K = int(kk.sum())
    o = default_opts()
    o.iters, o.tol, o.reg_covar, o.seed, o.lloyd_iters = iters, tol, reg_covar, seed, lloyd_iters
    if init is None:
        w, m, c = _new(points, (K,), np.float32), _new(points, (K, 3), np.float32), _new(points, (K, 3, 3), np.float32)
        o.init_mode = INIT_KMEANS
    else:
        w, m, c = (_f32_like(a, points) for a in init)
        if _is_torch(points):
            w, m, c = w.clone(), m.clone(), c.clone()
        else:
            w, m, c = w.copy(), m.copy(), c.copy()
        o.init_mode = INIT_PARAMS
    trace = np.full((B, max(iters, 1)), np.nan)
    done = np.zeros(B, np.int32)
    fll = np.full(B, np.nan)
    stat = np.zeros(B, np.int32)
    pp, kp, s = _ptr(points)
    wp, kw, _ = _ptr(w)
    mp, km, _ = _ptr(m)
    cp, kc, _ = _ptr(c)
    st = _lib.gira_gmm_fit_batched(pp, offs.ctypes.data, B, kk.ctypes.data, C.byref(o), wp, mp, cp,
                                   trace.ctypes.data if iters > 0 else None, done.ctypes.data,
                                   fll.ctypes.data if final_loglik else None, stat.ctypes.data, s)
    if raise_on_error:
        _check(st)
    return dict(weights=w, means=m, covs=c, iters_done=done, final_loglik=fll, trace=trace[:, :iters],
                status=stat)


def gira_gmm_loglik_grad_batched(points, offsets, ks, logits, means, chol, poses=None, want=GRADS,
                                 raise_on_error: bool = True):
    """gira_gmm_loglik_grad for a batch of scans (instance i = points[offsets[i]:offsets[i+1]]
    with its own model of ks[i] components, stacked, and pose poses[i] (12 values) or
    identity).  Returns a dict: loglik (batch,), status (batch,) and grad_<name> for each
    name in want: points (sum N,3), pose (batch,12), twist (batch,6), logits (sum K,),
    means (sum K,3), chol (sum K,3,3), on the points' side (torch device or numpy)."""
    total = _check_points(points)
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    kk = np.ascontiguousarray(ks, dtype=np.int32)
    B = len(kk)
    if offs.shape != (B + 1,) or offs[-1] != total:
        raise ValueError("offsets must hold batch + 1 entries ending at the number of points")
    K = int(kk.sum())
    lg, mu, ch = _f32_like(logits, points), _f32_like(means, points), _f32_like(chol, points)
    po = _f32_like(poses, points)
    shapes = {"points": ((total, 3), np.float32), "pose": ((B, 12), np.float64), "twist": ((B, 6), np.float64),
              "logits": ((K,), np.float32), "means": ((K, 3), np.float32), "chol": ((K, 3, 3), np.float32)}
    outs = {g: _new(points, *shapes[g]) for g in want}
    ll = np.full(B, np.nan)
    stat = np.zeros(B, np.int32)
    pp, kp, s = _ptr(points)
    keep = [kp]
    ptrs = []
    for x in (po, lg, mu, ch):
        p_, k_, _ = _ptr(x)
        ptrs.append(p_)
        keep.append(k_)
    optr = [(_ptr(outs[g])[0] if g in outs else None) for g in GRADS]
    st = _lib.gira_gmm_loglik_grad_batched(pp, offs.ctypes.data, B, kk.ctypes.data, ptrs[0], ptrs[1], ptrs[2],
                                           ptrs[3], ll.ctypes.data, *optr, stat.ctypes.data, s)
    if raise_on_error:
        _check(st)
    r = {"loglik": ll, "status": stat}
    for g in want:
        r["grad_" + g] = outs[g]
    return r


# ----------------------------------------------------------------------------- four dimensions
def gira_gmm_fit4(points, k: int, iters: int = 100, tol: float = 1e-3, reg_covar: float = 1e-6, seed: int = 0,
                  lloyd_iters: int = 10, init=None, final_loglik: bool = True):
    """EM fit of a D = 4 mixture to N x 4 points (x, y, z, intensity).  ``init`` =
    (weights, means K x 4, covs K x 4 x 4) starts from given parameters.  Returns a
    dict like gira_gmm_fit: weights, means, covs, trace, iters_done, final_loglik."""
    n = _check_points(points, 4)
    o = default_opts()
    o.iters, o.tol, o.reg_covar, o.seed, o.lloyd_iters = iters, tol, reg_covar, seed, lloyd_iters
    o.init_mode = INIT_KMEANS
    if init is None:
        w, m, c = _new(points, (k,), np.float32), _new(points, (k, 4), np.float32), _new(points, (k, 4, 4), np.float32)
    else:
        w, m, c = (_f32_like(a, points) for a in init)
        w, m, c = (a.clone() if _is_torch(a) else a.copy() for a in (w, m, c))
        o.init_mode = INIT_PARAMS
    tr = np.full(max(iters, 1), np.nan)
    pp, kp, s = _ptr(points)
    wp, kw, _ = _ptr(w)
    mp, km, _ = _ptr(m)
    cp, kc, _ = _ptr(c)
    done, fll = C.c_int(0), C.c_double(np.nan)
    _check(_lib.gira_gmm_fit4(pp, n, k, C.byref(o), wp, mp, cp, tr.ctypes.data_as(C.POINTER(C.c_double)),
                              C.byref(done), C.byref(fll) if final_loglik else None, s))
    return dict(weights=w, means=m, covs=c, trace=tr[:done.value], iters_done=done.value,
                final_loglik=fll.value if final_loglik else None)


def gira_gmm_loglik4(points, weights, means, covs, per_point: bool = False):
    """Mean (and optionally per-point) log-likelihood of N x 4 points under a D = 4 mixture."""
    n = _check_points(points, 4)
    k = int(weights.shape[0])
    w, m, c = (_f32_like(a, points) for a in (weights, means, covs))
    out = _new(points, (n,), np.float32) if per_point else None
    pp, kp, s = _ptr(points)
    wp, kw, _ = _ptr(w)
    mp, km, _ = _ptr(m)
    cp, kc, _ = _ptr(c)
    op, ko, _ = _ptr(out)
    mean = C.c_double(np.nan)
    _check(_lib.gira_gmm_loglik4(pp, n, k, wp, mp, cp, C.byref(mean), op, s))
    return (mean.value, out) if per_point else mean.value


def gira_gmm_conditional4(locs, weights, means, covs, want_var: bool = True):
    """Intensity regression (Sec. IV): E[I | xyz] and V[I | xyz] at M x 3 locations under a
    D = 4 mixture.  Returns (mean (M,), var (M,) or None) on the side of ``locs``."""
    m_ = _check_points(locs, 3)
    k = int(weights.shape[0])
    w, m, c = (_f32_like(a, locs) for a in (weights, means, covs))
    e = _new(locs, (m_,), np.float32)
    v = _new(locs, (m_,), np.float32) if want_var else None
    lp, kl, s = _ptr(locs)
    wp, kw, _ = _ptr(w)
    mp, km, _ = _ptr(m)
    cp, kc, _ = _ptr(c)
    ep, ke, _ = _ptr(e)
    vp_, kv, _ = _ptr(v)
    _check(_lib.gira_gmm_conditional4(lp, m_, k, wp, mp, cp, ep, vp_, s))
    return e, v


def gira_gmm_sample(m: int, weights, means, covs, seed: int = 0, device=None, want_components: bool = True):
    """m draws from a d-dimensional mixture (d = means.shape[1], 3 or 4).  Outputs live on
    ``device`` (a torch device) or, when None, on the side of ``means``.  Returns
    (points (m, d) float32, components (m,) int32 or None)."""
    like = means
    if device is not None:
        import torch
        like = torch.empty(0, device=device)
    d = int(means.shape[1])
    k = int(weights.shape[0])
    w, mu, c = (_f32_like(a, like) for a in (weights, means, covs))
    out = _new(like, (m, d), np.float32)
    comp = _new(like, (m,), np.int32) if want_components else None
    s = None
    if _is_torch(like) and like.is_cuda:
        import torch
        s = torch.cuda.current_stream(like.device).cuda_stream
    wp, kw, _ = _ptr(w)
    mp, km, _ = _ptr(mu)
    cp, kc, _ = _ptr(c)
    op, ko, _ = _ptr(out)
    qp, kq, _ = _ptr(comp)
    _check(_lib.gira_gmm_sample(m, k, d, wp, mp, cp, seed, op, qp, s))
    return out, comp


# ----------------------------------------------------------------------------- K from a bandwidth
def gira_gbms(points, bandwidth: float, max_iter: int = 300):
    """Mode seeking that sets K (Sec. V "Gaussian Blurring Mean Shift"): binned seeds
    moved to the average of the points within ``bandwidth`` until they stop; the
    distinct end points are the modes.  points: N x 3 or N x 4 float32.  Returns
    (modes (K, d) float64 in rank order, counts (K,) int32) on the side of the points."""
    if points.ndim != 2 or points.shape[1] not in (3, 4):
        raise ValueError("points must be N x 3 or N x 4")
    n, d = int(points.shape[0]), int(points.shape[1])
    modes = _new(points, (n, d), np.float64)
    counts = _new(points, (n,), np.int32)
    pp, kp, s = _ptr(points)
    mp, km, _ = _ptr(modes)
    cp, kc, _ = _ptr(counts)
    k = C.c_int(0)
    _check(_lib.gira_gbms(pp, n, d, float(bandwidth), max_iter, C.byref(k), mp, cp, s))
    return modes[:k.value], counts[:k.value]


# ----------------------------------------------------------------------------- test hooks
def gira_test_fail_next_allocations(count: int):
    """The next ``count`` workspace allocations fail with ERR_OOM (0 clears)."""
    _lib.gira_test_fail_next_allocations(count)


def gira_test_point_order(points, offsets=None):
    """The order the fits' E-steps visit the points in (torch int32 on the points' device)."""
    import torch
    n = int(points.shape[0])
    offs = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)
    batch = 1 if offs is None else len(offs) - 1
    order = torch.empty(n, dtype=torch.int32, device=points.device)
    s = torch.cuda.current_stream(points.device).cuda_stream
    _check(_lib.gira_test_point_order(points.data_ptr(), n, batch, None if offs is None else offs.ctypes.data,
                                      order.data_ptr(), s))
    return order


def gira_test_bounded_wait(mode: int, limit: int) -> int:
    """Run one device wait that nothing ends (0: mbarrier, limit in ns; 1: global counter,
    limit in polls) and return the status it recorded (ERR_TIMEOUT when the bound fired)."""
    import torch
    s = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    return _lib.gira_test_bounded_wait(mode, limit, s)
