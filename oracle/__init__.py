"""FP64 CPU oracle for GMM-EM (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; the
oracle shares no code with the CUDA path.  The arithmetic lives in
``gira_oracle.c`` (plain single-threaded C, binary64); this module only
marshals numpy arrays.  See the header of ``gira_oracle.c`` for the passages
of GIRA (arXiv 2307.00071, Sec. V) each function follows.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

OK, ERR_INVALID_ARG, ERR_NONFINITE, ERR_NOT_PD, ERR_OOM = 0, 1, 2, 3, 5


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"oracle {where} failed with status {code}")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp, fp, i64p, i32p = (C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int64),
                              C.POINTER(C.c_int32))
        L.oracle_splitmix64.restype = C.c_uint64
        L.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.oracle_uniform.restype = C.c_double
        L.oracle_uniform.argtypes = [C.c_uint64, C.c_uint64]
        L.oracle_cholesky3.argtypes = [dp, dp]
        L.oracle_tri_inverse3.argtypes = [dp, dp]
        L.oracle_log_gaussian.restype = C.c_double
        L.oracle_log_gaussian.argtypes = [dp, dp, dp]
        L.oracle_estep.argtypes = [fp, C.c_int64, C.c_int, dp, dp, dp, dp, dp, dp]
        L.oracle_mstep.argtypes = [fp, C.c_int64, C.c_int, dp, C.c_double, dp, dp, dp]
        L.oracle_dist2_f32.restype = C.c_float
        L.oracle_dist2_f32.argtypes = [fp, fp]
        L.oracle_kmeanspp.argtypes = [fp, C.c_int64, C.c_int, C.c_uint64, fp, i64p]
        L.oracle_lloyd.argtypes = [fp, C.c_int64, C.c_int, fp, C.c_int, i32p, C.POINTER(C.c_int)]
        L.oracle_init_from_labels.argtypes = [fp, C.c_int64, C.c_int, i32p, C.c_double, dp, dp, dp]
        L.oracle_em.argtypes = [fp, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_double, dp, dp, dp, dp,
                                C.POINTER(C.c_int), dp]
        L.oracle_gmm_fit.argtypes = [fp, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint64,
                                     C.c_int, dp, dp, dp, dp, C.POINTER(C.c_int), dp]
        L.oracle_last_bad_component.restype = C.c_int
        u64p = C.POINTER(C.c_uint64)
        L.oracle_fx48_parts.argtypes = [C.c_float, u64p, u64p]
        L.oracle_fx_threshold.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, u64p, u64p]
        L.oracle_loglik_grad.argtypes = [fp, C.c_int64, C.c_int, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        ci = C.c_int
        L.oracle_cholesky_d.argtypes = [dp, dp, ci]
        L.oracle_tri_inverse_d.argtypes = [dp, dp, ci]
        L.oracle_log_gaussian_d.restype = C.c_double
        L.oracle_log_gaussian_d.argtypes = [dp, dp, dp, ci]
        L.oracle_estep_d.argtypes = [fp, C.c_int64, ci, ci, dp, dp, dp, dp, dp, dp]
        L.oracle_mstep_d.argtypes = [fp, C.c_int64, ci, ci, dp, C.c_double, dp, dp, dp]
        L.oracle_dist2_f32_d.restype = C.c_float
        L.oracle_dist2_f32_d.argtypes = [fp, fp, ci]
        L.oracle_kmeanspp_d.argtypes = [fp, C.c_int64, ci, ci, C.c_uint64, fp, i64p]
        L.oracle_lloyd_d.argtypes = [fp, C.c_int64, ci, ci, fp, ci, i32p, C.POINTER(ci)]
        L.oracle_init_from_labels_d.argtypes = [fp, C.c_int64, ci, ci, i32p, C.c_double, dp, dp, dp]
        L.oracle_em_d.argtypes = [fp, C.c_int64, ci, ci, ci, C.c_double, C.c_double, dp, dp, dp, dp, C.POINTER(ci),
                                  dp]
        L.oracle_gmm_fit_d.argtypes = [fp, C.c_int64, ci, ci, ci, C.c_double, C.c_double, C.c_uint64, ci, dp, dp, dp,
                                       dp, C.POINTER(ci), dp]
        L.oracle_conditional4.argtypes = [fp, C.c_int64, ci, dp, dp, dp, dp, dp]
        L.oracle_sample_d.argtypes = [C.c_int64, ci, ci, dp, dp, dp, C.c_uint64, fp, i32p]
        L.oracle_gbms_d.argtypes = [fp, C.c_int64, ci, C.c_double, ci, C.POINTER(ci), dp, i32p]
        L.oracle_max_threads.restype = ci
        L.oracle_estep_par_d.argtypes = [fp, C.c_int64, ci, ci, dp, dp, dp, dp, dp, ci]
        L.oracle_em_par_d.argtypes = [fp, C.c_int64, ci, ci, ci, C.c_double, C.c_double, dp, dp, dp, dp,
                                      C.POINTER(ci), dp, ci]
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def _check(st, where):
    if st != OK:
        raise OracleError(st, where)


def last_bad_component() -> int:
    return int(lib().oracle_last_bad_component())


# ----------------------------------------------------------------------------- RNG
def splitmix64(seed: int, j: int) -> int:
    return int(lib().oracle_splitmix64(seed, j))


def uniform(seed: int, j: int) -> float:
    return float(lib().oracle_uniform(seed, j))


# ----------------------------------------------------------------------------- algebra
# The dimension d (3, or 4 for xyz + intensity) is taken from the arrays.
def cholesky3(S):
    S = _f64(S)
    d = int(round(np.sqrt(S.size)))
    S = S.reshape(d, d).copy()
    L = np.zeros((d, d))
    st = lib().oracle_cholesky_d(_p(S, C.c_double), _p(L, C.c_double), d)
    if st != 0:
        raise OracleError(ERR_NOT_PD, "cholesky")
    return L


def tri_inverse3(L):
    L = _f64(L)
    d = int(round(np.sqrt(L.size)))
    L = L.reshape(d, d).copy()
    P = np.zeros((d, d))
    lib().oracle_tri_inverse_d(_p(L, C.c_double), _p(P, C.c_double), d)
    return P


def log_gaussian(x, mu, cov) -> float:
    """Eq. (simplifiedGaussian) at one point."""
    P = tri_inverse3(cholesky3(cov))
    x, mu = _f64(x).copy(), _f64(mu).copy()
    return float(lib().oracle_log_gaussian_d(_p(x, C.c_double), _p(mu, C.c_double), _p(P, C.c_double), len(x)))


def fx48(d) -> int:
    """floor(d * 2^48) of a binary32 d >= 0 (k-means++ weight), as a Python int."""
    lo, hi = C.c_uint64(), C.c_uint64()
    lib().oracle_fx48_parts(float(np.float32(d)), C.byref(lo), C.byref(hi))
    return (hi.value << 64) | lo.value


def fx_threshold(k53: int, total: int) -> int:
    lo, hi = C.c_uint64(), C.c_uint64()
    lib().oracle_fx_threshold(k53, total & ((1 << 64) - 1), total >> 64, C.byref(lo), C.byref(hi))
    return (hi.value << 64) | lo.value


def dist2_f32(x, c) -> np.float32:
    x, c = _f32(x).copy(), _f32(c).copy()
    return np.float32(lib().oracle_dist2_f32_d(_p(x, C.c_float), _p(c, C.c_float), len(x)))


def _dim(pts):
    if pts.ndim != 2 or pts.shape[1] not in (3, 4):
        raise ValueError("points must be N x 3 or N x 4")
    return pts.shape[1]


# ----------------------------------------------------------------------------- EM steps
def estep(pts, weights, means, covs, want_resp: bool = True, want_lse: bool = False):
    """Returns (mean_ll, resp or None, lse or None)."""
    pts = _f32(pts)
    d = _dim(pts)
    N, K = pts.shape[0], len(weights)
    w, m, c = _f64(weights), _f64(means), _f64(covs)
    resp = np.empty((N, K)) if want_resp else None
    lse = np.empty(N) if want_lse else None
    ll = C.c_double()
    st = lib().oracle_estep_d(_p(pts, C.c_float), N, K, d, _p(w, C.c_double), _p(m, C.c_double),
                              _p(c, C.c_double), _p(resp, C.c_double), _p(lse, C.c_double), C.byref(ll))
    _check(st, "estep")
    return ll.value, resp, lse


def mstep(pts, resp, reg: float):
    pts, resp = _f32(pts), _f64(resp)
    d = _dim(pts)
    N, K = resp.shape
    w, m, c = np.empty(K), np.empty((K, d)), np.empty((K, d, d))
    st = lib().oracle_mstep_d(_p(pts, C.c_float), N, K, d, _p(resp, C.c_double), reg, _p(w, C.c_double),
                              _p(m, C.c_double), _p(c, C.c_double))
    _check(st, "mstep")
    return w, m, c


def kmeanspp(pts, K: int, seed: int):
    """Returns (centers (K,d) float32, chosen indices (K,) int64)."""
    pts = _f32(pts)
    d = _dim(pts)
    N = pts.shape[0]
    centers = np.empty((K, d), np.float32)
    chosen = np.empty(K, np.int64)
    st = lib().oracle_kmeanspp_d(_p(pts, C.c_float), N, K, d, seed, _p(centers, C.c_float), _p(chosen, C.c_int64))
    _check(st, "kmeanspp")
    return centers, chosen


def lloyd(pts, centers, lloyd_iters: int):
    """Returns (centers (K,d) float32, labels (N,) int32, iterations done)."""
    pts = _f32(pts)
    d = _dim(pts)
    centers = _f32(centers).copy()
    N, K = pts.shape[0], centers.shape[0]
    labels = np.empty(N, np.int32)
    done = C.c_int()
    st = lib().oracle_lloyd_d(_p(pts, C.c_float), N, K, d, _p(centers, C.c_float), lloyd_iters,
                              _p(labels, C.c_int32), C.byref(done))
    _check(st, "lloyd")
    return centers, labels, done.value


def init_from_labels(pts, labels, K: int, reg: float):
    pts = _f32(pts)
    d = _dim(pts)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    N = pts.shape[0]
    w, m, c = np.empty(K), np.empty((K, d)), np.empty((K, d, d))
    st = lib().oracle_init_from_labels_d(_p(pts, C.c_float), N, K, d, _p(labels, C.c_int32), reg,
                                         _p(w, C.c_double), _p(m, C.c_double), _p(c, C.c_double))
    _check(st, "init_from_labels")
    return w, m, c


def em(pts, weights, means, covs, iters: int, tol: float = 0.0, reg: float = 1e-6):
    """EM from explicit parameters.  Returns a dict (weights, means, covs, trace, iters_done, final_ll)."""
    pts = _f32(pts)
    d = _dim(pts)
    N = pts.shape[0]
    w, m, c = _f64(weights).copy(), _f64(means).copy(), _f64(covs).copy()
    K = w.shape[0]
    trace = np.full(max(iters, 1), np.nan)
    done, fll = C.c_int(), C.c_double()
    st = lib().oracle_em_d(_p(pts, C.c_float), N, K, d, iters, tol, reg, _p(w, C.c_double), _p(m, C.c_double),
                           _p(c, C.c_double), _p(trace, C.c_double), C.byref(done), C.byref(fll))
    _check(st, "em")
    return dict(weights=w, means=m, covs=c, trace=trace[:done.value], iters_done=done.value, final_ll=fll.value)


def max_threads() -> int:
    """Threads the parallel oracle uses by default (OpenMP: OMP_NUM_THREADS, else every core)."""
    return int(lib().oracle_max_threads())


def em_par(pts, weights, means, covs, iters: int, tol: float = 0.0, reg: float = 1e-6, threads: int = 0,
           final: bool = True):
    """``em`` over all host cores (``gira_oracle_par.c``): the same iteration, point
    arithmetic and stopping rule; sums over fixed chunks of points added in chunk
    order, so the result does not depend on ``threads`` (0 = every core).
    ``final=False`` skips the log-likelihood of the returned model (final_ll = nan)."""
    pts = _f32(pts)
    d = _dim(pts)
    N = pts.shape[0]
    w, m, c = _f64(weights).copy(), _f64(means).copy(), _f64(covs).copy()
    K = w.shape[0]
    trace = np.full(max(iters, 1), np.nan)
    done, fll = C.c_int(), C.c_double()
    st = lib().oracle_em_par_d(_p(pts, C.c_float), N, K, d, iters, tol, reg, _p(w, C.c_double),
                               _p(m, C.c_double), _p(c, C.c_double), _p(trace, C.c_double), C.byref(done),
                               C.byref(fll) if final else None, int(threads))
    _check(st, "em_par")
    return dict(weights=w, means=m, covs=c, trace=trace[:done.value], iters_done=done.value,
                final_ll=fll.value if final else float("nan"))


def loglik_par(pts, weights, means, covs, per_point: bool = False, threads: int = 0):
    """Mean per-point log-likelihood (and the per-point values) over all host cores."""
    pts = _f32(pts)
    d = _dim(pts)
    N, K = pts.shape[0], len(weights)
    w, m, c = _f64(weights), _f64(means), _f64(covs)
    lse = np.empty(N) if per_point else None
    ll = C.c_double()
    st = lib().oracle_estep_par_d(_p(pts, C.c_float), N, K, d, _p(w, C.c_double), _p(m, C.c_double),
                                  _p(c, C.c_double), _p(lse, C.c_double), C.byref(ll), int(threads))
    _check(st, "estep_par")
    return (ll.value, lse) if per_point else ll.value


def gmm_fit(pts, K: int, iters: int, tol: float = 0.0, reg: float = 1e-6, seed: int = 0, lloyd_iters: int = 10):
    pts = _f32(pts)
    d = _dim(pts)
    N = pts.shape[0]
    w, m, c = np.empty(K), np.empty((K, d)), np.empty((K, d, d))
    trace = np.full(max(iters, 1), np.nan)
    done, fll = C.c_int(), C.c_double()
    st = lib().oracle_gmm_fit_d(_p(pts, C.c_float), N, K, d, iters, tol, reg, seed, lloyd_iters,
                                _p(w, C.c_double), _p(m, C.c_double), _p(c, C.c_double), _p(trace, C.c_double),
                                C.byref(done), C.byref(fll))
    _check(st, "gmm_fit")
    return dict(weights=w, means=m, covs=c, trace=trace[:done.value], iters_done=done.value, final_ll=fll.value)


def kinit(pts, K: int, seed: int, lloyd_iters: int, reg: float):
    """k-means++ + Lloyd + one-hot M-step: the initial parameters gmm_fit starts EM from."""
    centers, chosen = kmeanspp(pts, K, seed)
    centers, labels, done = lloyd(pts, centers, lloyd_iters)
    w, m, c = init_from_labels(pts, labels, K, reg)
    return dict(weights=w, means=m, covs=c, centers=centers, labels=labels, chosen=chosen, lloyd_done=done)


def conditional4(locs, weights, means, covs):
    """E[I | xyz] and V[I | xyz] of a D = 4 mixture at locs (M x 3): Gaussian-mixture regression."""
    locs = _f32(locs)
    M, K = locs.shape[0], len(weights)
    w, m, c = _f64(weights), _f64(means).reshape(K, 4), _f64(covs).reshape(K, 16)
    e, v = np.empty(M), np.empty(M)
    st = lib().oracle_conditional4(_p(locs, C.c_float), M, K, _p(w, C.c_double), _p(m, C.c_double),
                                   _p(c, C.c_double), _p(e, C.c_double), _p(v, C.c_double))
    _check(st, "conditional4")
    return e, v


def sample(M: int, weights, means, covs, seed: int):
    """M draws from the mixture (d from means): (points (M,d) float32, components (M,) int32)."""
    w, m, c = _f64(weights), _f64(means), _f64(covs)
    K, d = m.shape
    out = np.empty((M, d), np.float32)
    comp = np.empty(M, np.int32)
    st = lib().oracle_sample_d(M, K, d, _p(w, C.c_double), _p(m, C.c_double), _p(c, C.c_double), seed,
                               _p(out, C.c_float), _p(comp, C.c_int32))
    _check(st, "sample")
    return out, comp


def loglik_grad(pts, logits, means, chol, pose=None, want_points: bool = True):
    """Summed log-likelihood of the moved scan R x + t and its gradient.

    pose: (R (3,3), t (3,)) or None.  Returns a dict: loglik, grad_points (N,3)
    or None, grad_twist (6,) = (omega, v), grad_logits (K,), grad_means (K,3),
    grad_chol (K,3,3) lower triangular."""
    pts = _f32(pts)
    N, K = pts.shape[0], len(logits)
    lg, m, ch = _f64(logits), _f64(means), _f64(chol).reshape(K, 9).copy()
    p12 = None
    if pose is not None:
        p12 = np.concatenate([_f64(pose[0]).reshape(9), _f64(pose[1]).reshape(3)])
    gp = np.empty((N, 3)) if want_points else None
    gt, gl, gm, gc = np.empty(6), np.empty(K), np.empty((K, 3)), np.empty((K, 3, 3))
    ll = C.c_double()
    st = lib().oracle_loglik_grad(_p(pts, C.c_float), N, K, _p(p12, C.c_double), _p(lg, C.c_double),
                                  _p(m, C.c_double), _p(ch, C.c_double), C.byref(ll), _p(gp, C.c_double),
                                  _p(gt, C.c_double), _p(gl, C.c_double), _p(gm, C.c_double), _p(gc, C.c_double))
    _check(st, "loglik_grad")
    return dict(loglik=ll.value, grad_points=gp, grad_twist=gt, grad_logits=gl, grad_means=gm, grad_chol=gc)


def gbms(pts, bandwidth: float, max_iter: int = 300):
    """Mode seeking that sets K (Sec. V GBMS): (modes (K,d) float64 in rank order,
    counts (K,) int32).  d from the points (3 or 4)."""
    pts = _f32(pts)
    d = _dim(pts)
    N = pts.shape[0]
    modes = np.empty((N, d))
    counts = np.empty(N, np.int32)
    k = C.c_int(0)
    st = lib().oracle_gbms_d(_p(pts, C.c_float), N, d, float(bandwidth), max_iter, C.byref(k),
                             _p(modes, C.c_double), _p(counts, C.c_int32))
    _check(st, "gbms")
    return modes[:k.value].copy(), counts[:k.value].copy()
