"""gira_gmm_loglik_noalloc, the entry point for callers that cannot allocate.

Real-time loops that forbid device allocation after start-up (cudaMalloc can
block for an unbounded time or fail mid-run), and hosts whose device memory
belongs to a pool they do not control, cannot let the library cudaMalloc its
scratch.  This entry point keeps its scratch in a static device array instead.
Here it is called through the C ABI and checked against gira_gmm_loglik, the
allocating entry point, on two calls in a row (different inputs, so stale
scratch contents would show), at the largest size the array is documented to
hold (n = GIRA_NOALLOC_MAX_N, k = 1024), and with the per-point output left
out.  While it runs, the library's workspace allocator is set to fail every
allocation, so a call that reached it would return GIRA_ERR_OOM.  The file is
named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from _parity import LL_ABS, per_point_bound

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_N = 524288   # GIRA_NOALLOC_MAX_N


def _noalloc(lib):
    f = lib.gira_gmm_loglik_noalloc
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                  C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def _case(seed, n, k):
    rng = np.random.default_rng(seed)
    w = rng.dirichlet(np.ones(k)).astype(np.float32)
    mu = rng.uniform(-2, 2, (k, 3)).astype(np.float32)
    a = rng.standard_normal((k, 3, 3))
    cov = (0.02 * (a @ a.transpose(0, 2, 1) + 0.3 * np.eye(3))).astype(np.float32)
    pts = rng.uniform(-2.2, 2.2, (n, 3)).astype(np.float32)
    return pts, w, mu, cov


def _call_without_allocations(gira, f, args):
    """The call with the library's workspace allocator failing every request."""
    gira._lib.gira_test_fail_next_allocations(1000)
    try:
        return f(*args)
    finally:
        gira._lib.gira_test_fail_next_allocations(0)


@pytest.mark.parametrize("cases", [((1, 40_011, 37), (2, 9_000, 512)), ((3, MAX_N, 1024), (4, 77_777, 200))])
def test_noalloc_matches_allocating_entry_point_on_two_calls(cases):
    from paper_2307_00071_gb300 import gira
    f = _noalloc(gira._lib)
    stream = torch.cuda.current_stream().cuda_stream
    for seed, n, k in cases:
        host = _case(seed, n, k)
        pts, w, mu, cov = [torch.as_tensor(x, device="cuda") for x in host]
        ref_mean, ref_pp = gira.gira_gmm_loglik(pts, w, mu, cov, per_point=True)
        out = torch.full((n,), float("nan"), device="cuda")
        mean = C.c_double(float("nan"))
        st = _call_without_allocations(gira, f, (pts.data_ptr(), n, k, w.data_ptr(), mu.data_ptr(), cov.data_ptr(),
                                                 C.byref(mean), out.data_ptr(), stream))
        assert st == gira.OK, gira._lib.gira_last_error_message()
        assert abs(mean.value - ref_mean) <= LL_ABS + 1e-7 * abs(ref_mean)
        got = out.double().cpu().numpy()
        assert np.all(np.isfinite(got))   # every point written
        err = np.abs(got - ref_pp.double().cpu().numpy())
        # the per-point tolerance at up to 16k sampled points (the bound costs N x K work on the host)
        idx = np.random.default_rng(seed).choice(n, min(n, 16_384), replace=False)
        bound = per_point_bound(host[0][idx], *host[1:])
        assert np.all(err[idx] <= bound), np.max(err[idx] / bound)


def test_noalloc_mean_only():
    from paper_2307_00071_gb300 import gira
    f = _noalloc(gira._lib)
    pts, w, mu, cov = [torch.as_tensor(x, device="cuda") for x in _case(5, 123_457, 300)]
    ref_mean = gira.gira_gmm_loglik(pts, w, mu, cov)
    mean = C.c_double(float("nan"))
    st = _call_without_allocations(gira, f, (pts.data_ptr(), len(pts), 300, w.data_ptr(), mu.data_ptr(),
                                             cov.data_ptr(), C.byref(mean), None,
                                             torch.cuda.current_stream().cuda_stream))
    assert st == gira.OK, gira._lib.gira_last_error_message()
    assert abs(mean.value - ref_mean) <= LL_ABS + 1e-7 * abs(ref_mean)


def test_noalloc_rejects_what_it_cannot_hold():
    from paper_2307_00071_gb300 import gira
    f = _noalloc(gira._lib)
    pts, w, mu, cov = [torch.as_tensor(x, device="cuda") for x in _case(3, 100, 4)]
    assert f(pts.data_ptr(), MAX_N + 1, 4, w.data_ptr(), mu.data_ptr(), cov.data_ptr(), None, None,
             None) == gira.ERR_INVALID_ARG
    assert f(pts.data_ptr(), 100, 1025, w.data_ptr(), mu.data_ptr(), cov.data_ptr(), None, None,
             None) == gira.ERR_INVALID_ARG
    host = np.zeros((100, 3), np.float32)
    assert f(host.ctypes.data, 100, 4, w.data_ptr(), mu.data_ptr(), cov.data_ptr(), None, None,
             None) == gira.ERR_INVALID_ARG


def test_noalloc_refuses_a_capturing_stream():
    """On a stream under capture the call returns GIRA_ERR_INVALID_ARG before any CUDA call
    that could break the capture (it synchronises its stream); the caller's graph still
    completes and replays."""
    from paper_2307_00071_gb300 import gira
    f = _noalloc(gira._lib)
    pts, w, mu, cov = [torch.as_tensor(x, device="cuda") for x in _case(6, 1_000, 8)]
    y = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st = f(pts.data_ptr(), len(pts), 8, w.data_ptr(), mu.data_ptr(), cov.data_ptr(), None, None, s.cuda_stream)
        y += 1
    assert st == gira.ERR_INVALID_ARG
    msg = gira._lib.gira_last_error_message()
    assert "captur" in (msg.decode() if isinstance(msg, bytes) else str(msg))
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(y == 1)
