"""gira_gmm_loglik_noalloc, the entry point for callers that cannot allocate.

Callers running inside CUDA-graph capture, real-time loops that forbid
allocation after start-up, or hosts whose device memory belongs to a pool they
do not control cannot let the library cudaMalloc its scratch.  This entry point
keeps its scratch in a static device array instead; here it is called through
the C ABI and checked against gira_gmm_loglik, the allocating entry point, on
two calls in a row (different inputs, so stale scratch contents would show).
The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from _parity import LL_ABS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
    return [torch.as_tensor(x, device="cuda") for x in (pts, w, mu, cov)]


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    from paper_2307_00071_gb300 import gira
    f = _noalloc(gira._lib)
    stream = torch.cuda.current_stream().cuda_stream
    for seed, n, k in ((1, 40_011, 37), (2, 9_000, 512)):
        pts, w, mu, cov = _case(seed, n, k)
        ref_mean, ref_pp = gira.gira_gmm_loglik(pts, w, mu, cov, per_point=True)
        out = torch.full((n,), float("nan"), device="cuda")
        mean = C.c_double(float("nan"))
        st = f(pts.data_ptr(), n, k, w.data_ptr(), mu.data_ptr(), cov.data_ptr(), C.byref(mean), out.data_ptr(),
               stream)
        assert st == gira.OK, gira._lib.gira_last_error_message()
        assert abs(mean.value - ref_mean) <= LL_ABS + 1e-7 * abs(ref_mean)
        err = (out - ref_pp).abs().max().item()
        assert err <= 2e-3 + 1e-5 * ref_pp.abs().max().item(), err


def test_noalloc_rejects_what_it_cannot_hold():
    from paper_2307_00071_gb300 import gira
    f = _noalloc(gira._lib)
    pts, w, mu, cov = _case(3, 100, 4)
    too_many = 524288 + 1
    assert f(pts.data_ptr(), too_many, 4, w.data_ptr(), mu.data_ptr(), cov.data_ptr(), None, None,
             None) == gira.ERR_INVALID_ARG
    host = np.zeros((100, 3), np.float32)
    assert f(host.ctypes.data, 100, 4, w.data_ptr(), mu.data_ptr(), cov.data_ptr(), None, None,
             None) == gira.ERR_INVALID_ARG
