"""The C ABI library: builds for sm_103a, loads, exports every declared symbol,
and rejects invalid arguments before touching a GPU (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "gira.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gira_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_00071_gb300 import build_lib
    return C.CDLL(build_lib.build())


def test_library_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert {"gira_gmm_fit", "gira_gmm_loglik", "gira_kmeans_init"} <= set(syms)
    for s in syms:
        assert hasattr(lib, s), s


def test_binary_targets_sm103a():
    from paper_2307_00071_gb300 import build_lib
    assert "arch=compute_103a,code=sm_103a" in " ".join(build_lib.ARCH)


def test_version_and_defaults():
    from paper_2307_00071_gb300 import gira
    assert "sm_103a" in gira.version()
    o = gira.default_opts()
    assert (o.iters, o.tol, o.reg_covar, o.lloyd_iters, o.init_mode) == (100, 1e-3, 1e-6, 10, gira.INIT_KMEANS)


@pytest.mark.parametrize("n,k", [(0, 1), (5, 0), (5, 6), (9000, 8193)])
def test_invalid_sizes_rejected_without_gpu(n, k):
    from paper_2307_00071_gb300 import gira
    pts = np.zeros((max(n, 1), 3), np.float32)
    w, m, c = np.ones(max(k, 1), np.float32), np.zeros((max(k, 1), 3), np.float32), np.tile(np.eye(3, dtype=np.float32), (max(k, 1), 1, 1))
    L = gira._lib
    o = gira.default_opts()
    st = L.gira_gmm_fit(pts.ctypes.data, n, k, C.byref(o), w.ctypes.data, m.ctypes.data, c.ctypes.data, None, None,
                        None, None)
    assert st == gira.ERR_INVALID_ARG
    assert L.gira_last_error_message()
    assert L.gira_gmm_loglik(pts.ctypes.data, n, k, w.ctypes.data, m.ctypes.data, c.ctypes.data, None, None,
                             None) == gira.ERR_INVALID_ARG
    assert L.gira_kmeans_init(pts.ctypes.data, n, k, 0, 1, m.ctypes.data, None, None, None) == gira.ERR_INVALID_ARG


def test_invalid_options_rejected_without_gpu():
    from paper_2307_00071_gb300 import gira
    L = gira._lib
    pts = np.zeros((10, 3), np.float32)
    w, m, c = np.ones(2, np.float32), np.zeros((2, 3), np.float32), np.tile(np.eye(3, dtype=np.float32), (2, 1, 1))
    for field, val in (("iters", -1), ("tol", float("nan")), ("tol", -1.0), ("reg_covar", -1e-6),
                       ("reg_covar", float("inf")), ("lloyd_iters", -2), ("init_mode", 7)):
        o = gira.default_opts()
        setattr(o, field, val)
        st = L.gira_gmm_fit(pts.ctypes.data, 10, 2, C.byref(o), w.ctypes.data, m.ctypes.data, c.ctypes.data, None,
                            None, None, None)
        assert st == gira.ERR_INVALID_ARG, field
    assert L.gira_gmm_fit(pts.ctypes.data, 10, 2, None, w.ctypes.data, m.ctypes.data, c.ctypes.data, None, None,
                          None, None) == gira.ERR_INVALID_ARG
    o = gira.default_opts()
    assert L.gira_gmm_fit(None, 10, 2, C.byref(o), w.ctypes.data, m.ctypes.data, c.ctypes.data, None, None, None,
                          None) == gira.ERR_INVALID_ARG
    assert L.gira_kmeans_init(pts.ctypes.data, 10, 2, 0, -1, m.ctypes.data, None, None, None) == gira.ERR_INVALID_ARG


def test_binding_raises_typed_error():
    from paper_2307_00071_gb300 import gira
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_fit(np.zeros((3, 3), np.float32), 5)
    assert e.value.status == gira.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        gira.gira_gmm_fit(np.zeros((3, 2), np.float32), 1)


def test_loglik_grad_invalid_arguments_rejected_without_gpu():
    from paper_2307_00071_gb300 import gira
    L = gira._lib
    pts = np.zeros((4, 3), np.float32)
    lg, mu, ch = np.zeros(2, np.float32), np.zeros((2, 3), np.float32), np.tile(np.eye(3, dtype=np.float32), (2, 1, 1))
    args = lambda n, k, lgp: (pts.ctypes.data, n, k, None, lgp, mu.ctypes.data, ch.ctypes.data, None, None, None,
                             None, None, None, None, None)
    assert L.gira_gmm_loglik_grad(*args(0, 2, lg.ctypes.data)) == gira.ERR_INVALID_ARG
    assert L.gira_gmm_loglik_grad(*args(4, 0, lg.ctypes.data)) == gira.ERR_INVALID_ARG
    assert L.gira_gmm_loglik_grad(*args(4, 2, None)) == gira.ERR_INVALID_ARG
    assert b"NULL" in L.gira_last_error_message()


def test_batched_invalid_arguments_rejected_without_gpu():
    from paper_2307_00071_gb300 import gira
    L = gira._lib
    pts = np.zeros((10, 3), np.float32)
    w, m, c = np.ones(4, np.float32), np.zeros((4, 3), np.float32), np.tile(np.eye(3, dtype=np.float32), (4, 1, 1))
    o = gira.default_opts()

    def call(offs, ks, batch):
        offs = np.asarray(offs, np.int64)
        ks = np.asarray(ks, np.int32)
        return L.gira_gmm_fit_batched(pts.ctypes.data, offs.ctypes.data, batch, ks.ctypes.data, C.byref(o),
                                      w.ctypes.data, m.ctypes.data, c.ctypes.data, None, None, None, None, None)

    assert call([0, 5, 10], [2, 2], 0) == gira.ERR_INVALID_ARG        # empty batch
    assert call([1, 5, 10], [2, 2], 2) == gira.ERR_INVALID_ARG        # offsets[0] != 0
    assert call([0, 5, 5], [2, 2], 2) == gira.ERR_INVALID_ARG         # an empty instance
    assert call([0, 5, 10], [2, 6], 2) == gira.ERR_INVALID_ARG        # k > n
    assert call([0, 5, 10], [0, 2], 2) == gira.ERR_INVALID_ARG        # k < 1
    assert b"instance" in L.gira_last_error_message()


def test_d4_invalid_arguments_rejected_without_gpu():
    from paper_2307_00071_gb300 import gira
    L = gira._lib
    pts = np.zeros((10, 4), np.float32)
    w, m, c = np.ones(2, np.float32), np.zeros((2, 4), np.float32), np.tile(np.eye(4, dtype=np.float32), (2, 1, 1))
    o = gira.default_opts()
    fit = lambda n, k: L.gira_gmm_fit4(pts.ctypes.data, n, k, C.byref(o), w.ctypes.data, m.ctypes.data,
                                       c.ctypes.data, None, None, None, None)
    assert fit(0, 1) == gira.ERR_INVALID_ARG
    assert fit(10, 11) == gira.ERR_INVALID_ARG
    assert fit(9000, 8193) == gira.ERR_INVALID_ARG                     # above GIRA_MAX_K4
    assert L.gira_gmm_loglik4(pts.ctypes.data, 10, 0, w.ctypes.data, m.ctypes.data, c.ctypes.data, None, None,
                              None) == gira.ERR_INVALID_ARG
    loc = np.zeros((3, 3), np.float32)
    out = np.zeros(3, np.float32)
    assert L.gira_gmm_conditional4(loc.ctypes.data, 0, 2, w.ctypes.data, m.ctypes.data, c.ctypes.data,
                                   out.ctypes.data, None, None) == gira.ERR_INVALID_ARG
    assert L.gira_gmm_conditional4(loc.ctypes.data, 3, 2, w.ctypes.data, m.ctypes.data, c.ctypes.data, None, None,
                                   None) == gira.ERR_INVALID_ARG
    so = np.zeros((4, 4), np.float32)
    assert L.gira_gmm_sample(4, 2, 5, w.ctypes.data, m.ctypes.data, c.ctypes.data, 0, so.ctypes.data, None,
                             None) == gira.ERR_INVALID_ARG                 # d not 3 or 4
    assert L.gira_gmm_sample(0, 2, 4, w.ctypes.data, m.ctypes.data, c.ctypes.data, 0, so.ctypes.data, None,
                             None) == gira.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        gira.gira_gmm_fit4(np.zeros((5, 3), np.float32), 1)


def test_gbms_invalid_arguments_rejected_without_gpu():
    from paper_2307_00071_gb300 import gira
    L = gira._lib
    pts = np.zeros((10, 3), np.float32)
    k = C.c_int(0)
    assert L.gira_gbms(pts.ctypes.data, 10, 5, 0.1, 10, C.byref(k), None, None, None) == gira.ERR_INVALID_ARG
    assert L.gira_gbms(pts.ctypes.data, 10, 3, 0.0, 10, C.byref(k), None, None, None) == gira.ERR_INVALID_ARG
    assert L.gira_gbms(pts.ctypes.data, 10, 3, float("nan"), 10, C.byref(k), None, None, None) == gira.ERR_INVALID_ARG
    assert L.gira_gbms(pts.ctypes.data, 10, 3, 0.1, 0, C.byref(k), None, None, None) == gira.ERR_INVALID_ARG
    assert L.gira_gbms(pts.ctypes.data, 0, 3, 0.1, 10, C.byref(k), None, None, None) == gira.ERR_INVALID_ARG
    assert L.gira_gbms(pts.ctypes.data, 10, 3, 0.1, 10, None, None, None, None) == gira.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        gira.gira_gbms(np.zeros((4, 2), np.float32), 0.1)


def test_test_hooks_check_arguments_without_gpu():
    from paper_2307_00071_gb300 import gira
    L = gira._lib
    assert L.gira_test_bounded_wait(2, 10, None) == gira.ERR_INVALID_ARG
    assert L.gira_test_bounded_wait(0, 0, None) == gira.ERR_INVALID_ARG
    gira.gira_test_fail_next_allocations(0)   # clearing is a no-op without a GPU


def test_profile_levels_without_gpu():
    """Profiling is host state: off, phase events only (the EM loop keeps its
    dependent launches), or phase events plus an event pair per E-step launch;
    reading and resetting the accumulated profile needs no GPU."""
    from paper_2307_00071_gb300 import gira
    gira.gira_profile_read(reset=True)   # whatever earlier calls in this process left
    for on, launches in ((True, False), (True, True), (False, True)):
        gira.gira_profile_enable(on, launches=launches)
        p = gira.gira_profile_read(reset=True)
        assert p["calls"] == 0 and p["estep_launches"] == 0 and p["estep_ms"] == 0.0
    gira.gira_profile_enable(False)


def test_debug_build_compiles_and_exports_the_same_symbols():
    """The build with device-side index checks (GIRA_DEBUG) cross-compiles for sm_103a."""
    from paper_2307_00071_gb300 import build_lib
    dbg = C.CDLL(build_lib.build(debug=True))
    for s in declared_symbols():
        assert hasattr(dbg, s), s
