"""The oracle's all-core EM (oracle/gira_oracle_par.c) against the single-threaded
oracle it restates (CPU only).

The parallel form takes every per-point value with the single-threaded
oracle's own expressions and changes only the order of the binary64 sums
(fixed chunks of points, added in chunk order) and recomputes the
responsibilities in the M-step's second pass instead of storing them.  So:
per-point log-likelihoods are bit-identical; EM results agree to the
rounding of reordered binary64 sums; and nothing depends on the number of
threads.  A sum of n non-negative terms taken in two different orders
differs by at most 2 (n - 1) u of its value (u = 2^-53, the standard bound
for recursive summation), which is the tolerance per component (norm-wise):
1e-12 on 20,000 points (the bound is 4.4e-12), 2 N u = 6.1e-11 on the
frame.  Pinned on the 20k-point K = 8
cloud (20 iterations) and on the 276k-point depth frame at K = 512 (two
iterations), the sizes the GPU parity tests use it at.
"""
import numpy as np
import pytest

import oracle
from paper_2307_00071_gb300 import synth

REL = 1e-12
U = 2.0 ** -53


def close(a, b, rel=REL):
    K = len(a["weights"])
    dw = np.abs(a["weights"] - b["weights"]) / a["weights"]
    dm = np.linalg.norm(a["means"] - b["means"], axis=1) / np.linalg.norm(a["means"], axis=1)
    dc = (np.linalg.norm((a["covs"] - b["covs"]).reshape(K, -1), axis=1)
          / np.linalg.norm(a["covs"].reshape(K, -1), axis=1))
    assert dw.max() <= rel and dm.max() <= rel and dc.max() <= rel, (dw.max(), dm.max(), dc.max())
    assert a["iters_done"] == b["iters_done"]
    assert np.max(np.abs(a["trace"] - b["trace"])) <= rel * np.max(np.abs(a["trace"]))
    assert abs(a["final_ll"] - b["final_ll"]) <= rel * abs(a["final_ll"])


@pytest.fixture(scope="module")
def cloud():
    cl = synth.gmm_cloud(20_000, 8, seed=0)
    ki = oracle.kinit(cl.points, 8, seed=0, lloyd_iters=10, reg=1e-6)
    return cl.points, (ki["weights"], ki["means"], ki["covs"])


def test_parallel_em_matches_single_threaded_oracle_small_cloud(cloud):
    pts, init = cloud
    ref = oracle.em(pts, *init, iters=20, tol=0.0, reg=1e-6)
    par = oracle.em_par(pts, *init, iters=20, tol=0.0, reg=1e-6)
    close(ref, par)


def test_parallel_em_does_not_depend_on_the_thread_count(cloud):
    pts, init = cloud
    runs = [oracle.em_par(pts, *init, iters=5, tol=0.0, reg=1e-6, threads=t) for t in (1, 3, 0)]
    for r in runs[1:]:
        for key in ("weights", "means", "covs", "trace"):
            assert np.array_equal(r[key], runs[0][key]), key
        assert r["final_ll"] == runs[0]["final_ll"]


def test_parallel_em_stops_at_the_same_iteration(cloud):
    pts, init = cloud
    ref = oracle.em(pts, *init, iters=100, tol=1e-3, reg=1e-6)
    par = oracle.em_par(pts, *init, iters=100, tol=1e-3, reg=1e-6)
    assert ref["iters_done"] < 100
    close(ref, par)


def test_parallel_per_point_loglik_is_bit_identical(cloud):
    pts, init = cloud
    mean, _, lse = oracle.estep(pts, *init, want_resp=False, want_lse=True)
    pmean, plse = oracle.loglik_par(pts, *init, per_point=True)
    assert np.array_equal(lse, plse)
    assert abs(mean - pmean) <= 1e-14 * abs(mean)


def test_parallel_em_reports_the_same_failing_component():
    rng = np.random.default_rng(7)
    pts = rng.normal(size=(300, 3)).astype(np.float32)
    w = np.full(3, 1 / 3)
    m = rng.normal(size=(3, 3))
    c = np.stack([np.eye(3)] * 3)
    c[1] = np.diag([1.0, -1.0, 1.0])
    with pytest.raises(oracle.OracleError) as e1:
        oracle.em(pts, w, m, c, iters=1)
    b1 = oracle.last_bad_component()
    with pytest.raises(oracle.OracleError) as e2:
        oracle.em_par(pts, w, m, c, iters=1)
    assert e1.value.code == e2.value.code == oracle.ERR_NOT_PD
    assert oracle.last_bad_component() == b1 == 1


def test_parallel_em_matches_single_threaded_oracle_on_the_frame():
    """The 276,348-point depth frame, K = 512, two iterations from a model of
    thin discs centred on frame points (any valid start serves: the pin is
    about the arithmetic, not the fit)."""
    pts = synth.depth_frame(seed=1).points
    rng = np.random.default_rng(5)
    K = 512
    idx = rng.choice(len(pts), K, replace=False)
    m = pts[idx].astype(np.float64)
    c = np.empty((K, 3, 3))
    for b in range(K):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        c[b] = Q @ np.diag([0.2 ** 2, 0.1 ** 2, 0.01 ** 2]) @ Q.T
    w = rng.dirichlet(np.ones(K))
    ref = oracle.em(pts, w, m, c, iters=2, tol=0.0, reg=1e-6)
    par = oracle.em_par(pts, w, m, c, iters=2, tol=0.0, reg=1e-6)
    close(ref, par, rel=2 * len(pts) * U)
