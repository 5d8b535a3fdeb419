"""K above 1024: the chunked E-step (two-level log-sum-exp over chunks of 512
components) against the FP64 oracle.  Same tolerances as the direct path."""
import numpy as np
import pytest

import oracle
from paper_2307_00071_gb300 import synth
from tests._parity import LL_ABS, assert_model_close, per_point_bound, to_np

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def gira():
    from paper_2307_00071_gb300 import gira as g
    return g


@pytest.fixture(scope="module")
def frame():
    return synth.depth_frame(seed=3).points


def subset(frame, n, seed):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(frame[np.sort(rng.choice(len(frame), n, replace=False))])


def test_chunked_em_from_given_init_matches_oracle(gira, frame):
    # ~65 points per component, like the paper's configurations (K = 512 on ~276k
    # points, K = 8192 on 4M); with < 10 points per component binary32 alone moves
    # a covariance by ~1e-4 in three iterations, on the direct path as well
    pts = subset(frame, 80_000, 1)
    K = 1236   # chunks of 512, 512, 212
    ki = oracle.kinit(pts, K, seed=0, lloyd_iters=5, reg=1e-6)
    w0, m0, c0 = (ki[a].astype(np.float32) for a in ("weights", "means", "covs"))
    r = gira.gira_gmm_fit(pts, K, iters=3, tol=0.0, init=(w0, m0, c0))
    ref = oracle.em(pts, w0, m0, c0, iters=3, tol=0.0, reg=1e-6)
    assert r["iters_done"] == 3
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert abs(r["final_loglik"] - ref["final_ll"]) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_chunked_fit_with_kmeans_init_matches_oracle(gira, frame):
    pts = subset(frame, 20_000, 2)
    K = 1100
    r = gira.gira_gmm_fit(pts, K, iters=2, tol=0.0, seed=5, lloyd_iters=3)
    ref = oracle.gmm_fit(pts, K, iters=2, tol=0.0, reg=1e-6, seed=5, lloyd_iters=3)
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def large_model(pts, K, rng):
    """K components centred on scan points, thin disc-like covariances (1-5 cm, 5 mm)."""
    idx = rng.choice(len(pts), K, replace=False)
    means = pts[idx].astype(np.float64) + rng.normal(scale=0.01, size=(K, 3))
    covs = []
    for _ in range(K):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = np.array([rng.uniform(0.01, 0.05), rng.uniform(0.01, 0.05), 0.005]) ** 2
        covs.append(Q @ np.diag(lam) @ Q.T)
    w = rng.dirichlet(np.ones(K))
    return w.astype(np.float32), means.astype(np.float32), np.stack(covs).astype(np.float32)


def test_chunked_loglik_k8192_with_outliers(gira, frame):
    rng = np.random.default_rng(3)
    pts = subset(frame, 50_000, 3)
    w, m, c = large_model(pts, 8192, rng)
    # outliers: far from every component, so the sum over components underflows the
    # common reference and the exact per-point maximum takes over
    far = (rng.normal(size=(20, 3)) * 5.0 + np.array([0.0, 0.0, 300.0])).astype(np.float32)
    allp = np.concatenate([pts, far])
    mean, pp = gira.gira_gmm_loglik(allp, w, m, c, per_point=True)
    pp = to_np(pp).astype(np.float64)
    assert np.all(np.isfinite(pp))
    assert mean == pytest.approx(pp.mean(), rel=1e-6)
    sample = np.concatenate([rng.choice(len(pts), 300, replace=False), np.arange(len(pts), len(allp))])
    _, _, lse = oracle.estep(allp[sample], w, m, c, want_resp=False, want_lse=True)
    err = np.abs(pp[sample] - lse)
    bound = per_point_bound(allp[sample], w, m, c)
    assert np.all(err <= bound), np.max(err / bound)


def test_chunked_loglik_equals_direct_where_both_apply(gira, frame):
    """K = 1024 runs the direct path, K = 1025 the chunked one: adding a component of
    negligible weight far away changes the log-likelihood by (almost) nothing."""
    rng = np.random.default_rng(4)
    pts = subset(frame, 30_000, 4)
    w, m, c = large_model(pts, 1024, rng)
    direct = gira.gira_gmm_loglik(pts, w, m, c)
    w2 = np.concatenate([w * (1 - 1e-7), [1e-7]]).astype(np.float32)
    m2 = np.concatenate([m, [[0.0, 0.0, 500.0]]]).astype(np.float32)
    c2 = np.concatenate([c, [np.eye(3, dtype=np.float32) * 1e-4]])
    chunked = gira.gira_gmm_loglik(pts, w2, m2, c2)
    assert abs(chunked - direct) <= LL_ABS


def test_full_size_map_sampled_points_match_oracle(gira):
    """The large-map size: 16 depth frames under random poses, the first 4M points,
    K = 8192 from means at random points.  Per-point log-likelihoods are checked on
    sampled points against the oracle; one EM iteration keeps every property that
    holds at any size (weights summing to 1, finite PD covariances, trace finite)."""
    import torch
    rng = np.random.default_rng(11)
    parts = []
    for i in range(16):
        f = synth.depth_frame(seed=100 + i).points.astype(np.float64)
        th = rng.uniform(0, 2 * np.pi)
        R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
        parts.append(f @ R.T + np.array([rng.uniform(-10, 10), rng.uniform(-10, 10), 0.0]))
    pts = np.concatenate(parts)[:4_000_000].astype(np.float32)
    K = 8192
    w, m, c = large_model(pts, K, rng)
    x = torch.as_tensor(pts, device="cuda")
    mean, pp = gira.gira_gmm_loglik(x, torch.as_tensor(w, device="cuda"), torch.as_tensor(m, device="cuda"),
                                    torch.as_tensor(c, device="cuda"), per_point=True)
    pp = pp.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(pp)) and mean == pytest.approx(pp.mean(), rel=1e-6)
    sample = rng.choice(len(pts), 400, replace=False)
    _, _, lse = oracle.estep(pts[sample], w, m, c, want_resp=False, want_lse=True)
    err = np.abs(pp[sample] - lse)
    bound = per_point_bound(pts[sample], w, m, c)
    assert np.all(err <= bound), np.max(err / bound)
    r = gira.gira_gmm_fit(x, K, iters=1, tol=0.0, init=(w, m, c), final_loglik=False)
    wr, cr = r["weights"].cpu().numpy().astype(np.float64), r["covs"].cpu().numpy().astype(np.float64)
    assert abs(wr.sum() - 1.0) < 1e-4 and np.all(np.isfinite(r["trace"]))
    live = wr > 1e-6
    assert np.all(np.linalg.eigvalsh(0.5 * (cr[live] + np.transpose(cr[live], (0, 2, 1)))) > 0)
