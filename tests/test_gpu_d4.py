"""Four dimensions (xyz + intensity, the paper's SOGMM data) on the GPU against
the FP64 oracle: the fit (KInit and EM), the log-likelihood, the regression of
intensity on position, and sampling.  Same tolerances as the 3D path
(tests/_parity.py); k-means decisions are exact, so a k-means start matches
the oracle's fit."""
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
def frame4():
    return synth.depth_frame4(seed=2)


def subset(a, n, seed):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(a[np.sort(rng.choice(len(a), n, replace=False))])


@pytest.mark.parametrize("n,k", [(20_000, 8), (9_001, 45)])   # 45: a partly filled second warp of components
def test_fit4_from_given_init_matches_oracle(gira, n, k):
    cl = synth.gmm_cloud4(n, min(k, 12), seed=k)
    ki = oracle.kinit(cl.points, k, seed=1, lloyd_iters=4, reg=1e-6)
    w0, m0, c0 = (ki[a].astype(np.float32) for a in ("weights", "means", "covs"))
    r = gira.gira_gmm_fit4(cl.points, k, iters=12, tol=0.0, init=(w0, m0, c0))
    ref = oracle.em(cl.points, w0, m0, c0, iters=12, tol=0.0, reg=1e-6)
    assert r["iters_done"] == 12
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert abs(r["final_loglik"] - ref["final_ll"]) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_fit4_kmeans_init_matches_oracle_fit(gira):
    cl = synth.gmm_cloud4(15_000, 10, seed=7)
    r = gira.gira_gmm_fit4(cl.points, 16, iters=8, tol=0.0, seed=5, lloyd_iters=6)
    ref = oracle.gmm_fit(cl.points, 16, iters=8, tol=0.0, reg=1e-6, seed=5, lloyd_iters=6)
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_fit4_on_depth_frame_with_intensity(gira, frame4):
    """A 40k-point subset of the frame with its intensity channel, K = 128 (~300 points
    per component, the paper's density), converged with tol as in its fits."""
    pts = subset(frame4, 40_000, 1)
    ki = oracle.kinit(pts, 128, seed=0, lloyd_iters=5, reg=1e-6)
    w0, m0, c0 = (ki[a].astype(np.float32) for a in ("weights", "means", "covs"))
    r = gira.gira_gmm_fit4(pts, 128, iters=6, tol=0.0, init=(w0, m0, c0))
    ref = oracle.em(pts, w0, m0, c0, iters=6, tol=0.0, reg=1e-6)
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


@pytest.mark.parametrize("n", [400_000, 700_000])   # persistent and per-centre seeding kernels
def test_fit4_kinit_on_large_clouds_matches_oracle(gira, n):
    f = np.concatenate([synth.depth_frame(seed=s).points for s in (1, 2, 3)])[:n]
    pts = np.ascontiguousarray(np.concatenate([f, synth.frame_intensity(f, 1)[:, None]], axis=1), np.float32)
    r = gira.gira_gmm_fit4(pts, 48, iters=0, seed=5, lloyd_iters=0)
    c0, _ = oracle.kmeanspp(pts, 48, 5)
    _, lab, _ = oracle.lloyd(pts, c0, 0)
    w, m, c = oracle.init_from_labels(pts, lab, 48, 1e-6)
    ll, _, _ = oracle.estep(pts, w, m, c, want_resp=False)
    assert abs(r["final_loglik"] - ll) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (w, m, c))


def test_fit4_device_tensors_and_convergence(gira):
    import torch
    cl = synth.gmm_cloud4(12_000, 6, seed=9)
    x = torch.as_tensor(cl.points, device="cuda")
    r = gira.gira_gmm_fit4(x, 6, iters=60, tol=1e-4, seed=2)
    ref = oracle.gmm_fit(cl.points, 6, iters=60, tol=1e-4, reg=1e-6, seed=2, lloyd_iters=10)
    assert r["weights"].is_cuda
    assert r["iters_done"] == len(ref["trace"])
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS


@pytest.mark.parametrize("k", [1, 33, 1024])
def test_loglik4_per_point_matches_oracle(gira, frame4, k):
    """k = 1, 33: the KInit model of the points (mean log-likelihood O(1), where the
    fit tolerance applies); k = 1024: a full block of narrow random components
    (log-likelihoods of -1e3 and below: per-point check only)."""
    pts = subset(frame4, 30_000, 3)
    rng = np.random.default_rng(k)
    if k <= 33:
        ki = oracle.kinit(pts, k, seed=0, lloyd_iters=3, reg=1e-6)
        w, m, c = (ki[a].astype(np.float32) for a in ("weights", "means", "covs"))
    else:
        idx = rng.choice(len(pts), k, replace=False)
        means = pts[idx].astype(np.float64) + rng.normal(scale=0.01, size=(k, 4))
        covs = []
        for _ in range(k):
            Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
            lam = np.array([rng.uniform(0.02, 0.1), rng.uniform(0.02, 0.1), 0.01, 0.03]) ** 2
            covs.append(Q @ np.diag(lam) @ Q.T)
        w = rng.dirichlet(np.ones(k)).astype(np.float32)
        m, c = means.astype(np.float32), np.stack(covs).astype(np.float32)
    mean, pp = gira.gira_gmm_loglik4(pts, w, m, c, per_point=True)
    pp = to_np(pp).astype(np.float64)
    sample = rng.choice(len(pts), 400, replace=False)
    _, _, lse = oracle.estep(pts[sample], w, m, c, want_resp=False, want_lse=True)
    err = np.abs(pp[sample] - lse)
    bound = per_point_bound(pts[sample], w, m, c, form="d")   # the 4-D E-step's d form
    assert np.all(err <= bound), np.max(err / bound)
    assert mean == pytest.approx(pp.mean(), rel=1e-6)
    if k <= 33:
        ll_ref, _, _ = oracle.estep(pts, w, m, c, want_resp=False)
        assert abs(mean - ll_ref) <= LL_ABS


@pytest.mark.parametrize("k", [12, 300])   # 300: two shared-memory tiles of components
def test_conditional4_matches_oracle(gira, k):
    cl = synth.gmm_cloud4(20_000, 12, seed=11)
    if k == 12:
        r = oracle.gmm_fit(cl.points, 12, iters=10, tol=0.0, reg=1e-6, seed=1, lloyd_iters=5)
    else:
        r = oracle.kinit(cl.points, k, seed=1, lloyd_iters=3, reg=1e-6)
    w, m, c = (r[a].astype(np.float32) for a in ("weights", "means", "covs"))
    rng = np.random.default_rng(0)
    locs = np.concatenate([cl.points[rng.choice(len(cl.points), 3000, replace=False), :3],
                           rng.uniform(-2, 2, size=(500, 3))]).astype(np.float32)
    e, v = gira.gira_gmm_conditional4(locs, w, m, c)
    re, rv = oracle.conditional4(locs, w, m, c)
    e, v = to_np(e).astype(np.float64), to_np(v).astype(np.float64)
    # binary32 log-weights (logits of size ~10-100 on far locations) move the weights by ~1e-5
    np.testing.assert_allclose(e, re, rtol=0, atol=2e-4)
    np.testing.assert_allclose(v, rv, rtol=2e-3, atol=2e-5)


@pytest.mark.parametrize("d", [3, 4])
def test_sample_matches_oracle(gira, d):
    cl = synth.gmm_cloud4(5_000, 7, seed=13) if d == 4 else synth.gmm_cloud(5_000, 7, seed=13)
    w, m, c = (np.asarray(a, np.float32) for a in (cl.weights, cl.means, cl.covs))
    x, comp = gira.gira_gmm_sample(50_000, w, m, c, seed=99)
    rx, rcomp = oracle.sample(50_000, w, m, c, seed=99)
    np.testing.assert_array_equal(to_np(comp), rcomp)   # the component draw is an exact decision
    # Box-Muller through CUDA's binary64 log/sincos vs the C library's: a few ulp
    np.testing.assert_allclose(to_np(x), rx, rtol=2e-6, atol=2e-6)


def test_sample_device_output(gira):
    import torch
    cl = synth.gmm_cloud(2_000, 4, seed=3)
    w, m, c = (np.asarray(a, np.float32) for a in (cl.weights, cl.means, cl.covs))
    x, comp = gira.gira_gmm_sample(10_000, w, m, c, seed=1, device="cuda")
    assert x.is_cuda and comp.is_cuda and x.shape == (10_000, 3)
    rx, rcomp = oracle.sample(10_000, w, m, c, seed=1)
    np.testing.assert_array_equal(comp.cpu().numpy(), rcomp)


def test_d4_errors(gira):
    cl = synth.gmm_cloud4(3_000, 4, seed=5)
    bad = cl.points.copy()
    bad[100, 3] = np.nan
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_fit4(bad, 4, iters=3)
    assert e.value.status == gira.ERR_NONFINITE_INPUT
    w, m, c = (np.asarray(a, np.float32) for a in (cl.weights, cl.means, cl.covs))
    c2 = c.copy()
    c2[2] = -np.eye(4)
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_loglik4(cl.points, w, m, c2)
    assert e.value.status == gira.ERR_NOT_PD and e.value.component == 2
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_sample(10, w, m, c2, seed=0)
    assert e.value.status == gira.ERR_NOT_PD


# ----------------------------------------------------------------------------- K above 1024 (chunks of 512)
def test_fit4_chunked_from_given_init_matches_oracle(gira, frame4):
    pts = subset(frame4, 30_000, 5)
    K = 1100   # chunks of 512, 512, 76
    ki = oracle.kinit(pts, K, seed=0, lloyd_iters=4, reg=1e-6)
    w0, m0, c0 = (ki[a].astype(np.float32) for a in ("weights", "means", "covs"))
    r = gira.gira_gmm_fit4(pts, K, iters=3, tol=0.0, init=(w0, m0, c0))
    ref = oracle.em(pts, w0, m0, c0, iters=3, tol=0.0, reg=1e-6)
    assert r["iters_done"] == 3
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert abs(r["final_loglik"] - ref["final_ll"]) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_fit4_chunked_kmeans_init_matches_oracle_fit(gira, frame4):
    pts = subset(frame4, 20_000, 6)
    K = 1030
    r = gira.gira_gmm_fit4(pts, K, iters=2, tol=0.0, seed=7, lloyd_iters=3)
    ref = oracle.gmm_fit(pts, K, iters=2, tol=0.0, reg=1e-6, seed=7, lloyd_iters=3)
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_loglik4_chunked_k2048_with_outliers(gira, frame4):
    rng = np.random.default_rng(8)
    pts = subset(frame4, 25_000, 8)
    K = 2048
    idx = rng.choice(len(pts), K, replace=False)
    means = pts[idx].astype(np.float64) + rng.normal(scale=0.01, size=(K, 4))
    covs = []
    for _ in range(K):
        Q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
        lam = np.array([rng.uniform(0.02, 0.1), rng.uniform(0.02, 0.1), 0.01, 0.03]) ** 2
        covs.append(Q @ np.diag(lam) @ Q.T)
    w = rng.dirichlet(np.ones(K)).astype(np.float32)
    m, c = means.astype(np.float32), np.stack(covs).astype(np.float32)
    # far points: every component's term underflows the common reference -> exact step
    far = np.concatenate([rng.normal(size=(15, 3)) * 5.0 + np.array([0.0, 0.0, 300.0]), rng.uniform(size=(15, 1))],
                         axis=1).astype(np.float32)
    allp = np.concatenate([pts, far])
    mean, pp = gira.gira_gmm_loglik4(allp, w, m, c, per_point=True)
    pp = to_np(pp).astype(np.float64)
    assert np.all(np.isfinite(pp))
    assert mean == pytest.approx(pp.mean(), rel=1e-6)
    sample = np.concatenate([rng.choice(len(pts), 300, replace=False), np.arange(len(pts), len(allp))])
    _, _, lse = oracle.estep(allp[sample], w, m, c, want_resp=False, want_lse=True)
    err = np.abs(pp[sample] - lse)
    bound = per_point_bound(allp[sample], w, m, c, form="d")
    assert np.all(err <= bound), np.max(err / bound)


def test_fit4_dependent_launches_give_the_same_fit(gira):
    """As in 3D: the 4D EM loop's dependent launches and plain launches (per-launch
    profiling) give the same bits."""
    cl = synth.gmm_cloud4(30_000, 10, seed=32)
    runs = []
    for launches in (False, True):
        gira.gira_profile_enable(True, launches=launches)
        try:
            runs.append(gira.gira_gmm_fit4(cl.points, 40, iters=12, tol=0.0, seed=6, lloyd_iters=4))
        finally:
            gira.gira_profile_enable(False)
    gira.gira_profile_read(reset=True)
    for key in ("weights", "means", "covs"):
        np.testing.assert_array_equal(to_np(runs[0][key]), to_np(runs[1][key]))
    assert runs[0]["final_loglik"] == runs[1]["final_loglik"]
