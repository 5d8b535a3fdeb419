"""Pins of the oracle in four dimensions (xyz + intensity, the paper's SOGMM data)
and of its mixture regression (intensity given xyz) and sampling (no GPU).

The four-dimensional code is the same generic code the three-dimensional pins
already fix; these pins fix what d = 4 adds: scipy's 4D log-density, the K = 1
closed form, scikit-learn's EM steps, the binary32 4D distance order; the
regression against closed forms and brute force; the sampler against the law
it must follow and a direct re-computation of its first draws.
"""
import warnings

import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

import oracle
from paper_2307_00071_gb300 import synth


@pytest.fixture(scope="module")
def cloud4():
    return synth.gmm_cloud4(3_000, 5, seed=4)


def test_log_density_4d_matches_scipy(cloud4):
    rng = np.random.default_rng(1)
    for b in range(3):
        x = rng.normal(size=4)
        want = stats.multivariate_normal(cloud4.means[b], cloud4.covs[b]).logpdf(x)
        assert oracle.log_gaussian(x, cloud4.means[b], cloud4.covs[b]) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_estep_4d_matches_scipy(cloud4):
    pts = cloud4.points[:400]
    w, m, c = cloud4.weights, cloud4.means, cloud4.covs
    ll, resp, lse = oracle.estep(pts, w, m, c, want_lse=True)
    comp = np.stack([np.log(w[b]) + stats.multivariate_normal(m[b], c[b]).logpdf(pts.astype(np.float64))
                     for b in range(len(w))], axis=1)
    want = logsumexp(comp, axis=1)
    np.testing.assert_allclose(lse, want, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(resp, np.exp(comp - want[:, None]), rtol=1e-10, atol=1e-13)
    assert ll == pytest.approx(want.mean(), rel=1e-12)


def test_single_component_4d_closed_form(cloud4):
    pts = cloud4.points.astype(np.float64)
    mu = pts.mean(0)
    S = (pts - mu).T @ (pts - mu) / len(pts)
    w, m, c = oracle.mstep(cloud4.points, np.ones((len(pts), 1)), 0.0)
    np.testing.assert_allclose(m[0], mu, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(c[0], S, rtol=1e-10, atol=1e-14)
    ll, _, _ = oracle.estep(cloud4.points, w, m, c, want_resp=False)
    want = stats.multivariate_normal(mu, S).logpdf(pts).mean()
    assert ll == pytest.approx(want, rel=1e-12)


def test_em_4d_matches_sklearn_steps(cloud4):
    skm = pytest.importorskip("sklearn.mixture")
    ki = oracle.kinit(cloud4.points, 5, seed=3, lloyd_iters=4, reg=1e-6)
    assert ki["means"].shape == (5, 4)
    for n in (1, 4):
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            g = skm.GaussianMixture(5, covariance_type="full", reg_covar=1e-6, tol=0.0, max_iter=n,
                                    weights_init=ki["weights"], means_init=ki["means"],
                                    precisions_init=np.linalg.inv(ki["covs"])).fit(cloud4.points.astype(np.float64))
        r = oracle.em(cloud4.points, ki["weights"], ki["means"], ki["covs"], iters=n, tol=0.0, reg=1e-6)
        assert g.n_iter_ == r["iters_done"] == n
        assert np.allclose(g.weights_, r["weights"], rtol=1e-10, atol=1e-13)
        assert np.allclose(g.means_, r["means"], rtol=1e-10, atol=1e-12)
        assert np.allclose(g.covariances_, r["covs"], rtol=1e-9, atol=1e-14)
        assert abs(g.lower_bound_ - r["trace"][-1]) < 1e-10


def test_dist2_4d_fixed_binary32_order():
    rng = np.random.default_rng(2)
    for _ in range(200):
        x, c = rng.normal(size=4).astype(np.float32), rng.normal(size=4).astype(np.float32)
        d = x - c
        p = d * d
        want = ((p[0] + p[1]) + p[2]) + p[3]   # binary32, left to right
        assert oracle.dist2_f32(x, c) == want


def test_lloyd_4d_fixed_point_and_means(cloud4):
    c0, _ = oracle.kmeanspp(cloud4.points, 6, seed=5)
    assert c0.shape == (6, 4)
    c, lab, done = oracle.lloyd(cloud4.points, c0, 50)
    assert done < 50   # converged
    d = ((cloud4.points[:, None, :].astype(np.float64) - c[None].astype(np.float64)) ** 2).sum(-1)
    assert np.all(lab == np.argmin(d, axis=1))
    for b in range(6):
        np.testing.assert_allclose(c[b], cloud4.points[lab == b].astype(np.float64).mean(0), rtol=1e-6, atol=1e-6)


# ------------------------------------------------------------------------ regression
def _single(rng):
    A = rng.normal(size=(4, 4))
    return rng.normal(size=4), A @ A.T + 0.5 * np.eye(4)


def test_conditional_single_component_closed_form():
    rng = np.random.default_rng(3)
    mu, S = _single(rng)
    locs = rng.normal(size=(50, 3)).astype(np.float32)
    e, v = oracle.conditional4(locs, [1.0], mu[None], S[None])
    g = np.linalg.solve(S[:3, :3], S[:3, 3])
    np.testing.assert_allclose(e, mu[3] + (locs.astype(np.float64) - mu[:3]) @ g, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(v, S[3, 3] - S[3, :3] @ g, rtol=1e-12)


def test_conditional_mixture_brute_force():
    rng = np.random.default_rng(4)
    K = 3
    mus, Ss = zip(*[_single(rng) for _ in range(K)])
    w = rng.dirichlet(np.ones(K))
    locs = rng.normal(size=(40, 3)).astype(np.float32)
    e, v = oracle.conditional4(locs, w, np.array(mus), np.array(Ss))
    x = locs.astype(np.float64)
    lw = np.stack([np.log(w[b]) + stats.multivariate_normal(mus[b][:3], Ss[b][:3, :3]).logpdf(x) for b in range(K)], 1)
    r = np.exp(lw - logsumexp(lw, axis=1, keepdims=True))
    m = np.stack([mus[b][3] + (x - mus[b][:3]) @ np.linalg.solve(Ss[b][:3, :3], Ss[b][:3, 3]) for b in range(K)], 1)
    vv = np.array([Ss[b][3, 3] - Ss[b][3, :3] @ np.linalg.solve(Ss[b][:3, :3], Ss[b][:3, 3]) for b in range(K)])
    want_e = (r * m).sum(1)
    np.testing.assert_allclose(e, want_e, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(v, (r * (vv[None] + m * m)).sum(1) - want_e ** 2, rtol=1e-9, atol=1e-12)


def test_conditional_uncorrelated_components_give_weighted_means():
    rng = np.random.default_rng(5)
    K = 4
    mus = rng.normal(size=(K, 4))
    Ss = np.array([np.diag(rng.uniform(0.5, 2.0, size=4)) for _ in range(K)])
    w = rng.dirichlet(np.ones(K))
    locs = rng.normal(size=(30, 3)).astype(np.float32)
    e, v = oracle.conditional4(locs, w, mus, Ss)
    x = locs.astype(np.float64)
    lw = np.stack([np.log(w[b]) + stats.multivariate_normal(mus[b][:3], Ss[b][:3, :3]).logpdf(x) for b in range(K)], 1)
    r = np.exp(lw - logsumexp(lw, axis=1, keepdims=True))
    np.testing.assert_allclose(e, r @ mus[:, 3], rtol=1e-11)
    assert np.all(v > 0)


# ------------------------------------------------------------------------ sampling
def test_sample_first_draws_recomputed(cloud4):
    pts, comp = oracle.sample(20, cloud4.weights, cloud4.means, cloud4.covs, seed=9)
    cum = np.cumsum(cloud4.weights)
    L = np.linalg.cholesky(cloud4.covs)
    for i in range(20):
        u = [oracle.uniform(9, 5 * i + j) for j in range(5)]
        b = int(np.argmax(cum > u[0] * cum[-1]))
        assert comp[i] == b
        z = []
        for p in range(2):
            r = np.sqrt(-2.0 * np.log(1.0 - u[1 + 2 * p]))
            z += [r * np.cos(2 * np.pi * u[2 + 2 * p]), r * np.sin(2 * np.pi * u[2 + 2 * p])]
        want = (cloud4.means[b] + L[b] @ np.array(z)).astype(np.float32)
        np.testing.assert_allclose(pts[i], want, rtol=1e-6, atol=1e-6)


def test_sample_follows_the_mixture(cloud4):
    M = 60_000
    pts, comp = oracle.sample(M, cloud4.weights, cloud4.means, cloud4.covs, seed=11)
    counts = np.bincount(comp, minlength=len(cloud4.weights))
    chi2 = ((counts - M * cloud4.weights) ** 2 / (M * cloud4.weights)).sum()
    assert chi2 < stats.chi2(len(counts) - 1).ppf(0.999)
    for b in range(len(cloud4.weights)):
        x = pts[comp == b].astype(np.float64)
        se = np.sqrt(np.diag(cloud4.covs[b]) / len(x))
        assert np.all(np.abs(x.mean(0) - cloud4.means[b]) < 5 * se)
        np.testing.assert_allclose(np.cov(x.T), cloud4.covs[b], atol=6 * np.abs(cloud4.covs[b]).max() / np.sqrt(len(x)))


def test_sample_three_dimensional_mixture():
    cl = synth.gmm_cloud(1_000, 3, seed=2)
    pts, comp = oracle.sample(5, cl.weights, cl.means, cl.covs, seed=1)
    assert pts.shape == (5, 3) and comp.shape == (5,)
