"""Pins of the FP64 oracle against things other than itself (no GPU).

Each test fixes the oracle to mathematics or to an independent computation:
closed forms, library routines run at test time (scipy, scikit-learn),
brute-force enumeration on tiny inputs, invariants, published RNG vectors and
recovery of known generating mixtures.  GIRA (arXiv 2307.00071) Sec. V gives
the E-step (Eq. estep / logestep / simplifiedGaussian); the M-step and
k-means initialisation are the standard ones the paper defers to.
"""
import itertools
import os
import warnings

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2307_00071_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------- RNG
def test_splitmix64_published_vectors():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 6
    for seed, j, want in rows:
        assert oracle.splitmix64(int(seed), int(j)) == int(want)


def test_uniform_is_top_53_bits():
    for seed in (0, 7, 2**63 + 5):
        for j in range(4):
            u = oracle.uniform(seed, j)
            assert 0.0 <= u < 1.0
            assert u == (oracle.splitmix64(seed, j) >> 11) / 2.0**53


# ------------------------------------------------------------------------------- log-density
def _random_spd(rng, scale=1.0):
    a = rng.standard_normal((3, 3))
    return scale * (a @ a.T + 0.3 * np.eye(3))


def _logpdf_cofactor_longdouble(x, mu, cov):
    """ln N via explicit adjugate inverse and determinant in long double."""
    c = cov.astype(np.longdouble)
    d = (x - mu).astype(np.longdouble)
    adj = np.empty((3, 3), dtype=np.longdouble)
    for i in range(3):
        for j in range(3):
            m = np.delete(np.delete(c, i, 0), j, 1)
            adj[j, i] = (-1) ** (i + j) * (m[0, 0] * m[1, 1] - m[0, 1] * m[1, 0])
    det = c[0, 0] * adj[0, 0] + c[0, 1] * adj[1, 0] + c[0, 2] * adj[2, 0]
    q = d @ (adj / det) @ d
    return float(-0.5 * (3 * np.log(np.longdouble(2) * np.pi) + np.log(det) + q))


def test_log_gaussian_matches_scipy_and_cofactor_form():
    rng = np.random.default_rng(11)
    for trial in range(50):
        cov = _random_spd(rng, scale=10.0 ** rng.uniform(-4, 1))
        mu = rng.uniform(-5, 5, 3)
        x = mu + rng.standard_normal(3) * 2 * np.sqrt(np.diag(cov))
        got = oracle.log_gaussian(x, mu, cov)
        ref = stats.multivariate_normal(mu, cov).logpdf(x)
        cof = _logpdf_cofactor_longdouble(x, mu, cov)
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (trial, got, ref)
        assert abs(got - cof) <= 1e-12 * max(1.0, abs(cof)), (trial, got, cof)


def test_cholesky_and_inverse_identities():
    rng = np.random.default_rng(3)
    for _ in range(20):
        S = _random_spd(rng)
        L = oracle.cholesky3(S)
        assert np.allclose(np.triu(L, 1), 0)
        assert np.all(np.diag(L) > 0)
        assert np.allclose(L @ L.T, S, rtol=1e-13, atol=1e-13)
        P = oracle.tri_inverse3(L)
        assert np.allclose(P @ L, np.eye(3), atol=1e-13)
        # sum ln diag(P) == ln |Sigma|^{-1/2}  (the paper's remark after Eq. simplifiedGaussian)
        assert abs(np.log(np.diag(P)).sum() + 0.5 * np.linalg.slogdet(S)[1]) < 1e-12
    with pytest.raises(oracle.OracleError):
        oracle.cholesky3(np.diag([1.0, -1.0, 1.0]))


# ------------------------------------------------------------------------------- E-step
def _params(rng, K, spread=2.0):
    w = rng.dirichlet(np.ones(K))
    mu = rng.uniform(-spread, spread, (K, 3))
    cov = np.stack([_random_spd(rng, 0.05) for _ in range(K)])
    return w, mu, cov


def test_estep_matches_scipy_responsibilities():
    rng = np.random.default_rng(5)
    K = 4
    w, mu, cov = _params(rng, K)
    pts = rng.uniform(-2.5, 2.5, (300, 3)).astype(np.float32)
    ll, resp, lse = oracle.estep(pts, w, mu, cov, want_lse=True)
    logp = np.stack([np.log(w[b]) + stats.multivariate_normal(mu[b], cov[b]).logpdf(pts.astype(np.float64))
                     for b in range(K)], axis=1)
    ref_lse = np.logaddexp.reduce(logp, axis=1)
    assert np.allclose(lse, ref_lse, rtol=0, atol=1e-10)
    assert np.allclose(resp, np.exp(logp - ref_lse[:, None]), rtol=1e-10, atol=1e-13)
    assert abs(ll - ref_lse.mean()) < 1e-11
    assert np.allclose(resp.sum(1), 1.0, atol=1e-12, rtol=0)


def test_estep_far_point_does_not_underflow():
    """Log-domain E-step (Eq. logestep): a point far from every component keeps a finite loglik."""
    w, mu, cov = np.array([0.5, 0.5]), np.zeros((2, 3)), np.stack([np.eye(3) * 1e-4] * 2)
    mu[1, 0] = 1.0
    pts = np.array([[50.0, 0, 0]], np.float32)
    ll, resp, _ = oracle.estep(pts, w, mu, cov)
    assert np.isfinite(ll) and ll < -1e6
    assert resp[0, 1] == pytest.approx(1.0)


# ------------------------------------------------------------------------------- M-step / K=1
def test_k1_single_step_is_sample_mean_and_covariance():
    rng = np.random.default_rng(8)
    pts = (rng.standard_normal((5000, 3)) @ np.array([[1, 0, 0], [0.3, 0.5, 0], [0.1, -0.2, 0.05]]).T
           + np.array([3.0, -1.0, 7.0])).astype(np.float32)
    reg = 1e-6
    r = oracle.em(pts, [1.0], np.zeros((1, 3)), np.eye(3)[None], iters=1, tol=0.0, reg=reg)
    x = pts.astype(np.longdouble)
    mean = x.mean(0)
    cov = ((x - mean).T @ (x - mean)) / len(x) + reg * np.eye(3)
    assert r["weights"][0] == 1.0
    assert np.allclose(r["means"][0], mean.astype(np.float64), rtol=0, atol=1e-12)
    assert np.allclose(r["covs"][0], cov.astype(np.float64), rtol=1e-11, atol=1e-14)
    ll = stats.multivariate_normal(mean.astype(np.float64), cov.astype(np.float64)).logpdf(pts.astype(np.float64))
    assert abs(r["final_ll"] - ll.mean()) < 1e-11
    # the E-step with K=1 gives responsibilities 1 whatever the parameters, so the trace is
    # the loglik of the (arbitrary) start and the final loglik is the one at the closed form
    assert r["iters_done"] == 1 and r["final_ll"] > r["trace"][0]


def test_mstep_matches_enumerated_sufficient_statistics():
    """Brute force: posterior-weighted enumeration over all K^N assignments."""
    rng = np.random.default_rng(21)
    N, K, reg = 6, 3, 1e-5
    w, mu, cov = _params(rng, K, spread=0.6)
    pts = rng.uniform(-0.8, 0.8, (N, 3)).astype(np.float32)
    x = pts.astype(np.float64)
    dens = np.stack([w[b] * stats.multivariate_normal(mu[b], cov[b]).pdf(x) for b in range(K)], axis=1)
    Z = 0.0
    S0, S1 = np.zeros(K), np.zeros((K, 3))
    for z in itertools.product(range(K), repeat=N):
        p = np.prod([dens[n, z[n]] for n in range(N)])
        Z += p
        for n in range(N):
            S0[z[n]] += p
            S1[z[n]] += p * x[n]
    S0, S1 = S0 / Z, S1 / Z
    ll, resp, _ = oracle.estep(pts, w, mu, cov)
    assert abs(np.log(Z) - N * ll) < 1e-10                      # sum over assignments = exp(N l)
    ww, mm, cc = oracle.mstep(pts, resp, reg)
    nb = S0 + 10 * np.finfo(float).eps
    mu_ref = S1 / nb[:, None]
    S2 = np.zeros((K, 3, 3))
    for z in itertools.product(range(K), repeat=N):
        p = np.prod([dens[n, z[n]] for n in range(N)]) / Z
        for n in range(N):
            d = x[n] - mu_ref[z[n]]
            S2[z[n]] += p * np.outer(d, d)
    cov_ref = S2 / nb[:, None, None] + reg * np.eye(3)
    assert np.allclose(ww, nb / nb.sum(), rtol=1e-10, atol=1e-14)
    assert np.allclose(mm, mu_ref, rtol=1e-10, atol=1e-12)
    assert np.allclose(cc, cov_ref, rtol=1e-9, atol=1e-13)


def test_dead_component_convention():
    """A component with no responsibility: N_b = 10 eps, so mu = 0 and Sigma = reg I (sklearn convention)."""
    pts = np.array([[1, 2, 3], [2, 3, 4], [1.5, 2, 3.5]], np.float32)
    resp = np.array([[1.0, 0.0], [1.0, 0.0], [1.0, 0.0]])
    w, m, c = oracle.mstep(pts, resp, 1e-3)
    assert np.allclose(m[1], 0.0) and np.allclose(c[1], 1e-3 * np.eye(3))
    assert w[1] < 1e-14 and abs(w.sum() - 1) < 1e-15


def test_mstep_reports_non_pd():
    pts = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], np.float32)   # collinear: singular covariance
    resp = np.ones((3, 1))
    with pytest.raises(oracle.OracleError) as e:
        oracle.mstep(pts, resp, 0.0)
    assert e.value.code == oracle.ERR_NOT_PD and oracle.last_bad_component() == 0
    oracle.mstep(pts, resp, 1e-6)   # regularised: fine


# ------------------------------------------------------------------------------- EM invariants
@pytest.fixture(scope="module")
def cloud0():
    return synth.gmm_cloud(20_000, 8, seed=0)


def test_em_monotone_and_valid(cloud0):
    pts = cloud0.points
    for reg, slack in ((0.0, 1e-12), (1e-6, 1e-10)):
        ki = oracle.kinit(pts, 8, seed=0, lloyd_iters=10, reg=max(reg, 1e-9))
        r = oracle.em(pts, ki["weights"], ki["means"], ki["covs"], iters=20, tol=0.0, reg=reg)
        tr = np.append(r["trace"], r["final_ll"])
        assert np.all(np.diff(tr) >= -slack), np.diff(tr).min()
        assert abs(r["weights"].sum() - 1) < 1e-14
        for c in r["covs"]:
            assert np.allclose(c, c.T, atol=0)
            assert np.all(np.linalg.eigvalsh(c) > 0)


def test_em_translation_invariance():
    # points on a 2^-18 grid inside [-4, 4]: adding v (also on the grid) is exact in binary32
    cl = synth.gmm_cloud(3000, 3, seed=9)
    pts = np.round(cl.points.astype(np.float64) * 2**18) / 2**18
    v = np.array([1.5, -2.25, 0.75])
    a, b = pts.astype(np.float32), (pts + v).astype(np.float32)
    assert np.array_equal(b.astype(np.float64) - v, a.astype(np.float64))
    # start from live components: with N_b near 10 eps the M-step convention
    # mu = sum r x / (sum r + 10 eps) is (correctly) not translation-equivariant
    w, mu, cov = cl.weights, cl.means, cl.covs
    ra = oracle.em(a, w, mu, cov, iters=5)
    rb = oracle.em(b, w, mu + v, cov, iters=5)
    assert np.allclose(ra["weights"], rb["weights"], rtol=1e-9, atol=1e-12)
    assert np.allclose(ra["means"] + v, rb["means"], rtol=0, atol=1e-9)
    assert np.allclose(ra["covs"], rb["covs"], rtol=1e-8, atol=1e-12)
    assert np.allclose(ra["trace"], rb["trace"], rtol=0, atol=1e-9)


def test_em_tol_stops_early(cloud0):
    ki = oracle.kinit(cloud0.points, 8, 0, 10, 1e-6)
    r = oracle.em(cloud0.points, ki["weights"], ki["means"], ki["covs"], iters=200, tol=1e-3)
    t = r["trace"]
    assert r["iters_done"] < 200
    assert abs(t[-1] - t[-2]) < 1e-3 and np.all(np.abs(np.diff(t[:-1])) >= 1e-3)


def test_em_matches_sklearn_steps():
    skm = pytest.importorskip("sklearn.mixture")
    c = synth.gmm_cloud(4000, 5, seed=13)
    ki = oracle.kinit(c.points, 5, seed=3, lloyd_iters=4, reg=1e-6)
    for n in (1, 3, 10):
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            g = skm.GaussianMixture(5, covariance_type="full", reg_covar=1e-6, tol=0.0, max_iter=n,
                                    weights_init=ki["weights"], means_init=ki["means"],
                                    precisions_init=np.linalg.inv(ki["covs"])).fit(c.points.astype(np.float64))
        r = oracle.em(c.points, ki["weights"], ki["means"], ki["covs"], iters=n, tol=0.0, reg=1e-6)
        assert g.n_iter_ == r["iters_done"] == n
        assert np.allclose(g.weights_, r["weights"], rtol=1e-10, atol=1e-13)
        assert np.allclose(g.means_, r["means"], rtol=1e-10, atol=1e-12)
        assert np.allclose(g.covariances_, r["covs"], rtol=1e-9, atol=1e-14)
        assert abs(g.lower_bound_ - r["trace"][-1]) < 1e-10


def test_recovers_generating_mixture(cloud0):
    r = oracle.gmm_fit(cloud0.points, 8, iters=100, tol=1e-10, reg=1e-6, seed=0, lloyd_iters=10)
    used = set()
    for b in range(8):
        j = min((j for j in range(8) if j not in used), key=lambda j: np.linalg.norm(r["means"][j] - cloud0.means[b]))
        used.add(j)
        nb = r["weights"][j] * len(cloud0.points)
        bound = 4 * np.sqrt(np.linalg.eigvalsh(cloud0.covs[b]).max() / nb)
        assert np.linalg.norm(r["means"][j] - cloud0.means[b]) < bound
        assert abs(r["weights"][j] - cloud0.weights[b]) < 5 * np.sqrt(cloud0.weights[b] / len(cloud0.points)) + 1e-3
        rel = np.linalg.norm(r["covs"][j] - cloud0.covs[b]) / np.linalg.norm(cloud0.covs[b])
        assert rel < 0.15


# ------------------------------------------------------------------------------- k-means
def test_dist2_f32_is_binary32_fixed_order():
    rng = np.random.default_rng(2)
    for _ in range(200):
        x = rng.uniform(-9, 9, 3).astype(np.float32)
        c = rng.uniform(-9, 9, 3).astype(np.float32)
        d = (x - c).astype(np.float32)
        p = (d * d).astype(np.float32)
        want = np.float32(np.float32(p[0] + p[1]) + p[2])
        assert oracle.dist2_f32(x, c) == want
        # and it is the squared distance up to binary32 rounding
        assert abs(float(want) - float(((x.astype(float) - c) ** 2).sum())) <= 4e-7 * float(want) + 1e-30


def test_kmeanspp_first_centre_uniform_and_draw_proportional_to_d2():
    """Empirical check of the k-means++ sampling law on a tiny cloud (chi-square)."""
    pts = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0], [3, 3, 3], [0.5, 0.5, 0.5]], np.float32)
    N, trials = len(pts), 6000
    first = np.zeros(N)
    second = np.zeros((N, N))
    for s in range(trials):
        _, ch = oracle.kmeanspp(pts, 2, seed=s)
        first[ch[0]] += 1
        second[ch[0], ch[1]] += 1
    chi = ((first - trials / N) ** 2 / (trials / N)).sum()
    assert chi < stats.chi2.ppf(0.999, N - 1)
    for a in range(N):
        d2 = ((pts.astype(float) - pts[a]) ** 2).sum(1)
        p = d2 / d2.sum()
        cnt = second[a]
        assert cnt[a] == 0
        m = p > 0
        exp_ = p[m] * cnt.sum()
        assert (((cnt[m] - exp_) ** 2) / exp_).sum() < stats.chi2.ppf(0.999, m.sum() - 1)


def test_kmeanspp_picks_distinct_points_and_duplicates_fallback():
    pts = synth.uniform_cloud(500, seed=1)
    _, ch = oracle.kmeanspp(pts, 50, seed=4)
    assert len(set(ch.tolist())) == 50
    dup = np.repeat(pts[:3], 4, axis=0)           # 12 points, 3 distinct locations
    cen, ch = oracle.kmeanspp(dup, 5, seed=1)      # more centres than distinct points
    assert len({tuple(c) for c in cen[:3]}) == 3    # the first three cover every location
    for j in range(3, 5):                           # then D^2 == 0 everywhere: uniform index
        assert ch[j] == min(int(np.floor(oracle.uniform(1, j) * 12)), 11)


def test_lloyd_fixed_point_and_monotone_sse(cloud0):
    pts = cloud0.points
    c0, _ = oracle.kmeanspp(pts, 8, seed=0)
    sse = []
    for it in range(0, 8):
        c, lab, done = oracle.lloyd(pts, c0, it)
        sse.append(((pts.astype(float) - c[lab].astype(float)) ** 2).sum())
    assert np.all(np.diff(sse) <= 1e-9 * sse[0])
    c, lab, done = oracle.lloyd(pts, c0, 100)
    assert done < 100                                   # converged: no label changed
    d = ((pts.astype(float)[:, None, :] - c.astype(float)[None]) ** 2).sum(-1)
    best = np.sort(d, 1)
    clear = (best[:, 1] - best[:, 0]) > 1e-5 * best[:, 1]
    assert np.array_equal(lab[clear], d.argmin(1)[clear])
    for b in range(8):
        assert np.array_equal(c[b], pts[lab == b].astype(np.float64).mean(0).astype(np.float32))


def test_lloyd_ties_go_to_lowest_index():
    pts = np.array([[0, 0, 0], [2, 0, 0], [1, 0, 0]], np.float32)
    c, lab, _ = oracle.lloyd(pts, np.array([[0, 0, 0], [2, 0, 0]], np.float32), 0)
    assert lab.tolist() == [0, 1, 0]


def test_init_from_labels_is_per_cluster_sample_moments():
    pts = synth.gmm_cloud(2000, 4, seed=2).points
    lab = np.random.default_rng(0).integers(0, 4, len(pts)).astype(np.int32)
    w, m, c = oracle.init_from_labels(pts, lab, 4, 1e-6)
    for b in range(4):
        x = pts[lab == b].astype(np.float64)
        assert abs(w[b] - len(x) / len(pts)) < 1e-12
        assert np.allclose(m[b], x.mean(0), atol=1e-12)
        assert np.allclose(c[b], np.cov(x.T, bias=True) + 1e-6 * np.eye(3), rtol=1e-10, atol=1e-14)


def test_invalid_arguments_and_nonfinite():
    pts = synth.uniform_cloud(10)
    with pytest.raises(oracle.OracleError) as e:
        oracle.kmeanspp(pts, 11, 0)
    assert e.value.code == oracle.ERR_INVALID_ARG
    bad = pts.copy()
    bad[3, 1] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.estep(bad, [1.0], np.zeros((1, 3)), np.eye(3)[None])
    assert e.value.code == oracle.ERR_NONFINITE


# ------------------------------------------------------------------------------- fixed-point draw
def test_fx48_is_exact_floor():
    from fractions import Fraction
    rng = np.random.default_rng(7)
    vals = np.concatenate([rng.uniform(0, 100, 300), 10.0 ** rng.uniform(-20, 14, 300), [0.0, 1e-30, 2.0**-48,
                                                                                           2.0**-49, 3.0]])
    for d in vals.astype(np.float32):
        want = int(Fraction(float(d)) * 2**48) if d < 2.0**47 else 2**95 - 1
        assert oracle.fx48(d) == want, d
    assert oracle.fx48(np.float32(2.0**47)) == 2**95 - 1


def test_fx_threshold_is_exact_floor():
    rng = np.random.default_rng(8)
    for _ in range(300):
        k = int(rng.integers(0, 2**53))
        T = int(rng.integers(1, 2**63)) << int(rng.integers(0, 64)) | int(rng.integers(0, 2**63))
        T &= (1 << 127) - 1
        assert oracle.fx_threshold(k, T) == (k * T) >> 53
    assert oracle.fx_threshold(2**53 - 1, 2**127 - 1) == ((2**53 - 1) * (2**127 - 1)) >> 53


def _kmeanspp_fp64_cumsum(pts, K, seed):
    """Independent k-means++: binary32 distances, binary64 cumsum, searchsorted."""
    x = pts.astype(np.float32)
    idx = min(int(np.floor(oracle.uniform(seed, 0) * len(x))), len(x) - 1)
    chosen = [idx]
    d2 = None
    for j in range(1, K):
        d = (x - x[chosen[-1]]).astype(np.float32)
        p = (d * d).astype(np.float32)
        dn = ((p[:, 0] + p[:, 1]).astype(np.float32) + p[:, 2]).astype(np.float32)
        d2 = dn if d2 is None else np.minimum(d2, dn)
        cs = np.cumsum(d2.astype(np.float64))
        t = oracle.uniform(seed, j) * cs[-1]
        chosen.append(int(np.searchsorted(cs, t, side="right")))
    return np.array(chosen)


def test_fixed_point_draw_matches_floating_point_sampling():
    """Away from measure-zero near-ties the exact draw equals the binary64 cumsum draw."""
    for seed in range(12):
        pts = synth.gmm_cloud(3000, 6, seed=seed).points
        _, ch = oracle.kmeanspp(pts, 25, seed)
        assert np.array_equal(ch, _kmeanspp_fp64_cumsum(pts, 25, seed)), seed
