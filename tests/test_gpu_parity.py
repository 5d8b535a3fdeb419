"""GPU parity: libgira (through the C ABI) against the FP64 oracle.

Same seeded inputs on both sides.  Integer decisions (k-means++ draws, Lloyd
labels) must agree bit for bit; floating-point results within the tolerances
of tests/_parity.py.  Sizes span several CTAs and a ragged tail; the 276k-point
depth frame with K=512 is the configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle
from paper_2307_00071_gb300 import synth

from _parity import LL_ABS, assert_model_close, max_rel_errors, model_mismatches, per_point_bound, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gira():
    from paper_2307_00071_gb300 import gira as g
    return g


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def random_model(rng, K, spread=2.0, scale=0.02):
    w = rng.dirichlet(np.ones(K))
    mu = rng.uniform(-spread, spread, (K, 3))
    cov = np.empty((K, 3, 3))
    for b in range(K):
        a = rng.standard_normal((3, 3))
        cov[b] = scale * (a @ a.T + 0.3 * np.eye(3))
    return w, mu, cov


def f32(*arrs):
    return [np.asarray(a, np.float32) for a in arrs]


# --------------------------------------------------------------------------- log-likelihood
@pytest.mark.parametrize("n,k", [(1, 1), (7, 3), (1237, 8), (5003, 64), (5003, 65), (4099, 200), (3001, 512),
                                 (2053, 1000)])
def test_loglik_matches_oracle(gira, n, k):
    rng = np.random.default_rng(n + k)
    w, mu, cov = f32(*random_model(rng, k))
    pts = rng.uniform(-2.2, 2.2, (n, 3)).astype(np.float32)
    ref_mean, _, ref_lse = oracle.estep(pts, w, mu, cov, want_resp=False, want_lse=True)
    mean, pp = gira.gira_gmm_loglik(dev(pts), dev(w), dev(mu), dev(cov), per_point=True)
    pp = to_np(pp).astype(np.float64)
    # random models put many points far from every component (|l| up to ~500), where the
    # binary32 value itself carries ~1e-7 relative rounding: allow that on top of 1e-5
    assert abs(mean - ref_mean) <= LL_ABS + 1e-7 * abs(ref_mean), (mean, ref_mean)
    err = np.abs(pp - ref_lse)
    bound = per_point_bound(pts, w, mu, cov)
    assert np.all(err <= bound), (err.max(), np.max(err / bound))


def test_loglik_host_and_device_pointers_agree(gira):
    rng = np.random.default_rng(1)
    w, mu, cov = f32(*random_model(rng, 16))
    pts = rng.uniform(-2, 2, (3000, 3)).astype(np.float32)
    m_host, pp_host = gira.gira_gmm_loglik(pts, w, mu, cov, per_point=True)
    m_dev, pp_dev = gira.gira_gmm_loglik(dev(pts), dev(w), dev(mu), dev(cov), per_point=True)
    assert m_host == m_dev
    assert np.array_equal(pp_host, to_np(pp_dev))


def test_loglik_far_outlier_takes_exact_max_path(gira):
    """A point > 100 binades below every component exercises the per-point max path."""
    w = np.array([0.5, 0.5], np.float32)
    mu = np.array([[0, 0, 0], [1, 0, 0]], np.float32)
    cov = np.stack([np.eye(3, dtype=np.float32) * 1e-4] * 2)
    pts = np.array([[0.01, 0, 0], [1.0, 0.02, 0], [3.0, 0, 0], [0.5, 0.5, 0.5]] * 5, np.float32)
    ref_mean, _, ref_lse = oracle.estep(pts, w, mu, cov, want_resp=False, want_lse=True)
    mean, pp = gira.gira_gmm_loglik(dev(pts), dev(w), dev(mu), dev(cov), per_point=True)
    pp = to_np(pp).astype(np.float64)
    assert np.all(np.abs(pp - ref_lse) <= per_point_bound(pts, w, mu, cov)), (pp, ref_lse)
    assert abs(mean - ref_mean) <= 1e-5 * abs(ref_mean)


# --------------------------------------------------------------------------- one EM step
@pytest.mark.parametrize("n,k", [(20_000, 8), (9_999, 3), (12_345, 64), (20_011, 100), (30_000, 256)])
def test_one_em_step_matches_oracle(gira, n, k):
    cl = synth.gmm_cloud(n, min(k, 16), seed=k)
    pts = cl.points
    ki = oracle.kinit(pts, k, seed=1, lloyd_iters=3, reg=1e-6)
    init = f32(ki["weights"], ki["means"], ki["covs"])
    ref = oracle.em(pts, *init, iters=1, tol=0.0, reg=1e-6)
    r = gira.gira_gmm_fit(dev(pts), k, iters=1, tol=0.0, reg_covar=1e-6, init=init)
    assert r["iters_done"] == 1
    assert abs(r["trace"][0] - ref["trace"][0]) <= LL_ABS
    assert abs(r["final_loglik"] - ref["final_ll"]) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_config0_full_run_matches_oracle(gira):
    """N=20k, K=8, 20 iterations from the oracle's k-means init (identical init)."""
    cl = synth.gmm_cloud(20_000, 8, seed=0)
    ki = oracle.kinit(cl.points, 8, seed=0, lloyd_iters=10, reg=1e-6)
    init = f32(ki["weights"], ki["means"], ki["covs"])
    ref = oracle.em(cl.points, *init, iters=20, tol=0.0, reg=1e-6)
    r = gira.gira_gmm_fit(dev(cl.points), 8, iters=20, tol=0.0, reg_covar=1e-6, init=init)
    assert r["iters_done"] == 20
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert abs(r["final_loglik"] - ref["final_ll"]) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_tol_stops_at_the_oracle_iteration(gira):
    cl = synth.gmm_cloud(20_000, 8, seed=0)
    ki = oracle.kinit(cl.points, 8, seed=0, lloyd_iters=10, reg=1e-6)
    init = f32(ki["weights"], ki["means"], ki["covs"])
    ref = oracle.em(cl.points, *init, iters=100, tol=1e-3, reg=1e-6)
    r = gira.gira_gmm_fit(dev(cl.points), 8, iters=100, tol=1e-3, reg_covar=1e-6, init=init)
    # the stopping iteration is an integer decided by floating point: equal unless the
    # change of the oracle's loglik lies within the loglik tolerance of tol
    tr = ref["trace"]
    near = np.any(np.abs(np.abs(np.diff(tr)) - 1e-3) < 2 * LL_ABS)
    assert r["iters_done"] == ref["iters_done"] or near
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


# --------------------------------------------------------------------------- k-means init
@pytest.mark.parametrize("n,k,seed", [(20_000, 8, 0), (5_001, 37, 3), (40_000, 256, 7), (2_048, 2_048 // 8, 11)])
def test_kmeanspp_centres_bit_exact(gira, n, k, seed):
    pts = synth.gmm_cloud(n, 8, seed=seed).points
    ref_c, _ = oracle.kmeanspp(pts, k, seed)
    c, _, done = gira.gira_kmeans_init(dev(pts), k, seed=seed, lloyd_iters=0)
    assert done == 0
    assert np.array_equal(to_np(c), ref_c)


@pytest.mark.parametrize("n,k,seed,iters", [(20_000, 8, 0, 10), (7_777, 50, 2, 4), (30_000, 512, 5, 10)])
def test_lloyd_labels_and_centres_bit_exact(gira, n, k, seed, iters):
    pts = synth.gmm_cloud(n, 12, seed=seed).points
    c0, _ = oracle.kmeanspp(pts, k, seed)
    ref_c, ref_lab, ref_done = oracle.lloyd(pts, c0, iters)
    c, lab, done = gira.gira_kmeans_init(dev(pts), k, seed=seed, lloyd_iters=iters)
    assert done == ref_done
    assert np.array_equal(to_np(lab), ref_lab)
    assert np.array_equal(to_np(c), ref_c)


def test_kmeans_duplicates_fallback(gira):
    pts = np.repeat(synth.uniform_cloud(3, seed=2), 40, axis=0)   # 120 points, 3 locations
    ref_c, _ = oracle.kmeanspp(pts, 6, 9)
    c, _, _ = gira.gira_kmeans_init(dev(pts), 6, seed=9, lloyd_iters=0)
    assert np.array_equal(to_np(c), ref_c)


def scan_cloud(n):
    """n points of three depth frames laid one after the other (N x 3)."""
    return np.ascontiguousarray(np.concatenate([synth.depth_frame(seed=s).points for s in (1, 2, 3)])[:n])


# On a 152-SM GPU that runs 16-CTA clusters these sizes take the three seeding
# kernels: one thread-block cluster (N <= 294,912), the persistent cooperative
# kernel (N <= 622,592), and one update + one select launch per centre.
@pytest.mark.parametrize("n", [200_000, 400_000, 700_000])
def test_kmeanspp_bit_exact_on_every_seeding_path(gira, n):
    pts = scan_cloud(n)
    ref_c, _ = oracle.kmeanspp(pts, 48, 5)
    c, _, _ = gira.gira_kmeans_init(dev(pts), 48, seed=5, lloyd_iters=0, want_labels=False)
    assert np.array_equal(to_np(c), ref_c)


def test_full_fit_with_kmeans_init_matches_oracle(gira):
    cl = synth.gmm_cloud(20_000, 8, seed=0)
    ref = oracle.gmm_fit(cl.points, 8, iters=20, tol=0.0, reg=1e-6, seed=0, lloyd_iters=10)
    r = gira.gira_gmm_fit(dev(cl.points), 8, iters=20, tol=0.0, reg_covar=1e-6, seed=0, lloyd_iters=10)
    assert r["iters_done"] == 20
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_host_buffers_give_the_same_fit(gira):
    cl = synth.gmm_cloud(6_000, 5, seed=4)
    rh = gira.gira_gmm_fit(cl.points, 5, iters=5, tol=0.0)
    rd = gira.gira_gmm_fit(dev(cl.points), 5, iters=5, tol=0.0)
    for key in ("weights", "means", "covs"):
        assert np.array_equal(rh[key], to_np(rd[key]))
    assert np.array_equal(rh["trace"], rd["trace"])


# --------------------------------------------------------------------------- edge cases
def test_k_equals_n_and_k1(gira):
    pts = synth.uniform_cloud(16, seed=3)
    r = gira.gira_gmm_fit(dev(pts), 16, iters=2, tol=0.0, reg_covar=1e-3)
    ref = oracle.gmm_fit(pts, 16, iters=2, tol=0.0, reg=1e-3, seed=0, lloyd_iters=10)
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))
    r1 = gira.gira_gmm_fit(dev(pts[:1]), 1, iters=3, tol=0.0, reg_covar=1e-4)
    assert np.allclose(to_np(r1["covs"])[0], 1e-4 * np.eye(3), rtol=1e-6)
    assert np.allclose(to_np(r1["means"])[0], pts[0])


def test_iters_zero_returns_init(gira):
    cl = synth.gmm_cloud(3_000, 4, seed=6)
    ki = oracle.kinit(cl.points, 4, seed=0, lloyd_iters=10, reg=1e-6)
    r = gira.gira_gmm_fit(dev(cl.points), 4, iters=0, tol=0.0)
    assert r["iters_done"] == 0 and len(r["trace"]) == 0
    assert_model_close((r["weights"], r["means"], r["covs"]), (ki["weights"], ki["means"], ki["covs"]))
    ll, _, _ = oracle.estep(cl.points, ki["weights"], ki["means"], ki["covs"], want_resp=False)
    assert abs(r["final_loglik"] - ll) <= LL_ABS


def test_nonfinite_points_rejected(gira):
    pts = synth.uniform_cloud(100)
    pts[17, 2] = np.nan
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_fit(dev(pts), 4, iters=3)
    assert e.value.status == gira.ERR_NONFINITE_INPUT
    pts[17, 2] = np.inf
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_loglik(dev(pts), dev(np.ones(1)), dev(np.zeros((1, 3))), dev(np.eye(3)[None]))
    assert e.value.status == gira.ERR_NONFINITE_INPUT


def test_not_pd_reports_component(gira):
    w, mu, cov = f32(*random_model(np.random.default_rng(0), 6))
    cov[4] = np.diag([1.0, -1.0, 1.0]).astype(np.float32)
    cov[5] = np.zeros((3, 3), np.float32)
    pts = synth.uniform_cloud(500)
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_loglik(dev(pts), dev(w), dev(mu), dev(cov))
    assert e.value.status == gira.ERR_NOT_PD and e.value.component == 4
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_fit(dev(pts), 6, iters=2, init=(w, mu, cov))
    assert e.value.status == gira.ERR_NOT_PD and e.value.component == 4


def test_collapsing_component_reports_not_pd_like_oracle(gira):
    pts = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [3, 0, 0]], np.float32)   # collinear
    init = (np.array([1.0], np.float32), np.zeros((1, 3), np.float32), np.eye(3, dtype=np.float32)[None])
    with pytest.raises(oracle.OracleError):
        oracle.em(pts, *init, iters=1, reg=0.0)
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_fit(dev(pts), 1, iters=1, reg_covar=0.0, init=init)
    assert e.value.status == gira.ERR_NOT_PD and e.value.component == 0


# --------------------------------------------------------------------------- full-size frame
@pytest.fixture(scope="module")
def frame():
    return synth.depth_frame(seed=1)


@pytest.fixture(scope="module")
def frame_init(frame):
    return oracle.kinit(frame.points, 512, seed=0, lloyd_iters=10, reg=1e-6)


def test_kmeanspp_cluster_exchange_is_stable_over_many_draws(gira, frame):
    """The cluster seeding kernel exchanges each centre's totals and chosen point
    as point-to-point messages on mbarriers that alternate by the parity of the
    centre: 48 seeds on the frame (K = 512, 511 exchanges each), each run twice,
    give the same centres run to run, and two of them equal the oracle's draws."""
    x = dev(frame.points)
    first = {}
    for rep in range(2):
        for seed in range(100, 148):
            c, _, _ = gira.gira_kmeans_init(x, 512, seed=seed, lloyd_iters=0, want_labels=False)
            c = to_np(c).copy()
            if rep == 0:
                first[seed] = c
            else:
                assert np.array_equal(c, first[seed]), seed
    for seed in (100, 129):
        ref_c, _ = oracle.kmeanspp(frame.points, 512, seed)
        assert np.array_equal(first[seed], ref_c), seed


def test_frame_kmeans_init_bit_exact(gira, frame, frame_init):
    c, lab, done = gira.gira_kmeans_init(dev(frame.points), 512, seed=0, lloyd_iters=10)
    assert done == frame_init["lloyd_done"]
    assert np.array_equal(to_np(c), frame_init["centers"])
    assert np.array_equal(to_np(lab), frame_init["labels"])


def test_frame_two_em_steps_match_oracle(gira, frame, frame_init):
    """276k points, K=512, in the launch configuration the benchmark times."""
    init = f32(frame_init["weights"], frame_init["means"], frame_init["covs"])
    ref = oracle.em(frame.points, *init, iters=2, tol=0.0, reg=1e-6)
    r = gira.gira_gmm_fit(dev(frame.points), 512, iters=2, tol=0.0, reg_covar=1e-6, init=init)
    assert np.max(np.abs(r["trace"] - ref["trace"])) <= LL_ABS
    assert abs(r["final_loglik"] - ref["final_ll"]) <= LL_ABS
    errs = max_rel_errors((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))
    bad = model_mismatches((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))
    assert not bad, (errs, bad[:10])


def test_frame_fit_is_valid_and_monotone(gira, frame):
    r = gira.gira_gmm_fit(dev(frame.points), 512, iters=30, tol=1e-4, reg_covar=1e-6, seed=0, lloyd_iters=10)
    tr = r["trace"]
    assert 1 <= r["iters_done"] <= 30
    assert np.all(np.diff(tr) >= -1e-5)
    w = to_np(r["weights"])
    assert abs(w.sum() - 1) < 1e-5 and np.all(w > 0)
    c = to_np(r["covs"]).astype(np.float64)
    assert np.all(np.linalg.eigvalsh(0.5 * (c + c.transpose(0, 2, 1))) > 0)


def test_resume_from_saved_parameters(gira):
    """Checkpoint / resume: a fit continued from the parameters it returned (the
    caller's saved binary32 model) follows the uninterrupted fit."""
    cl = synth.gmm_cloud(20_000, 8, seed=12)
    full = gira.gira_gmm_fit(dev(cl.points), 8, iters=16, tol=0.0, seed=3)
    first = gira.gira_gmm_fit(dev(cl.points), 8, iters=8, tol=0.0, seed=3)
    saved = tuple(to_np(first[a]).copy() for a in ("weights", "means", "covs"))
    rest = gira.gira_gmm_fit(dev(cl.points), 8, iters=8, tol=0.0, init=saved)
    np.testing.assert_allclose(first["trace"], full["trace"][:8], atol=1e-12)
    assert np.max(np.abs(rest["trace"] - full["trace"][8:])) <= LL_ABS
    assert_model_close((rest["weights"], rest["means"], rest["covs"]),
                       tuple(to_np(full[a]).astype(np.float64) for a in ("weights", "means", "covs")))


def test_calls_on_a_side_stream_match_the_default_stream(gira):
    """Every call runs on torch's current stream: on a side stream, with device inputs
    written on that stream, the results equal those on the default stream."""
    cl = synth.gmm_cloud(10_000, 6, seed=21)
    ref = gira.gira_gmm_fit(dev(cl.points), 6, iters=6, tol=0.0, seed=2)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        x = torch.as_tensor(cl.points, device="cuda")   # written on the side stream
        r = gira.gira_gmm_fit(x, 6, iters=6, tol=0.0, seed=2)
        ll = gira.gira_gmm_loglik(x, r["weights"], r["means"], r["covs"])
    side.synchronize()
    for key in ("weights", "means", "covs"):
        assert torch.equal(r[key], ref[key])
    np.testing.assert_array_equal(r["trace"], ref["trace"])
    assert abs(ll - r["final_loglik"]) < 1e-5


def test_dependent_launches_give_the_same_fit(gira):
    """The EM loop launches the E-step and the binary64 finalize as programmatic
    dependents of one another, except when per-launch profiling brackets every
    E-step with an event pair (plain launches): both orders of execution give
    the same bits, including a run that stops early on its tolerance."""
    cl = synth.gmm_cloud(30_000, 10, seed=31)
    x = dev(cl.points)
    for tol in (0.0, 1e-3):
        runs = []
        for launches in (False, True):
            gira.gira_profile_enable(True, launches=launches)
            try:
                runs.append(gira.gira_gmm_fit(x, 48, iters=14, tol=tol, seed=5, lloyd_iters=4))
            finally:
                gira.gira_profile_enable(False)
        prof = gira.gira_profile_read(reset=True)
        assert prof["estep_launches"] > 0   # the second run was timed launch by launch
        for key in ("weights", "means", "covs"):
            assert torch.equal(runs[0][key], runs[1][key])
        np.testing.assert_array_equal(runs[0]["trace"], runs[1]["trace"])
        assert runs[0]["iters_done"] == runs[1]["iters_done"]
