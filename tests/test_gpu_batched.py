"""Batched EM (gira_gmm_fit_batched) against the FP64 oracle, instance by instance.

Every instance must meet the single fit's tolerances (tests/_parity.py): the
batch only changes how the work is laid out on the GPU, not what is computed.
"""
import numpy as np
import pytest

import oracle
from paper_2307_00071_gb300 import synth
from tests._parity import LL_ABS, assert_model_close, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gira():
    from paper_2307_00071_gb300 import gira as g
    return g


def make_batch(sizes, ks, seed=0):
    clouds = [synth.gmm_cloud(n, max(2, min(k, 12)), seed=seed + i).points for i, (n, k) in enumerate(zip(sizes, ks))]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return clouds, np.concatenate(clouds), offsets, np.array(ks, np.int32)


def split(a, ks):
    a = to_np(a)
    return np.split(a, np.cumsum(ks)[:-1])


SIZES = [2_000, 7_500, 3_100, 12_000, 5_000]
KS = [3, 8, 40, 70, 130]


def test_batched_from_given_init_matches_oracle(gira):
    clouds, pts, offs, ks = make_batch(SIZES, KS, seed=10)
    inits = [oracle.kinit(c, int(k), seed=0, lloyd_iters=5, reg=1e-6) for c, k in zip(clouds, ks)]
    w0 = np.concatenate([i["weights"] for i in inits]).astype(np.float32)
    m0 = np.concatenate([i["means"] for i in inits]).astype(np.float32)
    c0 = np.concatenate([i["covs"] for i in inits]).astype(np.float32)
    import torch
    r = gira.gira_gmm_fit_batched(torch.as_tensor(pts, device="cuda"), offs, ks, iters=15, tol=0.0,
                                  init=(w0, m0, c0))
    assert np.all(r["status"] == 0)
    ws, ms, cs = split(r["weights"], ks), split(r["means"], ks), split(r["covs"], ks)
    for i, (cl, k) in enumerate(zip(clouds, ks)):
        sl = slice(offs[i], offs[i + 1])
        ref = oracle.em(pts[sl], w0[np.cumsum(np.r_[0, ks])[i]:np.cumsum(ks)[i]],
                        m0[np.cumsum(np.r_[0, ks])[i]:np.cumsum(ks)[i]], c0[np.cumsum(np.r_[0, ks])[i]:np.cumsum(ks)[i]],
                        iters=15, tol=0.0, reg=1e-6)
        assert r["iters_done"][i] == 15
        assert np.max(np.abs(r["trace"][i] - ref["trace"])) <= LL_ABS, i
        assert_model_close((ws[i], ms[i], cs[i]), (ref["weights"], ref["means"], ref["covs"]))
        assert abs(r["final_loglik"][i] - ref["final_ll"]) <= LL_ABS


def test_batched_kmeans_init_matches_oracle_fit(gira):
    # 40k points need a 4-CTA seeding cluster, the others one CTA: two seeding launches
    sizes, kk = [3_000, 6_000, 2_500, 40_000], [4, 16, 33, 64]
    clouds, pts, offs, ks = make_batch(sizes, kk, seed=20)
    r = gira.gira_gmm_fit_batched(pts, offs, ks, iters=10, tol=0.0, seed=3, lloyd_iters=6)
    assert np.all(r["status"] == 0)
    ws, ms, cs = split(r["weights"], ks), split(r["means"], ks), split(r["covs"], ks)
    for i, k in enumerate(ks):
        sl = slice(offs[i], offs[i + 1])
        ref = oracle.gmm_fit(pts[sl], int(k), iters=10, tol=0.0, reg=1e-6, seed=3, lloyd_iters=6)
        assert np.max(np.abs(r["trace"][i] - ref["trace"])) <= LL_ABS, i
        assert_model_close((ws[i], ms[i], cs[i]), (ref["weights"], ref["means"], ref["covs"]))


def test_batched_equals_single_fits_stopping(gira):
    """Per-instance convergence: each instance stops exactly where its own fit stops."""
    sizes, kk = [4_000, 8_000, 6_000], [5, 20, 9]
    clouds, pts, offs, ks = make_batch(sizes, kk, seed=30)
    r = gira.gira_gmm_fit_batched(pts, offs, ks, iters=40, tol=1e-3, seed=1)
    for i, k in enumerate(ks):
        single = gira.gira_gmm_fit(pts[offs[i]:offs[i + 1]], int(k), iters=40, tol=1e-3, seed=1)
        assert r["iters_done"][i] == single["iters_done"]
        n = single["iters_done"]
        assert np.all(np.isnan(r["trace"][i][n:]))
        np.testing.assert_allclose(r["trace"][i][:n], single["trace"], atol=1e-6)


def test_batched_error_is_isolated_to_its_instance(gira):
    sizes, kk = [3_000, 3_000, 3_000], [6, 6, 6]
    clouds, pts, offs, ks = make_batch(sizes, kk, seed=40)
    bad = pts.copy()
    bad[offs[1] + 17, 2] = np.nan
    r = gira.gira_gmm_fit_batched(bad, offs, ks, iters=8, tol=0.0, raise_on_error=False)
    assert list(r["status"]) == [0, gira.ERR_NONFINITE_INPUT, 0]
    good = gira.gira_gmm_fit_batched(pts, offs, ks, iters=8, tol=0.0)
    for i in (0, 2):
        sl = slice(int(np.sum(ks[:i])), int(np.sum(ks[:i + 1])))
        np.testing.assert_array_equal(to_np(r["means"])[sl], to_np(good["means"])[sl])
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_fit_batched(bad, offs, ks, iters=8, tol=0.0)
    assert e.value.status == gira.ERR_NONFINITE_INPUT


def test_batched_repeat_call_is_deterministic(gira):
    import torch
    clouds, pts, offs, ks = make_batch([5_000, 2_000, 11_000, 4_000], [12, 3, 100, 48], seed=50)
    x = torch.as_tensor(pts, device="cuda")
    a = gira.gira_gmm_fit_batched(x, offs, ks, iters=12, tol=0.0, seed=2)
    b = gira.gira_gmm_fit_batched(x, offs, ks, iters=12, tol=0.0, seed=2)
    for key in ("weights", "means", "covs"):
        assert torch.equal(a[key], b[key])
    np.testing.assert_array_equal(a["trace"], b["trace"])


def test_batched_single_instance_large_k(gira):
    """One instance of the largest shape class (K in (512, 1024])."""
    cl = synth.gmm_cloud(30_000, 8, seed=60)
    offs = np.array([0, 30_000], np.int64)
    r = gira.gira_gmm_fit_batched(cl.points, offs, [600], iters=3, tol=0.0, seed=4, lloyd_iters=2)
    ref = oracle.gmm_fit(cl.points, 600, iters=3, tol=0.0, reg=1e-6, seed=4, lloyd_iters=2)
    assert np.max(np.abs(r["trace"][0] - ref["trace"])) <= LL_ABS
    assert_model_close((r["weights"], r["means"], r["covs"]), (ref["weights"], ref["means"], ref["covs"]))


def test_full_size_batch_sampled_instances_match_oracle(gira):
    """The benchmark's batch at full size (256 clouds, N log-uniform in [2k, 200k],
    about 11 M points, K in {16 ... 512}) in one call; the six instances with the
    smallest N x K are checked against the oracle's own fit of each."""
    rng = np.random.default_rng(7)
    sizes = np.exp(rng.uniform(np.log(2_000), np.log(200_000), size=256)).astype(np.int64)
    kk = rng.choice((16, 32, 64, 128, 256, 512), size=256).astype(np.int32)
    clouds = [synth.gmm_cloud(int(n), 8, seed=1000 + i).points for i, n in enumerate(sizes)]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    import torch
    r = gira.gira_gmm_fit_batched(torch.as_tensor(np.concatenate(clouds), device="cuda"), offs, kk, iters=3, tol=0.0,
                                  seed=0, lloyd_iters=5)
    assert np.all(r["status"] == 0)
    ws, ms, cs = split(r["weights"], kk), split(r["means"], kk), split(r["covs"], kk)
    for i in np.argsort(sizes * kk)[:6]:
        ref = oracle.gmm_fit(clouds[i], int(kk[i]), iters=3, tol=0.0, reg=1e-6, seed=0, lloyd_iters=5)
        assert np.max(np.abs(r["trace"][i] - ref["trace"])) <= LL_ABS, i
        assert_model_close((ws[i], ms[i], cs[i]), (ref["weights"], ref["means"], ref["covs"]))


def test_single_fit_equals_batch_of_one(gira):
    """From the same start model, a single fit (its E-step's CTAs reordered by their
    previous work from the third iteration on) and a batch holding that one instance
    (launch order) give the same bits: the CTA order changes which SM runs which
    point blocks, never an addition's order."""
    import torch
    cl = synth.depth_frame(seed=3).points[::3].copy()
    k = 96
    init = oracle.kinit(cl, k, seed=0, lloyd_iters=5, reg=1e-6)
    w0, m0, c0 = (init[key].astype(np.float32) for key in ("weights", "means", "covs"))
    x = torch.as_tensor(cl, device="cuda")
    one = gira.gira_gmm_fit(x, k, iters=12, tol=0.0, init=(w0, m0, c0))
    bat = gira.gira_gmm_fit_batched(x, np.array([0, len(cl)], np.int64), np.array([k], np.int32), iters=12,
                                    tol=0.0, init=(w0, m0, c0))
    assert one["iters_done"] == 12 and bat["iters_done"][0] == 12
    for key in ("weights", "means", "covs"):
        np.testing.assert_array_equal(to_np(one[key]), to_np(bat[key]))
    np.testing.assert_array_equal(np.asarray(one["trace"]), np.asarray(bat["trace"][0]))
