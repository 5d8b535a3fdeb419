"""Mode seeking that sets K (Sec. V "Gaussian Blurring Mean Shift") on the GPU
against the oracle: the same modes bit for bit (fixed-point means, the same
binary32 ball test and binary64 merge test), the same counts and the same rank
order; at the frame's full size, properties that hold at any size."""
import numpy as np
import pytest

import oracle
from paper_2307_00071_gb300 import synth
from tests._parity import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gira():
    from paper_2307_00071_gb300 import gira as g
    return g


def check_equal(gira, pts, h, max_iter=300):
    modes, counts = gira.gira_gbms(pts, h, max_iter=max_iter)
    ref_m, ref_c = oracle.gbms(pts, h, max_iter=max_iter)
    assert len(modes) == len(ref_m)
    np.testing.assert_array_equal(to_np(counts), ref_c)
    np.testing.assert_array_equal(to_np(modes), ref_m)
    return len(ref_m)


@pytest.mark.parametrize("h", [0.05, 0.1, 0.2])
def test_gmm_cloud_3d_bit_exact(gira, h):
    pts = synth.gmm_cloud(20_000, 8, seed=1).points
    assert check_equal(gira, pts, h) >= 8


@pytest.mark.parametrize("h", [0.08, 0.15])
def test_gmm_cloud_4d_bit_exact(gira, h):
    pts = synth.gmm_cloud4(15_000, 10, seed=2).points
    check_equal(gira, pts, h)


def test_frame_subset_with_intensity_bit_exact(gira):
    f = synth.depth_frame4(seed=1)
    rng = np.random.default_rng(0)
    pts = np.ascontiguousarray(f[np.sort(rng.choice(len(f), 12_000, replace=False))])
    check_equal(gira, pts, 0.25)


def test_iteration_limit_and_tiny_inputs(gira):
    pts = synth.gmm_cloud(5_000, 4, seed=3).points
    check_equal(gira, pts, 0.1, max_iter=2)        # most seeds stop on the limit
    check_equal(gira, pts[:1], 0.1)                # one point: one mode
    check_equal(gira, pts[:7], 1e-4)               # every point its own seed and mode


def test_device_tensors(gira):
    import torch
    pts = synth.gmm_cloud(8_000, 6, seed=4).points
    m, c = gira.gira_gbms(torch.as_tensor(pts, device="cuda"), 0.12)
    assert m.is_cuda and c.is_cuda
    ref_m, ref_c = oracle.gbms(pts, 0.12)
    np.testing.assert_array_equal(m.cpu().numpy(), ref_m)


def test_full_frame_properties(gira):
    """The 276k-point frame with intensity: modes more than h apart, each mode close
    to the mean of its own ball (a mode is the mean of the ball of the previous
    position, at most 1e-3 h away; the two balls differ only in a thin shell),
    ranks by count, and the same bits on a second run."""
    pts = synth.depth_frame4(seed=1)
    h = 0.3
    m, c = gira.gira_gbms(pts, h)
    m2, c2 = gira.gira_gbms(pts, h)
    np.testing.assert_array_equal(m, m2)
    np.testing.assert_array_equal(c, c2)
    K = len(m)
    assert 10 < K < len(pts)
    assert np.all(np.diff(c) <= 0)
    rng = np.random.default_rng(0)
    sample = rng.choice(K, min(K, 40), replace=False)
    for r in sample:
        a = m[r]
        # merge: no kept mode within h of another
        dd = np.sum((m - a) ** 2, axis=1)
        dd[r] = np.inf
        assert np.all(dd > h * h)
        # the ball of the mode (same binary32 test): its mean is within the stop slack
        mf = a.astype(np.float32)
        d = pts - mf
        s = ((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]) + d[:, 3] * d[:, 3]
        ball = pts[s <= np.float32(h * h)].astype(np.float64)
        assert len(ball) > 0
        assert np.linalg.norm(ball.mean(0) - a) <= 0.05 * h


def test_errors(gira):
    pts = synth.gmm_cloud(1_000, 3, seed=5).points.copy()
    pts[5, 1] = np.nan
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gbms(pts, 0.1)
    assert e.value.status == gira.ERR_NONFINITE_INPUT
    far = np.array([[5000.0, 0.0, 0.0], [0.0, 0.0, 0.0]], np.float32)
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gbms(far, 1.0)
    assert e.value.status == gira.ERR_INVALID_ARG
