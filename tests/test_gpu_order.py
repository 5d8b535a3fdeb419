"""The spatial order the fits' E-steps visit points in (a stable radix sort by
Morton code), through the test hook gira_test_point_order.

The expected order is computed here from the hook's documented rule: per
instance, the bounding box of its points, cells of (largest extent) / 64 on
every axis, cell index floor((x - lo) * (64 / extent)) clamped to [0, 63] in
binary32, the three 6-bit indices interleaved (bit 3b + a = bit b of axis a),
and a stable sort by (instance, code).  The E-step's results do not depend on
the order beyond the rounding of its sums; this pins the order itself.
"""
import numpy as np
import pytest

from paper_2307_00071_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def codes(pts):
    x = np.asarray(pts, np.float32)
    lo, hi = x.min(0), x.max(0)
    ext = np.float32(max(hi - lo))
    scale = np.float32(64.0) / ext if ext > 0 else np.float32(0.0)
    q = np.clip(np.floor((x - lo[None]).astype(np.float32) * scale), 0, 63).astype(np.int64)
    code = np.zeros(len(x), np.int64)
    for b in range(6):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return code


def expected(pts, offsets):
    out = []
    for i in range(len(offsets) - 1):
        a, b = offsets[i], offsets[i + 1]
        out.append(a + np.argsort(codes(pts[a:b]), kind="stable"))
    return np.concatenate(out)


def run(pts, offsets=None):
    from paper_2307_00071_gb300 import gira
    x = torch.as_tensor(np.ascontiguousarray(pts, np.float32), device="cuda")
    got = gira.gira_test_point_order(x, offsets).cpu().numpy()
    want = expected(np.asarray(pts, np.float32), [0, len(pts)] if offsets is None else list(offsets))
    np.testing.assert_array_equal(got, want)


def test_frame_order():
    run(synth.depth_frame(seed=1).points)


@pytest.mark.parametrize("n", [1, 31, 2049, 100_003])
def test_uniform_clouds_ragged_sizes(n):
    run(synth.uniform_cloud(n, seed=n, scale=3.0))


def test_repeated_and_degenerate_points():
    pts = np.zeros((5000, 3), np.float32)   # one point repeated: zero extent, every code 0
    run(pts)
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 3, size=(7000, 3)).astype(np.float32)   # many equal codes: stability
    run(pts)
    flat = rng.uniform(-1, 1, size=(9000, 3)).astype(np.float32)
    flat[:, 2] = 0.25                                  # a plane: one axis of zero extent
    run(flat)


def test_batch_keeps_instances_in_place():
    rng = np.random.default_rng(5)
    sizes = [1, 4096, 7, 12_345, 2048, 300]
    parts = [synth.gmm_cloud(n, 3, seed=i).points if n > 8 else rng.normal(size=(n, 3)).astype(np.float32)
             for i, n in enumerate(sizes)]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    run(np.concatenate(parts), offs)
