"""The E-step's reach test against a binary32 emulation of its logits (CPU only).

The point-stationary E-step skips a component for a block of points when a lower
bound of q' = |P'(x - mu)|^2 + (cmax - c) over the block's box exceeds 128 (two
units above 126, where ex2.approx.ftz(-q') is exactly 0).  The bounds, taken in
binary32 with relative slack:

    |P'(x - mu)| >= |P'(ctr - mu)| - sum_j h_j |column j of P'|
    |P'(x - mu)|^2 >= sigma_min(P')^2 dist(mu, box)^2

Here both the test and the kernel's q' (d-form, fused multiply-adds, each step
rounded to binary32) are emulated, and every skipped (block, component) must
have q' > 126 at every point of the block, with margin, on: the depth frame in
Morton order and in sensor order with thin-disc models, needle components at the
conditioning limit, random models in a cube, and the frame 47 m from the origin.
"""
import numpy as np
import pytest

from paper_2307_00071_gb300 import synth

f32 = np.float32
ALPHA = np.sqrt(np.log2(np.e) / 2)


def fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def params(w, mu, cov):
    """The E-step's binary32 parameters: P' = alpha L^-1 (lower), c, -mu, sigma_min(P')^2 bound."""
    L = np.linalg.cholesky(cov.astype(np.float64))
    Pi = np.linalg.inv(L)
    Q = ALPHA * Pi
    p = np.stack([Q[:, 0, 0], Q[:, 1, 0], Q[:, 1, 1], Q[:, 2, 0], Q[:, 2, 1], Q[:, 2, 2]], 1).astype(f32)
    c = (np.log2(w * np.prod(np.diagonal(Pi, axis1=1, axis2=2), axis=1)) - 1.5 * np.log2(2 * np.pi)).astype(f32)
    lmax = np.linalg.eigvalsh(cov.astype(np.float64))[:, -1] * (1 + 1e-4)   # the kernel's upper bound
    s2 = (f32(ALPHA * ALPHA) / lmax.astype(f32) * f32(1 - 1e-4)).astype(f32)
    return p, c, (-mu).astype(f32), s2


def reach_mask(p, cp, nm, s2, xs):
    """Components the kernel keeps for the box of the points xs (binary32, as coded)."""
    lo, hi = xs.min(0), xs.max(0)
    ctr = (f32(0.5) * (lo + hi)).astype(f32)
    h = np.maximum(hi - ctr, ctr - lo).astype(f32)
    room = (f32(128) - cp).astype(f32)
    d = (ctr[None] + nm).astype(f32)
    y0 = (p[:, 0] * d[:, 0]).astype(f32)
    y1 = fma(p[:, 2], d[:, 1], (p[:, 1] * d[:, 0]).astype(f32))
    y2 = fma(p[:, 5], d[:, 2], fma(p[:, 4], d[:, 1], (p[:, 3] * d[:, 0]).astype(f32)))
    yy = fma(y2, y2, fma(y1, y1, (y0 * y0).astype(f32)))
    col0 = np.sqrt(fma(p[:, 0], p[:, 0], fma(p[:, 1], p[:, 1], (p[:, 3] * p[:, 3]).astype(f32)))).astype(f32)
    col1 = np.sqrt(fma(p[:, 2], p[:, 2], (p[:, 4] * p[:, 4]).astype(f32))).astype(f32)
    r = fma(h[0], col0, fma(h[1], col1, (h[2] * np.abs(p[:, 5])).astype(f32)))
    reach = ((r + np.sqrt(np.maximum(room, 0)).astype(f32)).astype(f32) * f32(1 + 1 / 256)).astype(f32)
    e = np.maximum(np.abs(d) - h[None], 0).astype(f32)
    iso = (s2 * fma(e[:, 2], e[:, 2], fma(e[:, 1], e[:, 1], (e[:, 0] * e[:, 0]).astype(f32)))).astype(f32)
    iso = (iso * f32(1 - 1 / 128)).astype(f32)
    return (room > 0) & (yy <= (reach * reach).astype(f32)) & (iso <= room)


def kernel_q(p, cp, nm, xs):
    """q' of every point and component, as the E-step forms it (binary32)."""
    D = (xs[:, None, :] + nm[None]).astype(f32)
    y0 = (p[None, :, 0] * D[:, :, 0]).astype(f32)
    y1 = fma(p[None, :, 2], D[:, :, 1], (p[None, :, 1] * D[:, :, 0]).astype(f32))
    y2 = fma(p[None, :, 5], D[:, :, 2], fma(p[None, :, 4], D[:, :, 1], (p[None, :, 3] * D[:, :, 0]).astype(f32)))
    return fma(y2, y2, fma(y1, y1, fma(y0, y0, cp[None])))


def check(X, w, mu, cov, blocks=160, seed=0):
    p, c, nm, s2 = params(w, mu, cov)
    cp = (c.max() - c).astype(f32)
    X = np.asarray(X, f32)
    rng = np.random.default_rng(seed)
    starts = rng.choice(len(X) // 128, size=min(blocks, len(X) // 128), replace=False) * 128
    skipped = total = 0
    for a in starts:
        xs = X[a:a + 128]
        keep = reach_mask(p, cp, nm, s2, xs)
        total += keep.size
        sk = np.nonzero(~keep)[0]
        skipped += len(sk)
        if len(sk):
            q = kernel_q(p[sk], cp[sk], nm[sk], xs)
            assert q.min() > 126.5, (a, float(q.min()))
    return skipped / total


def thin_discs(pts, K, rng, far=0.0):
    idx = rng.choice(len(pts), K, replace=False)
    mu = pts[idx].astype(np.float64) + rng.normal(scale=0.01, size=(K, 3))
    cov = np.empty((K, 3, 3))
    for b in range(K):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        cov[b] = Q @ np.diag([rng.uniform(0.01, 0.2) ** 2, rng.uniform(0.01, 0.2) ** 2, 0.005 ** 2]) @ Q.T
    return rng.dirichlet(np.ones(K)), mu, cov


def morton(pts):
    lo, hi = pts.min(0), pts.max(0)
    q = np.clip(((pts - lo) / (hi - lo).max() * 64).astype(np.int64), 0, 63)
    code = np.zeros(len(pts), np.int64)
    for b in range(6):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return np.argsort(code, kind="stable")


@pytest.fixture(scope="module")
def frame():
    return synth.depth_frame(seed=1).points


def test_reach_test_never_skips_a_reachable_pair_on_the_frame(frame):
    rng = np.random.default_rng(0)
    w, mu, cov = thin_discs(frame, 512, rng)
    frac_sorted = check(frame[morton(frame)], w, mu, cov)
    frac_raster = check(frame, w, mu, cov, seed=1)
    assert frac_sorted > 0.5 and frac_raster > 0.2   # the test does skip


def test_reach_test_needles_at_the_conditioning_limit(frame):
    rng = np.random.default_rng(1)
    K = 256
    mu = frame[rng.choice(len(frame), K, replace=False)].astype(np.float64)
    cov = np.empty((K, 3, 3))
    for b in range(K):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        cov[b] = Q @ np.diag([rng.uniform(0.5, 3.0) ** 2, 1e-6, 1e-6 * rng.uniform(1, 4)]) @ Q.T
    check(frame[morton(frame)], rng.dirichlet(np.ones(K)), mu, cov, seed=2)


def test_reach_test_random_models_and_far_points(frame):
    rng = np.random.default_rng(2)
    K = 300
    mu = rng.uniform(-2, 2, (K, 3))
    a = rng.standard_normal((K, 3, 3))
    cov = 0.02 * (a @ a.transpose(0, 2, 1) + 0.3 * np.eye(3))
    cube = rng.uniform(-2.2, 2.2, (40_000, 3))
    check(cube[morton(cube)], rng.dirichlet(np.ones(K)), mu, cov, seed=3)
    far = (frame.astype(np.float64) + np.array([40.0, -25.0, 3.0])).astype(f32)
    w, mu2, cov2 = thin_discs(far, 256, rng)
    check(far[morton(far)], w, mu2, cov2, seed=4)
