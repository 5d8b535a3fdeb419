"""The finalize's arithmetic, restated on the CPU (no GPU).

The binary64 update forms L^-1 of a 3x3 covariance from Schur complements and
three reciprocal square roots, the log-normaliser from an exact binary exponent
and log2 of a 24-bit significand, the statistics by compensated binary32 sums
joined in a fixed butterfly, and the E-step's CTA order by a counting sort of
8-bit work keys.  Each is checked here against what it must equal: the Cholesky
factor's inverse (numpy), log2 in binary64, the exact rational sum, and a stable
descending argsort.
"""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def chol_inv_schur(c):
    """P = L^-1 for c = (00, 01, 02, 11, 12, 22) by the finalize's formulas (binary64)."""
    a00, a01, a02, a11, a12, a22 = c
    u = 1.0 / np.sqrt(a00)
    r0 = u * u
    h0 = a01 * r0
    h1 = a02 * r0
    s11 = a11 - h0 * a01
    s12 = a12 - h0 * a02
    s22 = a22 - h1 * a02
    v = 1.0 / np.sqrt(s11)
    t = s12 * (v * v)
    a22p = s22 - t * s12
    z = 1.0 / np.sqrt(a22p)
    g = a02 - a01 * t
    P = np.zeros((3, 3))
    P[0, 0], P[1, 1], P[2, 2] = u, v, z
    P[1, 0] = -(h0 * v)
    P[2, 1] = -(t * z)
    P[2, 0] = -((r0 * g) * z)
    return P, (a00 > 0 and s11 > 0 and a22p > 0), u * v * z


def random_spd(rng, thin=False):
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    ev = rng.uniform(0.01, 3.0, 3) ** 2
    if thin:
        ev = np.array([rng.uniform(0.5, 3.0) ** 2, 1e-6, 1e-6 * rng.uniform(1, 4)])
    return Q @ np.diag(ev) @ Q.T


@pytest.mark.parametrize("thin", [False, True])
def test_schur_rsqrt_cholesky_inverse(thin):
    rng = np.random.default_rng(7 if thin else 3)
    for _ in range(300):
        S = random_spd(rng, thin)
        c = (S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2])
        P, pd, prod = chol_inv_schur(c)
        assert pd
        ref = np.linalg.inv(np.linalg.cholesky(S))
        cond = np.linalg.cond(S)
        assert np.max(np.abs(P - ref)) <= 1e-13 * cond * np.max(np.abs(ref))
        # P Sigma P^T = I and prod_j P_jj = det(Sigma)^(-1/2)
        assert np.allclose(P @ S @ P.T, np.eye(3), atol=1e-12 * cond)
        assert prod == pytest.approx(np.linalg.det(S) ** -0.5, rel=1e-12 * cond)


def test_schur_pivots_flag_indefinite_matrices():
    for S in (np.diag([1.0, -1.0, 1.0]), np.diag([0.0, 1.0, 1.0]), np.array([[1, 2, 0], [2, 1, 0], [0, 0, 1.0]])):
        c = (S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2])
        with np.errstate(invalid="ignore", divide="ignore"):
            assert not chol_inv_schur(c)[1]


def log2_norm(x):
    """log2(x) - 1.5 log2(2 pi) as the finalize forms it: exact exponent, log2 of the
    significand rounded to 24 bits, the constant 4 - 1.5 log2(2 pi) folded in (binary32)."""
    bits = np.frombuffer(np.float64(x).tobytes(), np.uint64)[0]
    e = int((bits >> np.uint64(52)) & np.uint64(0x7FF)) - 1023
    m24 = int(((bits & np.uint64(0xFFFFFFFFFFFFF)) + np.uint64(1 << 28)) >> np.uint64(29))
    m = np.frombuffer(np.uint32((127 << 23) + m24).tobytes(), np.float32)[0]
    lg = f32(np.log2(np.float64(m)))   # a correctly rounded log2f stands in for the device's
    return f32(f32(e - 4) + f32(lg + f32(0.0227558057915218)))


def test_log2_normaliser_within_a_few_1e8():
    rng = np.random.default_rng(11)
    xs = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 5000))
    xs = np.concatenate([xs, [1.0, 2.0, 0.5, 1.9999999999, 3.0, 1e-300 * 1e280]])
    for x in xs:
        ref = np.log2(x) - 1.5 * np.log2(2 * np.pi)
        got = float(log2_norm(x))
        ulp = float(np.spacing(f32(abs(ref)))) if ref != 0 else 1e-45
        assert abs(got - ref) <= 2.5e-7 + ulp, (x, got, ref)


def two_sum_acc(s, e, x):
    t = f32(s + x)
    bp = f32(t - s)
    err = f32(f32(s - f32(t - bp)) + f32(x - bp))
    return t, f32(e + err)


def compensated_slices(vals, nslices=64):
    """Slices of the list summed with TwoSum, a butterfly over 32 slices, then the two halves."""
    nl = len(vals)
    S = np.zeros(nslices, np.float32)
    E = np.zeros(nslices, np.float32)
    for q in range(nslices):
        s = e = f32(0)
        for v in vals[q * nl // nslices:(q + 1) * nl // nslices]:
            s, e = two_sum_acc(s, e, f32(v))
        S[q], E[q] = s, e
    for half in (slice(0, 32), slice(32, 64)):
        s_, e_ = S[half].copy(), E[half].copy()
        for d in (16, 8, 4, 2, 1):
            ns, ne = s_.copy(), e_.copy()
            for lane in range(32):
                p = lane ^ d
                ee = f32(e_[lane] + e_[p])
                ns[lane], ne[lane] = two_sum_acc(s_[lane], ee, s_[p])
            s_, e_ = ns, ne
        assert np.all(s_ == s_[0]) and np.all(e_ == e_[0])   # every lane ends with the same total
        S[half], E[half] = s_, e_
    s, e = S[0], f32(E[0] + E[32])
    s, e = two_sum_acc(s, e, S[32])
    return float(np.float64(s) + np.float64(e))


@pytest.mark.parametrize("n", [1, 7, 64, 208, 582, 3000])
def test_compensated_slice_sums_are_nearly_exact(n):
    rng = np.random.default_rng(n)
    vals = (rng.standard_normal(n) * np.exp(rng.uniform(-6, 6, n))).astype(np.float32)
    exact = sum(Fraction(float(v)) for v in vals)
    got = compensated_slices(vals)
    scale = float(sum(abs(Fraction(float(v))) for v in vals))
    assert abs(Fraction(got) - exact) <= Fraction(2 ** -40) * Fraction(scale) + Fraction(1, 10 ** 300)


def work_key(w):
    """The E-step's 8-bit key: 16 x the binary exponent of w plus its next 4 bits."""
    e = (int(w) | 1).bit_length() - 1
    m = ((w >> (e - 4)) if e >= 4 else (w << (4 - e))) & 15
    return min(255, e * 16 + m)


def test_work_key_is_monotone_and_logarithmic():
    ws = np.arange(0, 1 << 17, 7)
    keys = np.array([work_key(int(w)) for w in ws])
    assert np.all(np.diff(keys) >= 0)
    assert keys[-1] == 255
    for w in (1000, 5000, 20000):   # 16 steps per octave
        assert work_key(2 * w) - work_key(w) == 16


def cta_order(keys, threads=320):
    """The finalize's counting sort: position = keys above + equal keys before (per-chunk
    warp ranks by match_any, per-warp counts, running counts per key)."""
    grid = len(keys)
    above = np.zeros(256, np.int64)
    hist = np.bincount(keys, minlength=256)
    above[:] = np.concatenate([np.cumsum(hist[::-1])[::-1][1:], [0]])
    run = np.zeros(256, np.int64)
    out = np.full(grid, -1)
    for c0 in range(0, grid, threads):
        idx = np.arange(c0, min(grid, c0 + threads))
        k = keys[idx]
        warp = (idx - c0) // 32
        wc = np.zeros((threads // 32, 256), np.int64)
        rank = np.zeros(len(idx), np.int64)
        for w in np.unique(warp):
            sel = np.nonzero(warp == w)[0]
            for j, i in enumerate(sel):
                rank[i] = np.sum(k[sel[:j]] == k[i])
                wc[w, k[i]] += 1
        for i in range(len(idx)):
            pos = above[k[i]] + run[k[i]] + rank[i] + wc[:warp[i], k[i]].sum()
            assert out[pos] == -1
            out[pos] = idx[i]
        run += wc.sum(0)
    return out


@pytest.mark.parametrize("grid", [1, 33, 320, 1080, 2161])
def test_cta_order_is_a_stable_descending_sort(grid):
    rng = np.random.default_rng(grid)
    keys = rng.integers(0, 256, grid) if grid != 1080 else np.minimum(255, rng.poisson(120, grid))
    order = cta_order(keys)
    assert sorted(order.tolist()) == list(range(grid))
    np.testing.assert_array_equal(order, np.argsort(-keys, kind="stable"))


def whitened_mstep(S, q, s, reg):
    """The finalize's M-step from whitened statistics (binary64, the kernel's formulas):
    S = (S0, S1[3], S2[6]) of y = P'(x - s), q = P' (00, 10, 11, 20, 21, 22) in binary32."""
    q = np.asarray(q, np.float64)
    nbw = S[0] + 10 * np.finfo(np.float64).eps
    inv = 1.0 / nbw
    m00, m11, m22 = 1.0 / q[0], 1.0 / q[2], 1.0 / q[5]
    m10 = (-q[1] * m00) * m11
    m21 = (-q[4] * m11) * m22
    m20 = (q[4] * m10 + q[3] * m00) * (-m22)
    M = np.array([[m00, 0, 0], [m10, m11, 0], [m20, m21, m22]])
    yb = np.array(S[1:4]) * inv
    ij = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    C = np.zeros((3, 3))
    for u, (i, j) in enumerate(ij):
        C[i, j] = C[j, i] = -yb[i] * yb[j] + S[4 + u] * inv
    mu = s + M @ yb
    Sig = M @ C @ M.T + reg * np.eye(3)
    return nbw, mu, Sig


def test_whitened_mstep_equals_direct_weighted_moments():
    """mu = s + P'^-1 ybar and Sigma = P'^-1 C P'^-T + reg I from whitened statistics are
    the responsibility-weighted mean and covariance of the points (the standard M-step)."""
    rng = np.random.default_rng(5)
    alpha = np.sqrt(np.log2(np.e) / 2)
    for trial in range(50):
        n = int(rng.integers(5, 400))
        x = rng.normal(size=(n, 3)) * rng.uniform(0.01, 2.0, 3) + rng.uniform(-5, 5, 3)
        r = rng.uniform(0, 1, n) ** 3
        S_old = random_spd(rng, thin=trial % 3 == 0)
        q32 = (alpha * np.linalg.inv(np.linalg.cholesky(S_old))).astype(np.float32)
        q = np.array([q32[0, 0], q32[1, 0], q32[1, 1], q32[2, 0], q32[2, 1], q32[2, 2]])
        s = (x.mean(0) + rng.normal(size=3) * 0.1).astype(np.float32).astype(np.float64)
        P = q32.astype(np.float64)
        y = (x - s) @ P.T
        S = [r.sum(), *(r[:, None] * y).sum(0)]
        for i, j in [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]:
            S.append((r * y[:, i] * y[:, j]).sum())
        nbw, mu, Sig = whitened_mstep(S, q, s, 1e-6)
        Nb = r.sum() + 10 * np.finfo(np.float64).eps
        mu_ref = (r[:, None] * x).sum(0) / Nb
        d = x - mu_ref
        Sig_ref = (r[:, None, None] * d[:, :, None] * d[:, None, :]).sum(0) / Nb + 1e-6 * np.eye(3)
        assert nbw == pytest.approx(Nb, rel=1e-15)
        assert np.allclose(mu, mu_ref, rtol=0, atol=1e-9 * (1 + np.abs(mu_ref).max()))
        assert np.allclose(Sig, Sig_ref, rtol=1e-8, atol=1e-12)
