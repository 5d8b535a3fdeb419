"""The per-point error bound of tests/_parity.py against a binary32 emulation of
the E-step's arithmetic (CPU only).

The emulation takes the same steps as the GPU's E-step (Eq. logestep with the
log-density of Eq. simplifiedGaussian, base 2): parameters formed in binary64
and rounded to binary32, y = P' x + b' (or P' (x - mu)) by fused multiply-adds,
q' by fused multiply-adds, e = 2^-q', the sum over components, log2 and the
reference, each operation rounded to binary32 (a fused multiply-add is the
exact binary64 value a * b + c rounded once to binary32; exp2 and log2 are
rounded correctly here, inside the hardware's approximation errors the bound
allows).  Every emulated per-point value must lie within the bound of the
exact binary64 value, on the depth frame with a thin-disc model (points metres
from the origin: the b form's worst case) and on a random model.
"""
import numpy as np

from paper_2307_00071_gb300 import synth
from tests._parity import ALPHA, per_point_bound

f32 = np.float32


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def emulate(pts, w, mu, cov, form):
    X = pts.astype(f32)
    N, D = X.shape
    K = len(w)
    P = np.tril(np.linalg.inv(np.linalg.cholesky(cov.astype(np.float64))))
    Q64 = ALPHA * P
    Q = Q64.astype(f32)
    b = (-np.einsum("bij,bj->bi", Q64, mu.astype(np.float64))).astype(f32)
    c = (np.log2(w.astype(np.float64) * np.prod(np.diagonal(P, axis1=1, axis2=2), axis=1))
         - 0.5 * D * np.log2(2 * np.pi)).astype(f32)
    cmax = c.max()
    cp = (cmax - c).astype(f32)
    nmu = (-mu).astype(f32)
    out = np.empty(N)
    for a in range(0, N, 2048):
        x = X[a:a + 2048][:, None, :]                       # n x 1 x D
        if form == "b":
            y = []
            for i in range(D):
                acc = np.broadcast_to(b[None, :, i], (x.shape[0], K)).astype(f32)
                for j in range(i, -1, -1):
                    acc = fma32(Q[None, :, i, j], x[:, :, j], acc)
                y.append(acc)
        else:
            d = (x + nmu[None]).astype(f32)
            y = []
            for i in range(D):
                acc = (Q[None, :, i, 0] * d[:, :, 0]).astype(f32)
                for j in range(1, i + 1):
                    acc = fma32(Q[None, :, i, j], d[:, :, j], acc)
                y.append(acc)
        q = np.broadcast_to(cp[None], y[0].shape).astype(f32)
        for i in range(D):
            q = fma32(y[i], y[i], q)
        def tree_sum(e):
            tot = e.astype(np.float64)
            while tot.shape[1] > 1:                          # pairwise tree, binary32 each level
                if tot.shape[1] % 2:
                    tot = np.concatenate([tot, np.zeros((tot.shape[0], 1))], axis=1)
                tot = (tot[:, 0::2] + tot[:, 1::2]).astype(f32).astype(np.float64)
            return tot[:, 0]
        tot = tree_sum(np.exp2(-q.astype(np.float64)).astype(f32))
        ref = np.full(len(tot), f32(cmax), f32)
        rare = ~(tot >= 2.0 ** -100)                         # every e underflows: exact per-point maximum
        if np.any(rare):
            lq = (-q[rare]).astype(f32)
            mq = lq.max(1)
            tot[rare] = tree_sum(np.exp2((lq - mq[:, None]).astype(f32).astype(np.float64)).astype(f32))
            ref[rare] = (f32(cmax) + mq).astype(f32)
        lse2 = (np.log2(tot).astype(f32) + ref).astype(f32)
        out[a:a + 2048] = (lse2 * f32(np.log(2))).astype(f32)
    return out


def exact(pts, w, mu, cov):
    X = pts.astype(np.float64)
    D = X.shape[1]
    L = np.linalg.cholesky(cov.astype(np.float64))
    P = np.linalg.inv(L)
    d = X[:, None, :] - mu.astype(np.float64)[None]
    m2 = (np.einsum("bij,nbj->nbi", P, d) ** 2).sum(-1)
    logp = (np.log(w.astype(np.float64)) + np.log(np.diagonal(P, axis1=1, axis2=2)).sum(1)
            - 0.5 * D * np.log(2 * np.pi))[None] - 0.5 * m2
    m = logp.max(1, keepdims=True)
    return (m + np.log(np.exp(logp - m).sum(1, keepdims=True)))[:, 0]


def thin_model(pts, K, rng):
    idx = rng.choice(len(pts), K, replace=False)
    mu = pts[idx].astype(np.float64) + rng.normal(scale=0.01, size=(K, 3))
    cov = np.empty((K, 3, 3))
    for b in range(K):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        cov[b] = Q @ np.diag([rng.uniform(0.02, 0.2) ** 2, rng.uniform(0.02, 0.2) ** 2, 0.005 ** 2]) @ Q.T
    return rng.dirichlet(np.ones(K)).astype(f32), mu.astype(f32), cov.astype(f32)


def check(pts, w, mu, cov, form):
    got = emulate(pts, w, mu, cov, form)
    ref = exact(pts, w, mu, cov)
    bound = per_point_bound(pts, w, mu, cov, form=form)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (np.max(err / bound), np.argmax(err / bound))
    return err, bound


def test_bound_holds_on_frame_points_thin_discs():
    pts = synth.depth_frame(seed=1).points
    rng = np.random.default_rng(0)
    sample = pts[rng.choice(len(pts), 3000, replace=False)]
    w, mu, cov = thin_model(pts, 256, rng)
    for form in ("b", "d"):
        err, bound = check(sample, w, mu, cov, form)
    # the d form does not carry |P'||x|: its bound is far smaller on metre-scale points
    assert np.median(per_point_bound(sample, w, mu, cov, form="d")) < 0.1 * np.median(
        per_point_bound(sample, w, mu, cov, form="b"))


def test_bound_holds_on_random_models():
    rng = np.random.default_rng(1)
    K = 64
    w = rng.dirichlet(np.ones(K)).astype(f32)
    mu = rng.uniform(-2, 2, (K, 3)).astype(f32)
    a = rng.standard_normal((K, 3, 3))
    cov = (0.02 * (a @ a.transpose(0, 2, 1) + 0.3 * np.eye(3))).astype(f32)
    pts = rng.uniform(-2.2, 2.2, (4000, 3)).astype(f32)
    err, bound = check(pts, w, mu, cov, "b")
    assert np.max(bound) < 1e-3   # far tighter than a flat 2e-3 on this workload
