"""Why the E-step's logits stay on the FP32 pipe: the tensor-core form that lifts
points to 10 quadratic features (q_nb = phi(x_n) . m_b, an N x 10 by 10 x K GEMM)
cancels terms of size |P'x|^2 (a point metres away against a centimetre factor)
and misses the parity tolerance already with binary32 inputs; the tensor cores'
input types (TF32, BF16) are orders of magnitude worse.  Measured on a subset of
the depth frame with its KInit model (binary64 reference), no GPU."""
import numpy as np

import oracle
from paper_2307_00071_gb300 import synth


def _round_mantissa(a, bits):
    a = np.asarray(a, np.float64)
    e = np.floor(np.log2(np.abs(a) + 1e-300))
    s = 2.0 ** (e - bits)
    return np.round(a / s) * s


def test_lifted_quadratic_form_misses_the_tolerance():
    rng = np.random.default_rng(0)
    f = synth.depth_frame(seed=1).points
    pts = f[np.sort(rng.choice(len(f), 6000, replace=False))]
    ki = oracle.kinit(pts, 128, seed=0, lloyd_iters=5, reg=1e-6)
    mu, cov, w = ki["means"], ki["covs"], ki["weights"]
    x = pts.astype(np.float64) - pts.astype(np.float64).mean(0)   # frame-centred: the favourable case
    mu = mu - pts.astype(np.float64).mean(0)
    P = np.linalg.inv(np.linalg.cholesky(cov))
    Mq = np.einsum('kji,kjl->kil', P, P)
    y = np.einsum('kij,nkj->nki', P, x[:, None, :] - mu[None])
    q = np.sum(y * y, axis=2)                                      # binary64 Mahalanobis terms
    logit = np.log(w)[None] - 0.5 * q + np.log(np.abs(np.linalg.det(P)))[None]
    resp = np.exp(logit - logit.max(1, keepdims=True))
    resp /= resp.sum(1, keepdims=True)
    live = resp > 1e-6
    b = -np.einsum('kij,kj->ki', Mq, mu)
    c = np.einsum('ki,ki->k', mu, -b)
    m = np.stack([Mq[:, 0, 0], Mq[:, 1, 1], Mq[:, 2, 2], Mq[:, 0, 1], Mq[:, 0, 2], Mq[:, 1, 2],
                  b[:, 0], b[:, 1], b[:, 2], c], 1)
    phi = np.stack([x[:, 0] ** 2, x[:, 1] ** 2, x[:, 2] ** 2, 2 * x[:, 0] * x[:, 1], 2 * x[:, 0] * x[:, 2],
                    2 * x[:, 1] * x[:, 2], 2 * x[:, 0], 2 * x[:, 1], 2 * x[:, 2], np.ones(len(x))], 1)
    errs = {}
    for name, bits in (("fp32", 23), ("tf32", 10), ("bf16", 7)):
        ql = (_round_mantissa(phi, bits).astype(np.float32) @ _round_mantissa(m, bits).T.astype(np.float32))
        errs[name] = np.abs(ql.astype(np.float64) - q)[live]
    # a responsibility moves by about |dq| / 2 relative; the fit tolerance is 1e-4
    assert np.max(errs["fp32"]) / 2 > 1e-2
    assert np.median(errs["tf32"]) / 2 > 1e-1
    assert np.median(errs["bf16"]) > np.median(errs["tf32"])
    # the direct form the kernels use, |P'(x - mu)|^2 with binary32 operands, stays within it
    d32 = (x[:, None, :] - mu[None]).astype(np.float32)
    y32 = np.einsum('kij,nkj->nki', P.astype(np.float32), d32)
    q32 = np.sum(y32.astype(np.float64) ** 2, axis=2)
    assert np.max(np.abs(q32 - q)[live] / np.maximum(q[live], 1.0)) / 2 < 1e-5
