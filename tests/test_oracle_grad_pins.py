"""Pins of the oracle's differentiable log-likelihood (no GPU).

L = sum_n ln sum_b pi_b N(R x_n + t | mu_b, L_b L_b^T), pi = softmax(alpha).
The value is pinned to scipy's multivariate normal; the gradient to central
finite differences of that pinned value, to invariances of L (a common shift
of the scan and the means, a common shift of the logits) and to the K = 1
maximum-likelihood point, where every gradient but the points' vanishes.
"""
import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

import oracle


def rot(w):
    """Rotation matrix exp(w^) (Rodrigues)."""
    th = np.linalg.norm(w)
    if th == 0.0:
        return np.eye(3)
    k = np.asarray(w) / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx


def problem(n=30, k=3, seed=0):
    rng = np.random.default_rng(seed)
    pts = rng.normal(size=(n, 3)).astype(np.float32)
    logits = rng.normal(size=k)
    means = rng.normal(scale=0.7, size=(k, 3))
    chol = np.zeros((k, 3, 3))
    for b in range(k):
        A = np.tril(rng.normal(scale=0.3, size=(3, 3)))
        A[np.diag_indices(3)] = rng.uniform(0.5, 1.2, size=3)
        chol[b] = A
    R = rot(rng.normal(scale=0.3, size=3))
    t = rng.normal(scale=0.2, size=3)
    return pts, logits, means, chol, (R, t)


def scipy_loglik(pts, logits, means, chol, pose):
    R, t = pose
    xp = pts.astype(np.float64) @ R.T + t
    logpi = logits - logsumexp(logits)
    comp = np.stack([logpi[b] + stats.multivariate_normal(means[b], chol[b] @ chol[b].T).logpdf(xp)
                     for b in range(len(logits))], axis=1)
    return float(logsumexp(comp, axis=1).sum())


def test_loglik_matches_scipy():
    pts, logits, means, chol, pose = problem(n=200, k=5, seed=1)
    r = oracle.loglik_grad(pts, logits, means, chol, pose)
    assert r["loglik"] == pytest.approx(scipy_loglik(pts, logits, means, chol, pose), rel=1e-12)


def fd(f, x0, h):
    g = np.zeros_like(x0)
    for i in np.ndindex(x0.shape):
        xp, xm = x0.copy(), x0.copy()
        xp[i] += h
        xm[i] -= h
        g[i] = (f(xp) - f(xm)) / (2 * h)
    return g


def test_gradient_matches_central_differences():
    pts, logits, means, chol, pose = problem()
    r = oracle.loglik_grad(pts, logits, means, chol, pose)
    ll = lambda **kw: oracle.loglik_grad(kw.get("pts", pts), kw.get("logits", logits), kw.get("means", means),
                                         kw.get("chol", chol), kw.get("pose", pose), want_points=False)["loglik"]
    h = 1e-6
    np.testing.assert_allclose(r["grad_logits"], fd(lambda v: ll(logits=v), logits, h), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(r["grad_means"], fd(lambda v: ll(means=v), means, h), rtol=1e-6, atol=1e-7)
    gch = fd(lambda v: ll(chol=v), chol, h)
    low = np.tril(np.ones((3, 3), bool))
    np.testing.assert_allclose(r["grad_chol"][:, low], gch[:, low], rtol=1e-6, atol=1e-6)
    assert np.all(r["grad_chol"][:, ~low] == 0.0)
    # twist: left perturbation (omega, v) of the pose, rotation first
    R, t = pose

    def moved(xi):
        Rd = rot(xi[:3])
        return ll(pose=(Rd @ R, Rd @ t + xi[3:]))

    np.testing.assert_allclose(r["grad_twist"], fd(moved, np.zeros(6), h), rtol=1e-6, atol=1e-6)
    # points: perturb a few coordinates of the scan (binary32 input: perturb in binary64
    # through an equivalent translation of one point by the inverse rotation)
    for n in (0, 7, 29):
        def one(dx, n=n):
            R_, t_ = pose
            # move only point n: its image R x + t + R dx
            xp = pts.astype(np.float64) @ R_.T + t_
            xp[n] += R_ @ dx
            logpi = logits - logsumexp(logits)
            comp = np.stack([logpi[b] + stats.multivariate_normal(means[b], chol[b] @ chol[b].T).logpdf(xp)
                             for b in range(len(logits))], axis=1)
            return float(logsumexp(comp, axis=1).sum())
        np.testing.assert_allclose(r["grad_points"][n], fd(one, np.zeros(3), h), rtol=1e-6, atol=1e-6)


def test_invariances():
    pts, logits, means, chol, pose = problem(n=500, k=6, seed=4)
    r = oracle.loglik_grad(pts, logits, means, chol, pose)
    scale = np.abs(r["grad_means"]).max()
    # shifting every logit by the same amount leaves pi unchanged
    assert abs(r["grad_logits"].sum()) <= 1e-9 * len(pts)
    # translating the scan and every mean together leaves L unchanged
    np.testing.assert_allclose(r["grad_twist"][3:] + r["grad_means"].sum(0), 0.0, atol=1e-9 * scale)
    # the translation part of the twist is the sum of the per-point gradients in the moved frame
    R, _ = pose
    np.testing.assert_allclose(r["grad_twist"][3:], R @ r["grad_points"].sum(0), rtol=1e-10, atol=1e-9 * scale)


def test_single_component_at_the_mle():
    pts, _, _, _, pose = problem(n=400, k=1, seed=6)
    R, t = pose
    xp = pts.astype(np.float64) @ R.T + t
    mu = xp.mean(0)
    S = (xp - mu).T @ (xp - mu) / len(xp)
    L = np.linalg.cholesky(S)
    r = oracle.loglik_grad(pts, np.zeros(1), mu[None], L[None], pose)
    big = len(xp) * np.abs(np.linalg.inv(S)).max()
    np.testing.assert_allclose(r["grad_means"], 0.0, atol=1e-9 * big)
    np.testing.assert_allclose(r["grad_chol"], 0.0, atol=1e-9 * big)
    np.testing.assert_allclose(r["grad_twist"], 0.0, atol=1e-8 * big)
    np.testing.assert_allclose(r["grad_logits"], 0.0, atol=1e-9)
    # points: the closed form -Sigma^{-1}(x' - mu), rotated back
    g = -(xp - mu) @ np.linalg.inv(S)
    np.testing.assert_allclose(r["grad_points"], g @ R, rtol=1e-9, atol=1e-9 * np.abs(g).max())


def test_single_component_mean_gradient_closed_form():
    pts, _, means, chol, pose = problem(n=300, k=1, seed=8)
    R, t = pose
    xp = pts.astype(np.float64) @ R.T + t
    S = chol[0] @ chol[0].T
    want = np.linalg.solve(S, (xp - means[0]).sum(0))
    r = oracle.loglik_grad(pts, np.zeros(1), means, chol, pose)
    np.testing.assert_allclose(r["grad_means"][0], want, rtol=1e-10)


def test_rejects_non_positive_diagonal():
    pts, logits, means, chol, pose = problem()
    chol[1, 1, 1] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.loglik_grad(pts, logits, means, chol, pose)
    assert oracle.last_bad_component() == 1
