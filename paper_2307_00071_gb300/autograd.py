"""torch.autograd binding of the differentiable GMM log-likelihood.

    L = sum_n ln sum_b softmax(logits)_b N(R x_n + t | mu_b, L_b L_b^T)

The forward call runs the library's fused log-likelihood / adjoint kernel
(`gira_gmm_loglik_grad`): one pass over points x components that recomputes
the responsibilities instead of storing them and produces, with L, the
gradients of every input that requires one.  The backward step only scales
those by the incoming gradient.  Everything runs in the CUDA library; this
module marshals tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gira

_NAMES = ("points", "R", "t", "logits", "means", "chol")


class GmmLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, R, t, logits, means, chol):
        need = dict(zip(_NAMES, ctx.needs_input_grad))
        want = []
        if need["points"]:
            want.append("points")
        if need["R"] or need["t"]:
            want.append("pose")
        for name in ("logits", "means", "chol"):
            if need[name]:
                want.append(name)
        pose = torch.cat([R.reshape(9), t.reshape(3)]).to(torch.float32).contiguous()
        r = gira.gira_gmm_loglik_grad(points.detach().contiguous(), logits.detach().contiguous(),
                                      means.detach().contiguous(), chol.detach().contiguous(), pose, want=want)
        g = {name: None for name in _NAMES}
        if "points" in want:
            g["points"] = r["grad_points"]
        if "pose" in want:
            gp = r["grad_pose"]
            g["R"] = gp[:9].reshape(3, 3).to(R.dtype)
            g["t"] = gp[9:].to(t.dtype)
        for name in ("logits", "means", "chol"):
            if name in want:
                g[name] = r["grad_" + name]
        ctx.grads = g
        return torch.tensor(r["loglik"], dtype=torch.float64, device=points.device)

    @staticmethod
    def backward(ctx, gout):
        out = []
        for name in _NAMES:
            v = ctx.grads[name]
            out.append(None if v is None else v * gout.to(v.dtype))
        return tuple(out)


def gmm_loglik(points, logits, means, chol, R=None, t=None):
    """Differentiable L (binary64 scalar tensor); R, t default to the identity."""
    dev = points.device
    if R is None:
        R = torch.eye(3, dtype=torch.float32, device=dev)
    if t is None:
        t = torch.zeros(3, dtype=torch.float32, device=dev)
    return GmmLogLik.apply(points, R, t, logits, means, chol)


def hat(w):
    """Skew-symmetric matrix of a 3-vector (differentiable)."""
    z = torch.zeros((), dtype=w.dtype, device=w.device)
    return torch.stack([torch.stack([z, -w[2], w[1]]), torch.stack([w[2], z, -w[0]]),
                        torch.stack([-w[1], w[0], z])])


def se3_exp(xi):
    """(R, t) = exp(xi^) for the twist xi = (omega, v), rotation first (differentiable;
    series form near omega = 0)."""
    w, v = xi[:3], xi[3:]
    th2 = (w * w).sum()
    th = torch.sqrt(th2 + 1e-30)
    W = hat(w)
    W2 = W @ W
    small = th2 < 1e-8
    A = torch.where(small, 1 - th2 / 6, torch.sin(th) / th)
    B = torch.where(small, 0.5 - th2 / 24, (1 - torch.cos(th)) / (th2 + 1e-30))
    C = torch.where(small, 1.0 / 6 - th2 / 120, (th - torch.sin(th)) / (th2 * th + 1e-30))
    eye = torch.eye(3, dtype=xi.dtype, device=xi.device)
    R = eye + A * W + B * W2
    V = eye + B * W + C * W2
    return R, V @ v


def _exp_se3_np(xi):
    """(R, t) = exp(xi^) for xi = (omega, v), binary64 numpy (Rodrigues, series near 0)."""
    w, v = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    th2 = float(w @ w)
    th = np.sqrt(th2)
    W = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if th2 < 1e-8:
        A, B, Cc = 1 - th2 / 6, 0.5 - th2 / 24, 1.0 / 6 - th2 / 120
    else:
        A, B, Cc = np.sin(th) / th, (1 - np.cos(th)) / th2, (th - np.sin(th)) / (th2 * th)
    R = np.eye(3) + A * W + B * (W @ W)
    V = np.eye(3) + B * W + Cc * (W @ W)
    return R, V @ v


def register_scan(scan, logits, means, chol, steps=100, lr=0.02, decay=0.96, t0=None):
    """Likelihood-based rigid registration as a gradient solve: the pose (R, t)
    that maximises the mean log-likelihood of ``R scan + t`` under the mixture
    (logits, means, Cholesky factors).  Each of ``steps`` Adam steps takes one
    library call for L and its gradient with respect to a left perturbation
    (twist) of the current pose, and moves the pose by the exponential of the
    step: the optimiser itself is six numbers on the host.  The scan is rotated
    about its own centroid and the translation starts at ``t0`` (default: the
    mixture's weighted mean of the means), which keeps rotation and translation
    well scaled.  Returns (R (3, 3), t (3,)) in binary64 such that R scan + t lies
    on the mixture, and the final mean log-likelihood."""
    dev = scan.device
    c = scan.double().mean(0)
    s = (scan.double() - c).float().contiguous()
    if t0 is None:
        w = torch.softmax(logits.double(), 0)
        t0 = (w[:, None] * means.double()).sum(0)
    R = np.eye(3)
    t = np.asarray(torch.as_tensor(t0, dtype=torch.float64).cpu().numpy(), np.float64).copy()
    lg, mu, ch = logits.detach().contiguous(), means.detach().contiguous(), chol.detach().contiguous()
    n = len(scan)
    m1, m2 = np.zeros(6), np.zeros(6)
    b1, b2, eps = 0.9, 0.999, 1e-8
    step = lr
    for it in range(1, steps + 1):
        pose = torch.as_tensor(np.concatenate([R.reshape(9), t]).astype(np.float32), device=dev)
        r = gira.gira_gmm_loglik_grad(s, lg, mu, ch, pose, want=("twist",))
        g = -np.asarray(r["grad_twist"].cpu().numpy() if hasattr(r["grad_twist"], "cpu") else r["grad_twist"],
                        np.float64) / n
        m1 = b1 * m1 + (1 - b1) * g
        m2 = b2 * m2 + (1 - b2) * g * g
        d = -step * (m1 / (1 - b1 ** it)) / (np.sqrt(m2 / (1 - b2 ** it)) + eps)
        Rd, td = _exp_se3_np(d)
        R, t = Rd @ R, Rd @ t + td
        step *= decay
    pose = torch.as_tensor(np.concatenate([R.reshape(9), t]).astype(np.float32), device=dev)
    ll = gira.gira_gmm_loglik_grad(s, lg, mu, ch, pose, want=())["loglik"]
    cn = c.cpu().numpy()
    R_t, t_t = torch.as_tensor(R, device=dev), torch.as_tensor(t - R @ cn, device=dev)
    return R_t, t_t, float(ll) / n
