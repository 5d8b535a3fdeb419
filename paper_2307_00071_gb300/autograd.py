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


def register_scan(scan, logits, means, chol, steps=100, lr=0.02, decay=0.96, t0=None):
    """Likelihood-based rigid registration as a gradient solve: the pose (R, t)
    that maximises the mean log-likelihood of ``R scan + t`` under the mixture
    (logits, means, Cholesky factors), by ``steps`` Adam steps on the twist of a
    left perturbation.  The scan is rotated about its own centroid and the
    translation starts at ``t0`` (default: the mixture's weighted mean of the
    means), which keeps rotation and translation well scaled.  Every likelihood
    and gradient comes from the library's fused kernel; the optimiser updates six
    numbers.  Returns (R (3, 3), t (3,)) in binary64 such that R scan + t lies on
    the mixture, and the final mean log-likelihood."""
    dev = scan.device
    c = scan.double().mean(0)
    s = (scan.double() - c).float().contiguous()
    R0 = torch.eye(3, dtype=torch.float64, device=dev)
    if t0 is None:
        w = torch.softmax(logits.double(), 0)
        t0 = (w[:, None] * means.double()).sum(0)
    t_base = torch.as_tensor(t0, dtype=torch.float64, device=dev)
    xi = torch.zeros(6, dtype=torch.float64, device=dev, requires_grad=True)
    opt = torch.optim.Adam([xi], lr=lr)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=decay)
    n = len(scan)
    for _ in range(steps):
        opt.zero_grad()
        Rd, td = se3_exp(xi)
        L = gmm_loglik(s, logits, means, chol, Rd @ R0, Rd @ t_base + td)
        (-L / n).backward()
        opt.step()
        sched.step()
    with torch.no_grad():
        Rd, td = se3_exp(xi)
        R = Rd @ R0
        t = Rd @ t_base + td
        L = gmm_loglik(s, logits, means, chol, R, t)
    # R (scan - c) + t = R scan + (t - R c)
    return R, t - R @ c, float(L) / n
