"""Run a fixed number of fits on a synthetic workload (profiling driver).

    python -m paper_2307_00071_gb300.fit_once --workload frame --fits 1

``frame``: the 276k-point 640x480 depth frame, K=512, 30 iterations, tol 1e-4
(the benchmark's step).  ``gmm20k``: 20k points from a K=8 GMM, 20 iterations.
``grad1024``: L and all gradients of a 100k-point scan under a K=1024 GMM of the
frame (``--fits`` calls).  ``chunk2048``: the chunked E-step, K=2048 on the frame.
``frame4``: the frame with its intensity channel (N x 4), K=512, 30 iterations,
tol 1e-4.  ``gbms``: mode seeking on the frame with intensity, bandwidth 0.05.
Used under ncu, where a fixed, short launch sequence is wanted.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import gira, synth


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", choices=["frame", "gmm20k", "grad1024", "chunk2048", "frame4", "gbms"],
                   default="frame")
    p.add_argument("--fits", type=int, default=1)
    a = p.parse_args()
    if a.workload == "grad1024":
        grad_workload(a.fits)
        return
    if a.workload == "chunk2048":
        chunk_workload(a.fits)
        return
    if a.workload in ("frame4", "gbms"):
        x4 = torch.as_tensor(synth.depth_frame4(seed=1), device="cuda")
        for _ in range(a.fits):
            if a.workload == "frame4":
                r = gira.gira_gmm_fit4(x4, 512, iters=30, tol=1e-4, reg_covar=1e-6, seed=0, lloyd_iters=10)
                msg = f"iters_done={r['iters_done']} final_loglik={r['final_loglik']:.6f}"
            else:
                m, c = gira.gira_gbms(x4, 0.05)
                msg = f"K={len(m)}"
        torch.cuda.synchronize()
        print(f"{a.workload}: N={x4.shape[0]} {msg}")
        return
    if a.workload == "frame":
        pts, k, iters, tol = synth.depth_frame(seed=1).points, 512, 30, 1e-4
    else:
        pts, k, iters, tol = synth.gmm_cloud(20_000, 8, seed=0).points, 8, 20, 0.0
    x = torch.as_tensor(pts, device="cuda")
    for _ in range(a.fits):
        r = gira.gira_gmm_fit(x, k, iters=iters, tol=tol, reg_covar=1e-6, seed=0, lloyd_iters=10)
    torch.cuda.synchronize()
    print(f"{a.workload}: N={len(pts)} K={k} iters_done={r['iters_done']} final_loglik={r['final_loglik']:.6f}")


def grad_workload(calls):
    """L and all gradients for a 100k-point scan of the frame under a K=1024 GMM fitted to it."""
    frame = synth.depth_frame(seed=1).points
    x = torch.as_tensor(frame, device="cuda")
    fit = gira.gira_gmm_fit(x, 1024, iters=10, tol=1e-4, seed=0, lloyd_iters=5)
    logits = torch.log(fit["weights"])
    chol = torch.as_tensor(np.linalg.cholesky(fit["covs"].double().cpu().numpy()).astype(np.float32), device="cuda")
    rng = np.random.default_rng(5)
    scan = torch.as_tensor(frame[rng.choice(len(frame), 100_000, replace=False)], device="cuda")
    pose = torch.as_tensor(np.concatenate([np.eye(3).reshape(9), [0.01, 0.0, 0.0]]).astype(np.float32),
                           device="cuda")
    for _ in range(calls):
        r = gira.gira_gmm_loglik_grad(scan, logits, fit["means"], chol, pose)
    torch.cuda.synchronize()
    print(f"grad1024: loglik={r['loglik']:.3f}")


def chunk_workload(fits):
    """Chunked E-step: K=2048 on the frame from means at random points, 3 EM iterations."""
    frame = synth.depth_frame(seed=1).points
    x = torch.as_tensor(frame, device="cuda")
    rng = np.random.default_rng(3)
    idx = torch.as_tensor(rng.choice(len(frame), 2048, replace=False), device="cuda")
    for _ in range(fits):
        w0 = torch.full((2048,), 1.0 / 2048, device="cuda")
        c0 = (torch.eye(3, device="cuda") * 0.05 ** 2).expand(2048, 3, 3).contiguous()
        r = gira.gira_gmm_fit(x, 2048, iters=3, tol=0.0, init=(w0, x[idx].clone(), c0), final_loglik=False)
    torch.cuda.synchronize()
    print(f"chunk2048: trace={list(r['trace'])}")


if __name__ == "__main__":
    main()
