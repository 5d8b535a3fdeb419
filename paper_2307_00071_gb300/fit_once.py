"""Run a fixed number of fits on a synthetic workload (profiling driver).

    python -m paper_2307_00071_gb300.fit_once --workload frame --fits 1

``frame``: the 276k-point 640x480 depth frame, K=512, 30 iterations, tol 1e-4
(the benchmark's step).  ``gmm20k``: 20k points from a K=8 GMM, 20 iterations.
Used under ncu, where a fixed, short launch sequence is wanted.
"""
from __future__ import annotations

import argparse

import torch

from . import gira, synth


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", choices=["frame", "gmm20k"], default="frame")
    p.add_argument("--fits", type=int, default=1)
    a = p.parse_args()
    if a.workload == "frame":
        pts, k, iters, tol = synth.depth_frame(seed=1).points, 512, 30, 1e-4
    else:
        pts, k, iters, tol = synth.gmm_cloud(20_000, 8, seed=0).points, 8, 20, 0.0
    x = torch.as_tensor(pts, device="cuda")
    for _ in range(a.fits):
        r = gira.gira_gmm_fit(x, k, iters=iters, tol=tol, reg_covar=1e-6, seed=0, lloyd_iters=10)
    torch.cuda.synchronize()
    print(f"{a.workload}: N={len(pts)} K={k} iters_done={r['iters_done']} final_loglik={r['final_loglik']:.6f}")


if __name__ == "__main__":
    main()
