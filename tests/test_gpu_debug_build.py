"""The debug build (libgira_debug.so, -DGIRA_DEBUG) on small odd cases.

In that build the kernels check the indices they compute against their buffers
(points, listed pairs, partial and mask rows, log-likelihood slots, labels,
component permutations, the chosen seeding point) and record GIRA_ERR_BOUNDS
instead of making an access outside them.  Every entry point runs here on
cases with N <= 64 and K <= 4 (ragged tiles, single points, odd K) in a child
process that loads the debug library (GIRA_DEBUG=1) and in one that loads the
release library; every call must succeed in the debug build and give the same
bits as the release build (the checks change no arithmetic).
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, sys
import numpy as np, torch
from paper_2307_00071_gb300 import gira, synth

def cloud(n, d=3, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, d)).astype(np.float32) * np.float32(0.5)

def model(k, d=3, seed=1):
    rng = np.random.default_rng(seed)
    w = rng.dirichlet(np.ones(k)).astype(np.float32)
    mu = rng.normal(size=(k, d)).astype(np.float32) * np.float32(0.5)
    a = rng.normal(size=(k, d, d))
    cov = (0.05 * (a @ a.transpose(0, 2, 1) + 0.5 * np.eye(d))).astype(np.float32)
    return w, mu, cov

def dev(*a):
    return [torch.as_tensor(x, device="cuda") for x in a]

def flat(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        x = x.detach().cpu().numpy()
    return np.asarray(x, dtype=np.float64).ravel().tolist()

out = {"lib": gira.LIB_PATH}
for n, k in ((1, 1), (5, 2), (31, 3), (33, 4), (64, 4)):
    pts = cloud(n, seed=n)
    x = dev(pts)[0]
    c, lab, _ = gira.gira_kmeans_init(x, k, seed=3, lloyd_iters=4)
    out[f"kinit{n}_{k}"] = flat(c) + flat(lab)
    r = gira.gira_gmm_fit(x, k, iters=6, tol=0.0, seed=3, lloyd_iters=4)
    out[f"fit{n}_{k}"] = flat(r["weights"]) + flat(r["means"]) + flat(r["covs"]) + flat(r["trace"])
    w, mu, cov = model(k)
    m, pp = gira.gira_gmm_loglik(x, *dev(w, mu, cov), per_point=True)
    out[f"ll{n}_{k}"] = [m] + flat(pp)
    m2, pp2 = gira.gira_gmm_loglik_noalloc(x, *dev(w, mu, cov), per_point=True)
    out[f"llna{n}_{k}"] = [m2] + flat(pp2)
    chol = np.linalg.cholesky(cov.astype(np.float64)).astype(np.float32)
    g = gira.gira_gmm_loglik_grad(x, *dev(np.log(w), mu, chol))
    out[f"grad{n}_{k}"] = [g["loglik"]] + sum((flat(v) for kk, v in sorted(g.items()) if kk.startswith("grad_")), [])
    x4 = dev(cloud(n, 4, seed=n + 7))[0]
    r4 = gira.gira_gmm_fit4(x4, k, iters=4, tol=0.0, seed=2, lloyd_iters=3)
    out[f"fit4_{n}_{k}"] = flat(r4["weights"]) + flat(r4["means"]) + flat(r4["covs"])
    w4, mu4, cov4 = model(k, 4, seed=5)
    l4 = gira.gira_gmm_loglik4(x4, *dev(w4, mu4, cov4), per_point=True)
    out[f"ll4_{n}_{k}"] = [l4[0]] + flat(l4[1])
    e, v = gira.gira_gmm_conditional4(x, *dev(w4, mu4, cov4))
    out[f"cond{n}_{k}"] = flat(e) + flat(v)
    s, comp = gira.gira_gmm_sample(n, *dev(w, mu, cov), seed=9, device="cuda")
    out[f"sample{n}_{k}"] = flat(s) + flat(comp)
    modes = gira.gira_gbms(x4, 0.5, max_iter=20)
    out[f"gbms{n}_{k}"] = flat(modes[0]) + flat(modes[1])
# batches with ragged instances
sizes, ks = [1, 7, 64, 33, 5], [1, 3, 4, 2, 4]
pts = np.concatenate([cloud(s_, seed=100 + i) for i, s_ in enumerate(sizes)])
offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
x = dev(pts)[0]
rb = gira.gira_gmm_fit_batched(x, offs, ks, iters=5, tol=0.0, seed=4, lloyd_iters=3)
out["batched"] = flat(rb["weights"]) + flat(rb["means"]) + flat(rb["covs"]) + flat(rb["trace"])
mods = [model(k_, seed=20 + i) for i, k_ in enumerate(ks)]
lg = np.concatenate([np.log(m_[0]) for m_ in mods])
mu = np.concatenate([m_[1] for m_ in mods])
ch = np.concatenate([np.linalg.cholesky(m_[2].astype(np.float64)).astype(np.float32) for m_ in mods])
gb = gira.gira_gmm_loglik_grad_batched(x, offs, ks, *dev(lg, mu, ch))
out["grad_batched"] = flat(gb["loglik"]) + sum((flat(v) for kk, v in sorted(gb.items()) if kk.startswith("grad_")), [])
print(json.dumps(out))
'''


def run(debug: bool):
    env = dict(os.environ, GIRA_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_runs_every_entry_point_and_matches_release():
    from paper_2307_00071_gb300 import build_lib
    build_lib.build(debug=True)
    dbg, rel = run(True), run(False)
    assert dbg.pop("lib").endswith("libgira_debug.so")
    assert rel.pop("lib").endswith("libgira.so")
    assert dbg.keys() == rel.keys()
    for key in rel:
        assert dbg[key] == rel[key], key
