"""GPU parity of the differentiable log-likelihood (gira_gmm_loglik_grad and its
torch.autograd binding) against the FP64 oracle.

Tolerances (binary32 kernel with binary64 reductions vs the FP64 oracle):
  L                      |dL| <= 1e-5 * N + 4e-7 * |L|: the fit's 1e-5 mean
                         per-point bound, plus the binary32 storage of the
                         precision factors P' (relative 2^-24 per entry, about
                         3 entries per y) that scales |y|^2 ~ 2 |l_n| by up to
                         ~3.6e-7 for every point of a component alike
  per-component groups   max |d g| <= 1e-4 * max |g_ref| over the group (logits,
                         means, Cholesky factors, twist, pose), a norm-wise bound:
                         each entry is a sum over points of binary32 terms
  per-point gradients    |d g_n| <= 1e-3 * |g_n| + 1e-4 * rms_n |g_n|: one binary32
                         term per component, whose input y = P'(x' - mu) carries
                         the cancellation of a point metres from the origin
                         against a millimetre-scale Cholesky factor
"""
import math

import numpy as np
import pytest

import oracle
from paper_2307_00071_gb300 import synth
from tests._parity import to_np

pytestmark = pytest.mark.gpu

GRP_REL = 1e-4
PT_REL, PT_RMS = 1e-3, 1e-4


@pytest.fixture(scope="module")
def gira():
    from paper_2307_00071_gb300 import gira as g
    return g


def rot(w):
    th = np.linalg.norm(w)
    if th == 0.0:
        return np.eye(3)
    k = np.asarray(w) / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx


def model_from_mixture(cl, rng, jitter=0.05):
    """Logits, means, Cholesky factors near a generating mixture (binary32)."""
    K = len(cl.weights)
    logits = np.log(cl.weights) + rng.normal(scale=0.1, size=K)
    means = cl.means + rng.normal(scale=jitter, size=(K, 3))
    chol = np.stack([np.linalg.cholesky(c * rng.uniform(0.8, 1.25)) for c in cl.covs])
    return logits.astype(np.float32), means.astype(np.float32), chol.astype(np.float32)


def small_pose(rng, deg=10.0, trans=0.2):
    w = rng.normal(size=3)
    w *= math.radians(deg) / np.linalg.norm(w)
    return rot(w).astype(np.float32), rng.uniform(-trans, trans, size=3).astype(np.float32)


def pose12(R, t):
    return np.concatenate([np.asarray(R, np.float32).reshape(9), np.asarray(t, np.float32)])


def ref_grads(pts, logits, means, chol, R, t):
    r = oracle.loglik_grad(pts, logits.astype(np.float64), means.astype(np.float64), chol.astype(np.float64),
                           (np.float64(R), np.float64(t)))
    g = r["grad_points"] @ np.float64(R).T   # dL/dx'
    M = g.T @ pts.astype(np.float64)          # sum g x^T
    r["grad_pose"] = np.concatenate([M.reshape(9), g.sum(0)])
    return r


def ll_tol(L, n):
    return 1e-5 * n + 4e-7 * abs(L)


def assert_group(got, ref, name, rel=GRP_REL):
    got, ref = to_np(got).astype(np.float64), np.asarray(ref, np.float64)
    err = np.max(np.abs(got - ref))
    scale = np.max(np.abs(ref))
    assert err <= rel * scale, f"{name}: max err {err:.3e} vs max |ref| {scale:.3e} (rel {err / scale:.2e})"


def assert_points(got, ref):
    got, ref = to_np(got).astype(np.float64), np.asarray(ref, np.float64)
    d = np.linalg.norm(got - ref, axis=1)
    mag = np.linalg.norm(ref, axis=1)
    rms = np.sqrt(np.mean(mag ** 2))
    bad = d > PT_REL * mag + PT_RMS * rms
    assert not bad.any(), (f"{bad.sum()} points outside tolerance; worst rel {np.max(d / (mag + 1e-30)):.2e}, "
                           f"max err / rms {np.max(d) / rms:.2e}")


def check_all(r, ref, n):
    assert abs(r["loglik"] - ref["loglik"]) <= ll_tol(ref["loglik"], n), (r["loglik"], ref["loglik"])
    for g in ("logits", "means", "chol", "twist", "pose"):
        assert_group(r["grad_" + g], ref["grad_" + g], g)
    assert_points(r["grad_points"], ref["grad_points"])


@pytest.mark.parametrize("n,k,seed", [(20_000, 8, 0), (5_001, 37, 3), (3_000, 130, 5)])
def test_grad_matches_oracle(gira, n, k, seed):
    rng = np.random.default_rng(100 + seed)
    cl = synth.gmm_cloud(n, k, seed=seed)
    logits, means, chol = model_from_mixture(cl, rng)
    R, t = small_pose(rng)
    import torch
    dev = lambda a: torch.as_tensor(a, device="cuda")
    # the scan is the cloud moved by the inverse pose, so R x + t lands on the model
    scan = ((cl.points.astype(np.float64) - t) @ np.float64(R)).astype(np.float32)
    r = gira.gira_gmm_loglik_grad(dev(scan), dev(logits), dev(means), dev(chol), dev(pose12(R, t)))
    check_all(r, ref_grads(scan, logits, means, chol, R, t), n)


def test_grad_host_buffers_and_identity_pose(gira):
    rng = np.random.default_rng(7)
    cl = synth.gmm_cloud(4_000, 6, seed=7)
    logits, means, chol = model_from_mixture(cl, rng)
    r = gira.gira_gmm_loglik_grad(cl.points, logits, means, chol, None)
    check_all(r, ref_grads(cl.points, logits, means, chol, np.eye(3), np.zeros(3)), len(cl.points))


def test_grad_subsets_and_forward_only_agree(gira):
    import torch
    rng = np.random.default_rng(9)
    cl = synth.gmm_cloud(6_000, 12, seed=9)
    logits, means, chol = model_from_mixture(cl, rng)
    R, t = small_pose(rng)
    args = [torch.as_tensor(a, device="cuda") for a in (cl.points, logits, means, chol, pose12(R, t))]
    full = gira.gira_gmm_loglik_grad(*args)
    for want in (("points",), ("logits",), ("twist", "chol"), ()):
        part = gira.gira_gmm_loglik_grad(*args, want=want)
        assert part["loglik"] == pytest.approx(full["loglik"], rel=1e-12, abs=1e-9)
        for g in want:
            assert torch.equal(part["grad_" + g], full["grad_" + g])
    # forward-only equals the plain log-likelihood of the moved scan
    moved = (cl.points.astype(np.float64) @ np.float64(R).T + t).astype(np.float32)
    w = np.exp(logits - logits.max())
    w = (w / w.sum()).astype(np.float32)
    covs = np.einsum("kij,klj->kil", chol.astype(np.float64), chol.astype(np.float64)).astype(np.float32)
    mean = gira.gira_gmm_loglik(moved, w, means, covs)
    assert abs(full["loglik"] / len(moved) - mean) <= ll_tol(mean, 1)


def test_grad_single_point_single_component(gira):
    pts = np.array([[0.3, -0.2, 1.1]], np.float32)
    logits = np.zeros(1, np.float32)
    means = np.array([[0.25, -0.1, 1.0]], np.float32)
    chol = np.array([np.diag([0.1, 0.2, 0.05])], np.float32)
    chol[0, 2, 0] = 0.02
    r = gira.gira_gmm_loglik_grad(pts, logits, means, chol, None)
    check_all(r, ref_grads(pts, logits, means, chol, np.eye(3), np.zeros(3)), 1)


def test_grad_rejects_bad_cholesky(gira):
    pts = synth.gmm_cloud(1_000, 3, seed=1).points
    logits = np.zeros(3, np.float32)
    means = np.zeros((3, 3), np.float32)
    chol = np.tile(np.eye(3, dtype=np.float32), (3, 1, 1))
    chol[2, 1, 1] = -1.0
    with pytest.raises(gira.GiraError) as e:
        gira.gira_gmm_loglik_grad(pts, logits, means, chol, None)
    assert e.value.status == gira.ERR_NOT_PD
    assert e.value.component == 2


def frame_model(frame_pts, K, rng):
    """A K-component model on a depth frame from a seeded generator (not from a fit):
    means at random frame points, thin disc-like covariances (1-5 cm, 5 mm normal)."""
    idx = rng.choice(len(frame_pts), K, replace=False)
    means = frame_pts[idx].astype(np.float64) + rng.normal(scale=0.01, size=(K, 3))
    chol = []
    for _ in range(K):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = np.array([rng.uniform(0.01, 0.05), rng.uniform(0.01, 0.05), 0.005]) ** 2
        chol.append(np.linalg.cholesky(Q @ np.diag(lam) @ Q.T))
    logits = rng.normal(scale=0.3, size=K)
    return logits.astype(np.float32), means.astype(np.float32), np.stack(chol).astype(np.float32)


def test_grad_frame_scale_k1024(gira):
    """Registration-sized model (K = 1024) on depth-frame points metres from the origin."""
    import torch
    rng = np.random.default_rng(11)
    frame = synth.depth_frame(seed=1).points
    logits, means, chol = frame_model(frame, 1024, rng)
    scan = frame[rng.choice(len(frame), 20_000, replace=False)]
    R, t = small_pose(rng, deg=2.0, trans=0.02)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    r = gira.gira_gmm_loglik_grad(dev(scan), dev(logits), dev(means), dev(chol), dev(pose12(R, t)))
    check_all(r, ref_grads(scan, logits, means, chol, R, t), len(scan))


def test_autograd_matches_oracle_and_chains_through_se3(gira):
    import torch
    from paper_2307_00071_gb300 import autograd as ag
    rng = np.random.default_rng(13)
    cl = synth.gmm_cloud(8_000, 10, seed=13)
    logits, means, chol = model_from_mixture(cl, rng)
    R0, t0 = small_pose(rng)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    pts = dev(cl.points).requires_grad_(True)
    lg, mu, ch = (dev(a).requires_grad_(True) for a in (logits, means, chol))
    xi = torch.zeros(6, dtype=torch.float64, device="cuda", requires_grad=True)
    Rd, td = ag.se3_exp(xi)
    R = Rd @ dev(R0).double()
    t = Rd @ dev(t0).double() + td
    L = ag.gmm_loglik(pts, lg, mu, ch, R, t)
    L.backward()
    ref = ref_grads(cl.points, logits, means, chol, R0, t0)
    assert abs(L.item() - ref["loglik"]) <= ll_tol(ref["loglik"], len(cl.points))
    assert_group(lg.grad, ref["grad_logits"], "logits")
    assert_group(mu.grad, ref["grad_means"], "means")
    assert_group(ch.grad, ref["grad_chol"], "chol")
    assert_points(pts.grad, ref["grad_points"])
    # at xi = 0 the chain through exp gives the left-perturbation twist gradient
    assert_group(xi.grad, ref["grad_twist"], "twist via se3_exp")


def test_registration_recovers_pose(gira):
    """A scan of a frame moved by a random rigid offset (<= 15 deg, <= 0.5 m) plus
    5 mm noise is registered to a GMM of the frame by gradient steps on the twist."""
    import torch
    from paper_2307_00071_gb300 import autograd as ag
    rng = np.random.default_rng(17)
    frame = synth.depth_frame(seed=2).points
    x = torch.as_tensor(frame, device="cuda")
    fit = gira.gira_gmm_fit(x, 256, iters=20, tol=1e-4, seed=0, lloyd_iters=10)
    w, mu, cov = fit["weights"], fit["means"], fit["covs"]
    logits = torch.log(w)
    chol = torch.linalg.cholesky(cov.double()).float()
    w_off = rng.normal(size=3)
    w_off *= math.radians(rng.uniform(5, 15)) / np.linalg.norm(w_off)
    R_off = rot(w_off)
    t_off = rng.uniform(-0.5, 0.5, size=3)
    sub = frame[rng.choice(len(frame), 100_000, replace=False)].astype(np.float64)
    scan = (sub @ R_off.T + t_off + rng.normal(scale=0.005, size=sub.shape)).astype(np.float32)
    # rotate about the scan's centroid: s = scan - c_scan, x' = R s + t, t starts at the map's centroid
    c_scan = scan.astype(np.float64).mean(0)
    s = torch.as_tensor((scan - c_scan).astype(np.float32), device="cuda")
    R = torch.eye(3, dtype=torch.float64, device="cuda")
    t = torch.as_tensor(frame.astype(np.float64).mean(0), dtype=torch.float64, device="cuda")
    xi = torch.zeros(6, dtype=torch.float64, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([xi], lr=0.02)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=0.96)
    for step in range(100):
        opt.zero_grad()
        Rd, td = ag.se3_exp(xi)
        L = ag.gmm_loglik(s, logits, mu, chol, Rd @ R, Rd @ t + td)
        (-L / len(scan)).backward()
        opt.step()
        sched.step()
    with torch.no_grad():
        Rd, td = ag.se3_exp(xi)
        R_est, t_est = (Rd @ R).cpu().numpy(), (Rd @ t + td).cpu().numpy()
    # truth: map point = R_off^T (scan - t_off) = R_off^T s + R_off^T (c_scan - t_off)
    dR = R_est @ R_off
    ang = math.degrees(math.acos(np.clip((np.trace(dR) - 1) / 2, -1, 1)))
    dt = np.linalg.norm(t_est - R_off.T @ (c_scan - t_off))
    assert ang < 1.0 and dt < 0.03, (ang, dt)


def test_batched_grad_matches_oracle_per_instance(gira):
    """Five registrations of uneven size and K (three block shapes) in one call."""
    import torch
    rng = np.random.default_rng(21)
    sizes, kk = [3_000, 8_000, 2_500, 6_000, 4_000], [6, 40, 130, 9, 300]
    scans, models, poses = [], [], []
    for i, (n, k) in enumerate(zip(sizes, kk)):
        cl = synth.gmm_cloud(n, min(k, 12), seed=200 + i)
        if k > 12:   # more components than the generating mixture: centred on points
            idx = rng.choice(n, k, replace=False)
            mu = (cl.points[idx] + rng.normal(scale=0.01, size=(k, 3))).astype(np.float32)
            ch = np.stack([np.eye(3) * rng.uniform(0.02, 0.1) for _ in range(k)]).astype(np.float32)
            lg = rng.normal(scale=0.2, size=k).astype(np.float32)
        else:
            lg, mu, ch = model_from_mixture(cl, rng)
        R, t = small_pose(rng)
        scans.append(((cl.points.astype(np.float64) - t) @ np.float64(R)).astype(np.float32))
        models.append((lg, mu, ch))
        poses.append(pose12(R, t))
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    dev = lambda a: torch.as_tensor(a, device="cuda")
    r = gira.gira_gmm_loglik_grad_batched(dev(np.concatenate(scans)), offs, kk,
                                          dev(np.concatenate([m[0] for m in models])),
                                          dev(np.concatenate([m[1] for m in models])),
                                          dev(np.concatenate([m[2] for m in models])), dev(np.stack(poses)))
    assert np.all(r["status"] == 0)
    ck = np.concatenate([[0], np.cumsum(kk)])
    for i in range(len(kk)):
        R, t = poses[i][:9].reshape(3, 3), poses[i][9:]
        ref = ref_grads(scans[i], *models[i], R, t)
        got = {"loglik": r["loglik"][i],
               "grad_points": to_np(r["grad_points"])[offs[i]:offs[i + 1]],
               "grad_pose": to_np(r["grad_pose"])[i], "grad_twist": to_np(r["grad_twist"])[i],
               "grad_logits": to_np(r["grad_logits"])[ck[i]:ck[i + 1]],
               "grad_means": to_np(r["grad_means"])[ck[i]:ck[i + 1]],
               "grad_chol": to_np(r["grad_chol"])[ck[i]:ck[i + 1]]}
        check_all(got, ref, sizes[i])
    # a second call with new poses reuses the cached graph and follows the new inputs
    poses2 = [pose12(*small_pose(rng)) for _ in kk]
    r2 = gira.gira_gmm_loglik_grad_batched(dev(np.concatenate(scans)), offs, kk,
                                           dev(np.concatenate([m[0] for m in models])),
                                           dev(np.concatenate([m[1] for m in models])),
                                           dev(np.concatenate([m[2] for m in models])), dev(np.stack(poses2)),
                                           want=("twist",))
    for i in (0, 4):
        R, t = poses2[i][:9].reshape(3, 3), poses2[i][9:]
        ref = ref_grads(scans[i], *models[i], R, t)
        assert abs(r2["loglik"][i] - ref["loglik"]) <= ll_tol(ref["loglik"], sizes[i])
        assert_group(to_np(r2["grad_twist"])[i], ref["grad_twist"], "twist")


@pytest.mark.parametrize("offset_seed", [3, 4])
def test_registration_k1024_second_scan_of_the_scene(gira, offset_seed):
    """The differentiable-registration configuration: a K = 1024 GMM fitted to the
    depth frame; a second scan of the same scene (its own 5 mm sensor noise and
    dropout), 100k of its points under a random rigid offset (<= 15 deg, <= 0.5 m);
    100 Adam steps on the twist recover the offset."""
    import torch
    from paper_2307_00071_gb300 import autograd as ag
    frame = synth.depth_frame(seed=1).points
    fit = gira.gira_gmm_fit(torch.as_tensor(frame, device="cuda"), 1024, iters=30, tol=1e-4, seed=0, lloyd_iters=10)
    logits = torch.log(fit["weights"])
    chol = torch.linalg.cholesky(fit["covs"].double()).float()
    scan, R_off, t_off = synth.registration_scan(seed=1, offset_seed=offset_seed)
    R, t, ll = ag.register_scan(torch.as_tensor(scan, device="cuda"), logits, fit["means"], chol, steps=100)
    R, t = R.cpu().numpy(), t.cpu().numpy()
    # truth: x = R_off^T (scan - t_off)
    dR = R @ R_off
    ang = math.degrees(math.acos(np.clip((np.trace(dR) - 1) / 2, -1, 1)))
    dt = np.linalg.norm(t + R_off.T @ t_off)
    assert ang < 0.5 and dt < 0.02, (ang, dt, ll)
