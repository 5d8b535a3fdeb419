"""Seeded synthetic point clouds for the GMM-EM workloads.

This module only *generates inputs*; it contains none of the EM arithmetic (no
log-densities, responsibilities, k-means or sufficient statistics). Both the
CUDA path (tests, bench) and the FP64 oracle (tests) consume what it returns,
so it imports neither of them.

Workloads (all numpy PCG64 ``default_rng(seed)``):

* :func:`gmm_cloud` -- points drawn from a random full-covariance 3D GMM:
  means uniform in ``[-2, 2]^3`` m, covariance ``R diag(lam) R^T`` with
  ``lam`` log-uniform in ``[1e-4, 1e-2]`` m^2 and ``R`` Haar-random, weights
  Dirichlet(1), per-component counts multinomial.  The 20k-point, K=8 cloud is
  the small workload; it stands in for no dataset.
* :func:`depth_frame` -- a 640x480 pinhole depth image (fx = fy = 525,
  cx = 319.5, cy = 239.5) of a procedural scene (ground plane, far wall,
  20 boxes and spheres of 0.2-1.5 m at 0.5-8 m), with N(0, 5 mm) depth noise
  and 10 % pixel dropout, back-projected to ~276k camera-frame points.  It
  stands in for the Augmented ICL-NUIM ``livingroom1`` frame that the paper
  times SOGMM on (Sec. IV-A), which is not available here; only its image
  shape and intrinsics are reproduced.
"""
from __future__ import annotations

import dataclasses

import numpy as np

FX = FY = 525.0
CX, CY = 319.5, 239.5
WIDTH, HEIGHT = 640, 480


@dataclasses.dataclass
class GMMCloud:
    points: np.ndarray      # (N, 3) float32
    weights: np.ndarray     # (K,)   float64, generating weights
    means: np.ndarray       # (K, 3) float64
    covs: np.ndarray        # (K, 3, 3) float64
    labels: np.ndarray      # (N,)   int32 generating component of each point


def haar_rotation(rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal 3x3 matrix (QR of a Gaussian, sign-fixed)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.diag(r))[None, :]


def gmm_cloud(n: int = 20_000, k: int = 8, seed: int = 0, lam_lo: float = 1e-4, lam_hi: float = 1e-2,
              box: float = 2.0, shuffle: bool = True) -> GMMCloud:
    """Sample ``n`` points from a random K-component full-covariance GMM."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-box, box, size=(k, 3))
    covs = np.empty((k, 3, 3))
    factors = np.empty((k, 3, 3))
    for b in range(k):
        rot = haar_rotation(rng)
        lam = np.exp(rng.uniform(np.log(lam_lo), np.log(lam_hi), size=3))
        covs[b] = (rot * lam[None, :]) @ rot.T
        factors[b] = rot * np.sqrt(lam)[None, :]
    weights = rng.dirichlet(np.ones(k))
    counts = rng.multinomial(n, weights)
    pts = np.empty((n, 3))
    labels = np.empty(n, dtype=np.int32)
    at = 0
    for b in range(k):
        c = int(counts[b])
        z = rng.standard_normal((c, 3))
        pts[at:at + c] = means[b] + z @ factors[b].T
        labels[at:at + c] = b
        at += c
    if shuffle:
        perm = rng.permutation(n)
        pts, labels = pts[perm], labels[perm]
    return GMMCloud(pts.astype(np.float32), weights, means, covs, labels)


# --------------------------------------------------------------------------------------
# Procedural depth frame
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class DepthFrame:
    points: np.ndarray      # (N, 3) float32, camera frame (x right, y down, z forward), metres
    depth: np.ndarray       # (H, W) float32, 0 where dropped
    pitch_deg: float


def _rays_world(pitch: float):
    """Unit-free ray directions for every pixel, in a world frame with z up.

    Camera frame is OpenCV (x right, y down, z forward).  World: X right,
    Y forward (horizontal), Z up; the camera is pitched down by ``pitch``.
    Returns (dirs_world (H*W, 3), dirs_cam (H*W, 3)) with dirs_cam[:, 2] == 1.
    """
    u, v = np.meshgrid(np.arange(WIDTH, dtype=np.float64), np.arange(HEIGHT, dtype=np.float64))
    dc = np.stack([(u - CX) / FX, (v - CY) / FY, np.ones_like(u)], axis=-1).reshape(-1, 3)
    c, s = np.cos(pitch), np.sin(pitch)
    # camera axes expressed in world coordinates
    x_w = np.array([1.0, 0.0, 0.0])
    z_w = np.array([0.0, c, -s])            # forward, tilted down
    y_w = np.array([0.0, -s, -c])           # image-down axis
    rot = np.stack([x_w, y_w, z_w], axis=1)  # columns: camera axes in world
    return dc @ rot.T, dc, rot


def depth_frame(seed: int = 1, n_objects: int = 20, noise_sigma: float = 0.005, dropout: float = 0.1,
                wall_dist: float = 8.0, cam_height: float = 1.5, scan_seed: int | None = None) -> DepthFrame:
    """Ray-cast a procedural scene into a 640x480 depth image and back-project it.

    ``seed`` fixes the scene (camera pitch, objects) and, by default, the sensor
    noise and dropout; ``scan_seed`` draws the noise and dropout from a stream of
    their own instead, which gives another scan of the same scene."""
    rng = np.random.default_rng(seed)
    pitch = np.deg2rad(rng.uniform(20.0, 30.0))
    dw, dc, rot = _rays_world(pitch)
    origin = np.array([0.0, 0.0, cam_height])
    n_rays = dw.shape[0]
    t_best = np.full(n_rays, np.inf)

    def take(t):
        ok = (t > 1e-6) & (t < t_best)
        t_best[ok] = t[ok]

    # ground plane Z = 0
    with np.errstate(divide="ignore", invalid="ignore"):
        take(np.where(dw[:, 2] < 0, -origin[2] / dw[:, 2], np.inf))
        # far wall Y = wall_dist (tall enough to catch every upward ray)
        take(np.where(dw[:, 1] > 0, (wall_dist - origin[1]) / dw[:, 1], np.inf))
    half_fov = np.arctan(CX / FX)
    for _ in range(n_objects):
        size = rng.uniform(0.2, 1.5)
        dist = rng.uniform(0.5, wall_dist)
        lateral = rng.uniform(-1.0, 1.0) * np.tan(half_fov) * dist
        if rng.uniform() < 0.5:     # sphere resting on the ground
            r = 0.5 * size
            ctr = np.array([lateral, dist, r])
            oc = origin - ctr
            b = dw @ oc
            a = np.einsum("ij,ij->i", dw, dw)
            cc = oc @ oc - r * r
            disc = b * b - a * cc
            with np.errstate(invalid="ignore"):
                t = np.where(disc >= 0, (-b - np.sqrt(np.maximum(disc, 0))) / a, np.inf)
            take(t)
        else:                       # yawed box resting on the ground
            half = 0.5 * rng.uniform(0.2, 1.5, size=3)
            half[0] = 0.5 * size
            yaw = rng.uniform(0, np.pi)
            cy_, sy_ = np.cos(yaw), np.sin(yaw)
            rz = np.array([[cy_, -sy_, 0], [sy_, cy_, 0], [0, 0, 1.0]])
            ctr = np.array([lateral, dist, half[2]])
            o_l = rz.T @ (origin - ctr)
            d_l = dw @ rz             # (rz^T d) for every ray
            with np.errstate(divide="ignore", invalid="ignore"):
                t1 = (-half[None, :] - o_l[None, :]) / d_l
                t2 = (half[None, :] - o_l[None, :]) / d_l
            tmin = np.nanmax(np.minimum(t1, t2), axis=1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=1)
            take(np.where((tmax >= tmin) & (tmax > 0), tmin, np.inf))
    hit = np.isfinite(t_best)
    sensor = rng if scan_seed is None else np.random.default_rng(scan_seed)
    # depth along the optical axis: dirs_cam has z == 1, so z_cam == t
    z = np.where(hit, t_best, 0.0)
    z = z + sensor.normal(0.0, noise_sigma, size=n_rays) * hit
    keep = hit & (sensor.uniform(size=n_rays) >= dropout) & (z > 0)
    depth = np.where(keep, z, 0.0).reshape(HEIGHT, WIDTH).astype(np.float32)
    u, v = np.meshgrid(np.arange(WIDTH, dtype=np.float64), np.arange(HEIGHT, dtype=np.float64))
    zz = depth.astype(np.float64)
    m = zz > 0
    pts = np.stack([(u[m] - CX) * zz[m] / FX, (v[m] - CY) * zz[m] / FY, zz[m]], axis=1)
    n = pts.shape[0]
    if not 250_000 <= n <= 300_000:
        raise AssertionError(f"depth frame produced {n} points, outside [250k, 300k]")
    return DepthFrame(pts.astype(np.float32), depth, float(np.rad2deg(pitch)))


def gmm_cloud4(n: int = 20_000, k: int = 8, seed: int = 0, lam_lo: float = 1e-4, lam_hi: float = 1e-2,
               box: float = 2.0) -> GMMCloud:
    """xyz + intensity: ``n`` points from a random K-component full-covariance 4D GMM
    (means uniform in [-box, box]^3 x [0, 1], Haar-rotated covariances with
    eigenvalues log-uniform in [lam_lo, lam_hi], so intensity correlates with
    position inside each component)."""
    rng = np.random.default_rng(seed)
    means = np.concatenate([rng.uniform(-box, box, size=(k, 3)), rng.uniform(0, 1, size=(k, 1))], axis=1)
    covs = np.empty((k, 4, 4))
    factors = np.empty((k, 4, 4))
    for b in range(k):
        q, r = np.linalg.qr(rng.standard_normal((4, 4)))
        rot = q * np.sign(np.diag(r))[None, :]
        lam = np.exp(rng.uniform(np.log(lam_lo), np.log(lam_hi), size=4))
        covs[b] = (rot * lam[None, :]) @ rot.T
        factors[b] = rot * np.sqrt(lam)[None, :]
    weights = rng.dirichlet(np.ones(k))
    counts = rng.multinomial(n, weights)
    pts = np.empty((n, 4))
    labels = np.empty(n, dtype=np.int32)
    at = 0
    for b in range(k):
        c = int(counts[b])
        pts[at:at + c] = means[b] + rng.standard_normal((c, 4)) @ factors[b].T
        labels[at:at + c] = b
        at += c
    perm = rng.permutation(n)
    return GMMCloud(pts[perm].astype(np.float32), weights, means, covs, labels[perm])


def rigid_offset(rng: np.random.Generator, max_deg: float = 15.0, max_t: float = 0.5):
    """A random rigid motion: rotation about a uniformly random axis by an angle
    uniform in [0, max_deg] degrees, translation uniform in [-max_t, max_t]^3 m.
    Returns (R (3, 3), t (3,)) in binary64."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = np.deg2rad(rng.uniform(0.0, max_deg))
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * (K @ K)
    return R, rng.uniform(-max_t, max_t, size=3)


def registration_scan(seed: int = 1, scan_seed: int = 1001, n: int = 100_000, offset_seed: int = 3,
                      max_deg: float = 15.0, max_t: float = 0.5):
    """A second scan of the scene of ``depth_frame(seed)``: the same scene with its
    own sensor noise (5 mm) and dropout, ``n`` of its points at random, moved by a
    random rigid offset (``rigid_offset``).  Returns (scan (n, 3) float32, R, t):
    scan = R x + t for points x of the scene in the first scan's frame."""
    second = depth_frame(seed=seed, scan_seed=scan_seed).points.astype(np.float64)
    rng = np.random.default_rng(offset_seed)
    R, t = rigid_offset(rng, max_deg, max_t)
    sub = second[rng.choice(len(second), n, replace=False)]
    return (sub @ R.T + t).astype(np.float32), R, t


def frame_subsampled(frame: DepthFrame, step: int) -> np.ndarray:
    """The frame's points on every ``step``-th pixel row and column: the smaller image
    sizes the paper times (320x240 at step 2, 213x160 at step 3, 160x120 at step 4),
    back-projected with the full-size intrinsics (the same 3D points as those pixels)."""
    depth = frame.depth.astype(np.float64)
    v, u = np.meshgrid(np.arange(0, HEIGHT, step, dtype=np.float64), np.arange(0, WIDTH, step, dtype=np.float64),
                       indexing="ij")
    zz = depth[::step, ::step]
    m = zz > 0
    pts = np.stack([(u[m] - CX) * zz[m] / FX, (v[m] - CY) * zz[m] / FY, zz[m]], axis=1)
    return pts.astype(np.float32)


def frame_intensity(pts: np.ndarray, seed: int = 1, noise_sigma: float = 0.01) -> np.ndarray:
    """An intensity channel for a depth frame (the paper fits xyz + intensity): a smooth
    procedural texture of the 3D position plus N(0, noise_sigma), in [0, 1]."""
    rng = np.random.default_rng(seed + 7919)
    x, y, z = pts[:, 0].astype(np.float64), pts[:, 1].astype(np.float64), pts[:, 2].astype(np.float64)
    tex = 0.5 + 0.25 * np.sin(3.0 * x) * np.cos(2.0 * y) + 0.15 * np.sin(1.3 * z + 0.5 * x) - 0.02 * z
    return np.clip(tex + rng.normal(0.0, noise_sigma, size=len(pts)), 0.0, 1.0).astype(np.float32)


def depth_frame4(seed: int = 1) -> np.ndarray:
    """The depth frame's points with an intensity channel: N x 4 float32."""
    pts = depth_frame(seed=seed).points
    return np.concatenate([pts, frame_intensity(pts, seed)[:, None]], axis=1)


def uniform_cloud(n: int, seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """Plain uniform points in a cube (edge cases, ragged sizes)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(n, 3)).astype(np.float32)
