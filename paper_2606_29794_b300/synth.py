"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only: scenes of 3D Gaussians, camera views
and request streams. It contains none of the rasterizer's arithmetic, and both
the CUDA path and the FP64 oracle receive exactly the arrays it produces.

Scene recipe (per Gaussian): means uniform in the volume of the spherical shell
r in [r_min, r_max] around the origin; log-scales i.i.d. Normal(mu, sd) per
axis; rotations uniform unit quaternions (normalised 4-D Gaussians, (w,x,y,z));
opacity = sigmoid(Normal(0, 1)); colours either SH degree 0 with RGB uniform in
[0, 1] (stored as the DC coefficient (c - 0.5) / Y00) or SH degree 3 with all
48 coefficients Normal(0, 0.2). The paper trains on real captures (Sec. 5.1);
these scenes stand in for them with the same camera kinds, FoVs, HEALPix orders
and Gaussian counts.
"""
from __future__ import annotations

import math

import numpy as np

CAM_FULL, CAM_PINHOLE, CAM_FISHEYE = 0, 1, 2

_Y00 = 0.5 / math.sqrt(math.pi)   # value of the constant SH basis function


def make_scene(P: int, sh_degree: int = 0, seed: int = 0, r_min: float = 2.0, r_max: float = 6.0,
               logscale_mu: float = -2.5, logscale_sd: float = 0.5) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(P)
    rad = np.cbrt(r_min ** 3 + u * (r_max ** 3 - r_min ** 3))
    d = rng.standard_normal((P, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    means = d * rad[:, None]
    scales = np.exp(rng.normal(logscale_mu, logscale_sd, (P, 3)))
    q = rng.standard_normal((P, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = 1.0 / (1.0 + np.exp(-rng.standard_normal(P)))
    K = (sh_degree + 1) ** 2
    if sh_degree == 0:
        col = rng.random((P, 3))
        sh = ((col - 0.5) / _Y00).reshape(P, 1, 3)
    else:
        sh = rng.normal(0.0, 0.2, (P, K, 3))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(means=f32(means), scales=f32(scales), rotations=f32(q), opacities=f32(opac),
                sh=f32(sh), sh_degree=int(sh_degree))


def perturb_scene(scene: dict, seed: int) -> dict:
    """A perturbed copy (the target scene of the training-step workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = scene["means"].shape[0]
    means = scene["means"] + rng.normal(0, 0.02, (P, 3))
    scales = np.exp(np.log(scene["scales"]) + rng.normal(0, 0.1, (P, 3)))
    q = scene["rotations"] + rng.normal(0, 0.05, (P, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    o = np.clip(scene["opacities"].astype(np.float64), 1e-6, 1 - 1e-6)
    logit = np.log(o / (1 - o)) + rng.normal(0, 0.2, P)
    opac = 1.0 / (1.0 + np.exp(-logit))
    sh = scene["sh"] + rng.normal(0, 0.05, scene["sh"].shape)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return dict(means=f32(means), scales=f32(scales), rotations=f32(q), opacities=f32(opac),
                sh=f32(sh), sh_degree=scene["sh_degree"])


def random_rotation(rng) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def make_view(nside_log2: int, cam: int = CAM_FULL, fov_x: float = 360.0, fov_y: float | None = None,
              R: np.ndarray | None = None, position=(0.0, 0.0, 0.0), pp=(0.0, 0.0)) -> dict:
    """World-to-camera view V = [W | b] with W = R (rotation) and b = -R c (camera centre c).
    pp: a pinhole's principal point offset from the image centre, in half-image units
    (c_x = (W/2)(1 + pp[0]), c_y = (H/2)(1 + pp[1]))."""
    W = np.eye(3) if R is None else np.asarray(R, np.float64)
    c = np.asarray(position, np.float64)
    b = -W @ c
    return dict(W=np.ascontiguousarray(W, np.float32), b=np.ascontiguousarray(b, np.float32),
                nside_log2=int(nside_log2), cam=int(cam), fov_x=float(fov_x),
                fov_y=float(fov_x if fov_y is None else fov_y), pp=(float(pp[0]), float(pp[1])))


def random_pose_view(rng, nside_log2, cam, fov_x, fov_y=None, radius=1.0, pp=(0.0, 0.0)) -> dict:
    R = random_rotation(rng)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    pos = d * radius * np.cbrt(rng.random())
    return make_view(nside_log2, cam, fov_x, fov_y, R, pos, pp)


def multiview_set(seed: int) -> list:
    """16 views: 6 pinhole 90 deg at Nside 1024, 6 fisheye 180 deg at 512, 4 full at 256."""
    rng = np.random.Generator(np.random.PCG64(seed))
    views = []
    for _ in range(6):
        views.append(random_pose_view(rng, 10, CAM_PINHOLE, 90.0, 90.0))
    for _ in range(6):
        views.append(random_pose_view(rng, 9, CAM_FISHEYE, 180.0))
    for _ in range(4):
        views.append(random_pose_view(rng, 8, CAM_FULL, 360.0))
    return views


def request_stream(n: int, rate_hz: float, seed: int, nside_choices=(7, 8, 9, 10, 11)) -> list:
    """Poisson arrivals; each request picks Nside, camera kind, FoV and a random pose."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    reqs = []
    for i in range(n):
        k = int(rng.choice(nside_choices))
        kind = int(rng.integers(0, 3))
        if kind == CAM_PINHOLE:
            fov = float(rng.uniform(60.0, 100.0))
            v = random_pose_view(rng, k, CAM_PINHOLE, fov, fov)
        elif kind == CAM_FISHEYE:
            v = random_pose_view(rng, k, CAM_FISHEYE, float(rng.uniform(180.0, 220.0)))
        else:
            v = random_pose_view(rng, k, CAM_FULL, 360.0)
        reqs.append(dict(arrival=float(t[i]), view=v, id=i))
    return reqs
