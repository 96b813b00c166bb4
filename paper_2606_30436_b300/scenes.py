"""Seeded synthetic inputs for the Gaussian-splatting mapping step.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic, so the oracle-based tests and the CUDA path can share it.
Every generator takes an explicit seed (numpy ``default_rng``) and returns
float32 arrays, so the same values feed both sides exactly.

Parameter dictionaries (array-of-structures, as generated):
    means (n,3), log_scales (n,3), quats (n,4) as (w,x,y,z), opacity_logits (n,),
    sh (n,(D+1)^2,3) coefficient-major with RGB last, sh_degree D.
Cameras map world to camera coordinates (x right, y down, z forward):
    R (3,3), t (3,), fx, fy, cx, cy, width, height.

Workloads (the paper evaluates on outdoor driving sequences; these synthetic
scenes stand in for them):
    * ``uniform_scene``: camera-frame means with x, y ~ U[-5,5], depth ~ U[2,20],
      log-scales ~ N(-3, 0.5), random unit quaternions, opacity logits ~ N(0,1),
      degree-0 colour coefficients uniform on [-sqrt(pi), sqrt(pi)] (colours
      uniform on [0,1]); used for the 10k-Gaussian 320x240 single view, the 200
      Gaussian 64x48 gradient check and the multi-million batched chunk;
    * ``corridor_scene``: Gaussians strewn along a 1 km x 20 m road corridor,
      lateral offset exponential (scale 4 m, truncated at 10 m), 70% on the
      ground plane, SH degree 3 with coefficients ~ N(0, 0.1);
    * ``corridor_camera``: forward-moving camera 1.6 m above the road, 1 m per
      frame, 1280x720, fx = fy = 900.
"""
from __future__ import annotations

import math

import numpy as np


def _quats(rng, n):
    q = rng.standard_normal((n, 4)).astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def uniform_scene(n, seed=0, sh_degree=0, xy_range=5.0, z_range=(2.0, 20.0)):
    rng = np.random.default_rng(seed)
    K = (sh_degree + 1) ** 2
    means = np.empty((n, 3), np.float32)
    means[:, 0] = rng.uniform(-xy_range, xy_range, n)
    means[:, 1] = rng.uniform(-xy_range, xy_range, n)
    means[:, 2] = rng.uniform(z_range[0], z_range[1], n)
    log_scales = rng.normal(-3.0, 0.5, (n, 3)).astype(np.float32)
    quats = _quats(rng, n)
    opacity_logits = rng.standard_normal(n).astype(np.float32)
    sh = np.zeros((n, K, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, K - 1, 3))
    return dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits,
                sh=sh, sh_degree=sh_degree)


def corridor_scene(n, seed=0, length=1000.0, half_width=10.0, lateral_scale=4.0,
                   ground_fraction=0.7, max_height=8.0, sh_degree=3):
    rng = np.random.default_rng(seed)
    K = (sh_degree + 1) ** 2
    means = np.empty((n, 3), np.float32)
    # lateral |x| ~ Exponential(scale) truncated at half_width (resampled), random sign
    lat = rng.exponential(lateral_scale, n)
    bad = lat > half_width
    while bad.any():
        lat[bad] = rng.exponential(lateral_scale, int(bad.sum()))
        bad = lat > half_width
    means[:, 0] = lat * rng.choice([-1.0, 1.0], n)
    ground = rng.uniform(0.0, 1.0, n) < ground_fraction
    # y points down: the road surface is y = 0, elevated structure has y < 0
    means[:, 1] = np.where(ground, rng.normal(0.0, 0.05, n), -rng.uniform(0.0, max_height, n))
    means[:, 2] = rng.uniform(0.0, length, n)
    log_scales = rng.normal(-3.0, 0.5, (n, 3)).astype(np.float32)
    quats = _quats(rng, n)
    opacity_logits = rng.standard_normal(n).astype(np.float32)
    sh = rng.normal(0.0, 0.1, (n, K, 3)).astype(np.float32)
    return dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits,
                sh=sh, sh_degree=sh_degree)


def pinhole(width, height, fx, fy=None, cx=None, cy=None, R=None, t=None):
    fy = fx if fy is None else fy
    return dict(R=np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
                t=np.zeros(3, np.float32) if t is None else np.asarray(t, np.float32),
                fx=float(np.float32(fx)), fy=float(np.float32(fy)),
                cx=float(np.float32(width / 2 if cx is None else cx)),
                cy=float(np.float32(height / 2 if cy is None else cy)),
                width=int(width), height=int(height))


def yaw_matrix(deg):
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    # rotation about the camera's vertical (y) axis
    return np.array([[c, 0.0, -s], [0.0, 1.0, 0.0], [s, 0.0, c]], np.float32)


def world_to_camera(R_wc, centre):
    """t = -R c for a camera with world->camera rotation R at world position c."""
    R = np.asarray(R_wc, np.float64)
    t = -(R @ np.asarray(centre, np.float64))
    return np.asarray(R, np.float32), t.astype(np.float32)


def corridor_camera(frame, width=1280, height=720, f=900.0, height_above_road=1.6, yaw_deg=0.0):
    R, t = world_to_camera(yaw_matrix(yaw_deg), (0.0, -height_above_road, float(frame)))
    return pinhole(width, height, f, R=R, t=t)


CHUNK_RESOLUTIONS = ((640, 360), (960, 540), (1280, 720), (1600, 900))


def chunk_cameras(n_views, seed=2, resolutions=CHUNK_RESOLUTIONS):
    """Keyframes of a chunk: positions z ~ U[-2, 0], yaw ~ U[-5, 5] degrees,
    resolutions cycling through ``resolutions``, fx = fy = 0.9375 W."""
    rng = np.random.default_rng(seed)
    cams = []
    for k in range(n_views):
        W, H = resolutions[k % len(resolutions)]
        R, t = world_to_camera(yaw_matrix(rng.uniform(-5.0, 5.0)), (0.0, 0.0, rng.uniform(-2.0, 0.0)))
        cams.append(pinhole(W, H, 0.9375 * W, R=R, t=t))
    return cams


def random_rotation(seed):
    """A random proper rotation (QR of a Gaussian matrix, sign-fixed)."""
    rng = np.random.default_rng(seed)
    Q, Rr = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(Rr))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q.astype(np.float32)


def perturb(params, sigma=0.01, seed=1):
    """Adds N(0, sigma) to every parameter entry (a target scene near the map)."""
    rng = np.random.default_rng(seed)
    out = dict(params)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        a = np.asarray(params[k], np.float32)
        out[k] = (a + rng.normal(0.0, sigma, a.shape)).astype(np.float32)
    return out


def degraded_map(scene, remove=0.3, floaters=0.2, sigma=0.01, seed=2, length=1000.0, half_width=10.0,
                 max_height=8.0):
    """An initial map for the lifecycle workload: a random `remove` fraction of
    the scene dropped, `floaters` x n random Gaussians added uniformly in the
    corridor box (log-scales N(-3, 0.5), opacity logits N(0, 1), SH N(0, 0.1)),
    and every entry perturbed by N(0, sigma)."""
    rng = np.random.default_rng(seed)
    n = len(scene["means"])
    keep = rng.random(n) >= remove
    nf = int(round(floaters * n))
    K = (int(scene["sh_degree"]) + 1) ** 2
    fl = dict(means=np.stack([rng.uniform(-half_width, half_width, nf), -rng.uniform(0.0, max_height, nf),
                              rng.uniform(0.0, length, nf)], axis=1).astype(np.float32),
              log_scales=rng.normal(-3.0, 0.5, (nf, 3)).astype(np.float32), quats=_quats(rng, nf),
              opacity_logits=rng.standard_normal(nf).astype(np.float32),
              sh=rng.normal(0.0, 0.1, (nf, K, 3)).astype(np.float32))
    out = dict(scene)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        out[k] = np.concatenate([np.asarray(scene[k])[keep], fl[k]], axis=0)
    return perturb(out, sigma, seed=seed + 1)


def smooth_image(height, width, seed=3, channels=3):
    """A seeded image in [0,1]: a few random low-frequency waves plus fine noise."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    img = np.zeros((channels, height, width))
    for c in range(channels):
        for _ in range(4):
            fx, fy = rng.uniform(0.0, 0.1, 2)
            ph = rng.uniform(0, 2 * math.pi)
            img[c] += np.sin(fx * xx + fy * yy + ph)
        img[c] = 0.5 + 0.12 * img[c] + rng.normal(0.0, 0.05, (height, width))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def keyframe(height, width, seed=4, missing=0.0):
    """A synthetic driving keyframe for the anchor initialisation: image
    [3][H][W] in [0, 1] and metric depth [H][W] (0 marks the sky above the
    horizon).  The ground is a plane 1.6 m below a camera with fx = fy = 0.9 W
    (depth = 1.6 fy / (v - horizon)); axis-aligned boxes (facades, vehicles) at
    random depths have sharp colour and depth edges and some carry a fine
    checker texture; the sky is a smooth gradient.  With missing > 0 that
    fraction of the boxes is left out, as a render of an incomplete map would
    show it.  Also returns uniform [H][W] draws.  float32 throughout."""
    rng = np.random.default_rng(seed)
    H, W = int(height), int(width)
    f = 0.9 * W
    horizon = 0.45 * H
    v = np.arange(H, dtype=np.float64)[:, None] + 0.5
    u = np.arange(W, dtype=np.float64)[None, :] + 0.5
    ground = v > horizon + 1.0
    depth = np.where(ground, 1.6 * f / np.maximum(v - horizon, 1e-6), 0.0) * np.ones((1, W))
    depth = np.minimum(depth, 400.0)
    base = rng.uniform(0.25, 0.6, 3)
    img = np.empty((3, H, W))
    for c in range(3):
        sky = 0.55 + 0.35 * (1.0 - v / horizon) * (c == 2) + 0.05 * np.sin(u / W * 3.0 + c)
        road = base[c] + 0.05 * np.sin(u / 37.0 + v / 11.0 + c)
        img[c] = np.where(ground, road, sky)
    n_box = 24
    keep = rng.random(n_box) >= missing
    for b in range(n_box):
        d = float(np.exp(rng.uniform(np.log(4.0), np.log(150.0))))
        wpx = rng.uniform(0.5, 6.0) * f / d
        hpx = rng.uniform(0.8, 8.0) * f / d
        x0 = rng.uniform(-0.1 * W, 1.05 * W)
        foot = horizon + 1.6 * f / d  # the box stands on the ground at depth d
        colour = rng.uniform(0.05, 0.95, 3)
        checker = rng.random() < 0.4
        period = rng.integers(2, 6)
        if not keep[b]:
            continue
        m = (u >= x0) & (u < x0 + wpx) & (v >= foot - hpx) & (v < foot) & ((depth == 0.0) | (depth > d))
        if not m.any():
            continue
        depth = np.where(m, d, depth)
        for c in range(3):
            tex = colour[c]
            if checker:
                tex = tex + 0.15 * (((np.floor(u / period) + np.floor(v / period)) % 2) - 0.5)
            img[c] = np.where(m, tex, img[c])
    img = np.clip(img + rng.normal(0.0, 0.01, img.shape), 0.0, 1.0)
    uniform = rng.random((H, W))
    return img.astype(np.float32), depth.astype(np.float32), uniform.astype(np.float32)


def keyframe_camera(height, width, seed=5, centre=(0.0, 0.0, 0.0), yaw_deg=0.0):
    """Pinhole of keyframe(): fx = fy = 0.9 W, principal point at the centre."""
    rng = np.random.default_rng(seed)
    R_wc = yaw_matrix(yaw_deg + rng.uniform(-2.0, 2.0))
    R, t = world_to_camera(R_wc, np.asarray(centre, np.float64))
    return pinhole(int(width), int(height), 0.9 * width, R=R, t=t)
