"""Host logic of the initialisation and anchor bindings (no GPU): the seeded
keyframe generator (determinism, the ground-plane depth, the sky, the missing
boxes of a render), the camera centre of a keyframe camera, the level bands
handed to the decoder, and the initialisation constants."""
import math

import numpy as np

from paper_2606_30436_b300 import anchors, scenes, spawn


def test_keyframe_is_seeded_and_shaped():
    a = scenes.keyframe(48, 80, seed=3)
    b = scenes.keyframe(48, 80, seed=3)
    for x, y in zip(a, b):
        assert x.dtype == np.float32 and np.array_equal(x, y)
    img, depth, U = a
    assert img.shape == (3, 48, 80) and depth.shape == (48, 80) and U.shape == (48, 80)
    assert img.min() >= 0.0 and img.max() <= 1.0 and U.min() >= 0.0 and U.max() < 1.0


def test_keyframe_ground_plane_and_sky():
    H, W = 90, 160
    img, depth, _ = scenes.keyframe(H, W, seed=4)
    f, horizon = 0.9 * W, 0.45 * H
    v = np.arange(H) + 0.5
    # only the sky (above the horizon, where no box stands in front of it) has no depth
    sky_rows = v < horizon
    assert (depth[sky_rows] == 0).any()
    assert np.all(depth[v > horizon + 1.0] > 0)
    # the bottom row is road unless a box covers it: depth 1.6 f / (v - horizon)
    ground = 1.6 * f / (v[-1] - horizon)
    bottom = depth[-1]
    assert np.isclose(np.median(bottom), ground, rtol=1e-5)


def test_render_misses_boxes():
    img, depth, U = scenes.keyframe(120, 200, seed=5)
    img_r, depth_r, U_r = scenes.keyframe(120, 200, seed=5, missing=0.5)
    assert np.array_equal(U, U_r)  # the same draws
    differ = np.abs(depth - depth_r) > 0
    assert 0.0 < differ.mean() < 0.5
    # where nothing is missing the two views agree exactly
    same = ~differ & (np.abs(img - img_r).max(axis=0) == 0)
    assert same.mean() > 0.5


def test_keyframe_camera_centre():
    cam = scenes.keyframe_camera(64, 96, seed=7, centre=(2.0, -1.6, 30.0))
    c = anchors.camera_centre(cam)
    assert np.allclose(c, [2.0, -1.6, 30.0], atol=1e-5)
    # the camera maps its centre to the origin of the camera frame
    R, t = np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64)
    assert np.allclose(R @ c + t, 0.0, atol=1e-5)


def test_bands_and_init_constants():
    md, n = anchors._bands(anchors.MAX_DIST_DEFAULT)
    assert n == 5 and list(md)[:4] == [10.0, 25.0, 100.0, 500.0] and math.isfinite(md[4]) and md[4] > 1e37
    cfg = spawn.init_config()
    assert (cfg.sigma1, cfg.lam, cfg.scale, cfg.levels) == (1.0, np.float32(0.9), 255.0, 5)
    assert list(cfg.voxel)[:5] == [np.float32(x) for x in (0.1, 0.25, 1.0, 5.0, 25.0)]
    assert math.isinf(cfg.max_dist[4])
    # voxel size and band of level l: the band's upper edge is 100 eps_l below the last level
    for l in range(4):
        assert np.isclose(anchors.MAX_DIST_DEFAULT[l], 100 * anchors.VOXEL_DEFAULT[l])
