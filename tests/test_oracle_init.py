"""Pins of the oracle's probabilistic initialisation (Sec. 3.3.1, Supp. D.5;
readings R19-R24): the DoG against scipy's Gaussian filter (separable,
replicated borders), closed forms of the depth gradient of a quadratic bowl,
the probability map's special cases, the 3x3 selection against a pure-Python
brute force on tiny inputs, and the unprojection / voxel rule against a
projection round trip and the voxel bounds."""
import math

import numpy as np
import pytest
from scipy.ndimage import gaussian_filter
from scipy.spatial.transform import Rotation

import oracle as orc


def _scipy_blur(Y, s):
    r = math.ceil(3.0 * s)
    return gaussian_filter(Y, s, mode="nearest", truncate=r / s)


@pytest.mark.parametrize("s1,s2,scale", [(1.0, 1.6, 1.0), (2.3, 0.7, 30.0), (1.0, 1.6, 255.0)])
def test_dog_matches_scipy(s1, s2, scale):
    rng = np.random.default_rng(3)
    img = 0.2 * rng.random((3, 37, 53))
    img[1] *= 0.5  # channels differ, so a wrong channel weighting shows
    depth = np.ones((37, 53))
    dog, grad = orc.init_saliency(img, depth, s1, s2, scale)
    Y = img.mean(axis=0)
    ref = np.minimum(scale * np.abs(_scipy_blur(Y, s1) - _scipy_blur(Y, s2)), 1.0)
    assert np.abs(dog - ref).max() < 1e-12
    if scale > 1:
        assert (dog == 1.0).any() and (dog < 1.0).any()  # the clamp is exercised
    else:
        assert dog.max() < 0.1
    assert np.array_equal(grad, np.zeros_like(grad))


def test_dog_constant_and_linear_images():
    H, W = 30, 40
    dog, _ = orc.init_saliency(np.full((3, H, W), 0.37), np.ones((H, W)))
    assert np.abs(dog).max() < 1e-12
    # a symmetric normalised kernel reproduces a linear ramp away from the borders
    x = np.arange(W)[None, :] * 0.01 + np.arange(H)[:, None] * 0.003
    dog, _ = orc.init_saliency(np.stack([x, x, x]), np.ones((H, W)))
    r = math.ceil(3 * 1.6)
    assert np.abs(dog[r:H - r, r:W - r]).max() < 1e-12
    assert dog[:, 0].max() > 1e-4  # the replicated border bends the ramp


def test_depth_gradient_of_a_bowl():
    H, W, a = 12, 17, 0.25
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    depth = a * (xx ** 2 + yy ** 2) + 3.0
    _, g = orc.init_saliency(np.zeros((3, H, W)), depth)
    # central differences of a quadratic are exact: grad = 2 a (x, y)
    ref = 2 * a * np.hypot(xx, yy)
    assert np.abs(g[1:-1, 1:-1] - ref[1:-1, 1:-1]).max() < 1e-12
    # replicated borders: one-sided halves
    gx0, gy0 = a / 2.0, 2 * a * yy[1:-1, 0]
    assert np.allclose(g[1:-1, 0], np.hypot(gx0, gy0), atol=1e-12)
    gxw = a * ((W - 1) ** 2 - (W - 2) ** 2) / 2.0
    assert np.allclose(g[1:-1, W - 1], np.hypot(gxw, 2 * a * yy[1:-1, 0]), atol=1e-12)


def test_probability_special_cases():
    H, W, a, lam = 20, 28, 0.1, 0.9
    cfg = orc.InitCfg(lam=lam)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    bowl = a * (xx ** 2 + yy ** 2) + 2.0
    flat_img = np.full((3, H, W), 0.5)
    # texture-free keyframe: P = (1 - lambda) minmax(||grad D||)
    _, g = orc.init_saliency(flat_img, bowl)
    P = orc.init_probability(flat_img, bowl, cfg=cfg)
    assert np.allclose(P, (1 - lam) * (g - g.min()) / (g.max() - g.min()), atol=1e-12)
    assert abs(P.max() - (1 - lam)) < 1e-12 and P.min() < 1e-12
    # flat depth: the normalised gradient is 0, P = min(lambda DoG, 1)
    rng = np.random.default_rng(8)
    img = 0.3 * rng.random((3, H, W))
    Y = img.mean(axis=0)
    dog = np.minimum(255.0 * np.abs(_scipy_blur(Y, 1.0) - _scipy_blur(Y, 1.6)), 1.0)
    assert (dog == 1.0).any() and (dog < 1.0).any()
    P = orc.init_probability(img, np.full((H, W), 5.0), cfg=cfg)
    assert np.abs(P - np.minimum(lam * dog, 1.0)).max() < 1e-12
    # residual against itself is 0; against a blank render it is P
    assert np.array_equal(orc.init_probability(img, bowl, img, bowl, cfg), np.zeros((H, W)))
    P = orc.init_probability(img, bowl, cfg=cfg)
    Pk = orc.init_probability(img, bowl, flat_img, np.full((H, W), 5.0), cfg)
    assert np.abs(Pk - P).max() < 1e-12  # a blank render: P^ = lambda DoG of a constant = 0 up to rounding
    # the clamp at 1
    Pc = orc.init_probability(img, 40.0 * bowl, cfg=orc.InitCfg(lam=lam, scale=2550.0))
    assert Pc.max() == 1.0 and (Pc < 1.0).any()


def _camera(seed, H, W):
    rng = np.random.default_rng(seed)
    R = Rotation.from_rotvec(rng.normal(0, 0.3, 3)).as_matrix()
    t = rng.normal(0, 2.0, 3)
    return dict(R=R, t=t, fx=0.9 * W, fy=0.9 * W, cx=W / 2 + 0.3, cy=H / 2 - 0.2, width=W, height=H)


def _brute_select(prob, U, depth, near):
    """Pure-Python NMS: (value, -raster index) maximum of the 3x3 window, P > 0, U < P, depth > near."""
    H, W = prob.shape
    out = []
    for y in range(H):
        for x in range(W):
            p = prob[y, x]
            ok = p > 0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    yy, xx = y + dy, x + dx
                    if (dy, dx) == (0, 0) or not (0 <= yy < H and 0 <= xx < W):
                        continue
                    q = prob[yy, xx]
                    if q > p or (q == p and yy * W + xx < y * W + x):
                        ok = False
            if ok and U[y, x] < p and depth[y, x] > near:
                out.append((y, x))
    return out


def _project(cam, xw):
    xc = cam["R"] @ xw + cam["t"]
    return cam["fx"] * xc[0] / xc[2] + cam["cx"], cam["fy"] * xc[1] / xc[2] + cam["cy"], xc


def test_select_brute_force_and_round_trip():
    H, W = 9, 11
    rng = np.random.default_rng(4)
    prob = rng.choice([0.0, 0.2, 0.5, 0.7, 0.7001], size=(H, W)).astype(np.float64)
    prob[2:4, 3:6] = 0.9  # a plateau: only its first pixel in raster order survives
    U = rng.random((H, W)) * 0.8
    depth = rng.uniform(0.1, 40.0, (H, W))
    cam = _camera(1, H, W)
    cfg = orc.InitCfg(near_z=0.2, max_dist=(10.0, 25.0, 100.0, 500.0, float("inf")))
    r = orc.init_select(prob, U, depth, cam, cfg)
    sel = _brute_select(prob, U, depth, cfg.near_z)
    # the plateau keeps at most its first pixel
    assert not any(2 <= y < 4 and 3 <= x < 6 and (y, x) != (2, 3) for y, x in sel)
    assert sorted(zip(*np.nonzero(r["selected"]))) == sorted(sel)
    # every anchor: its pixel projects back, its voxel holds the point, its band holds the distance
    seen = {}
    for y, x in sel:  # first pixel per voxel in raster order
        d = depth[y, x]
        # the point the oracle unprojected must project to the pixel centre at depth d
        xc = np.array([(x + 0.5 - cam["cx"]) / cam["fx"] * d, (y + 0.5 - cam["cy"]) / cam["fy"] * d, d])
        xw = cam["R"].T @ (xc - cam["t"])
        u, v, xc2 = _project(cam, xw)
        assert abs(u - (x + 0.5)) < 1e-9 and abs(v - (y + 0.5)) < 1e-9 and abs(xc2[2] - d) < 1e-9
        l = next(k for k, m in enumerate(cfg.max_dist) if np.linalg.norm(xc) < m)
        key = (l, *np.floor(xw / cfg.voxel[l]).astype(np.int64))
        seen.setdefault(key, y * W + x)
    assert r["n_new"] == len(seen)
    assert [tuple(k) for k in r["keys"]] == list(seen.keys())
    assert list(r["pixel"]) == list(seen.values())
    assert np.all(np.diff(r["pixel"]) > 0)
    for k, p, l in zip(r["keys"], r["pos"], r["level"]):
        e = cfg.voxel[k[0]]
        assert k[0] == l and np.allclose(p, np.array(k[1:]) * e, rtol=0, atol=1e-12)


def test_select_old_keys_cap_and_levels():
    H, W = 40, 50
    rng = np.random.default_rng(6)
    prob = rng.random((H, W))
    U = np.zeros((H, W))  # every local maximum is drawn
    depth = np.exp(rng.uniform(np.log(0.5), np.log(800.0), (H, W)))
    cam = _camera(2, H, W)
    cfg = orc.InitCfg()
    full = orc.init_select(prob, U, depth, cam, cfg)
    assert full["n_new"] > 20
    assert set(full["level"]) == set(range(5))  # distances span every band
    # voxels already occupied are not spawned again
    again = orc.init_select(prob, U, depth, cam, cfg, old_keys=full["keys"])
    assert again["n_new"] == 0 and again["selected"].sum() == full["selected"].sum()
    # a capacity keeps the prefix and still counts every new voxel
    part = orc.init_select(prob, U, depth, cam, cfg, cap=7)
    assert part["n_new"] == full["n_new"]
    assert np.array_equal(part["keys"], full["keys"][:7]) and np.array_equal(part["pixel"], full["pixel"][:7])
    # a point beyond the last band is never inserted
    short = orc.InitCfg(max_dist=(10.0, 25.0, 100.0, 500.0, 600.0))
    cut = orc.init_select(prob, U, depth, cam, short)
    far = depth * np.sqrt(1 + ((np.arange(W)[None, :] + 0.5 - cam["cx"]) / cam["fx"]) ** 2 +
                          ((np.arange(H)[:, None] + 0.5 - cam["cy"]) / cam["fy"]) ** 2) >= 600.0
    assert not (cut["selected"].astype(bool) & far).any()
    assert (full["selected"].astype(bool) & far).any()


def test_uncertain_flags_mark_near_ties():
    H, W = 5, 5
    prob = np.full((H, W), 0.1)
    prob[2, 2] = 0.6
    U = np.zeros((H, W))
    U[2, 2] = 0.6 - 3e-6  # within tol of the draw threshold
    depth = np.full((H, W), 5.0)
    cam = dict(R=np.eye(3), t=np.zeros(3), fx=10.0, fy=10.0, cx=2.3, cy=2.4, width=W, height=H)
    r = orc.init_select(prob, U, depth, cam, orc.InitCfg(), tol=1e-5)
    assert r["selected"][2, 2] == 1 and r["uncertain"][2, 2] == 1
    # the centre pixel at depth 5 sits at x_w = (0.1, 0.05, 5): 5 / 0.25 = 20 is a voxel boundary
    U[2, 2] = 0.0
    r = orc.init_select(prob, U, depth, cam, orc.InitCfg(voxel=(0.25, 1.0, 1.0, 5.0, 25.0)), tol=1e-5)
    assert r["uncertain"][2, 2] == 1
    r = orc.init_select(prob, U, depth + 0.1, cam, orc.InitCfg(voxel=(0.25, 1.0, 1.0, 5.0, 25.0)), tol=1e-5)
    assert r["uncertain"][2, 2] == 0 and r["selected"][2, 2] == 1
