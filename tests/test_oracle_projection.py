"""Pins of the oracle's projection (readings R1-R7): rotation matrices, the
closed-form footprint of an axis-aligned Gaussian on the optical axis, the EWA
covariance against a finite-difference Jacobian of the perspective map, the
FP32 evaluation order, colours, tile rectangles and the pair order."""
import math

import numpy as np
import pytest

from paper_2606_30436_b300 import scenes


def _single(mean, log_scales, quat=(1, 0, 0, 0), logit=0.0, sh=None, D=0):
    K = (D + 1) ** 2
    if sh is None:
        sh = np.zeros((1, K, 3))
    return dict(means=np.array([mean], np.float64), log_scales=np.array([log_scales], np.float64),
                quats=np.array([quat], np.float64), opacity_logits=np.array([logit], np.float64),
                sh=np.asarray(sh, np.float64).reshape(1, K, 3), sh_degree=D)


def test_rotation_from_quaternion(orc):
    rng = np.random.default_rng(0)
    assert np.allclose(orc.quat_to_rot([1, 0, 0, 0]), np.eye(3), atol=0)
    for _ in range(20):
        axis = rng.standard_normal(3)
        axis /= np.linalg.norm(axis)
        th = rng.uniform(-math.pi, math.pi)
        s = rng.uniform(0.3, 3.0)  # unnormalised input
        q = s * np.array([math.cos(th / 2), *(math.sin(th / 2) * axis)])
        R = orc.quat_to_rot(q)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-14
        # Rodrigues: R v = v cos + (k x v) sin + k (k.v)(1 - cos)
        v = rng.standard_normal(3)
        ref = v * math.cos(th) + np.cross(axis, v) * math.sin(th) + axis * (axis @ v) * (1 - math.cos(th))
        assert np.abs(R @ v - ref).max() < 1e-13


def test_on_axis_closed_form(orc):
    W, H, f = 64, 48, 60.0
    cam = scenes.pinhole(W, H, f)
    for (sx, sy, z) in [(0.05, 0.02, 3.0), (0.2, 0.2, 5.0), (0.01, 0.3, 2.5)]:
        p = _single((0, 0, z), (math.log(sx), math.log(sy), math.log(0.1)))
        pr = orc.project(p, cam, orc.Cfg(fp32_positions=False))
        A = (f * sx / z) ** 2 + 0.3
        Cc = (f * sy / z) ** 2 + 0.3
        assert np.allclose(pr["cov2d"][0], [A, 0, Cc], rtol=1e-13, atol=1e-15)
        assert np.allclose(pr["conic"][0], [1 / A, 0, 1 / Cc], rtol=1e-13, atol=1e-15)
        lam = 0.5 * (A + Cc) + math.sqrt(max(0.1, (0.5 * (A - Cc)) ** 2))
        assert pr["radius"][0] == math.ceil(3 * math.sqrt(lam))
        assert pr["u"][0] == W / 2 and pr["v"][0] == H / 2 and pr["z"][0] == z


def _persp_jacobian_fd(p, fx, fy, h=1e-6):
    def proj(q):
        return np.array([fx * q[0] / q[2], fy * q[1] / q[2]])
    J = np.zeros((2, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        J[:, a] = (proj(p + e) - proj(p - e)) / (2 * h)
    return J


@pytest.mark.parametrize("clamped", [False, True])
def test_ewa_against_numeric_jacobian(orc, clamped):
    rng = np.random.default_rng(1 + clamped)
    W, H, f = 320, 240, 300.0
    Rc = scenes.random_rotation(5).astype(np.float64)
    t = np.array([0.3, -0.2, 1.0])
    cam = scenes.pinhole(W, H, f, R=Rc, t=t)
    cam["R"], cam["t"] = Rc, t
    lim = 1.3 * W / (2 * f)
    for _ in range(10):
        z = rng.uniform(2, 10)
        x = (rng.uniform(1.5, 3.0) if clamped else rng.uniform(-0.9, 0.9)) * lim * z
        y = rng.uniform(-0.5, 0.5) * z * H / (2 * f)
        mean = Rc.T @ (np.array([x, y, z]) - t)
        x, y, z = Rc @ mean + t  # Rc is float32-valued, so orthonormal only to ~1e-7
        ls = rng.normal(-2, 0.5, 3)
        q = rng.standard_normal(4)
        pr = orc.project(_single(mean, ls, q), cam, orc.Cfg(fp32_positions=False))
        Rq = orc.quat_to_rot(q)
        Sig = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
        pj = np.array([np.clip(x / z, -lim, lim) * z, y, z])  # Jacobian taken at the clamped point
        J = _persp_jacobian_fd(pj, f, f)
        S2 = J @ Rc @ Sig @ Rc.T @ J.T + 0.3 * np.eye(2)
        got = pr["cov2d"][0]
        ref = np.array([S2[0, 0], S2[0, 1], S2[1, 1]])
        assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max()
        assert abs(pr["u"][0] - (f * x / z + W / 2)) < 1e-9


def test_cull_near_plane(orc):
    cam = scenes.pinhole(64, 48, 60.0)
    for z, culled in [(0.1, True), (0.2, True), (0.21, False)]:
        pr = orc.project(_single((0, 0, z), (-3, -3, -3)), cam, orc.Cfg())
        assert (pr["radius"][0] == 0) == culled


def test_fp32_evaluation_order(orc):
    """u, v, z in the FP32 mode equal the same expression evaluated with numpy
    float32 scalars, left to right (so no compiler contraction crept in)."""
    p = scenes.uniform_scene(500, seed=4)
    R = scenes.random_rotation(7)
    cam = scenes.pinhole(320, 240, 300.0, R=R, t=np.array([0.1, 0.2, 0.3], np.float32))
    pr = orc.project(p, cam, orc.Cfg())
    f32 = np.float32
    Rf = cam["R"].astype(f32)
    tf = cam["t"].astype(f32)
    m = p["means"].astype(f32)
    with np.errstate(all="ignore"):
        xc = Rf[0, 0] * m[:, 0] + Rf[0, 1] * m[:, 1] + Rf[0, 2] * m[:, 2] + tf[0]
        yc = Rf[1, 0] * m[:, 0] + Rf[1, 1] * m[:, 1] + Rf[1, 2] * m[:, 2] + tf[1]
        zc = Rf[2, 0] * m[:, 0] + Rf[2, 1] * m[:, 1] + Rf[2, 2] * m[:, 2] + tf[2]
        u = (f32(cam["fx"]) * xc) / zc + f32(cam["cx"])
        v = (f32(cam["fy"]) * yc) / zc + f32(cam["cy"])
    assert np.array_equal(pr["z32"], zc)
    assert np.array_equal(pr["u32"], u)
    assert np.array_equal(pr["v32"], v)


def test_colour_and_opacity(orc):
    rng = np.random.default_rng(3)
    cam = scenes.pinhole(64, 48, 60.0, R=scenes.random_rotation(2), t=np.array([0.0, 0.0, 0.5], np.float32))
    cam["R"] = cam["R"].astype(np.float64)
    centre = -cam["R"].T @ cam["t"]
    for D in (0, 1, 3):
        K = (D + 1) ** 2
        for _ in range(5):
            pc = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(2, 5)])
            mean = cam["R"].T @ (pc - cam["t"])
            sh = rng.normal(0, 0.5, (K, 3))
            logit = rng.normal()
            pr = orc.project(_single(mean, (-3, -3, -3), sh=sh, logit=logit, D=D), cam, orc.Cfg(fp32_positions=False))
            d = (mean - centre) / np.linalg.norm(mean - centre)
            Y, _ = orc.sh_eval(D, d)
            raw = 0.5 + Y @ sh
            assert np.allclose(pr["rgb"][0], np.maximum(raw, 0), atol=1e-14)
            assert abs(pr["opacity"][0] - 1 / (1 + math.exp(-logit))) < 1e-15


def test_tile_rect_and_pairs_brute_force(orc):
    """Tile rectangles equal the tiles whose pixel span meets [u-r, u+r] x
    [v-r, v+r]; the pair list equals an enumeration sorted by (tile, depth, id)."""
    p = scenes.uniform_scene(300, seed=5)
    cam = scenes.pinhole(100, 70, 90.0)  # ragged grid: 7 x 5 tiles of 16
    cfg = orc.Cfg()
    pr = orc.project(p, cam, cfg)
    GW, GH = orc.grid(cam, cfg)
    pairs = []
    for i in range(pr.n):
        r = int(pr["radius"][i])
        if r == 0:
            continue
        u, v = float(pr["u32"][i]), float(pr["v32"][i])
        tiles = [(tx, ty) for ty in range(GH) for tx in range(GW)
                 if tx * 16 <= u + r and (tx + 1) * 16 > u - r and ty * 16 <= v + r and (ty + 1) * 16 > v - r]
        xs = sorted({a for a, _ in tiles})
        ys = sorted({b for _, b in tiles})
        rect = pr["rect"][i]
        if tiles:
            assert (rect[0], rect[1], rect[2], rect[3]) == (xs[0], ys[0], xs[-1] + 1, ys[-1] + 1)
        for tx, ty in tiles:
            pairs.append((ty * GW + tx, float(pr["z32"][i]), i))
    pairs.sort()
    keys, vals, ranges = orc.bin_pairs(pr, cam, cfg)
    assert list(vals) == [g for _, _, g in pairs]
    zb = np.array([z for _, z, _ in pairs], np.float32).view(np.uint32).astype(np.uint64)
    assert np.array_equal(keys, (np.array([t for t, _, _ in pairs], np.uint64) << np.uint64(32)) | zb)
    for t in range(GW * GH):
        idx = [k for k, (tt, _, _) in enumerate(pairs) if tt == t]
        if idx:
            assert tuple(ranges[t]) == (idx[0], idx[-1] + 1)
        else:
            assert ranges[t][0] == ranges[t][1]
