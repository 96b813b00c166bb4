"""Pins of the oracle's compositing (Supp. D.2 and reading R8): the closed-form
image of a single Gaussian, a two-Gaussian closed form, the transmittance
identity sum_j T_j alpha_j + T_final = 1, and brute-force unsorted
compositing in pure Python on tiny scenes."""
import math

import numpy as np

from paper_2606_30436_b300 import scenes

SH0 = 2.0 * math.sqrt(math.pi)  # colour c needs DC coefficient (c - 0.5) * 2 sqrt(pi)


def _scene(means, log_scales, logits, rgb, quats=None):
    n = len(means)
    return dict(means=np.array(means, np.float64), log_scales=np.array(log_scales, np.float64),
                quats=np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None else np.array(quats, np.float64),
                opacity_logits=np.array(logits, np.float64),
                sh=((np.array(rgb, np.float64) - 0.5) * SH0).reshape(n, 1, 3), sh_degree=0)


def test_single_gaussian_closed_form(orc):
    W, H, f = 64, 48, 60.0
    cam = scenes.pinhole(W, H, f)
    sx, sy, z, o, c = 0.08, 0.05, 3.0, 0.8, np.array([0.9, 0.4, 0.2])
    cfg = orc.Cfg(fp32_positions=False)
    p = _scene([(0, 0, z)], [(math.log(sx), math.log(sy), -3)], [math.log(o / (1 - o))], [c])
    f_ = orc.forward(p, cam, cfg)
    A, Cc = (f * sx / z) ** 2 + 0.3, (f * sy / z) ** 2 + 0.3
    lam = 0.5 * (A + Cc) + math.sqrt(max(0.1, (0.5 * (A - Cc)) ** 2))
    r = math.ceil(3 * math.sqrt(lam))
    tx0, tx1 = math.floor((32 - r) / 16), math.floor((32 + r) / 16) + 1
    ty0, ty1 = math.floor((24 - r) / 16), math.floor((24 + r) / 16) + 1
    for j in range(H):
        for i in range(W):
            dx, dy = i + 0.5 - W / 2, j + 0.5 - H / 2
            a = min(0.99, o * math.exp(-0.5 * (dx * dx / A + dy * dy / Cc)))
            inside = tx0 <= i // 16 < tx1 and ty0 <= j // 16 < ty1
            if a < 1 / 255 or not inside:
                a = 0.0
            assert np.allclose(f_["img"][:, j, i], c * a, atol=1e-14)
            assert abs(f_["T_final"][j, i] - (1 - a)) < 1e-14
            assert abs(f_["depth"][j, i] - z * a) < 1e-13


def test_two_gaussian_closed_form(orc):
    cam = scenes.pinhole(32, 32, 40.0)
    cfg = orc.Cfg(fp32_positions=False)
    c1, c2 = np.array([1.0, 0.2, 0.1]), np.array([0.1, 0.7, 0.9])
    p = _scene([(0.05, 0.0, 2.0), (-0.05, 0.02, 4.0)], [(-2.5, -2.5, -3), (-2.0, -2.2, -3)],
               [0.5, 1.5], [c1, c2])
    f_ = orc.forward(p, cam, cfg)
    pr = f_["proj"]
    for (i, j) in [(16, 16), (14, 15), (18, 17), (10, 20)]:
        a = []
        for g in range(2):
            dx, dy = i + 0.5 - pr["u"][g], j + 0.5 - pr["v"][g]
            q = pr["conic"][g]
            a.append(min(0.99, pr["opacity"][g] * math.exp(-0.5 * (q[0] * dx * dx + q[2] * dy * dy) - q[1] * dx * dy)))
        a = [x if x >= 1 / 255 else 0.0 for x in a]
        ref = c1 * a[0] + c2 * a[1] * (1 - a[0])  # Gaussian 0 is nearer
        assert np.allclose(f_["img"][:, j, i], ref, atol=1e-14)


def test_transmittance_identity(orc):
    """With every colour and the background equal to 1 the image is exactly
    sum_j T_j alpha_j + T_final = 1 at every pixel."""
    p = scenes.uniform_scene(2000, seed=11)
    p["sh"] = p["sh"].astype(np.float64)
    p["sh"][:, 0, :] = 0.5 * SH0  # colour 1
    cam = scenes.pinhole(96, 80, 100.0)
    cfg = orc.Cfg(bg=(1.0, 1.0, 1.0))
    f_ = orc.forward(p, cam, cfg)
    assert np.abs(f_["img"] - 1.0).max() < 1e-12
    assert f_["n_contrib"].max() > 5
    assert f_["T_final"].min() < 0.5


def _brute_force(pr, cam, cfg, W, H):
    """Per pixel: every Gaussian whose tile rectangle holds the pixel's tile,
    sorted by (depth, index), composited front to back under reading R8."""
    img = np.zeros((3, H, W))
    Tf = np.ones((H, W))
    nb = np.zeros((H, W), np.int64)
    n = pr.n
    for j in range(H):
        for i in range(W):
            tx, ty = i // cfg.tile_w, j // cfg.tile_h
            members = [g for g in range(n) if pr["radius"][g] > 0 and pr["rect"][g][0] <= tx < pr["rect"][g][2]
                       and pr["rect"][g][1] <= ty < pr["rect"][g][3]]
            members.sort(key=lambda g: (pr["z"][g], g))
            T, C = 1.0, np.zeros(3)
            for g in members:
                dx, dy = i + 0.5 - pr["u"][g], j + 0.5 - pr["v"][g]
                q = pr["conic"][g]
                power = -0.5 * (q[0] * dx * dx + q[2] * dy * dy) - q[1] * dx * dy
                if power > 0:
                    continue
                a = min(cfg.alpha_max, pr["opacity"][g] * math.exp(power))
                if a < cfg.alpha_min:
                    continue
                if T * (1 - a) < cfg.t_min:
                    break
                C += pr["rgb"][g] * a * T
                T *= 1 - a
                nb[j, i] += 1
            img[:, j, i] = C + T * np.array(cfg.bg)
            Tf[j, i] = T
    return img, Tf, nb


def test_brute_force_unsorted_compositing(orc):
    for seed, fp32 in [(21, False), (22, True)]:
        p = scenes.uniform_scene(50, seed=seed, xy_range=1.5)
        p["log_scales"] += 1.0  # larger footprints: many overlaps at 64x48
        cam = scenes.pinhole(64, 48, 60.0)
        cfg = orc.Cfg(fp32_positions=fp32, bg=(0.1, 0.2, 0.3))
        f_ = orc.forward(p, cam, cfg)
        img, Tf, nb = _brute_force(f_["proj"], cam, cfg, 64, 48)
        assert np.abs(f_["img"] - img).max() < 1e-12
        assert np.abs(f_["T_final"] - Tf).max() < 1e-12
        assert np.array_equal(f_["n_contrib"], nb)
        assert nb.max() >= 4


def test_early_termination(orc):
    """A stack of Gaussians whose alpha is clamped to 0.99 at the centre pixel:
    after two of them T = 1e-4 (plus rounding), the third would bring T below
    the cut, so compositing stops before it."""
    k = 4
    p = _scene([(0, 0, 2 + 0.1 * g) for g in range(k)], [(-0.5, -0.5, -3)] * k, [8.0] * k,
               [[g / k, 0.5, 1 - g / k] for g in range(k)])
    cam = scenes.pinhole(16, 16, 20.0)
    f_ = orc.forward(p, cam, orc.Cfg(fp32_positions=False))
    assert f_["T_final"].min() >= 1e-4
    assert f_["n_contrib"][8, 8] == 2
    assert abs(f_["T_final"][8, 8] - 1e-4) < 1e-15
