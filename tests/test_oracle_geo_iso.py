"""Pins of the oracle's geometric and isotropic terms (Supp. D.4): closed
forms, the isotropic special case, and central finite differences; and of the
depth channel D^ = sum_j T_j alpha_j z_j with its backward."""
import math

import numpy as np

from paper_2606_30436_b300 import scenes


def test_iso_closed_form(orc):
    ls = np.log(np.array([[1.0, 2.0, 3.0], [0.5, 0.5, 0.5]]))
    L, g = orc.iso_loss(ls)
    # scales (1,2,3): mean 2, |-1| + 0 + |1| = 2; isotropic Gaussian: 0; mean over 2 Gaussians
    assert abs(L - 1.0) < 1e-15
    assert np.all(g[1] == 0)
    # d/dlog s_k of |s_k - m| summed: e = (-1, 0, 1), sum 0 -> e_k s_k / n
    assert np.allclose(g[0], np.array([-1.0, 0.0, 3.0]) / 2, atol=1e-15)


def test_iso_fd(orc):
    rng = np.random.default_rng(0)
    ls = rng.normal(-3, 0.5, (50, 3))
    L, g = orc.iso_loss(ls)
    h = 1e-7
    for i, k in [(0, 0), (3, 2), (17, 1), (49, 0)]:
        lp, lm = ls.copy(), ls.copy()
        lp[i, k] += h
        lm[i, k] -= h
        fd = (orc.iso_loss(lp, grad=False)[0] - orc.iso_loss(lm, grad=False)[0]) / (2 * h)
        assert abs(fd - g[i, k]) < 1e-7


def test_geo_closed_form_and_fd(orc):
    rng = np.random.default_rng(1)
    depth = rng.uniform(2, 20, (12, 15))
    prior = depth + rng.normal(0, 0.5, depth.shape)
    prior[0, :] = 0.0  # no prior on the first row
    L, g = orc.geo_loss(depth, prior)
    valid = prior > 0
    assert abs(L - np.abs(depth - prior)[valid].sum() / depth.size) < 1e-13
    assert np.all(g[~valid] == 0)
    assert np.array_equal(g[valid], np.sign(depth - prior)[valid] / depth.size)


def test_depth_channel_gradient_fd(orc):
    """Loss = sum w * D^ (depth only): the oracle backward with dL/dD^ = w
    against central differences of the forward (FP64, decision flips excluded)."""
    s = scenes.uniform_scene(60, seed=71, xy_range=1.5)
    s = {k: (np.asarray(v, np.float64) if k != "sh_degree" else v) for k, v in s.items()}
    cam = scenes.pinhole(48, 40, 50.0)
    cfg = orc.Cfg(fp32_positions=False)
    rng = np.random.default_rng(2)
    w = rng.standard_normal((40, 48))
    f = orc.forward(s, cam, cfg)
    g2, _, _ = orc.render_backward(f["proj"], f["vals"], f["ranges"], cam, cfg, np.zeros((3, 40, 48)),
                                   f["img"], f["img"], dL_ddepth=w)
    g = orc.project_backward(f["params"], cam, cfg, f["proj"], g2)

    def val(q):
        ff = orc.forward(q, cam, cfg)
        return float((ff["depth"] * w).sum()), ff["n_contrib"].tobytes() + ff["vals"].tobytes()

    h = 1e-6
    fd, an = [], []
    for grp, idx in [("means", (3, 2)), ("means", (10, 0)), ("log_scales", (5, 1)), ("opacity_logits", (7,)),
                     ("quats", (2, 1)), ("means", (20, 1))]:
        qp, qm = dict(s), dict(s)
        qp[grp], qm[grp] = s[grp].copy(), s[grp].copy()
        qp[grp][idx] += h
        qm[grp][idx] -= h
        (vp, sp), (vm, sm) = val(qp), val(qm)
        if sp != sm:
            continue
        fd.append((vp - vm) / (2 * h))
        an.append(g[grp][idx])
    fd, an = np.array(fd), np.array(an)
    assert len(fd) >= 4
    assert np.linalg.norm(fd - an) <= 1e-5 * np.linalg.norm(an)
