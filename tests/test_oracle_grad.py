"""Pin of the oracle's analytic backward: central finite differences (h = 1e-6,
FP64) of the full chain parameters -> projection -> compositing -> loss on the
gradient-check scene (200 Gaussians, 64x48, fx = fy = 60), for every parameter
group.  Coordinates whose +-h evaluations cross a discrete decision (pair list,
blended set, early stop, radius, colour clamp) are excluded and counted."""
import numpy as np
import pytest

from paper_2606_30436_b300 import scenes

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _setup(sh_degree, seed):
    p = scenes.uniform_scene(200, seed=seed, sh_degree=sh_degree)
    p = {k: (np.asarray(v, np.float64) if k != "sh_degree" else v) for k, v in p.items()}
    R = scenes.random_rotation(seed + 10).astype(np.float64)
    # rotate the scene with the camera so the visible set is unchanged
    t = np.array([0.05, -0.03, 0.1])
    p["means"] = (p["means"] - t) @ R
    cam = scenes.pinhole(64, 48, 60.0)
    cam["R"], cam["t"] = R, t
    target = scenes.smooth_image(48, 64, seed=seed + 1).astype(np.float64)
    return p, cam, target


def _signature(f_):
    pr = f_["proj"]
    return (f_["vals"].tobytes(), f_["ranges"].tobytes(), f_["n_contrib"].tobytes(), f_["last_pos"].tobytes(),
            pr["radius"].tobytes(), pr["rect"].tobytes(), pr["rgb_clamped"].tobytes())


@pytest.mark.parametrize("sh_degree,seed", [(0, 40), (3, 41)])
def test_gradients_central_differences(orc, sh_degree, seed):
    p, cam, target = _setup(sh_degree, seed)
    cfg = orc.Cfg(fp32_positions=False)
    lam = 0.2
    ref = orc.loss_and_grads(p, cam, cfg, target, lam)
    assert ref["n_contrib"].max() >= 3
    rng = np.random.default_rng(seed)
    visible = np.nonzero(ref["proj"]["radius"] > 0)[0]
    chosen = rng.choice(visible, size=min(60, visible.size), replace=False)
    h = 1e-6
    excluded = 0
    for grp in GROUPS:
        fd, an = [], []
        for g in chosen:
            for idx in np.ndindex(p[grp][g].shape):
                full = (g,) + idx
                vals = []
                sigs = []
                for s in (+1, -1):
                    q = dict(p)
                    q[grp] = p[grp].copy()
                    q[grp][full] += s * h
                    f_ = orc.forward(q, cam, cfg)
                    vals.append(orc.loss(f_["img"], target, lam, grad=False)[0])
                    sigs.append(_signature(f_))
                if sigs[0] != sigs[1] or sigs[0] != _signature(ref):
                    excluded += 1
                    continue
                fd.append((vals[0] - vals[1]) / (2 * h))
                an.append(ref["grads"][grp][full])
        fd, an = np.array(fd), np.array(an)
        err = np.linalg.norm(fd - an) / np.linalg.norm(an)
        assert err < 1e-5, (grp, err)
    assert excluded < 20
