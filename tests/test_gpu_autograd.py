"""The autograd.Function (recompute-in-backward) against the FP64 oracle
gradient and against central finite differences of the FP64 oracle forward."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2606_30436_b300 import gs, scenes
from paper_2606_30436_b300.autograd import rasterize

from _parity import GROUPS, ocfg, rel_l2

pytestmark = pytest.mark.gpu


def _scene():
    s = scenes.uniform_scene(200, seed=60, sh_degree=2)
    cams = [scenes.pinhole(64, 48, 60.0), scenes.pinhole(48, 40, 50.0, t=np.array([0.1, 0.0, 0.2], np.float32))]
    return s, cams


def test_autograd_matches_oracle_gradient():
    s, cams = _scene()
    cfg = gs.Config()
    model = gs.GaussianModel.from_scene(s)
    params = model.data.clone().requires_grad_(True)
    img = rasterize(params, model.n, model.sh_degree, cams, cfg)
    rng = np.random.default_rng(0)
    Wt = torch.from_numpy(rng.standard_normal(img.numel()).astype(np.float32)).cuda()
    (img * Wt).sum().backward()
    g = gs.unpack_planes(params.grad.cpu().numpy(), model.n, model.sh_degree)
    oc = ocfg(cfg)
    ref = {k: 0.0 for k in GROUPS}
    off = 0
    for cam in cams:
        H, W = cam["height"], cam["width"]
        wv = Wt[off:off + 3 * H * W].cpu().numpy().reshape(3, H, W).astype(np.float64)
        off += 3 * H * W
        f = orc.forward(s, cam, oc)
        g2, _, _ = orc.render_backward(f["proj"], f["vals"], f["ranges"], cam, oc, wv, f["img"], f["img"])
        go = orc.project_backward(f["params"], cam, oc, f["proj"], g2)
        for k in GROUPS:
            ref[k] = ref[k] + go[k]
    for k in GROUPS:
        assert rel_l2(g[k], ref[k]) < 1e-3, k


def _entry(scene, plane):
    """The oracle scene's array and column of a parameter plane of the GPU layout."""
    if plane < 3:
        return scene["means"], (slice(None), plane)
    if plane < 6:
        return scene["log_scales"], (slice(None), plane - 3)
    if plane < 10:
        return scene["quats"], (slice(None), plane - 6)
    if plane == 10:
        return scene["opacity_logits"], (slice(None),)
    return scene["sh"], (slice(None), (plane - 11) // 3, (plane - 11) % 3)


def test_autograd_finite_differences():
    """The autograd gradient against central differences of the FP64 oracle's
    forward (sum over both views of W . image, projected positions kept in
    FP64 so that the function is smooth in the means) at the three largest
    entries of eight parameter planes.  In FP64 a step of 1e-6 (relative)
    leaves the truncation and rounding error of the difference far below the
    check (the oracle's own analytic gradient agrees with these differences to
    1e-6 of the tolerance), and crosses one of the forward's discrete cuts
    (alpha >= 1/255, T >= 1e-4, the 3-sigma radius) with negligible
    probability, so every entry must agree within 2e-3 relative (the FP32
    backward) plus 1e-5 of the plane's largest gradient."""
    s, cams = _scene()
    model = gs.GaussianModel.from_scene(s)
    params = model.data.clone().requires_grad_(True)
    rng = np.random.default_rng(1)
    img = rasterize(params, model.n, model.sh_degree, cams)
    Wt = torch.from_numpy(rng.standard_normal(img.numel()).astype(np.float32)).cuda()
    (img * Wt).sum().backward()
    grad = params.grad.clone()
    oc = ocfg(gs.Config(), fp32=False)  # smooth in the means: no FP32 rounding of the projected positions
    sizes = [3 * c["height"] * c["width"] for c in cams]
    wv = np.split(Wt.cpu().numpy().astype(np.float64), np.cumsum(sizes)[:-1])
    base = {k: (np.asarray(v, np.float64).copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}

    def f(scene):
        return sum(float((orc.forward(scene, cam, oc)["img"].reshape(-1) * w).sum()) for cam, w in zip(cams, wv))

    bad = []
    n_checked = 0
    for plane in (0, 1, 2, 3, 5, 10, 11, 14):
        row = grad[plane, :model.n].abs()
        scale = float(row.max())
        for g_idx in torch.topk(row, 3).indices.tolist():
            arr, col = _entry(base, plane)
            idx = (g_idx,) + tuple(col[1:])
            v0 = float(arr[idx])
            h = 1e-6 * max(1.0, abs(v0))
            sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
            sm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
            ap, _ = _entry(sp, plane)
            am, _ = _entry(sm, plane)
            ap[idx] = v0 + h
            am[idx] = v0 - h
            fd = (f(sp) - f(sm)) / (2 * h)
            an = float(grad[plane, g_idx])
            n_checked += 1
            if abs(fd - an) > 2e-3 * abs(an) + 1e-5 * scale:
                bad.append((plane, g_idx, fd, an))
    assert n_checked == 24
    assert not bad, bad
