"""The projection backward fused with Adam (gs_project_bwd_adam) against the
unfused sequence (gs_render_bwd with a gradient buffer, gs_iso_loss, gs_adam)
on the same inputs, single- and multi-view, with and without the isotropic
term, eager and graph-replayed; and against the FP64 oracle's gradient and
Adam through the first moment (m = (1 - b1) g after one step)."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2606_30436_b300 import gs, scenes

from _parity import GROUPS, ocfg, rel_l2

pytestmark = pytest.mark.gpu


def _case(multi):
    if multi:
        s = scenes.uniform_scene(3000, seed=7, sh_degree=3, xy_range=3.0)
        cams = [scenes.pinhole(100, 70, 90.0),
                scenes.pinhole(150, 90, 140.0, R=scenes.yaw_matrix(4.0), t=np.array([0.2, -0.1, 0.3], np.float32)),
                scenes.pinhole(64, 48, 60.0, t=np.array([-0.1, 0.05, -0.5], np.float32))]
    else:
        s = scenes.uniform_scene(10000, seed=0, sh_degree=3)
        cams = [scenes.pinhole(320, 240, 300.0)]
    return s, cams


def _target(scene, cams, cfg):
    tm = gs.GaussianModel.from_scene(scenes.perturb(scene, 0.02, seed=9))
    st = gs.MappingStep(tm, cams, cfg, with_stats=False)
    st.fit_capacity()
    return st.buf.img.clone()


def _run(scene, cams, cfg, target, fused, iters, lambda_iso, graph=False):
    model = gs.GaussianModel.from_scene(scene)
    st = gs.MappingStep(model, cams, cfg, lambda_iso=lambda_iso, lr=gs.default_lr(extent=5.0), fused_adam=fused)
    st.fit_capacity(slack=2.0)
    if graph:
        g = st.capture(target)
        for _ in range(iters):
            st.replay(g)
    else:
        for _ in range(iters):
            st.step(target)
    torch.cuda.synchronize()
    st.check_status()
    return st


@pytest.mark.parametrize("multi,lambda_iso,graph", [(False, 0.0, False), (True, 10.0, False), (False, 10.0, True)])
def test_fused_matches_unfused(multi, lambda_iso, graph):
    scene, cams = _case(multi)
    cfg = gs.Config()
    target = _target(scene, cams, cfg)
    p0 = gs.GaussianModel.from_scene(scene).data.clone()
    a = _run(scene, cams, cfg, target, True, 3, lambda_iso, graph)
    b = _run(scene, cams, cfg, target, False, 3, lambda_iso, graph)
    n = a.model.n
    # moments are linear (m) and quadratic (v) in the gradients: FP32 summation order only
    assert rel_l2(a.exp_avg.data[:, :n].cpu().numpy(), b.exp_avg.data[:, :n].cpu().numpy()) < 1e-4
    assert rel_l2(a.exp_avg_sq.data[:, :n].cpu().numpy(), b.exp_avg_sq.data[:, :n].cpu().numpy()) < 1e-4
    # the updates agree except where a gradient sums to ~0 and its sign depends on rounding
    da = (a.model.data - p0)[:, :n].cpu().numpy()
    db = (b.model.data - p0)[:, :n].cpu().numpy()
    close = np.abs(da - db) <= 1e-6 + 1e-4 * np.abs(db)
    assert close.mean() > 0.999, close.mean()
    assert rel_l2(da, db) < 2e-2
    # padding rows untouched
    assert torch.equal(a.model.data[:, n:], p0[:, n:])
    # the statistics are folded by the fused kernel as by the unfused one
    assert rel_l2(a.buf.stats_acc[:, :n].cpu().numpy(), b.buf.stats_acc[:, :n].cpu().numpy()) < 1e-5


def test_fused_first_moment_matches_oracle_gradient():
    """One fused step from zero moments: m = (1 - b1) g with g the oracle's FP64 gradient (L1 + D-SSIM)."""
    scene = scenes.uniform_scene(200, seed=41, sh_degree=3)
    cams = [scenes.pinhole(64, 48, 60.0)]
    cfg = gs.Config()
    oc = ocfg(cfg)
    tscene = scenes.perturb(scene, 0.01, seed=141)
    tgt_np = orc.forward(tscene, cams[0], oc)["img"].astype(np.float32)
    target = torch.from_numpy(tgt_np.reshape(-1)).cuda()
    model = gs.GaussianModel.from_scene(scene)
    st = gs.MappingStep(model, cams, cfg, lambda_dssim=0.2, fused_adam=True)
    st.fit_capacity(slack=2.0)
    st.step(target)
    torch.cuda.synchronize()
    st.check_status()
    f = orc.loss_and_grads(scene, cams[0], oc, tgt_np, 0.2)
    m = gs.unpack_planes(st.exp_avg.data.cpu().numpy(), model.n, model.sh_degree)
    for k in GROUPS:
        e = rel_l2(m[k] / 0.1, f["grads"][k])
        assert e < 1e-3, (k, e)
