"""The stored per-pixel-list backward against the FP64 oracle (whose own
backward walks stored contributor lists) and against the recompute-in-
backward path: the lists forward renders bit for bit like the unsplit
forward, each pixel's list holds exactly the Gaussians the oracle blends
there, the gradients of every group match the oracle within 1e-3 relative L2
and the lifecycle statistics match the recompute path; a list buffer that is
too small is reported and never overrun."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2606_30436_b300 import gs, scenes

from _parity import GROUPS, ocfg, rel_l2

pytestmark = pytest.mark.gpu


def _step(scene, cams, stored, lam=0.2, target=None, with_stats=True, cfg=None):
    cfg = cfg or gs.Config(segment=0)
    model = gs.GaussianModel.from_scene(scene)
    st = gs.MappingStep(model, cams, cfg, lambda_dssim=lam, stored_lists=stored, with_stats=with_stats)
    st.fit_capacity()
    if target is not None:
        st.buf.stats_acc.zero_() if with_stats else None
        st.step(target, optimize=False)
        torch.cuda.synchronize()
        st.check_status()
    return st


def _targets(scene, cams, cfg, seed):
    ts = scenes.perturb(scene, 0.01, seed=seed)
    oc = ocfg(cfg)
    imgs = [orc.forward(ts, c, oc)["img"].astype(np.float32) for c in cams]
    return imgs, torch.from_numpy(np.concatenate([t.reshape(-1) for t in imgs])).cuda()


@pytest.mark.parametrize("case", ["cfg1", "multiview"])
def test_lists_forward_matches_unsplit_forward_and_oracle(case):
    if case == "cfg1":
        scene, cams = scenes.uniform_scene(10000, seed=0, sh_degree=0), [scenes.pinhole(320, 240, 300.0)]
    else:
        scene = scenes.uniform_scene(2000, seed=7, sh_degree=1, xy_range=3.0)
        cams = [scenes.pinhole(100, 70, 90.0), scenes.pinhole(64, 48, 60.0, t=np.array([-0.1, 0.05, -0.5], np.float32))]
    cfg = gs.Config(segment=0)
    a = _step(scene, cams, stored=True)
    b = _step(scene, cams, stored=False)
    a.forward()
    b.forward()
    torch.cuda.synchronize()
    assert torch.equal(a.buf.img, b.buf.img) and torch.equal(a.buf.T_final, b.buf.T_final)
    assert torch.equal(a.buf.last, b.buf.last)
    off = a.lists.offsets.cpu().numpy()
    ids = a.lists.ids.cpu().numpy()
    alpha = a.lists.alpha.cpu().numpy()
    assert off[-1] == a.lists.events() <= a.lists.capacity
    oc = ocfg(cfg)
    ld = a.buf.ld
    for v, cam in enumerate(cams):
        f = orc.forward(scene, cam, oc)
        W, H = cam["width"], cam["height"]
        p0 = int(a.buf.pixel_offset[v])
        n = np.diff(off[p0:p0 + W * H + 1]).reshape(H, W)
        mask = f["flags"] & (orc.OR_FLAG_NEAR_ALPHA_MIN | orc.OR_FLAG_NEAR_T_CUT) != 0
        # the number of blended Gaussians per pixel equals the oracle's away from near-threshold pixels
        assert np.array_equal(n[~mask], f["n_contrib"][~mask])
        # the events belong to this view's records and have alpha in [alpha_min, alpha_max]
        sl = slice(int(off[p0]), int(off[p0 + W * H]))
        assert np.all(ids[sl] // ld == v)
        assert np.all((alpha[sl] >= cfg.alpha_min) & (alpha[sl] <= cfg.alpha_max))


@pytest.mark.parametrize("D,seed", [(0, 40), (3, 41)])
def test_lists_backward_gradcheck_scene(D, seed):
    scene = scenes.uniform_scene(200, seed=seed, sh_degree=D)
    cams = [scenes.pinhole(64, 48, 60.0)]
    cfg = gs.Config(segment=0)
    imgs, tgt = _targets(scene, cams, cfg, seed + 100)
    st = _step(scene, cams, stored=True, target=tgt)
    ref = orc.loss_and_grads(scene, cams[0], ocfg(cfg), imgs[0], 0.2)
    assert abs(st.buf.loss.item() - ref["loss"]) < 1e-4 * abs(ref["loss"]) + 1e-7
    g = gs.unpack_planes(st.grads.data.cpu().numpy(), st.model.n, D)
    for k in GROUPS:
        assert rel_l2(g[k], ref["grads"][k]) < 1e-3, k


def test_lists_backward_config1_and_stats_match_recompute():
    scene, cams = scenes.uniform_scene(10000, seed=0, sh_degree=0), [scenes.pinhole(320, 240, 300.0)]
    cfg = gs.Config(segment=0)
    imgs, tgt = _targets(scene, cams, cfg, 1)
    a = _step(scene, cams, stored=True, target=tgt)
    b = _step(scene, cams, stored=False, target=tgt)
    ref = orc.loss_and_grads(scene, cams[0], ocfg(cfg), imgs[0], 0.2)
    ga = gs.unpack_planes(a.grads.data.cpu().numpy(), a.model.n, 0)
    gb = gs.unpack_planes(b.grads.data.cpu().numpy(), b.model.n, 0)
    for k in GROUPS:
        assert rel_l2(ga[k], ref["grads"][k]) < 1e-3, k
        assert rel_l2(ga[k], gb[k]) < 1e-3, k
    sa = a.buf.stats_acc[:, :a.model.n].cpu().numpy()
    sb = b.buf.stats_acc[:, :b.model.n].cpu().numpy()
    # |Omega|, kappa and the view count are the same event counts; max blend weight and gamma agree
    assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1]) and np.array_equal(sa[5], sb[5])
    assert np.abs(sa[3] - sb[3]).max() < 1e-5 and rel_l2(sa[2], sb[2]) < 1e-5


def test_lists_capacity_overflow_reported():
    scene, cams = scenes.uniform_scene(3000, seed=3, sh_degree=0), [scenes.pinhole(128, 96, 120.0)]
    model = gs.GaussianModel.from_scene(scene)
    st = gs.MappingStep(model, cams, gs.Config(segment=0), stored_lists=True)
    st.fit_capacity()
    need = st.lists.events()
    assert need > 100
    # a capacity of 100 slots over buffers of 200: nothing at or past slot 100 may be written
    st.lists.capacity = 100
    st.lists.ids = torch.full((200,), -7, dtype=torch.int32, device="cuda")
    st.lists.alpha = torch.full((200,), -7.0, dtype=torch.float32, device="cuda")
    st.forward()
    torch.cuda.synchronize()
    assert st.buf.status.item() & (1 << gs.GS_ERR_CAPACITY)
    assert st.lists.events() == need
    with pytest.raises(gs.GSError):
        st.check_status()
    ids, alpha = st.lists.ids.cpu().numpy(), st.lists.alpha.cpu().numpy()
    assert np.all(ids[:100] >= 0) and np.all(alpha[:100] > 0)
    assert np.all(ids[100:] == -7) and np.all(alpha[100:] == -7.0)
    st.fit_capacity()
    assert st.lists.capacity >= need and st.lists.events() == need
