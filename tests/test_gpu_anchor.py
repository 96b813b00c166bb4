"""Parity of the Scaffold-GS anchor decoding (Supp. D.1, D.3) with the FP64
oracle: the decoded Gaussians (keep decisions outside the oracle's near-tie
set), the decoder's backward, a whole anchor mapping iteration (decode,
render, L1 + D-SSIM, backward, decoder backward) against the oracle's chain,
the flat Adam, and a few iterations lowering the loss."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2606_30436_b300 import anchors, gs, scenes

from _parity import ocfg, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda"
BANDS = anchors.MAX_DIST_DEFAULT


def _anchor_set(n, seed, near=(2.5, 9.0), far=(11.0, 22.0), spread=2.0):
    rng = np.random.default_rng(seed)
    lv = (rng.random(n) < 0.3).astype(np.int32)
    z = np.where(lv == 0, rng.uniform(*near, n), rng.uniform(*far, n))
    pos = np.column_stack([rng.uniform(-spread, spread, n) * z / 5, rng.uniform(-spread, spread, n) * z / 8, z])
    A = dict(pos=pos.astype(np.float32).astype(np.float64), level=lv,
             feat=rng.normal(0, 0.5, (n, 32)).astype(np.float32).astype(np.float64),
             log_l=(np.log(np.where(lv == 0, 0.1, 0.25))[:, None] + rng.normal(0, 0.2, (n, 3))).astype(
                 np.float32).astype(np.float64),
             offs=rng.normal(0, 1.0, (n, 10, 3)).astype(np.float32).astype(np.float64))
    w = anchors.init_weights(seed, device="cpu").numpy().astype(np.float64)
    w[anchors.W2:anchors.B2] += rng.normal(0, 0.05, anchors.B2 - anchors.W2)
    w[anchors.B2:] += rng.normal(0, 0.3, 140)
    return A, w.astype(np.float32).astype(np.float64)


def _model(A, w):
    return anchors.AnchorModel.from_arrays(A["pos"], A["level"], A["feat"], A["log_l"], A["offs"], w)


def _gpu_rows(g: gs.GaussianModel, n, ld):
    """Decoded planes [14][10 ld] -> rows [10 n][14] in the oracle's order (slot k n + i)."""
    d = g.data.cpu().numpy().astype(np.float64)
    cols = np.concatenate([k * ld + np.arange(n) for k in range(10)])
    return d[:, cols].T


@pytest.mark.parametrize("n", [1, 1000])
def test_decode_parity(n):
    A, w = _anchor_set(n, 3 + n)
    m = _model(A, w)
    cc = np.array([0.2, -0.1, 0.05])
    out = m.decoded()
    anchors.gs_anchor_decode(m, cc, out)
    torch.cuda.synchronize()
    rows, keep, unsure = orc.anchor_decode(A, w, cc, BANDS, tol=1e-5)
    got = _gpu_rows(out, n, m.ld)
    gkeep = got[:, 10] > -29.0
    sure = ~unsure
    assert np.array_equal(gkeep[sure], keep[sure])
    both = keep & gkeep
    assert both.sum() > 0.3 * keep.size * (n > 1)
    # positions, log-scales, rotations, colour coefficients: FP32 evaluation of the decoder
    for lo, hi, tol in ((0, 3, 2e-5), (3, 6, 2e-5), (6, 10, 2e-5), (11, 14, 2e-5)):
        err = np.abs(got[both, lo:hi] - rows[both, lo:hi]).max() if both.any() else 0.0
        assert err <= tol * max(1.0, np.abs(rows[both, lo:hi]).max()), (lo, err)
    # opacity compared as alpha = sigmoid(logit) (the logit is ill-conditioned near alpha = 1)
    a_gpu = 1 / (1 + np.exp(-got[both, 10]))
    a_ref = 1 / (1 + np.exp(-rows[both, 10]))
    assert np.abs(a_gpu - a_ref).max() <= 2e-6
    # padding anchors and dropped Gaussians are culled placeholders
    pad = out.data[10].view(10, m.ld)[:, n:]
    assert torch.all(pad == -30.0)


def test_decode_backward_parity():
    n = 1000
    A, w = _anchor_set(n, 7)
    m = _model(A, w)
    cc = np.array([0.0, 0.1, -0.2])
    rows, keep, unsure = orc.anchor_decode(A, w, cc, BANDS, tol=1e-5)
    rng = np.random.default_rng(8)
    G = (rng.normal(size=rows.shape) * keep[:, None]).astype(np.float32).astype(np.float64)
    # gradient planes in the decoded layout; the anchors with a near-tie slot get no gradient on either side
    bad = unsure.reshape(10, n).any(axis=0)
    G.reshape(10, n, 14)[:, bad, :] = 0.0
    gout = m.decoded()
    gd = np.zeros((14, 10 * m.ld), np.float32)
    for k in range(10):
        gd[:, k * m.ld:k * m.ld + n] = G.reshape(10, n, 14)[k].T
    gout.data.copy_(torch.from_numpy(gd))
    gA = torch.zeros_like(m.data)
    gW = torch.zeros_like(m.weights)
    anchors.gs_anchor_decode_bwd(m, cc, gout, gA, gW)
    torch.cuda.synchronize()
    gf, gl, go, gw = orc.anchor_decode_backward(A, w, cc, BANDS, G)
    a = gA[:, :n].cpu().numpy().astype(np.float64)
    assert rel_l2(a[0:32].T, gf) < 1e-4
    assert rel_l2(a[32:35].T, gl) < 1e-4
    assert rel_l2(a[35:65].T.reshape(n, 10, 3), go) < 1e-4
    g = gW.cpu().numpy().astype(np.float64)
    for lo, hi in ((anchors.W1, anchors.B1), (anchors.B1, anchors.W2), (anchors.W2, anchors.B2), (anchors.B2, 11468)):
        assert rel_l2(g[lo:hi], gw[lo:hi]) < 1e-4, (lo, hi)
    assert torch.all(gA[:, n:] == 0)


def _step_case(seed=11):
    A, w = _anchor_set(150, seed, near=(3.0, 8.0), far=(12.0, 18.0), spread=1.6)
    cam = scenes.pinhole(64, 48, 60.0)
    cc = np.zeros(3)
    # target: the oracle's render of the same anchors with perturbed features and offsets
    rng = np.random.default_rng(seed + 1)
    At = dict(A, feat=A["feat"] + rng.normal(0, 0.1, A["feat"].shape),
              offs=A["offs"] + rng.normal(0, 0.1, A["offs"].shape))
    rows_t, _, _ = orc.anchor_decode(At, w, cc, BANDS)
    oc = ocfg(gs.Config())
    target = orc.forward(orc.rows_to_params(rows_t), cam, oc)["img"].astype(np.float32)
    return A, w, cam, cc, oc, target


def test_anchor_iteration_gradients_match_oracle():
    A, w, cam, cc, oc, target = _step_case()
    m = _model(A, w)
    st = anchors.AnchorStep(m, cam, gs.Config(), lambda_dssim=0.2)
    st.fit_capacity(slack=2.0)
    tgt = torch.from_numpy(target.reshape(-1)).to(DEV)
    st.gradients(tgt)
    torch.cuda.synchronize()
    st.map.check_status()
    rows, keep, unsure = orc.anchor_decode(A, w, cc, BANDS, tol=1e-5)
    assert not unsure[keep].any()
    f = orc.loss_and_grads(orc.rows_to_params(rows), cam, oc, target, 0.2)
    assert abs(st.map.buf.loss.item() - f["loss"]) <= 1e-4 * abs(f["loss"])
    gf, gl, go, gw = orc.anchor_decode_backward(A, w, cc, BANDS, orc.grads_to_rows(f["grads"]))
    n = len(A["level"])
    a = st.g_anchor[:, :n].cpu().numpy().astype(np.float64)
    for name, got, ref in (("feat", a[0:32].T, gf), ("log_l", a[32:35].T, gl),
                           ("offs", a[35:65].T.reshape(n, 10, 3), go)):
        assert rel_l2(got, ref) < 1e-3, (name, rel_l2(got, ref))
    g = st.g_w.cpu().numpy().astype(np.float64)
    assert rel_l2(g, gw) < 1e-3, rel_l2(g, gw)


def test_adam_flat_matches_oracle():
    rng = np.random.default_rng(2)
    p, g = rng.normal(size=1003).astype(np.float32), rng.normal(size=1003).astype(np.float32)
    m, v = (0.1 * rng.normal(size=1003)).astype(np.float32), rng.random(1003).astype(np.float32)
    t = [torch.from_numpy(x.copy()).to(DEV) for x in (p, g, m, v)]
    anchors.gs_adam_flat(t[0], t[1], t[2], t[3], 1e-3, 5, eps=1e-8)
    pw, pm, pv = (x.astype(np.float64) for x in (p, m, v))
    orc.adam(pw, g.astype(np.float64), pm, pv, np.full(1003, 1e-3), 5, eps=1e-8)
    assert np.abs(t[0].cpu().double().numpy() - pw).max() < 1e-6
    assert np.abs(t[3].cpu().double().numpy() - pv).max() < 1e-6


def test_anchor_steps_lower_the_loss():
    A, w, cam, cc, oc, target = _step_case(21)
    m = _model(A, w)
    st = anchors.AnchorStep(m, cam, gs.Config(), lambda_dssim=0.2)
    st.fit_capacity(slack=3.0)
    tgt = torch.from_numpy(target.reshape(-1)).to(DEV)
    first = float(st.step(tgt).item())
    for _ in range(30):
        last = st.step(tgt)
    torch.cuda.synchronize()
    st.map.check_status()
    assert float(last.item()) < 0.8 * first


def test_keyframe_to_anchor_mapping():
    """The chain of a new keyframe: probability, voxel insertion, anchors from the
    inserted voxels (zero features, voxel-size scales), then anchor mapping on the
    keyframe's own image lowers the loss."""
    from paper_2606_30436_b300 import spawn
    H, W = 120, 200
    img, depth, U = scenes.keyframe(H, W, seed=51)
    cam = scenes.keyframe_camera(H, W, seed=52, centre=(0.0, -1.6, 20.0))
    prob = spawn.gs_init_probability(torch.from_numpy(img).to(DEV), torch.from_numpy(depth).to(DEV))
    amap = spawn.AnchorMap(8192)
    amap.insert(prob, torch.from_numpy(U).to(DEV), torch.from_numpy(depth).to(DEV), cam)
    torch.cuda.synchronize()
    amap.check_status()
    m = anchors.AnchorModel.from_anchor_map(amap)
    n = m.n
    assert n > 50
    assert torch.equal(m.pos[:, :n], amap.pos[:, :n]) and torch.equal(m.level[:n], amap.level[:n])
    eps = np.log(np.asarray(anchors.VOXEL_DEFAULT))[amap.level[:n].cpu().numpy()]
    assert np.allclose(m.data[32:35, :n].cpu().numpy(), eps[None, :], atol=1e-6)
    assert torch.all(m.data[:32, :n] == 0) and torch.all(m.data[35:, :n] == 0)
    st = anchors.AnchorStep(m, cam, gs.Config(), lambda_dssim=0.2)
    st.fit_capacity(slack=3.0)
    tgt = torch.from_numpy(img.reshape(-1)).to(DEV)
    first = float(st.step(tgt).item())
    for _ in range(40):
        last = st.step(tgt)
    torch.cuda.synchronize()
    st.map.check_status()
    assert np.isfinite(float(last.item())) and float(last.item()) < first
    assert torch.isfinite(m.data).all() and torch.isfinite(m.weights).all()
