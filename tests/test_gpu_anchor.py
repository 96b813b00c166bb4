"""Parity of the Scaffold-GS anchor decoding (Supp. D.1, D.3) with the FP64
oracle's bfloat16-operand decoder (the tensor cores' operand precision): the
decoded Gaussians (keep decisions outside the oracle's near-tie set), the
decoder's backward with tolerances derived from its bfloat16 roundings, the
bounded tensor-core waits, a whole anchor mapping iteration (decode, render,
L1 + D-SSIM, backward, decoder backward) against the oracle's chain, the flat
Adam, and a few iterations lowering the loss."""
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


U_BF16 = 2.0 ** -8  # unit roundoff of bfloat16 (8 significant bits, round to nearest)


def _bf16(v):
    b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _near_midpoint(v, rtol):
    b = np.asarray(v, np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    mid = (b + np.uint32(0x8000)).view(np.float32).astype(np.float64)
    return np.abs(v - mid) <= rtol * np.abs(v)


def bf16_ties(A, w, cc):
    """Anchors where the kernel's FP32 evaluation and the oracle's FP64 one may
    round a decoder operand to neighbouring bfloat16 values: a direction or
    log-distance input within 1e-6 (relative) of a rounding midpoint, a hidden
    pre-activation within 2e-6 of one, or a pre-activation within 1e-5 of the
    ReLU's kink."""
    x, pre = orc.anchor_hidden(A, w, cc, bf16=True)
    return (_near_midpoint(x[:, 32:36], 1e-6).any(axis=1) | _near_midpoint(np.maximum(pre, 0.0), 2e-6).any(axis=1)
            | (np.abs(pre) < 1e-5).any(axis=1))


@pytest.mark.parametrize("n", [1, 1000, 40000])
def test_decode_parity(n):
    """Decoded Gaussians against the oracle's bfloat16-operand decoder (the
    tensor cores' operand precision, FP64 sums): keep decisions away from the
    oracle's near-tie set, values within FP32 rounding away from anchors with a
    bfloat16 rounding tie, and within the size of one rounding step at those."""
    A, w = _anchor_set(n, 3 + n)
    m = _model(A, w)
    cc = np.array([0.2, -0.1, 0.05])
    out = m.decoded()
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    anchors.gs_anchor_decode(m, cc, out, status=status)
    torch.cuda.synchronize()
    assert status.item() == 0
    rows, keep, unsure = orc.anchor_decode(A, w, cc, BANDS, tol=1e-5, bf16=True)
    tie = np.tile(bf16_ties(A, w, cc), 10)
    assert tie.mean() < 0.1
    got = _gpu_rows(out, n, m.ld)
    gkeep = got[:, 10] > -29.0
    sure = ~unsure & ~tie
    assert np.array_equal(gkeep[sure], keep[sure])
    both = keep & gkeep & ~tie
    assert both.sum() > 0.3 * keep.size * (n > 1)
    # positions, log-scales, rotations, colour coefficients: FP32 evaluation of the decoder
    for lo, hi, tol in ((0, 3, 2e-5), (3, 6, 2e-5), (6, 10, 2e-5), (11, 14, 2e-5)):
        err = np.abs(got[both, lo:hi] - rows[both, lo:hi]).max() if both.any() else 0.0
        assert err <= tol * max(1.0, np.abs(rows[both, lo:hi]).max()), (lo, err)
        at_tie = keep & gkeep & tie
        if at_tie.any():
            assert np.abs(got[at_tie, lo:hi] - rows[at_tie, lo:hi]).max() <= 2e-2 * max(
                1.0, np.abs(rows[at_tie, lo:hi]).max())
    # opacity compared as alpha = tanh(z) = sigmoid(logit) (the logit is ill-conditioned near alpha = 1):
    # the tensor core sums z's 64 exact products in FP32, an error of at most 64 x 2^-23 x sum |W2 h|
    # (one unit in the last place of the running sum per addition), which alpha sees times 1 - alpha^2
    x, pre = orc.anchor_hidden(A, w, cc, bf16=True)
    w2b = _bf16(w[anchors.W2:anchors.B2].reshape(140, 64))
    S = (_bf16(np.maximum(pre, 0.0)) @ np.abs(w2b).T)[:, 3::14].T.reshape(-1)  # rows k n + i
    a_gpu = 1 / (1 + np.exp(-got[both, 10]))
    a_ref = 1 / (1 + np.exp(-rows[both, 10]))
    bound = (1 - a_ref ** 2) * (64 * 2.0 ** -23 * S[both] + 2.0 ** -23 * np.abs(np.arctanh(a_ref))) + 2e-7
    assert np.all(np.abs(a_gpu - a_ref) <= bound), np.max(np.abs(a_gpu - a_ref) / bound)
    # padding anchors and dropped Gaussians are culled placeholders
    pad = out.data[10].view(10, m.ld)[:, n:]
    assert torch.all(pad == -30.0)


def bf16_backward_envelope(A, w, cc, dz, dp):
    """Expected size (root of the summed variances) of the error the kernel
    makes when it rounds each anchor's dL/dz and dL/dpre to bfloat16 before its
    tensor-core products, which the oracle's plain FP64 backward does not: each
    rounding is a relative error of at most u, of variance at most u^2 / 3,
    independent across anchors and units; dL/dpre carries dL/dz's errors
    through W2 plus its own.  Returns {block: envelope}."""
    var = U_BF16 ** 2 / 3.0
    x, pre = orc.anchor_hidden(A, w, cc, bf16=True)
    hb, xb = _bf16(np.maximum(pre, 0.0)), _bf16(x)
    w1b = _bf16(w[anchors.W1:anchors.B1].reshape(64, 36))
    w2b = _bf16(w[anchors.W2:anchors.B2].reshape(140, 64))
    mask = (pre > 0).astype(np.float64)
    v_dp = var * ((dz ** 2) @ (w2b ** 2) * mask + dp ** 2)      # [r][c]
    return {"W1": np.sqrt((v_dp.T @ (xb ** 2)).sum()), "b1": np.sqrt(v_dp.sum()),
            "W2": np.sqrt(var * ((dz ** 2).T @ (hb ** 2)).sum()), "b2": np.sqrt(var * (dz ** 2).sum()),
            "feat": np.sqrt((v_dp @ (w1b[:, :32] ** 2)).sum())}


@pytest.mark.parametrize("n", [1000, 40000])
def test_decode_backward_parity(n):
    """The decoder's backward against the oracle's plain FP64 chain rule of the
    bfloat16-operand forward.  The offset and log-scale gradients are FP32 on
    both sides (1e-4); the feature and weight gradients pass through the
    tensor cores with dL/dz and dL/dpre rounded to bfloat16, so each block's
    tolerance is three times the envelope those roundings imply for these
    anchors plus 2e-5 for FP32 sums.  Anchors with a near-tie keep decision or
    a bfloat16 rounding tie get no gradient on either side."""
    A, w = _anchor_set(n, 7 + n)
    m = _model(A, w)
    cc = np.array([0.0, 0.1, -0.2])
    rows, keep, unsure = orc.anchor_decode(A, w, cc, BANDS, tol=1e-5, bf16=True)
    rng = np.random.default_rng(8)
    G = (rng.normal(size=rows.shape) * keep[:, None]).astype(np.float32).astype(np.float64)
    bad = unsure.reshape(10, n).any(axis=0) | bf16_ties(A, w, cc)
    G.reshape(10, n, 14)[:, bad, :] = 0.0
    gout = m.decoded()
    gd = np.zeros((14, 10 * m.ld), np.float32)
    for k in range(10):
        gd[:, k * m.ld:k * m.ld + n] = G.reshape(10, n, 14)[k].T
    gout.data.copy_(torch.from_numpy(gd))
    gA = torch.full_like(m.data, 7.0)
    gW = torch.full_like(m.weights, 7.0)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    anchors.gs_anchor_decode_bwd(m, cc, gout, gA, gW, status=status)
    torch.cuda.synchronize()
    assert status.item() == 0
    gf, gl, go, gw, dz, dp = orc.anchor_decode_backward(A, w, cc, BANDS, G, bf16=True, rows=True)
    env = bf16_backward_envelope(A, w, cc, dz, dp)
    a = gA[:, :n].cpu().numpy().astype(np.float64)

    def close(name, got, ref, tol):
        err, nrm = np.linalg.norm(got - ref), np.linalg.norm(ref)
        assert err <= tol * nrm, (name, err / nrm, tol)

    close("feat", a[0:32].T, gf, 3.0 * env["feat"] / np.linalg.norm(gf) + 2e-5)
    close("log_l", a[32:35].T, gl, 1e-4)
    close("offs", a[35:65].T.reshape(n, 10, 3), go, 1e-4)
    g = gW.cpu().numpy().astype(np.float64)
    for name, (lo, hi) in {"W1": (anchors.W1, anchors.B1), "b1": (anchors.B1, anchors.W2),
                           "W2": (anchors.W2, anchors.B2), "b2": (anchors.B2, 11468)}.items():
        close(name, g[lo:hi], gw[lo:hi], 3.0 * env[name] / np.linalg.norm(gw[lo:hi]) + 2e-5)
    assert torch.all(gA[:, n:] == 0)


def test_decode_wait_timeout():
    """A poll budget of zero makes the first wait for the tensor core give up
    in both directions: the kernels flag GS_ERR_TIMEOUT, write no decoded
    Gaussian and add nothing to the weight gradient, and the next call with
    the default budget is correct."""
    n = 3000
    A, w = _anchor_set(n, 5)
    m = _model(A, w)
    cc = np.zeros(3)
    out = m.decoded()
    out.data.fill_(5.0)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    anchors.gs_anchor_decode(m, cc, out, status=status, max_polls=0)
    torch.cuda.synchronize()
    assert status.item() == 1 << gs.GS_ERR_TIMEOUT
    assert torch.all(out.data == 5.0)
    gA, gW = torch.zeros_like(m.data), torch.full_like(m.weights, 3.0)
    status.zero_()
    anchors.gs_anchor_decode_bwd(m, cc, out, gA, gW, status=status, max_polls=0)
    torch.cuda.synchronize()
    assert status.item() == 1 << gs.GS_ERR_TIMEOUT
    assert torch.all(gW == 0)  # zeroed by the call, nothing added
    status.zero_()
    anchors.gs_anchor_decode(m, cc, out, status=status)
    torch.cuda.synchronize()
    assert status.item() == 0
    rows, keep, unsure = orc.anchor_decode(A, w, cc, BANDS, tol=1e-5, bf16=True)
    ok = ~unsure & ~np.tile(bf16_ties(A, w, cc), 10)
    got = _gpu_rows(out, n, m.ld)
    assert np.array_equal((got[:, 10] > -29.0)[ok], keep[ok])


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
    """One anchor mapping iteration (decode, render, L1 + D-SSIM, backward,
    decoder backward) against the oracle's chain with the bfloat16-operand
    decoder: the loss within 1e-4, the anchors' gradients within 1e-3 (the
    FP32 rasteriser) plus three times the bfloat16 envelope of the decoder's
    backward where its tensor-core products enter."""
    A, w, cam, cc, oc, target = _step_case()
    m = _model(A, w)
    st = anchors.AnchorStep(m, cam, gs.Config(), lambda_dssim=0.2)
    st.fit_capacity(slack=2.0)
    tgt = torch.from_numpy(target.reshape(-1)).to(DEV)
    st.gradients(tgt)
    torch.cuda.synchronize()
    st.map.check_status()
    rows, keep, unsure = orc.anchor_decode(A, w, cc, BANDS, tol=1e-5, bf16=True)
    assert not unsure[keep].any()
    f = orc.loss_and_grads(orc.rows_to_params(rows), cam, oc, target, 0.2)
    assert abs(st.map.buf.loss.item() - f["loss"]) <= 1e-4 * abs(f["loss"])
    gf, gl, go, gw, dz, dp = orc.anchor_decode_backward(A, w, cc, BANDS, orc.grads_to_rows(f["grads"]), bf16=True,
                                                       rows=True)
    env = bf16_backward_envelope(A, w, cc, dz, dp)
    n = len(A["level"])
    a = st.g_anchor[:, :n].cpu().numpy().astype(np.float64)
    for name, got, ref, e in (("feat", a[0:32].T, gf, env["feat"]), ("log_l", a[32:35].T, gl, 0.0),
                              ("offs", a[35:65].T.reshape(n, 10, 3), go, 0.0)):
        tol = 1e-3 + 3.0 * e / np.linalg.norm(ref)
        assert rel_l2(got, ref) < tol, (name, rel_l2(got, ref), tol)
    g = st.g_w.cpu().numpy().astype(np.float64)
    e = np.sqrt(sum(env[k] ** 2 for k in ("W1", "b1", "W2", "b2")))
    tol = 1e-3 + 3.0 * e / np.linalg.norm(gw)
    assert rel_l2(g, gw) < tol, (rel_l2(g, gw), tol)


@pytest.mark.parametrize("n", [1003, 1004])  # the scalar and the float4 path
def test_adam_flat_matches_oracle(n):
    rng = np.random.default_rng(2)
    p, g = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    m, v = (0.1 * rng.normal(size=n)).astype(np.float32), rng.random(n).astype(np.float32)
    t = [torch.from_numpy(x.copy()).to(DEV) for x in (p, g, m, v)]
    anchors.gs_adam_flat(t[0], t[1], t[2], t[3], 1e-3, 5, eps=1e-8)
    pw, pm, pv = (x.astype(np.float64) for x in (p, m, v))
    orc.adam(pw, g.astype(np.float64), pm, pv, np.full(n, 1e-3), 5, eps=1e-8)
    assert np.abs(t[0].cpu().double().numpy() - pw).max() < 1e-6
    assert np.abs(t[3].cpu().double().numpy() - pv).max() < 1e-6


def test_adam_flat_device_step_matches_host_step():
    rng = np.random.default_rng(4)
    x = [rng.normal(size=776).astype(np.float32) for _ in range(3)] + [rng.random(776).astype(np.float32)]
    a = [torch.from_numpy(v.copy()).to(DEV) for v in x]
    b = [torch.from_numpy(v.copy()).to(DEV) for v in x]
    anchors.gs_adam_flat(a[0], a[1], a[2], a[3], 1e-3, 7)
    anchors.gs_adam_flat(b[0], b[1], b[2], b[3], 1e-3, 1, step_device=torch.full((1,), 7, dtype=torch.int64,
                                                                                 device=DEV))
    torch.cuda.synchronize()
    for u, w in zip(a, b):
        assert torch.equal(u, w)


def test_anchor_graph_replay_matches_eager_steps():
    A, w, cam, cc, oc, target = _step_case(23)
    tgt = torch.from_numpy(target.reshape(-1)).to(DEV)
    runs = []
    for graph in (False, True):
        st = anchors.AnchorStep(_model(A, w), cam, gs.Config(), lambda_dssim=0.2)
        st.fit_capacity(slack=3.0)
        losses = []
        g = st.capture(tgt) if graph else None
        for _ in range(4):
            losses.append(float((st.replay(g) if graph else st.step(tgt)).item()))
        torch.cuda.synchronize()
        st.map.check_status()
        runs.append((losses, st.model.data.clone(), st.model.weights.clone(), st.step_count))
    (la, pa, wa, ca), (lb, pb, wb, cb) = runs
    assert ca == cb == 4
    # the compositing backward sums with atomics, so two runs differ in the last bits of their
    # gradients, and Adam (eps 1e-15) turns such differences in near-zero gradients into
    # full-size steps: over four steps the losses drift apart by up to ~1e-4.  The first loss
    # is exact; a wrong step counter or bias correction moves the later ones by far more.
    assert la[0] == lb[0]
    assert np.allclose(la, lb, rtol=2e-3, atol=0.0), (la, lb)
    assert rel_l2(pa.cpu().numpy(), pb.cpu().numpy()) < 1e-4
    assert rel_l2(wa.cpu().numpy(), wb.cpu().numpy()) < 1e-4


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
