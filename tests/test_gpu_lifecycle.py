"""GPU versus the FP64 oracle for the lifecycle actions and the learned
predictor: densify / prune compaction (index work bit-exact, split children
within FP32 rounding), the predictor's inputs, the tensor-core MLP forward and
its BCE gradient, plus a training run on a known rule."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2606_30436_b300 import gs, scenes

from _parity import rel_l2

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _features(n, seed):
    """Inputs with the ranges of the predictor's features (opacity, log-scales,
    log counts, blend weights, log distances)."""
    rng = np.random.default_rng(seed)
    x = np.empty((n, 16))
    x[:, 0] = rng.random(n)
    x[:, 1:4] = rng.normal(-3.0, 0.5, size=(n, 3))
    x[:, 4] = np.log1p(rng.integers(0, 100, n))
    x[:, 5] = np.log1p(rng.exponential(3.0, n))
    x[:, 6:14] = rng.random((n, 8)) * (rng.random((n, 1)) < 0.7)
    x[:, 14] = np.log1p(rng.uniform(1.0, 200.0, n))
    x[:, 15] = np.log1p(rng.exponential(50.0, n))
    return x


def _weights(seed):
    w = gs.mlp_init(seed, device="cpu").double().numpy()
    rng = np.random.default_rng(seed + 100)
    w[1024:1088] = rng.normal(0.0, 0.1, 64)
    w[5184:5248] = rng.normal(0.0, 0.1, 64)
    w[5376:5378] = rng.normal(0.0, 0.5, 2)
    return w


def near_bf16_tie(h, rtol=1e-5):
    """Rows with an element within rtol of a bfloat16 rounding midpoint: there
    the FP32 (GPU) and FP64 (oracle) sums may round to neighbouring values."""
    b = np.asarray(h, np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    mid = (b + np.uint32(0x8000)).view(np.float32).astype(np.float64)
    return (np.abs(h - mid) <= rtol * np.abs(h)).any(axis=1)


def _planes(x, ld):
    f = torch.zeros(x.shape[1], ld, dtype=torch.float32)
    f[:, :x.shape[0]] = torch.from_numpy(x.T.astype(np.float32))
    return f.to(DEV)


@pytest.mark.parametrize("n", [1, 128, 1000, 5003])
def test_mlp_forward_parity(n):
    x = _features(n, n).astype(np.float32).astype(np.float64)
    w = _weights(3).astype(np.float32).astype(np.float64)
    ld = gs.padded(n)
    feat = _planes(x, ld)
    wd = torch.from_numpy(w.astype(np.float32)).to(DEV)
    prob = torch.full((2, ld), -1.0, device=DEV)
    dens = torch.full((n,), 7, dtype=torch.uint8, device=DEV)
    prn = torch.full((n,), 7, dtype=torch.uint8, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    gs.gs_mlp_forward(feat, n, wd, prob, dens, prn, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    p_gpu = prob[:, :n].cpu().double().numpy().T
    p_ref, h1_ref, _ = orc.mlp_forward(x, w, bf16=True)
    # both sides round inputs, weights and h1 to bfloat16 and differ by FP32 vs FP64 accumulation (~1e-7);
    # where a pre-rounding h1 sits at a bfloat16 midpoint the two may round one bfloat16 ulp apart (2^-8
    # relative of that element), which moves a probability by up to ~1e-2
    tie = near_bf16_tie(h1_ref, 2e-6)
    err = np.abs(p_gpu - p_ref).max(axis=1)
    assert err[~tie].max(initial=0.0) < 2e-6, (err[~tie].max(), tie.mean())
    assert err[tie].max(initial=0.0) < 2e-2
    # 64 elements, each within 2e-6 of a midpoint with probability ~4e-6 / 2^-7
    assert tie.mean() < 0.1
    assert np.all(prob[:, n:].cpu().numpy() == -1.0)  # padding untouched
    d_gpu, pr_gpu = dens.cpu().numpy(), prn.cpu().numpy()
    assert set(np.unique(d_gpu)) <= {0, 1} and set(np.unique(pr_gpu)) <= {0, 1}
    # the kernel decides on the FP32 logit (z > 0); its FP32 sigmoid can round to exactly 1/2 next to z = 0
    for k, dec in ((0, d_gpu), (1, pr_gpu)):
        odd = dec != (p_gpu[:, k] > 0.5)
        assert np.all(p_gpu[odd, k] == 0.5)
    clear = np.abs(p_ref - 0.5) > 1e-3
    assert np.array_equal(d_gpu[clear[:, 0]], (p_ref[clear[:, 0], 0] > 0.5).astype(np.uint8))
    assert np.array_equal(pr_gpu[clear[:, 1]], (p_ref[clear[:, 1], 1] > 0.5).astype(np.uint8))


def test_mlp_forward_wait_timeout():
    """A poll budget of zero makes the first wait for the tensor core give up:
    every CTA stops, drains the product it issued, frees its tensor memory and
    flags GS_ERR_TIMEOUT; the call returns normally, nothing is written, and
    the next call with the default budget matches the oracle."""
    n = 1000
    x = _features(n, 31).astype(np.float32).astype(np.float64)
    w = _weights(3).astype(np.float32).astype(np.float64)
    feat = _planes(x, gs.padded(n))
    wd = torch.from_numpy(w.astype(np.float32)).to(DEV)
    prob = torch.full((2, gs.padded(n)), -1.0, device=DEV)
    dens = torch.full((n,), 7, dtype=torch.uint8, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    gs.gs_mlp_forward(feat, n, wd, prob, dens, None, status, max_polls=0)
    torch.cuda.synchronize()
    assert status.item() == 1 << gs.GS_ERR_TIMEOUT
    assert torch.all(prob == -1.0) and torch.all(dens == 7)
    status.zero_()
    gs.gs_mlp_forward(feat, n, wd, prob, dens, None, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    p_ref, h1_ref, _ = orc.mlp_forward(x, w, bf16=True)
    tie = near_bf16_tie(h1_ref, 2e-6)
    err = np.abs(prob[:, :n].cpu().double().numpy().T - p_ref).max(axis=1)
    assert err[~tie].max(initial=0.0) < 2e-6


def _bf16(v):
    b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


U_BF16 = 2.0 ** -8  # unit roundoff of bfloat16 (8 significant bits, round to nearest)


def bf16_backward_envelope(x, w, h1, dh2, dh1):
    """Expected size (root of the summed variances) of the error a kernel
    makes in the hidden layers' weight and bias gradients when it rounds the
    backward's per-row gradients dh2 and dh1 to bfloat16 before its tensor-core
    sums, which the oracle's plain FP64 backward does not: each rounding is a
    relative error of at most u, of variance at most u^2 / 3, independent
    across rows and units; dh1 carries dh2's errors through W2 plus its own.
    Returns {block: envelope} for W1, b1, W2, b2."""
    var = U_BF16 ** 2 / 3.0
    h1b, xb, w2b = _bf16(h1), _bf16(x), _bf16(w[1088:5184].reshape(64, 64))
    v_w2 = var * (dh2 ** 2).T @ (h1b ** 2)                       # [o][c]: sum_r (dh2 h1b)^2
    v_b2 = var * (dh2 ** 2).sum(0)
    mask = (h1 > 0).astype(np.float64)
    v_dh1 = var * ((dh2 ** 2) @ (w2b ** 2) * mask + dh1 ** 2)    # [r][c]
    v_w1 = v_dh1.T @ (xb ** 2)                                   # [o][c]
    v_b1 = v_dh1.sum(0)
    return {"W1": np.sqrt(v_w1.sum()), "b1": np.sqrt(v_b1.sum()), "W2": np.sqrt(v_w2.sum()),
            "b2": np.sqrt(v_b2.sum())}


@pytest.mark.parametrize("n", [1, 1000, 40000])
def test_mlp_train_grad_parity(n):
    """The kernel's gradient against the oracle's plain FP64 backward of the
    BF16-operand forward.  The kernel rounds dh2 and dh1 to bfloat16 for its
    tensor-core sums; the tolerance of each hidden-layer block is three times
    the error envelope those roundings imply for these rows (from u = 2^-8 and
    the per-row terms the oracle returns), plus 1e-5 for FP32 accumulation
    over the rows.  The output layer is FP32 on both sides."""
    x = _features(n, 20 + n).astype(np.float32).astype(np.float64)
    w = _weights(5).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(n)
    y = (rng.random((n, 2)) < 0.3).astype(np.float64)
    ld = gs.padded(n)
    feat = _planes(x, ld)
    wd = torch.from_numpy(w.astype(np.float32)).to(DEV)
    yd = torch.from_numpy(y[:, 0].astype(np.uint8)).to(DEV)
    yp = torch.from_numpy(y[:, 1].astype(np.uint8)).to(DEV)
    grad = torch.full((gs.MLP_WEIGHTS,), 9.0, device=DEV)
    loss = torch.full((1,), 9.0, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    gs.gs_mlp_train_grad(feat, yd, yp, n, wd, grad, loss, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    L_ref, g_ref, dh2, dh1 = orc.mlp_bce_grad(x, y, w, bf16=True, rows=True)
    _, h1, _ = orc.mlp_forward(x, w, bf16=True)
    env = bf16_backward_envelope(x, w, h1, dh2, dh1)
    g = grad.cpu().double().numpy()
    assert abs(loss.item() - L_ref) < 1e-5 * max(1.0, abs(L_ref))
    blocks = {"W1": (0, 1024), "b1": (1024, 1088), "W2": (1088, 5184), "b2": (5184, 5248),
              "W3": (5248, 5376), "b3": (5376, 5378)}
    for name, (lo, hi) in blocks.items():
        err = np.linalg.norm(g[lo:hi] - g_ref[lo:hi])
        ref = np.linalg.norm(g_ref[lo:hi])
        if name in env:
            tol = 3.0 * env[name] / ref + 1e-5
        else:
            tol = 1e-4  # FP32 head on both sides; the forward's operands are rounded alike
        assert err <= tol * ref, (name, err / ref, tol)


def test_mlp_learns_a_rule():
    """Labels from a fixed rule of two inputs; Adam on the GPU gradient reaches high accuracy."""
    n = 8192
    x = _features(n, 77).astype(np.float32)
    yd = (x[:, 5] > np.log1p(3.0)).astype(np.uint8)       # large accumulated gradient -> densify
    yp = ((x[:, 0] < 0.2) & (x[:, 4] > 2.0)).astype(np.uint8)  # faint and seen often -> prune
    ld = gs.padded(n)
    feat = _planes(x.astype(np.float64), ld)
    w = gs.mlp_init(1, device=DEV)
    m, v, grad = torch.zeros_like(w), torch.zeros_like(w), torch.zeros_like(w)
    loss = torch.zeros(1, device=DEV)
    ydt, ypt = torch.from_numpy(yd).to(DEV), torch.from_numpy(yp).to(DEV)
    first = None
    for step in range(1, 401):
        gs.gs_mlp_train_grad(feat, ydt, ypt, n, w, grad, loss)
        gs.gs_mlp_adam(w, grad, m, v, 3e-3, step)
        if first is None:
            first = loss.item()
    dens = torch.zeros(n, dtype=torch.uint8, device=DEV)
    prn = torch.zeros(n, dtype=torch.uint8, device=DEV)
    gs.gs_mlp_forward(feat, n, w, None, dens, prn)
    acc_d = (dens.cpu().numpy() == yd).mean()
    acc_p = (prn.cpu().numpy() == yp).mean()
    assert loss.item() < 0.5 * first
    assert acc_d > 0.95 and acc_p > 0.95, (acc_d, acc_p)


def test_mlp_adam_matches_oracle():
    rng = np.random.default_rng(9)
    w = rng.normal(size=gs.MLP_WEIGHTS).astype(np.float32)
    g = rng.normal(size=gs.MLP_WEIGHTS).astype(np.float32)
    m = (0.1 * rng.normal(size=gs.MLP_WEIGHTS)).astype(np.float32)
    v = rng.random(gs.MLP_WEIGHTS).astype(np.float32)
    t = [torch.from_numpy(a.copy()).to(DEV) for a in (w, g, m, v)]
    gs.gs_mlp_adam(t[0], t[1], t[2], t[3], 1e-3, 7, eps=1e-8)
    pw, pm, pv = (a.astype(np.float64) for a in (w, m, v))
    orc.adam(pw, g.astype(np.float64), pm, pv, np.full(gs.MLP_WEIGHTS, 1e-3), 7, eps=1e-8)
    assert np.abs(t[0].cpu().double().numpy() - pw).max() < 1e-6
    assert np.abs(t[2].cpu().double().numpy() - pm).max() < 1e-6


def _stats(n, ld, seed):
    rng = np.random.default_rng(seed)
    st = np.zeros((6, ld), np.float32)
    views = rng.integers(0, 40, n)
    st[0, :n] = views * rng.exponential(30.0, n)
    st[1, :n] = rng.exponential(2.0, n)
    st[2, :n] = rng.exponential(1.0, n)
    st[3, :n] = rng.random(n)
    st[4, :n] = rng.exponential(1e-3, n) * views
    st[5, :n] = views
    return st


def test_features_and_ring_parity():
    n = 3001
    scene = scenes.uniform_scene(n, seed=4, sh_degree=1)
    model = gs.GaussianModel.from_scene(scene, device=DEV)
    st = _stats(n, model.ld, 4)
    ring = np.random.default_rng(5).random((8, model.ld)).astype(np.float32)
    stats_d, ring_d = torch.from_numpy(st).to(DEV), torch.from_numpy(ring).to(DEV)
    # push: plane 3 moves into slot 6 and restarts at zero
    gs.gs_mlp_push_blend(stats_d, n, ring_d, 6)
    ring[6, :n] = st[3, :n]
    st[3, :n] = 0.0
    torch.cuda.synchronize()
    assert np.array_equal(ring_d.cpu().numpy(), ring) and np.array_equal(stats_d.cpu().numpy(), st)
    feat = torch.zeros(16, model.ld, device=DEV)
    cam = [0.5, -1.0, 2.0]
    gs.gs_mlp_features(model, stats_d, ring_d, 6, cam, feat)
    f_ref = orc.mlp_features(scene["means"], scene["log_scales"], scene["opacity_logits"], st[:, :n].T,
                             ring[:, :n], 6, cam)
    f = feat[:, :n].cpu().double().numpy().T
    assert np.array_equal(f[:, 1:4], f_ref[:, 1:4]) and np.array_equal(f[:, 6:14], f_ref[:, 6:14])
    assert np.abs(f - f_ref).max() < 2e-5, np.abs(f - f_ref).max(axis=0)


def _actions_case(n, D, seed, p_prune=0.25, p_dens=0.3):
    scene = scenes.uniform_scene(n, seed=seed, sh_degree=D)
    model = gs.GaussianModel.from_scene(scene, device=DEV)
    rng = np.random.default_rng(seed)
    prune = (rng.random(n) < p_prune).astype(np.uint8)
    dens = (rng.random(n) < p_dens).astype(np.uint8)
    noise = np.zeros((6, model.ld), np.float32)
    noise[:, :n] = rng.normal(size=(6, n))
    m = rng.normal(size=(model.K, model.ld)).astype(np.float32)
    v = rng.random((model.K, model.ld)).astype(np.float32)
    return scene, model, prune, dens, noise, m, v


@pytest.mark.parametrize("n,D,cap", [(1000, 3, None), (777, 0, None), (5000, 1, 4000), (1, 0, None)])
def test_densify_prune_parity(n, D, cap):
    scene, model, prune, dens, noise, m, v = _actions_case(n, D, n + D)
    ma, va = model.like(), model.like()
    ma.data.copy_(torch.from_numpy(m))
    va.data.copy_(torch.from_numpy(v))
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    split_ls = -3.0
    out, mo, vo, n_out = gs.gs_densify_prune(model, torch.from_numpy(dens).to(DEV), torch.from_numpy(prune).to(DEV),
                                             torch.from_numpy(noise).to(DEV), split_ls, 1.6, exp_avg=ma,
                                             exp_avg_sq=va, capacity=cap, status=status)
    torch.cuda.synchronize()
    P = gs.pack_planes(scene, model.ld)[:, :n].T.astype(np.float64)
    Po, mref, vref, need = orc.densify_prune(P, dens, prune, noise[:, :n].T, split_ls, 1.6, m=m[:, :n].T,
                                             v=v[:, :n].T, cap=out.ld)
    assert int(n_out.item()) == need
    assert status.item() == (1 << 3 if need > out.ld else 0)
    k = min(need, out.ld)
    assert out.n == k
    got = out.data[:, :k].cpu().double().numpy().T
    # every plane except split children's means and log-scales is a copy: bit-exact
    split = np.zeros(k, bool)
    o = 0
    for i in range(n):
        c = 0 if prune[i] else (2 if dens[i] else 1)
        if c == 2 and P[i, 3:6].max() > split_ls:
            split[o:o + 2] = True
        o += c
    split = split[:k]
    assert np.array_equal(got[:, 6:], Po[:, 6:])
    assert np.array_equal(got[~split, :6], Po[~split, :6])
    assert np.abs(got[split, :6] - Po[split, :6]).max(initial=0.0) < 1e-5
    assert np.array_equal(mo.data[:, :k].cpu().double().numpy().T, mref)
    assert np.array_equal(vo.data[:, :k].cpu().double().numpy().T, vref)


def test_densify_prune_all_pruned_and_no_moments():
    n = 300
    scene, model, _, dens, noise, _, _ = _actions_case(n, 0, 3)
    prune = torch.ones(n, dtype=torch.uint8, device=DEV)
    out, mo, vo, n_out = gs.gs_densify_prune(model, torch.from_numpy(dens).to(DEV), prune,
                                             torch.from_numpy(noise).to(DEV), -3.0)
    assert int(n_out.item()) == 0 and out.n == 0 and mo is None and vo is None
    keep = torch.zeros(n, dtype=torch.uint8, device=DEV)
    out, _, _, n_out = gs.gs_densify_prune(model, keep, keep, torch.from_numpy(noise).to(DEV), -3.0)
    assert int(n_out.item()) == n
    assert torch.equal(out.data[:, :n], model.data[:, :n])


def test_lifecycle_chunks_plain_and_learned():
    """Two chunks of the corridor with each decider: row counts follow the bits, moments follow the rows, the
    learned decider reports its agreement with the plain criterion."""
    from paper_2606_30436_b300 import lifecycle
    gt = scenes.corridor_scene(20000, seed=0, sh_degree=1, length=60.0)
    init = scenes.degraded_map(gt, seed=2, length=60.0)
    cfg = gs.Config()
    cams = {f0: [scenes.corridor_camera(f0 + j, 160, 90, 112.5) for j in range(2)] for f0 in (10, 20)}
    gtm = gs.GaussianModel.from_scene(gt, device=DEV)
    targets = {}
    for f0, cs in cams.items():
        st = gs.MappingStep(gtm, cs, cfg, with_stats=False)
        st.fit_capacity()
        targets[f0] = st.buf.img.clone()
    pred = lifecycle.Predictor(seed=1, device=DEV)
    for mode in ("plain", "learned"):
        model = gs.GaussianModel.from_scene(init, device=DEV)
        lc = lifecycle.Lifecycle(mode, tau_d=1.0, tau_p=0.9, predictor=pred, collect=(mode == "plain"))
        moments, steps = None, 0
        for f0 in (10, 20):
            step = gs.MappingStep(model, cams[f0], cfg, moments=moments, step_count=steps)
            step.fit_capacity(slack=1.5)
            lc.start(step)
            for _ in range(3):
                step.step(targets[f0])
                lc.after_iteration(step)
            step.check_status()
            n = model.n
            dens, prune = lc.decide(step, [0.0, -1.6, float(f0 + 1)])
            d, p = dens.cpu().numpy().astype(bool), prune.cpu().numpy().astype(bool)
            rec = lc.assess(step)
            assert rec["densify"] == d.sum() and rec["prune"] == p.sum()
            model, moments = lc.apply(step, dens, prune)
            assert model.n == n - p.sum() + (d & ~p).sum()
            assert moments[0].ld == model.ld and moments[0].n == model.n
            assert torch.isfinite(model.data[:, :model.n]).all()
            steps = step.step_count
        assert len(lc.history) == 2
        if mode == "plain":
            assert len(lc.samples) == 2 and any(h["densify"] + h["prune"] > 0 for h in lc.history)
            pred.train(lifecycle.future_labels(lc.samples, DEV), epochs=20)
        else:
            assert all("prune_recall" in h for h in lc.history)
