"""Pins of the oracle's Scaffold-GS anchor decoding (Supp. D.1, D.3; readings
R25-R29) and of the opacity cull (R2): closed forms with the hidden layer
switched off, the LoD band, dropped Gaussians, the view-direction and
distance inputs, and the backward against central finite differences of the
forward (FP64); the cull against renders with and without the culled
Gaussian."""
import math

import numpy as np

import oracle as orc
from paper_2606_30436_b300 import scenes

K, F, H, IN = 10, 32, 64, 36
NW = H * IN + H + 14 * K * H + 14 * K
W1, B1, W2, B2 = 0, H * IN, H * IN + H, H * IN + H + 14 * K * H
BANDS = (10.0, 25.0, 100.0, 500.0, math.inf)


def _anchors(n, seed, dist=(3.0, 8.0), level=0):
    rng = np.random.default_rng(seed)
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    d = rng.uniform(*dist, n)
    return dict(pos=dirs * d[:, None], level=np.full(n, level, np.int32), feat=rng.normal(0, 0.5, (n, F)),
                log_l=rng.normal(-1.0, 0.3, (n, 3)), offs=rng.normal(0, 1.0, (n, K, 3)))


def _weights(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, scale, NW)
    w[B1:B1 + H] = rng.uniform(0.05, 0.3, H)  # most hidden units active
    w[B2:] = rng.normal(0, 0.3, 14 * K)
    w[B2 + 3:B2 + 14 * K:14] = rng.uniform(0.2, 0.8, K)  # opacities mostly kept
    return w


def test_weights_layout():
    assert orc.anchor_num_weights() == NW == 11468


def test_closed_form_with_hidden_layer_off():
    A = _anchors(3, 1)
    w = np.zeros(NW)
    b2 = w[B2:].reshape(K, 14)
    b2[:, 3] = math.atanh(0.5)  # opacity 1/2: logit 0
    rows, keep, _ = orc.anchor_decode(A, w, np.zeros(3), BANDS)
    assert keep.all()
    r = rows.reshape(K, 3, 14)
    for k in range(K):
        for i in range(3):
            l = np.exp(A["log_l"][i])
            assert np.allclose(r[k, i, 0:3], A["pos"][i] + A["offs"][i, k] * l, atol=1e-14)
            assert np.allclose(r[k, i, 3:6], A["log_l"][i] + math.log(0.5), atol=1e-14)  # scale l / 2
            assert np.allclose(r[k, i, 6:10], [1, 0, 0, 0])  # identity rotation
            assert abs(r[k, i, 10]) < 1e-14 and np.allclose(r[k, i, 11:14], 0.0)  # colour 1/2
    # a negative opacity pre-activation drops every Gaussian: a culled placeholder
    b2[:, 3] = -0.1
    rows, keep, _ = orc.anchor_decode(A, w, np.zeros(3), BANDS)
    assert not keep.any() and np.all(rows[:, 10] == -30.0)


def test_lod_band_of_the_level():
    w = np.zeros(NW)
    w[B2 + 3:B2 + 14 * K:14] = 0.5
    A = dict(pos=np.array([[0.0, 0.0, 5.0], [0.0, 0.0, 15.0], [0.0, 0.0, 30.0], [0.0, 0.0, 9.999]]),
             level=np.array([1, 1, 1, 0], np.int32), feat=np.zeros((4, F)), log_l=np.zeros((4, 3)),
             offs=np.zeros((4, K, 3)))
    _, keep, unsure = orc.anchor_decode(A, w, np.zeros(3), BANDS, tol=1e-3)
    keep = keep.reshape(K, 4)
    # level 1 takes [10, 25): 5 and 30 are outside; level 0 takes [0, 10)
    assert list(keep[0]) == [False, True, False, True]
    assert unsure.reshape(K, 4)[0, 3] and not unsure.reshape(K, 4)[0, 1]


def test_view_direction_and_distance_inputs():
    # hidden unit 0 = relu(dir_x), unit 1 = relu(log(1 + d)); colour red of Gaussian 0 reads unit 0,
    # its opacity reads unit 1 with weight 1: a = tanh(log(1 + d))
    w = np.zeros(NW)
    w[W1 + 0 * IN + F + 0] = 1.0
    w[W1 + 1 * IN + F + 3] = 1.0
    w[W2 + 0 * H + 0] = 2.0
    w[W2 + 3 * H + 1] = 1.0
    w[B2 + 3 + 14:B2 + 14 * K:14] = 0.5  # the other Gaussians kept by their bias
    A = dict(pos=np.array([[3.0, 0.0, 4.0]]), level=np.zeros(1, np.int32), feat=np.zeros((1, F)),
             log_l=np.zeros((1, 3)), offs=np.zeros((1, K, 3)))
    rows, keep, _ = orc.anchor_decode(A, w, np.zeros(3), BANDS)
    a = math.tanh(math.log(6.0))  # d = 5
    assert keep[0] and abs(rows[0, 10] - math.log(a / (1 - a))) < 1e-12
    red = 1.0 / (1.0 + math.exp(-2.0 * 0.6))  # dir_x = 3/5
    assert abs(rows[0, 11] - (red - 0.5) / 0.28209479177387814) < 1e-12
    # seen from the other side the direction's x is negative: the unit is off, red = 1/2
    rows, _, _ = orc.anchor_decode(A, w, np.array([6.0, 0.0, 0.0]), BANDS)
    assert abs(rows[0, 11]) < 1e-15


def test_backward_matches_finite_differences():
    A = _anchors(4, 3)
    w = _weights(4)
    cc = np.array([0.3, -0.2, 0.1])
    rows, keep, _ = orc.anchor_decode(A, w, cc, BANDS)
    assert 0.3 < keep.mean() < 1.0
    rng = np.random.default_rng(5)
    G = rng.normal(size=rows.shape) * keep[:, None]  # the loss reads the kept Gaussians only
    gf, gl, go, gw = orc.anchor_decode_backward(A, w, cc, BANDS, G)

    def loss(A2, w2):
        r, k2, _ = orc.anchor_decode(A2, w2, cc, BANDS)
        assert np.array_equal(k2, keep)
        return float((r * G).sum())

    # h = 1e-5: large enough for FP64 rounding of sums ~10, small enough to cross no ReLU kink
    h = 1e-5
    for name, g in (("feat", gf), ("log_l", gl), ("offs", go)):
        fd = np.zeros_like(A[name])
        for idx in np.ndindex(A[name].shape):
            Ap, Am = {**A, name: A[name].copy()}, {**A, name: A[name].copy()}
            Ap[name][idx] += h
            Am[name][idx] -= h
            fd[idx] = (loss(Ap, w) - loss(Am, w)) / (2 * h)
        assert np.linalg.norm(fd - g) <= 1e-5 * np.linalg.norm(fd), name
    sel = rng.choice(NW, 400, replace=False)
    sel = np.concatenate([sel, np.arange(B2, NW)])  # every output bias
    fd = np.zeros(len(sel))
    for j, idx in enumerate(sel):
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd[j] = (loss(A, wp) - loss(A, wm)) / (2 * h)
    assert np.linalg.norm(fd - gw[sel]) <= 1e-5 * np.linalg.norm(fd)


def test_opacity_cull_never_changes_an_image():
    scene = scenes.uniform_scene(60, seed=12, sh_degree=0)
    cam = scenes.pinhole(64, 48, 60.0)
    cfg = orc.Cfg()
    base = orc.forward(scene, cam, cfg)
    seen = np.nonzero(base["proj"].arrays["radius"] > 0)[0]
    assert len(seen) >= 12
    faint = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    faint["opacity_logits"][seen[:10]] = -6.0    # sigmoid = 0.0025 < 1/255: culled
    faint["opacity_logits"][seen[10:12]] = -5.0  # 0.0067 > 1/255: kept
    f = orc.forward(faint, cam, cfg)
    rad = f["proj"].arrays["radius"]
    assert np.all(rad[seen[:10]] == 0) and np.all(rad[seen[10:12]] > 0)
    # the culled ones never blended: removing them leaves the image unchanged
    keep = np.ones(60, bool)
    keep[seen[:10]] = False
    rest = {k: (v[keep] if isinstance(v, np.ndarray) else v) for k, v in faint.items()}
    g = orc.forward(rest, cam, cfg)
    assert np.abs(f["img"] - g["img"]).max() < 1e-12


def _bf16(v):
    """Round to the nearest bfloat16 (ties to even) through float32 bits, independently of the oracle."""
    b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_mode_two_unit_closed_form():
    """Reading R30 by hand: two hidden units feed the opacity output of
    Gaussian 0.  In bfloat16 mode the forward multiplies rounded operands
    (input, W1, the hidden activation, W2) and sums exactly; the backward is
    the exact chain rule of that forward, with the rounded factors."""
    A = _anchors(1, 5)
    A["pos"] = np.array([[0.3, -0.2, 4.0]])
    w = np.zeros(NW)
    rng = np.random.default_rng(6)
    w[W1:W1 + IN] = rng.normal(0, 0.3, IN)            # unit 0 sees every input
    w[W1 + IN:W1 + 2 * IN] = rng.normal(0, 0.3, IN)   # unit 1 too
    w[B1], w[B1 + 1] = 0.7, 0.9
    w[W2 + 3 * H], w[W2 + 3 * H + 1] = 0.61, -0.27     # z[3] (opacity of Gaussian 0) = ...
    w[B2 + 3] = 0.4
    w[B2 + 3 + 14:B2 + 14 * K:14] = -1.0               # the other Gaussians dropped
    cam = np.zeros(3)
    rows, keep, _ = orc.anchor_decode(A, w, cam, BANDS, bf16=True)
    rows64, _, _ = orc.anchor_decode(A, w, cam, BANDS, bf16=False)
    v = A["pos"][0]
    d = np.linalg.norm(v)
    x = np.concatenate([A["feat"][0], v / d, [math.log1p(d)]])
    xb = _bf16(x)
    pre = np.array([w[B1 + u] + _bf16(w[W1 + u * IN:W1 + (u + 1) * IN]) @ xb for u in range(2)])
    assert np.all(pre > 0)
    hb = _bf16(pre)
    w2b = _bf16(w[W2 + 3 * H:W2 + 3 * H + 2])
    z3 = w[B2 + 3] + w2b @ hb
    a = math.tanh(z3)
    assert keep[0] and not keep[1:].any()
    assert abs(rows[0, 10] - math.log(a / (1 - a))) < 1e-12
    assert abs(rows[0, 10] - rows64[0, 10]) > 1e-6  # the rounding acts
    # backward of a loss = 2.5 x (opacity logit of Gaussian 0)
    g_rows = np.zeros_like(rows)
    g_rows[0, 10] = 2.5
    gf, gl, go, gw = orc.anchor_decode_backward(A, w, cam, BANDS, g_rows, bf16=True)
    dz3 = 2.5 * (1 + a) / a
    assert abs(gw[B2 + 3] - dz3) < 1e-12
    assert np.allclose(gw[W2 + 3 * H:W2 + 3 * H + 2], dz3 * hb, atol=1e-12)
    dp = dz3 * w2b
    assert np.allclose(gw[B1:B1 + 2], dp, atol=1e-12)
    for u in range(2):
        assert np.allclose(gw[W1 + u * IN:W1 + (u + 1) * IN], dp[u] * xb, atol=1e-12)
    w1b = np.stack([_bf16(w[W1 + u * IN:W1 + (u + 1) * IN]) for u in range(2)])
    assert np.allclose(gf[0], dp @ w1b[:, :F], atol=1e-12)


def test_bf16_mode_is_fp64_mode_on_bfloat16_values():
    """With inputs, weights and every hidden activation representable in
    bfloat16 (small dyadic values; the direction and distance inputs carry
    zero weight), the two modes decode identically and the feature and
    decoder-weight gradients agree to rounding."""
    A = _anchors(4, 7)
    rng = np.random.default_rng(8)
    A["feat"] = rng.integers(-4, 5, (4, F)) / 4.0
    w = np.zeros(NW)
    W1m = (rng.integers(-2, 3, (H, IN)) / 8.0)
    W1m[:, F:] = 0.0
    w[W1:W1 + H * IN] = W1m.ravel()
    w[B1:B1 + H] = rng.integers(0, 3, H) / 8.0
    w[W2:W2 + 14 * K * H] = rng.integers(-2, 3, 14 * K * H) / 64.0
    w[B2:] = rng.integers(-2, 3, 14 * K) / 8.0
    w[B2 + 3:B2 + 14 * K:14] = 0.5
    cam = np.zeros(3)
    r16, k16, _ = orc.anchor_decode(A, w, cam, BANDS, bf16=True)
    r64, k64, _ = orc.anchor_decode(A, w, cam, BANDS, bf16=False)
    assert np.array_equal(k16, k64) and k16.any()
    assert np.array_equal(r16, r64)
    g_rows = rng.normal(size=r16.shape)
    g16 = orc.anchor_decode_backward(A, w, cam, BANDS, g_rows, bf16=True)
    g64 = orc.anchor_decode_backward(A, w, cam, BANDS, g_rows, bf16=False)
    assert np.allclose(g16[0], g64[0], rtol=1e-12, atol=1e-12)  # features
    gw16, gw64 = g16[3], g64[3]
    feat_cols = np.zeros(NW, bool)
    feat_cols[W1:W1 + H * IN] = np.tile(np.arange(IN) < F, H)
    feat_cols[B1:] = True
    assert np.allclose(gw16[feat_cols], gw64[feat_cols], rtol=1e-12, atol=1e-12)


def test_hidden_inputs_and_pre_activations():
    """The decoder input is (feature, unit direction from the camera, log(1 + d))
    and the pre-activation is W1 x + b1 (a matrix product); in bf16 mode the
    pre-activation is that product over bfloat16-rounded x and W1, while the
    returned input stays unrounded."""
    A = _anchors(7, 31, dist=(2.0, 40.0))
    w = _weights(32)
    cc = np.array([0.3, -0.2, 0.1])
    x, pre = orc.anchor_hidden(A, w, cc)
    v = A["pos"] - cc
    d = np.linalg.norm(v, axis=1)
    assert np.array_equal(x[:, :F], A["feat"])
    assert np.allclose(x[:, F:F + 3], v / d[:, None], atol=1e-15)
    assert np.allclose(np.expm1(x[:, F + 3]), d, rtol=1e-13)
    W1m, b1 = w[W1:B1].reshape(H, IN), w[B1:B1 + H]
    assert np.allclose(pre, x @ W1m.T + b1, atol=1e-12)
    xb, preb = orc.anchor_hidden(A, w, cc, bf16=True)
    assert np.array_equal(xb, x)
    assert np.allclose(preb, _bf16(x) @ _bf16(W1m).T + b1, atol=1e-12)
    assert np.abs(preb - pre).max() > 1e-4  # the rounding is visible


def test_backward_row_terms_assemble_the_gradients():
    """The per-anchor dL/dz and dL/dpre the backward returns assemble its
    weight and feature gradients as matrix products: dW2 = dz^T relu(pre),
    db2 = sum dz, dW1 = dpre^T x, db1 = sum dpre, dfeat = dpre W1 (bf16 mode:
    with the rounded operands), and dpre vanishes where pre <= 0."""
    A = _anchors(9, 41)
    w = _weights(42)
    cc = np.array([0.1, 0.0, -0.2])
    rng = np.random.default_rng(43)
    g = rng.normal(size=(K * 9, 14))
    for bf16 in (False, True):
        gf, gl, go, gw, dz, dp = orc.anchor_decode_backward(A, w, cc, BANDS, g, bf16=bf16, rows=True)
        x, pre = orc.anchor_hidden(A, w, cc, bf16=bf16)
        r = _bf16 if bf16 else (lambda v: v)
        h = r(np.maximum(pre, 0.0))
        W1m = r(w[W1:B1].reshape(H, IN))
        assert np.abs(dz).max() > 0 and np.all(dp[pre <= 0] == 0)
        assert np.allclose(gw[W2:B2].reshape(14 * K, H), dz.T @ h, atol=1e-11)
        assert np.allclose(gw[B2:], dz.sum(0), atol=1e-11)
        assert np.allclose(gw[W1:B1].reshape(H, IN), dp.T @ r(x), atol=1e-11)
        assert np.allclose(gw[B1:B1 + H], dp.sum(0), atol=1e-11)
        assert np.allclose(gf, dp @ W1m[:, :F], atol=1e-11)
