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
