"""Pins of the oracle's prune / densify MLP: closed forms (zero hidden
weights; a one-unit network), central finite differences of the mean BCE in
FP64 for every weight block, and the bfloat16 rounding of operands."""
import math

import numpy as np


def _w(orc, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, orc.mlp_num_weights())


def test_layout_and_zero_hidden(orc):
    assert orc.mlp_num_weights() == 64 * 16 + 64 + 64 * 64 + 64 + 2 * 64 + 2
    w = np.zeros(orc.mlp_num_weights())
    w[-2:] = [0.7, -1.2]  # b3
    x = np.random.default_rng(0).standard_normal((5, 16))
    p, h1, h2 = orc.mlp_forward(x, w, bf16=False)
    assert np.allclose(p, 1 / (1 + np.exp(-np.array([0.7, -1.2]))), atol=0)
    assert np.all(h1 == 0) and np.all(h2 == 0)


def test_one_unit_closed_form(orc):
    """Only unit 0 of each layer connected: p = sigmoid(w3 relu(w2 relu(w1 . x + b1) + b2) + b3)."""
    n = orc.mlp_num_weights()
    w = np.zeros(n)
    W1, B1, W2, B2, W3, B3 = 0, 1024, 1088, 5184, 5248, 5376
    w[W1:W1 + 16] = np.linspace(-0.5, 0.5, 16)
    w[B1] = 0.1
    w[W2] = 1.5
    w[B2] = -0.2
    w[W3] = 2.0
    w[W3 + 64] = -1.0
    w[B3:B3 + 2] = [0.3, 0.4]
    x = np.random.default_rng(1).standard_normal((7, 16))
    p, _, _ = orc.mlp_forward(x, w, bf16=False)
    a = np.maximum(x @ w[W1:W1 + 16] + 0.1, 0)
    b = np.maximum(1.5 * a - 0.2, 0)
    ref = 1 / (1 + np.exp(-np.stack([2.0 * b + 0.3, -1.0 * b + 0.4], 1)))
    assert np.abs(p - ref).max() < 1e-15


def test_bce_gradient_fd(orc):
    rng = np.random.default_rng(2)
    w = _w(orc, 3)
    x = rng.standard_normal((40, 16))
    y = (rng.uniform(size=(40, 2)) < 0.4).astype(float)
    L, g = orc.mlp_bce_grad(x, y, w, bf16=False)
    p, _, _ = orc.mlp_forward(x, w, bf16=False)
    ref = -np.mean(y * np.log(p) + (1 - y) * np.log(1 - p))
    assert abs(L - ref) < 1e-14
    h = 1e-6
    idx = [0, 5, 1023, 1024, 1030, 1088, 2000, 5183, 5184, 5200, 5248, 5300, 5376, 5377]
    fd = []
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd.append((orc.mlp_bce_grad(x, y, wp, bf16=False)[0] - orc.mlp_bce_grad(x, y, wm, bf16=False)[0]) / (2 * h))
    fd = np.array(fd)
    assert np.linalg.norm(fd - g[idx]) <= 1e-7 * np.linalg.norm(g[idx])


def test_bf16_rounding(orc):
    """bfloat16 mode differs from FP64 mode only through the rounding of the
    tensor-core operands: a weight of 1 + 2^-9 (below the midpoint between the
    bf16 neighbours 1 and 1 + 2^-7) acts as exactly 1 in bf16 mode."""
    n = orc.mlp_num_weights()
    w = np.zeros(n)
    w[0] = 1.0 + 2 ** -9  # W1[0][0]
    w[1088] = 1.0         # W2[0][0]
    w[5248] = 1.0         # W3[0][0]
    x = np.zeros((1, 16))
    x[0, 0] = 1.0
    pb, _, _ = orc.mlp_forward(x, w, bf16=True)
    pf, _, _ = orc.mlp_forward(x, w, bf16=False)
    assert abs(pb[0, 0] - 1 / (1 + math.exp(-1.0))) < 1e-15
    assert abs(pf[0, 0] - 1 / (1 + math.exp(-(1.0 + 2 ** -9)))) < 1e-15
    # above the midpoint it rounds up to 1 + 2^-7
    w[0] = 1.0 + 3 * 2 ** -9
    pb, _, _ = orc.mlp_forward(x, w, bf16=True)
    assert abs(pb[0, 0] - 1 / (1 + math.exp(-(1.0 + 2 ** -7)))) < 1e-15


def _bf16(v):
    """Round to the nearest bfloat16 (ties to even) through float32 bits, independently of the oracle."""
    b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_gradient_one_unit_closed_form(orc):
    """One connected unit per layer and one row: in bfloat16 mode the
    forward multiplies rounded operands (x, W1, W2, h1) and the backward is
    the exact chain rule of that forward, written out by hand here: the
    gradient of a rounded operand's product uses the rounded factor it was
    multiplied by, and no backward quantity is rounded."""
    n = orc.mlp_num_weights()
    W1, B1, W2, B2, W3, B3 = 0, 1024, 1088, 5184, 5248, 5376
    w = np.zeros(n)
    w[W1:W1 + 16] = np.linspace(-0.31, 0.47, 16)
    w[B1] = 0.113
    w[W2] = 1.37
    w[B2] = -0.071
    w[W3], w[W3 + 64] = 1.93, -0.87
    w[B3:B3 + 2] = [0.3, -0.2]
    x = (np.linspace(0.2, 1.1, 16) + 0.01 * np.random.default_rng(3).standard_normal(16))[None, :]
    y = np.array([[1.0, 0.0]])
    L, g, dh2_rows, dh1_rows = orc.mlp_bce_grad(x, y, w, bf16=True, rows=True)
    scale = 1.0 / 2.0  # one row, two outputs
    xb, w1b, w2b = _bf16(x[0]), _bf16(w[W1:W1 + 16]), _bf16(w[W2])
    h1 = max(xb @ w1b + w[B1], 0.0)
    h2 = max(w2b * _bf16(h1) + w[B2], 0.0)
    assert h1 > 0.1 and h2 > 0.1  # both units active
    assert _bf16(h1) != h1 and w2b != w[W2]  # the forward's rounding acts
    z = np.array([w[W3] * h2 + w[B3], w[W3 + 64] * h2 + w[B3 + 1]])
    p = 1 / (1 + np.exp(-z))
    assert abs(L - (-np.log(p[0]) - np.log(1 - p[1])) * scale) <= 1e-15
    dz = (p - y[0]) * scale
    assert np.abs(g[B3:B3 + 2] - dz).max() <= 1e-16 and abs(g[W3] - dz[0] * h2) <= 1e-16
    dh2 = dz[0] * w[W3] + dz[1] * w[W3 + 64]
    assert abs(g[B2] - dh2) <= 1e-16 and abs(g[W2] - dh2 * _bf16(h1)) <= 1e-16
    dh1 = dh2 * w2b
    assert abs(g[B1] - dh1) <= 1e-16
    assert np.abs(g[W1:W1 + 16] - dh1 * xb).max() <= 1e-16
    assert abs(dh2_rows[0, 0] - dh2) <= 1e-16 and abs(dh1_rows[0, 0] - dh1) <= 1e-16
    assert np.all(dh2_rows[0, 1:] == 0) and np.all(dh1_rows[0, 1:] == 0)


def test_bf16_output_layer_finite_differences(orc):
    """The parameters the bfloat16 forward does not round and that feed no
    rounded operand (b2, W3, b3) have their exact derivatives in bfloat16
    mode: central differences of the bfloat16-mode loss agree."""
    rng = np.random.default_rng(12)
    w = _w(orc, 13)
    x = rng.standard_normal((30, 16))
    y = (rng.uniform(size=(30, 2)) < 0.5).astype(float)
    _, g = orc.mlp_bce_grad(x, y, w, bf16=True)
    h = 1e-6
    idx = [5184, 5190, 5247, 5248, 5290, 5375, 5376, 5377]
    fd = []
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd.append((orc.mlp_bce_grad(x, y, wp, bf16=True)[0] - orc.mlp_bce_grad(x, y, wm, bf16=True)[0]) / (2 * h))
    fd = np.array(fd)
    assert np.linalg.norm(fd - g[idx]) <= 1e-7 * np.linalg.norm(g[idx])
