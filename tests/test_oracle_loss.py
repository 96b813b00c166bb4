"""Pins of the oracle's photometric loss L = 0.8 L1 + 0.2 (1 - SSIM) (Supp. D.4,
reading R9): SSIM against scipy's 2D correlation, identical images, constant
images in the interior, the L1 gradient and finite differences of the full
gradient."""
import numpy as np
from scipy import signal

from paper_2606_30436_b300 import scenes


def _window():
    k = np.arange(-5, 6)
    g = np.exp(-k * k / (2 * 1.5 ** 2))
    g /= g.sum()
    return np.outer(g, g)


def _ssim_scipy(x, y, C1=0.01 ** 2, C2=0.03 ** 2):
    w = _window()
    out = np.zeros_like(x)
    for c in range(x.shape[0]):
        f = lambda a: signal.correlate2d(a, w, mode="same", boundary="fill", fillvalue=0.0)
        mx, my = f(x[c]), f(y[c])
        sxx, syy, sxy = f(x[c] * x[c]) - mx * mx, f(y[c] * y[c]) - my * my, f(x[c] * y[c]) - mx * my
        out[c] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return out


def test_ssim_matches_scipy(orc):
    x = scenes.smooth_image(23, 31, seed=1).astype(np.float64)
    y = scenes.smooth_image(23, 31, seed=2).astype(np.float64)
    assert np.abs(orc.ssim_map(x, y) - _ssim_scipy(x, y)).max() < 1e-12


def test_identical_images(orc):
    x = scenes.smooth_image(20, 24, seed=3).astype(np.float64)
    L, dL, ssim = orc.loss(x, x, 0.2)
    assert abs(ssim - 1.0) < 1e-14 and abs(L) < 1e-14
    assert np.abs(dL).max() < 1e-14


def test_constant_images_interior(orc):
    a, b = 0.3, 0.7
    x, y = np.full((3, 30, 30), a), np.full((3, 30, 30), b)
    m = orc.ssim_map(x, y)
    ref = (2 * a * b + 0.01 ** 2) / (a * a + b * b + 0.01 ** 2)
    # E[x^2] - mu^2 cancels to ~1e-16, divided by C2 = 9e-4
    assert np.abs(m[:, 5:-5, 5:-5] - ref).max() < 1e-11


def test_l1_gradient(orc):
    x = scenes.smooth_image(10, 12, seed=4).astype(np.float64)
    y = scenes.smooth_image(10, 12, seed=5).astype(np.float64)
    L, dL, _ = orc.loss(x, y, 0.0)
    assert abs(L - np.abs(x - y).mean()) < 1e-15
    assert np.array_equal(dL, np.sign(x - y) / x.size)


def test_loss_gradient_fd(orc):
    rng = np.random.default_rng(6)
    x = scenes.smooth_image(14, 17, seed=6).astype(np.float64)
    y = scenes.smooth_image(14, 17, seed=7).astype(np.float64)
    L, dL, _ = orc.loss(x, y, 0.2)
    h = 1e-6
    idx = [tuple(rng.integers(0, s) for s in x.shape) for _ in range(60)]
    idx += [(0, 0, 0), (2, 13, 16), (1, 0, 16)]  # corners: zero padding
    fd, an = [], []
    for i in idx:
        if abs(x[i] - y[i]) < 1e-4:
            continue  # |x - y| kink
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd.append((orc.loss(xp, y, 0.2, grad=False)[0] - orc.loss(xm, y, 0.2, grad=False)[0]) / (2 * h))
        an.append(dL[i])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) / np.linalg.norm(an) < 1e-6
