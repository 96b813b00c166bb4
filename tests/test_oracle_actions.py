"""Pins of the oracle's predictor inputs and densify / prune actions against
closed forms, library routines (boolean masking, scipy's rotation) and sample
statistics, independent of the oracle's own arithmetic."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as orc


def _rows(n, K_row, seed):
    rng = np.random.default_rng(seed)
    P = rng.normal(size=(n, K_row))
    P[:, 3:6] = rng.normal(-3.0, 0.5, size=(n, 3))
    return P


def test_features_closed_forms():
    n = 3
    means = np.array([[3.0, 4.0, 0.0], [1.0, 2.0, 2.0], [0.0, 0.0, 0.0]]) + np.array([1.0, 1.0, 1.0])
    ls = np.array([[-1.0, -2.0, -3.0], [0.0, 0.5, 1.0], [2.0, 2.0, 2.0]])
    logit = np.array([0.0, np.log(3.0), -np.log(3.0)])
    stats = np.zeros((n, 6))
    stats[:, 0] = [40.0, 0.0, 7.0]   # |Omega| summed over views
    stats[:, 4] = [1e-4, 0.0, 2e-4]  # accumulated ||dL/d(u,v)||
    stats[:, 5] = [4.0, 0.0, 1.0]    # views seen
    ring = np.tile(np.arange(8.0)[:, None], (1, n)) + 0.1 * np.arange(n)[None, :]
    f = orc.mlp_features(means, ls, logit, stats, ring, 2, [1.0, 1.0, 1.0])
    assert f.shape == (n, 16)
    assert np.allclose(f[:, 0], [0.5, 0.75, 0.25], atol=1e-15)
    assert np.array_equal(f[:, 1:4], ls)
    assert np.allclose(f[:, 4], np.log([5.0, 1.0, 2.0]), atol=1e-15)
    assert np.allclose(f[:, 5], np.log([2.0, 1.0, 3.0]), atol=1e-15)
    # most recent slot first: head 2 -> slots 2, 1, 0, 7, 6, 5, 4, 3
    assert np.allclose(f[0, 6:14], [2, 1, 0, 7, 6, 5, 4, 3])
    assert np.allclose(f[2, 6:14], np.array([2, 1, 0, 7, 6, 5, 4, 3]) + 0.2)
    assert np.allclose(f[:, 14], np.log([6.0, 4.0, 1.0]), atol=1e-15)
    # mean |Omega_v| = 40 / 4, and a Gaussian never seen has mean 0
    assert np.allclose(f[:, 15], np.log([11.0, 1.0, 8.0]), atol=1e-15)


def test_actions_counts_and_order_without_densify():
    rng = np.random.default_rng(1)
    n, K = 500, 59
    P = _rows(n, K, 2)
    prune = rng.random(n) < 0.3
    dens = np.zeros(n, bool)
    m, v = rng.normal(size=(n, K)), rng.random((n, K))
    Po, mo, vo, need = orc.densify_prune(P, dens, prune, np.zeros((n, 6)), 10.0, m=m, v=v)
    assert need == int((~prune).sum())
    assert np.array_equal(Po, P[~prune]) and np.array_equal(mo, m[~prune]) and np.array_equal(vo, v[~prune])


def test_actions_clone_and_split_rows():
    n, K = 6, 14
    P = _rows(n, K, 3)
    P[:, 3:6] = [[-1.0, -4.0, -4.0], [-4.0, -4.0, -4.0], [-4.0, -4.0, -0.5]] * 2
    dens = np.array([1, 1, 1, 0, 1, 0], np.uint8)
    prune = np.array([0, 0, 0, 0, 1, 1], np.uint8)
    m = np.full((n, K), 7.0)
    Po, mo, _, need = orc.densify_prune(P, dens, prune, np.zeros((n, 6)), -2.0, 1.6, m=m)
    # counts 2, 2, 2, 1, 0, 0
    assert need == 7 and Po.shape == (7, K)
    # Gaussian 1 (max log-scale -4 <= -2) is cloned: two identical rows, moments on the first only
    assert np.array_equal(Po[2], P[1]) and np.array_equal(Po[3], P[1])
    assert np.all(mo[2] == 7.0) and np.all(mo[3] == 0.0)
    # Gaussians 0 and 2 are split; zero noise puts both children at the mean, scales / 1.6
    for o, i in ((0, 0), (1, 0), (4, 2), (5, 2)):
        assert np.array_equal(Po[o, :3], P[i, :3])
        assert np.allclose(np.exp(Po[o, 3:6]), np.exp(P[i, 3:6]) / 1.6, rtol=1e-14)
        assert np.array_equal(Po[o, 6:], P[i, 6:])
        assert np.all(mo[o] == 0.0)
    assert np.array_equal(Po[6], P[3]) and np.all(mo[6] == 7.0)


def test_split_children_sample_the_gaussian():
    # children mu + R S xi with xi ~ N(0, I) have covariance R S^2 R^T; R from scipy's
    # rotation of the (w, x, y, z) quaternion, so a transposed R or a swapped scale fails
    n, K = 20000, 11
    q = np.array([0.8, 0.3, -0.4, 0.2])
    row = np.concatenate([[1.0, -2.0, 3.0], np.log([0.5, 0.1, 0.02]), q, [0.0]])
    P = np.tile(row, (n, 1))
    rng = np.random.default_rng(4)
    xi = rng.normal(size=(n, 6))
    Po, _, _, need = orc.densify_prune(P, np.ones(n), np.zeros(n), xi, -3.0, 1.6)
    assert need == 2 * n
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sigma = R @ np.diag([0.25, 0.01, 0.0004]) @ R.T
    d = Po[:, :3] - row[:3]
    C = d.T @ d / d.shape[0]
    assert np.abs(C - Sigma).max() < 0.02 * np.abs(Sigma).max()
    # both children of one parent use their own noise: first child of row 0 is mu + R S xi_0
    assert np.allclose(Po[0, :3], row[:3] + R @ (np.array([0.5, 0.1, 0.02]) * xi[0, :3]), atol=1e-12)
    assert np.allclose(Po[1, :3], row[:3] + R @ (np.array([0.5, 0.1, 0.02]) * xi[0, 3:]), atol=1e-12)


@pytest.mark.parametrize("cap", [0, 1, 5, 12])
def test_actions_capacity_keeps_prefix(cap):
    n, K = 10, 11
    P = _rows(n, K, 5)
    dens = np.array([1, 0, 1, 0, 0, 1, 1, 0, 0, 1], np.uint8)
    prune = np.array([0, 1, 0, 0, 0, 0, 1, 0, 0, 0], np.uint8)
    full, _, _, need = orc.densify_prune(P, dens, prune, np.ones((n, 6)), -2.5)
    part, _, _, need2 = orc.densify_prune(P, dens, prune, np.ones((n, 6)), -2.5, cap=cap)
    assert need == need2 == 12
    assert np.array_equal(part, full[:cap])
