"""Pins of the oracle's real spherical harmonics (reading R6): orthonormality on
the sphere by quadrature, agreement with scipy's complex spherical harmonics,
the degree-0 constant, and finite differences of the Cartesian derivatives."""
import math

import numpy as np
import pytest
from scipy import special


def _dirs_quadrature(nt=24, nphi=48):
    # Gauss-Legendre in cos(theta), uniform in phi: exact for polynomials of degree <= 2*nt-1
    x, w = np.polynomial.legendre.leggauss(nt)
    phi = np.arange(nphi) * 2 * math.pi / nphi
    dirs, wts = [], []
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for p in phi:
            dirs.append((st * math.cos(p), st * math.sin(p), ct))
            wts.append(wt * 2 * math.pi / nphi)
    return np.array(dirs), np.array(wts)


def test_sh_orthonormal(orc):
    D = 3
    dirs, wts = _dirs_quadrature()
    Y = np.stack([orc.sh_eval(D, d)[0] for d in dirs])
    G = (Y * wts[:, None]).T @ Y
    assert np.abs(G - np.eye((D + 1) ** 2)).max() < 1e-12


def test_sh_degree0_constant(orc):
    Y, dY = orc.sh_eval(0, np.array([0.3, -0.4, math.sqrt(1 - 0.25)]))
    assert abs(Y[0] - 1.0 / (2.0 * math.sqrt(math.pi))) < 1e-15
    assert np.all(dY == 0)


def test_sh_matches_scipy(orc):
    """real Y_l^m = sqrt(2) Re Y_l^m (m > 0), sqrt(2) Im Y_l^|m| (m < 0), Y_l^0,
    with scipy's complex harmonics (Condon-Shortley phase included)."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y, _ = orc.sh_eval(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                yc = special.sph_harm_y(l, abs(m), theta, phi)
                ref = yc.real if m == 0 else math.sqrt(2) * (yc.real if m > 0 else yc.imag)
                assert abs(Y[l * l + l + m] - ref) < 1e-12, (l, m)


def test_sh_derivative_fd(orc):
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        d = rng.standard_normal(3)
        _, dY = orc.sh_eval(3, d)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (orc.sh_eval(3, d + e)[0] - orc.sh_eval(3, d - e)[0]) / (2 * h)
            assert np.abs(fd - dY[:, a]).max() < 1e-7
