"""Pins for oracle.fd: exact weights, Taylor moments, plane-wave symbol, analytic derivatives."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fd

pytestmark = pytest.mark.filterwarnings("ignore")


def test_weights_match_published_rationals():
    # Order-12 centred second-derivative weights (Fornberg 1988 tables).
    expected = [Fraction(-5369, 1800), Fraction(12, 7), Fraction(-15, 56), Fraction(10, 189),
                Fraction(-1, 112), Fraction(2, 1925), Fraction(-1, 16632)]
    assert fd.fd_weights_exact(6) == expected


@pytest.mark.parametrize("p", [1, 2, 3, 6])
def test_weights_taylor_moments(p):
    # sum_r w_|r| r^(2j) = 2 for j = 1 and 0 for every other j <= p: the unique order-2p stencil.
    w = fd.fd_weights_exact(p)
    for j in range(0, p + 1):
        m = sum((w[abs(r)] * Fraction(r) ** (2 * j) for r in range(-p, p + 1)), Fraction(0))
        assert m == (2 if j == 1 else 0), (j, m)
    if p == 1:
        assert w == [Fraction(-2), Fraction(1)]


def test_laplacian_of_smooth_function_matches_analytic_derivative():
    # u = sin(2 pi x/L) cos(4 pi y/L) exp(sin(2 pi z/L)): order-12 FD error ~ (k h)^12.
    n, L = (40, 36, 32), (6.0, 6.0, 6.0)
    h = tuple(L[d] / n[d] for d in range(3))
    x, y, z = [np.arange(n[d]) * h[d] for d in range(3)]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    k = 2 * np.pi / 6.0
    u = np.sin(k * X) * np.cos(2 * k * Y) * np.exp(np.sin(k * Z))
    ez = np.exp(np.sin(k * Z))
    d2z = ez * (k * k * np.cos(k * Z) ** 2 - k * k * np.sin(k * Z))
    exact = (-k * k - 4 * k * k) * u + np.sin(k * X) * np.cos(2 * k * Y) * d2z
    got = fd.laplacian(u, h)
    assert np.max(np.abs(got - exact)) < 1e-7 * np.max(np.abs(exact))


def test_bloch_plane_wave_eigenfunction():
    # exp(i (2 pi (m + kappa)/L) . x) with the Bloch wrap phase exp(2 pi i kappa) is an
    # eigenfunction; its eigenvalue tends to -|G + k|^2 with order-12 accuracy.
    n = (12, 10, 14)
    L = (5.0, 4.0, 6.0)
    h = tuple(L[d] / n[d] for d in range(3))
    kappa = (0.25, -0.375, 0.5)
    m = (1, 0, -2)
    x, y, z = [np.arange(n[d]) * h[d] for d in range(3)]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    G = [2 * np.pi * (m[d] + kappa[d]) / L[d] for d in range(3)]
    u = np.exp(1j * (G[0] * X + G[1] * Y + G[2] * Z))
    ph = tuple(np.exp(2j * np.pi * kk) for kk in kappa)
    lu = fd.laplacian(u, h, ph)
    ratio = lu / u
    assert np.allclose(ratio, ratio.flat[0], rtol=0, atol=1e-10)
    cont = -sum(g * g for g in G)
    assert abs(ratio.flat[0].real - cont) < 1e-4 * abs(cont)
    assert abs(ratio.flat[0].imag) < 1e-10
