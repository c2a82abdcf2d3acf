"""Centred finite differences on a uniform periodic grid (Sec. 2.1: "high-order centered
finite-difference approximation for differential operators").

The paper names neither the order nor the weights.  Order 12 (radius 6) is used; the
weights are the standard centred second-derivative formula
    w_k = 2 (-1)^(k+1) (p!)^2 / (k^2 (p-k)! (p+k)!),   w_0 = -2 sum_{k>=1} w_k,
so that u''(x) ~ sum_{r=-p..p} w_|r| u(x + r h) / h^2.

Pinned by tests/test_oracle_fd.py (exact rationals, Taylor moments, empty-lattice symbol).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

FD_RADIUS = 6


def fd_weights_exact(p: int = FD_RADIUS) -> list:
    """Second-derivative weights w_0..w_p as exact fractions."""
    w = [Fraction(0)] * (p + 1)
    for k in range(1, p + 1):
        w[k] = Fraction(2 * (-1) ** (k + 1) * factorial(p) ** 2,
                        k * k * factorial(p - k) * factorial(p + k))
    w[0] = -2 * sum(w[1:])
    return w


def fd_weights(p: int = FD_RADIUS) -> np.ndarray:
    return np.array([float(x) for x in fd_weights_exact(p)])


def bloch_pad(u: np.ndarray, axis: int, p: int, phase: complex) -> np.ndarray:
    """Extend u by p ghost layers on both sides of `axis` using the Bloch condition
    u(x + L e_d) = phase * u(x) (phase = 1 for periodic, Sec. 2: Bloch-periodic BCs)."""
    n = u.shape[axis]
    idx = np.arange(-p, n + p)
    src = np.mod(idx, n)
    wraps = np.floor_divide(idx, n)
    v = np.take(u, src, axis=axis)
    if phase != 1.0:
        shape = [1] * u.ndim
        shape[axis] = idx.size
        v = v * (np.asarray(phase, complex) ** wraps).reshape(shape)
    return v


def laplacian(u: np.ndarray, h: tuple, phases=(1.0, 1.0, 1.0), p: int = FD_RADIUS,
              dirichlet: bool = False) -> np.ndarray:
    """(L_h u)(x) = sum_d sum_{r=-p..p} w_|r| u(x + r h_d e_d) / h_d^2.

    u has shape (..., n3, n2, n1) with x (d = 0) the last axis.  phases[d] is the Bloch
    factor exp(i k_d L_d) applied when a shift wraps around the cell along d.  dirichlet: u is zero
    outside the grid (isolated systems) instead of periodic."""
    w = fd_weights(p)
    out = np.zeros_like(u, dtype=np.result_type(u, *[np.asarray(ph) for ph in phases]))
    for d in range(3):
        axis = u.ndim - 1 - d
        n = u.shape[axis]
        if dirichlet:
            widths = [(0, 0)] * u.ndim
            widths[axis] = (p, p)
            pad = np.pad(u, widths)
        else:
            pad = bloch_pad(u, axis, p, phases[d])
        acc = w[0] * u

        def sl(a, b):
            s = [slice(None)] * u.ndim
            s[axis] = slice(a, b)
            return tuple(s)

        for r in range(1, p + 1):
            acc = acc + w[r] * (pad[sl(p + r, p + r + n)] + pad[sl(p - r, p - r + n)])
        out = out + acc / (h[d] * h[d])
    return out


def laplacian_symbol(n: tuple, h: tuple, kred=(0.0, 0.0, 0.0), p: int = FD_RADIUS) -> np.ndarray:
    """Eigenvalues of L_h on plane waves exp(i (2 pi m/L + k) x):
    sum_d (w_0 + 2 sum_r w_r cos(r theta_d)) / h_d^2, theta_d = 2 pi (m_d + kred_d) / n_d.
    Returned with shape (n3, n2, n1), m_d in FFT order."""
    w = fd_weights(p)
    sym = []
    for d in range(3):
        m = np.fft.fftfreq(n[d]) * n[d]
        th = 2.0 * np.pi * (m + kred[d]) / n[d]
        s = w[0] + 2.0 * sum(w[r] * np.cos(r * th) for r in range(1, p + 1))
        sym.append(s / (h[d] * h[d]))
    return sym[2][:, None, None] + sym[1][None, :, None] + sym[0][None, None, :]
