"""GGA exchange-correlation: PBE, spin-unpolarized (test infrastructure: only tests/, the smoke
check and the benchmark's CPU baseline may use the oracle).

The paper's code offers GGA (PBE) beside LDA (Sec. 2.2 functionalities; the TiO2, MoS2 and Co runs of
Sec. 3).  Definitions (J. P. Perdew, K. Burke, M. Ernzerhof, Phys. Rev. Lett. 77, 3865 (1996)):

    f(rho, sigma) = rho [eps_x^unif(rho) F_x(s) + eps_c^PW92(r_s) + H(r_s, t)],   sigma = |grad rho|^2
    F_x = 1 + kappa - kappa / (1 + mu s^2 / kappa),      s = |grad rho| / (2 k_F rho)
    H   = gamma ln(1 + (beta/gamma) t^2 (1 + A t^2) / (1 + A t^2 + A^2 t^4)),
    A   = (beta/gamma) / (exp(-eps_c^PW92 / gamma) - 1),  t = |grad rho| / (2 k_s rho)
    k_F = (3 pi^2 rho)^(1/3),  k_s = (4 k_F / pi)^(1/2),  gamma = (1 - ln 2)/pi^2,
    beta = 0.06672455060314922,  mu = beta pi^2 / 3,  kappa = 0.804,
with eps_c^PW92 the Perdew-Wang 1992 fit (Phys. Rev. B 45, 13244, Eq. 10, unpolarized row).

Discretisation (the same order-12 centred stencils as the Laplacian, periodic): D_d is the order-12
first-derivative stencil along axis d, sigma_g = sum_d (D_d rho)_g^2 and

    E_xc = dV sum_g f(rho_g, sigma_g),
    v_xc = (1/dV) dE_xc/drho_g = f_rho - 2 sum_d D_d (f_sigma D_d rho)       (D_d^T = -D_d),

the exact derivative of the discrete energy.  f_rho and f_sigma are taken by complex-step
differentiation of f (Im f(x + i h) / h with h = 1e-30: exact to rounding, no cancellation), so the
functional is written down once.  The density is floored at 1e-14 inside this module only.

Pinned by tests/test_oracle_gga.py: first-derivative weights (Taylor moments, plane-wave symbol),
the uniform-gas limit (LDA exchange + PW92 correlation), the gradient-expansion limit H / t^2 -> beta,
the large-gradient limits F_x -> 1 + kappa and H -> -eps_c, the high-density PW92 coefficient, PW92
against the independent PZ81 fit of the same data, the complex-step derivatives against central
differences, and v_xc against finite differences of the discrete E_xc on a small grid.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

from . import fd

RHO_FLOOR = 1e-14
KAPPA = 0.804
BETA = 0.06672455060314922
MU = BETA * np.pi ** 2 / 3.0
GAMMA = (1.0 - np.log(2.0)) / np.pi ** 2
# PW92 unpolarized: A, alpha1, beta1..beta4
PW92_U = (0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294)
_H = 1e-30   # complex step


def d1_weights_exact(p: int = fd.FD_RADIUS) -> list:
    """Centred first-derivative weights c_1..c_p: u'(x) ~ sum_k c_k (u(x + k h) - u(x - k h)) / h,
    c_k = (-1)^(k+1) (p!)^2 / (k (p-k)! (p+k)!)."""
    return [Fraction((-1) ** (k + 1) * factorial(p) ** 2, k * factorial(p - k) * factorial(p + k))
            for k in range(1, p + 1)]


def d1_weights(p: int = fd.FD_RADIUS) -> np.ndarray:
    return np.array([float(x) for x in d1_weights_exact(p)])


def derivative(cell, u: np.ndarray, axis_d: int) -> np.ndarray:
    """(D_d u) on the periodic grid, u of shape (ngrid,) (x fastest) -> (ngrid,)."""
    n1, n2, n3 = cell.n
    g = u.reshape(n3, n2, n1)
    ax = 2 - axis_d
    c = d1_weights()
    out = np.zeros_like(g)
    for k in range(1, len(c) + 1):
        out = out + c[k - 1] * (np.roll(g, -k, axis=ax) - np.roll(g, k, axis=ax))
    return (out / cell.h[axis_d]).reshape(-1)


def pw92(rs):
    A, a1, b1, b2, b3, b4 = PW92_U
    s = np.sqrt(rs)
    q = 2.0 * A * (b1 * s + b2 * rs + b3 * rs * s + b4 * rs * rs)
    return -2.0 * A * (1.0 + a1 * rs) * np.log(1.0 + 1.0 / q)


def pbe_parts(rho, sigma):
    """(eps_x^unif, F_x, eps_c^PW92, H) for arrays (real or complex) rho > 0, sigma >= 0."""
    kf = (3.0 * np.pi ** 2 * rho) ** (1.0 / 3.0)
    ex_unif = -3.0 * kf / (4.0 * np.pi)
    s2 = sigma / (4.0 * kf * kf * rho * rho)
    fx = 1.0 + KAPPA - KAPPA / (1.0 + MU * s2 / KAPPA)
    rs = (3.0 / (4.0 * np.pi * rho)) ** (1.0 / 3.0)
    ec = pw92(rs)
    ks2 = 4.0 * kf / np.pi
    t2 = sigma / (4.0 * ks2 * rho * rho)
    A = (BETA / GAMMA) / (np.exp(-ec / GAMMA) - 1.0)
    y = A * t2
    H = GAMMA * np.log(1.0 + (BETA / GAMMA) * t2 * (1.0 + y) / (1.0 + y + y * y))
    return ex_unif, fx, ec, H


def pbe_f(rho, sigma):
    """Energy density per volume f = rho eps_xc(rho, sigma)."""
    ex_unif, fx, ec, H = pbe_parts(rho, sigma)
    return rho * (ex_unif * fx + ec + H)


def pbe_point(rho, sigma):
    """(eps_xc, f_rho, f_sigma) per grid point; derivatives by complex step."""
    rho = np.maximum(np.asarray(rho, float), RHO_FLOOR)
    sigma = np.asarray(sigma, float)
    f = pbe_f(rho, sigma)
    f_rho = np.imag(pbe_f(rho + 1j * _H, sigma + 0j)) / _H
    f_sigma = np.imag(pbe_f(rho + 0j, sigma + 1j * _H)) / _H
    return f / rho, f_rho, f_sigma


def pbe_unpolarized(cell, rho):
    """(eps_xc per electron, v_xc) of the discrete PBE functional for a spin-unpolarized density."""
    rho = np.asarray(rho, float)
    grads = [derivative(cell, rho, d) for d in range(3)]
    sigma = sum(gd * gd for gd in grads)
    exc, f_rho, f_sigma = pbe_point(rho, sigma)
    v = f_rho.copy()
    for d in range(3):
        v -= 2.0 * derivative(cell, f_sigma * grads[d], d)
    return exc, v


def exc_energy(cell, rho):
    """E_xc = dV sum_g rho eps_xc (used by the pins)."""
    exc, _ = pbe_unpolarized(cell, rho)
    return float(np.prod(cell.h)) * float(np.dot(np.maximum(rho, RHO_FLOOR), exc))
