"""Pins of the PBE GGA oracle (oracle/gga.py) against facts that do not come from its own formulas:
Taylor moments of the first-derivative stencil, the known limits of the PBE functional, the PZ81 fit
of the same correlation data, central differences of its complex-step derivatives, and finite
differences of the discrete exchange-correlation energy for the potential."""
from fractions import Fraction

import numpy as np
import pytest

import workloads
from oracle import fd, gga, xc


def test_first_derivative_weights_taylor_moments():
    # sum_k c_k (k^m - (-k)^m) = [m == 1] for m = 1..2p (odd m only: even moments cancel by symmetry)
    c = gga.d1_weights_exact()
    for m in range(1, 2 * fd.FD_RADIUS + 1, 2):
        mom = sum(ck * 2 * Fraction(k) ** m for k, ck in enumerate(c, start=1))
        assert mom == (1 if m == 1 else 0)
    assert c[0] == Fraction(6, 7) and c[5] == Fraction(-1, 5544)


def test_derivative_of_plane_wave_matches_symbol():
    c = workloads.small_cell(npts=16, L=5.0)
    c.n = (16, 12, 10)
    c.L = (5.0, 4.0, 3.5)
    z, y, x = np.meshgrid(*[np.arange(c.n[d]) * c.h[d] for d in (2, 1, 0)], indexing="ij")
    for d, (m, coord) in enumerate(((3, x), (2, y), (1, z))):
        G = 2 * np.pi * m / c.L[d]
        u = np.sin(G * coord).reshape(-1)
        th = G * c.h[d]
        sym = 2 * sum(ck * np.sin((k + 1) * th) for k, ck in enumerate(gga.d1_weights())) / c.h[d]
        got = gga.derivative(c, u, d)
        assert np.max(np.abs(got - sym * np.cos(G * coord).reshape(-1))) < 1e-12
        assert abs(sym - G) < 0.2 * th ** 12 * G   # order-12 accuracy: relative error O(theta^12)


def test_uniform_gas_limit_is_lda_exchange_plus_pw92():
    rho = np.logspace(-4, 1, 25)
    exc, _, _ = gga.pbe_point(rho, np.zeros_like(rho))
    ex = xc.CX * np.cbrt(rho)
    rs = xc.wigner_seitz_radius(rho)
    assert np.max(np.abs(exc - ex - gga.pw92(rs))) < 1e-14


def test_exchange_enhancement_limits():
    ex_unif, fx, _, _ = gga.pbe_parts(np.array([0.1]), np.array([0.0]))
    assert abs(fx[0] - 1.0) < 1e-15
    _, fx, _, _ = gga.pbe_parts(np.array([0.1]), np.array([1e12]))
    assert abs(fx[0] - (1 + gga.KAPPA)) < 1e-6
    # small s: F_x = 1 + mu s^2 + O(s^4), mu = beta pi^2 / 3
    rho = 0.1
    kf = (3 * np.pi ** 2 * rho) ** (1 / 3)
    s2 = 1e-6
    _, fx, _, _ = gga.pbe_parts(np.array([rho]), np.array([s2 * 4 * kf * kf * rho * rho]))
    assert abs((fx[0] - 1.0) / s2 - gga.MU) < 1e-5
    assert abs(gga.MU - 0.2195149727645171) < 1e-15


def test_correlation_gradient_limits():
    rho = np.array([0.02, 0.2, 2.0])
    kf = (3 * np.pi ** 2 * rho) ** (1 / 3)
    ks2 = 4 * kf / np.pi

    def parts_at_t2(t2):
        return gga.pbe_parts(rho, t2 * 4 * ks2 * rho * rho)

    # gradient expansion: H -> beta t^2 (phi = 1) as t -> 0
    _, _, ec, H = parts_at_t2(1e-8)
    assert np.max(np.abs(H / 1e-8 - gga.BETA)) < 1e-5
    # large gradients: H -> -eps_c (correlation energy vanishes)
    _, _, ec, H = parts_at_t2(1e8)
    assert np.max(np.abs(H + ec)) < 1e-6 * np.max(np.abs(ec))
    assert abs(gga.GAMMA - 0.031090690869654895) < 1e-15


def test_pw92_high_density_coefficient_and_agreement_with_pz81():
    # eps_c -> A ln rs + const as rs -> 0, A = (1 - ln 2)/pi^2 (Gell-Mann-Brueckner)
    r1, r2 = 1e-6, 1e-5
    slope = (gga.pw92(r2) - gga.pw92(r1)) / (np.log(r2) - np.log(r1))
    assert abs(slope - (1 - np.log(2)) / np.pi ** 2) < 2e-4
    # PW92 and PZ81 fit the same Ceperley-Alder data independently: within 1.5 mHa
    rs = np.array([0.3, 0.7, 1.0, 2.0, 5.0, 10.0, 20.0])
    ez, _ = xc.pz_correlation(rs, xc.PZ_U)
    assert np.max(np.abs(gga.pw92(rs) - ez)) < 1.5e-3


def test_complex_step_derivatives_match_central_differences():
    rng = np.random.default_rng(3)
    rho = 10 ** rng.uniform(-3, 0.5, 30)
    # reduced gradients s^2 in [0.008, 0.8], where the gradient part of f is a sizeable fraction of f
    # (for tiny s a difference in sigma cancels to rounding; that limit is pinned analytically above)
    sigma = rho ** (8 / 3) * 10 ** rng.uniform(-0.5, 1.5, 30)
    _, f_rho, f_sigma = gga.pbe_point(rho, sigma)
    for which, d in ((0, 1e-4 * rho), (1, 1e-3 * sigma)):
        def f(t):
            return gga.pbe_f(rho + (t if which == 0 else 0), sigma + (t if which == 1 else 0))
        cd = (-f(2 * d) + 8 * f(d) - 8 * f(-d) + f(-2 * d)) / (12 * d)
        ref = f_rho if which == 0 else f_sigma
        assert np.max(np.abs(cd - ref) / np.abs(ref)) < 1e-7


def test_potential_is_derivative_of_discrete_energy():
    c = workloads.small_cell(npts=10, L=4.0, natom=1)
    c.n = (10, 9, 8)
    c.L = (4.0, 3.6, 3.2)
    rng = np.random.default_rng(4)
    z, y, x = np.meshgrid(*[np.arange(c.n[d]) * c.h[d] for d in (2, 1, 0)], indexing="ij")
    rho = (0.05 + 0.03 * np.cos(2 * np.pi * x / c.L[0]) * np.sin(2 * np.pi * y / c.L[1])
           + 0.01 * rng.uniform(size=x.shape)).reshape(-1)
    _, v = gga.pbe_unpolarized(c, rho)
    dV = float(np.prod(c.h))
    for g in rng.choice(c.ngrid, 8, replace=False):
        h = 1e-5 * rho[g]

        def e(t):
            r = rho.copy()
            r[g] += t
            return gga.exc_energy(c, r)

        fdv = (-e(2 * h) + 8 * e(h) - 8 * e(-h) + e(-2 * h)) / (12 * h) / dV
        assert abs(fdv - v[g]) < 1e-7 * max(1.0, abs(v[g]))
