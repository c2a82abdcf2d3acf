"""Pins for oracle.xc (Perdew-Zunger 1981 LDA)."""
import numpy as np
import pytest

from oracle import xc


def _pw92_g(rs, A, a1, b1, b2, b3, b4):
    # Perdew & Wang, PRB 45, 13244 (1992), Eq. 10 with p = 1: an independent fit of the
    # same Ceperley-Alder data that PZ81 parametrises.
    s = np.sqrt(rs)
    den = 2 * A * (b1 * s + b2 * rs + b3 * rs * s + b4 * rs * rs)
    return -2 * A * (1 + a1 * rs) * np.log1p(1.0 / den)


def test_high_density_coefficient_is_gell_mann_brueckner():
    # eps_c -> A ln rs + B as rs -> 0 with A = (1 - ln 2)/pi^2 (unpolarized), half of it polarized.
    a_gmb = (1 - np.log(2)) / np.pi ** 2
    assert abs(xc.PZ_U["A"] - a_gmb) < 1e-4
    assert abs(xc.PZ_P["A"] - a_gmb / 2) < 1e-4


@pytest.mark.parametrize("rs", [0.3, 0.7, 1.0, 1.5, 2.0, 3.0, 5.0, 8.0, 12.0, 20.0])
def test_correlation_agrees_with_pw92(rs):
    eu, _ = xc.pz_correlation(np.array([rs]), xc.PZ_U)
    ep, _ = xc.pz_correlation(np.array([rs]), xc.PZ_P)
    pu = _pw92_g(rs, 0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294)
    pp = _pw92_g(rs, 0.015545, 0.20548, 14.1189, 6.1977, 3.3662, 0.62517)
    assert abs(eu[0] - pu) < 1.5e-3
    assert abs(ep[0] - pp) < 1.5e-3


def test_continuity_at_rs_one():
    for c in (xc.PZ_U, xc.PZ_P):
        e, m = xc.pz_correlation(np.array([1 - 1e-12, 1 + 1e-12]), c)
        assert abs(e[0] - e[1]) < 1e-4
        assert abs(m[0] - m[1]) < 2e-3


def test_exchange_constants():
    # Dirac exchange: eps_x = -(3/4)(3 rho/pi)^(1/3); 0.7385587663820224 = (3/4)(3/pi)^(1/3).
    e, _ = xc.lda_pz_unpolarized(np.array([1.0]))
    ec, _ = xc.pz_correlation(xc.wigner_seitz_radius(np.array([1.0])), xc.PZ_U)
    assert abs((e[0] - ec[0]) + 0.7385587663820224) < 1e-14
    # Fully polarized exchange is 2^(1/3) times the unpolarized value at the same density.
    ep, _, _ = xc.lda_pz_polarized(np.array([1.0]), np.array([0.0]))
    ecp, _ = xc.pz_correlation(xc.wigner_seitz_radius(np.array([1.0])), xc.PZ_P)
    assert abs((ep[0] - ecp[0]) - 2 ** (1 / 3) * (e[0] - ec[0])) < 1e-13


def test_unpolarized_potential_is_derivative():
    rho = np.logspace(-5, 1.5, 40)
    d = 1e-6 * rho
    e_p, _ = xc.lda_pz_unpolarized(rho + d)
    e_m, _ = xc.lda_pz_unpolarized(rho - d)
    _, v = xc.lda_pz_unpolarized(rho)
    fd = ((rho + d) * e_p - (rho - d) * e_m) / (2 * d)
    assert np.max(np.abs(fd - v) / np.abs(v)) < 1e-7


def test_polarized_potential_is_derivative():
    rng = np.random.default_rng(0)
    ru = 10 ** rng.uniform(-4, 1, 50)
    rd = 10 ** rng.uniform(-4, 1, 50)
    e, vu, vd = xc.lda_pz_polarized(ru, rd)
    for which, v in ((0, vu), (1, vd)):
        # fourth-order central difference with a step relative to the varied spin density
        d = 1e-3 * (ru if which == 0 else rd)

        def g(t):
            a, b = (ru + t, rd) if which == 0 else (ru, rd + t)
            e_, _, _ = xc.lda_pz_polarized(a, b)
            return (a + b) * e_

        fd = (-g(2 * d) + 8 * g(d) - 8 * g(-d) + g(-2 * d)) / (12 * d)
        assert np.max(np.abs(fd - v) / np.abs(v)) < 1e-7


def test_zero_moment_polarized_equals_unpolarized():
    rho = np.logspace(-4, 1, 30)
    e0, v0 = xc.lda_pz_unpolarized(rho)
    e1, vu, vd = xc.lda_pz_polarized(rho / 2, rho / 2)
    assert np.allclose(e0, e1, rtol=1e-14, atol=0)
    assert np.allclose(v0, vu, rtol=1e-14, atol=0) and np.allclose(v0, vd, rtol=1e-14, atol=0)
