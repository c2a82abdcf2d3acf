"""Perdew-Zunger LDA exchange-correlation (Sec. 3: "Perdew-Zunger parametrization for LDA";
J. P. Perdew and A. Zunger, Phys. Rev. B 23, 5048 (1981), Appendix C).

Exchange is the Dirac/Slater form with exact spin scaling.  Correlation is the PZ81 fit to
the Ceperley-Alder data, unpolarized (U) and fully polarized (P) phases, joined by the
von Barth-Hedin interpolation f(zeta).  The density is floored at RHO_FLOOR inside this
module only.

Pinned by tests/test_oracle_xc.py: the Gell-Mann-Brueckner high-density coefficient, the
Perdew-Wang 1992 fit of the same Ceperley-Alder data, continuity at r_s = 1, and V_xc
against a finite difference of rho*eps_xc.
"""
from __future__ import annotations

import numpy as np

RHO_FLOOR = 1e-14

#            gamma    beta1   beta2    A        B        C       D
PZ_U = dict(g=-0.1423, b1=1.0529, b2=0.3334, A=0.0311, B=-0.048, C=0.0020, D=-0.0116)
PZ_P = dict(g=-0.0843, b1=1.3981, b2=0.2611, A=0.01555, B=-0.0269, C=0.0007, D=-0.0048)

CX = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0)   # eps_x = CX rho^(1/3) for the unpolarized gas


def wigner_seitz_radius(rho):
    return (3.0 / (4.0 * np.pi * rho)) ** (1.0 / 3.0)


def pz_correlation(rs, c):
    """(eps_c, mu_c) of one PZ81 phase, mu_c = eps_c - (rs/3) d eps_c / d rs."""
    rs = np.asarray(rs, float)
    eps = np.empty_like(rs)
    mu = np.empty_like(rs)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + c["b1"] * s + c["b2"] * rs[hi]
    eps[hi] = c["g"] / den
    mu[hi] = eps[hi] * (1.0 + 7.0 / 6.0 * c["b1"] * s + 4.0 / 3.0 * c["b2"] * rs[hi]) / den
    lo = ~hi
    r = rs[lo]
    lr = np.log(r)
    eps[lo] = c["A"] * lr + c["B"] + c["C"] * r * lr + c["D"] * r
    mu[lo] = c["A"] * lr + (c["B"] - c["A"] / 3.0) + 2.0 / 3.0 * c["C"] * r * lr \
        + (2.0 * c["D"] - c["C"]) / 3.0 * r
    return eps, mu


def _f_zeta(z):
    return ((1 + z) ** (4 / 3) + (1 - z) ** (4 / 3) - 2.0) / (2.0 ** (4 / 3) - 2.0)


def _df_zeta(z):
    return 4.0 / 3.0 * (np.cbrt(1 + z) - np.cbrt(1 - z)) / (2.0 ** (4 / 3) - 2.0)


def lda_pz_unpolarized(rho):
    """Returns (eps_xc per electron, v_xc) for a spin-unpolarized density."""
    r = np.maximum(np.asarray(rho, float), RHO_FLOOR)
    ex = CX * np.cbrt(r)
    vx = 4.0 / 3.0 * ex
    ec, vc = pz_correlation(wigner_seitz_radius(r), PZ_U)
    return ex + ec, vx + vc


def lda_pz_polarized(rho_up, rho_dn):
    """Returns (eps_xc, v_xc_up, v_xc_dn) for spin densities (Sec. 2.1 spin-polarized case)."""
    r = np.maximum(np.asarray(rho_up, float) + np.asarray(rho_dn, float), RHO_FLOOR)
    z = np.clip((np.asarray(rho_up, float) - np.asarray(rho_dn, float)) / r, -1.0, 1.0)
    exu = CX * np.cbrt(r)
    ex = exu * 0.5 * ((1 + z) ** (4 / 3) + (1 - z) ** (4 / 3))
    vx_up = 4.0 / 3.0 * exu * np.cbrt(1 + z)
    vx_dn = 4.0 / 3.0 * exu * np.cbrt(1 - z)
    rs = wigner_seitz_radius(r)
    eu, mu_u = pz_correlation(rs, PZ_U)
    ep, mu_p = pz_correlation(rs, PZ_P)
    f = _f_zeta(z)
    df = _df_zeta(z)
    ec = eu + f * (ep - eu)
    vc_common = mu_u + f * (mu_p - mu_u)
    vc_up = vc_common + (ep - eu) * df * (1.0 - z)
    vc_dn = vc_common + (ep - eu) * df * (-1.0 - z)
    return ex + ec, vx_up + vc_up, vx_dn + vc_dn
