"""Density extrapolation between molecular-dynamics steps (test infrastructure: only tests/, the smoke
check and the benchmark's CPU baseline may use the oracle).

Sec. 2.1: for QMD, the starting density of later MD steps comes from an extrapolation of earlier ones
(the cited scheme: D. Alfe, Comput. Phys. Commun. 118 (1999) 31).  With positions R_0 (newest), R_1, R_2
of the last SCF runs and their density corrections D_i = rho_i - rho_SAD(R_i):

    alpha, beta = argmin | (R - R_0) - alpha (R_0 - R_1) - beta (R_1 - R_2) |^2     (minimum image),
    rho_guess  = rho_SAD(R) + D_0 + alpha (D_0 - D_1) + beta (D_1 - D_2),

then clamped at zero and renormalised to N_e.  With two past runs beta = 0, with one alpha = beta = 0.

Pinned by tests/test_oracle_extrapolation.py: constant-velocity and uniformly accelerated motion (where
the displacement fit is exact with (1, 0) and (2, -1)), periodic-image invariance, a static density
correction passing through unchanged, and electron-count conservation.
"""
from __future__ import annotations

import numpy as np


def _min_image(d, L):
    L = np.asarray(L, float)
    return d - L * np.round(d / L)


def alfe_coefficients(R, hist, L):
    """R: (natom, 3) new positions; hist: newest-first list of up to three (natom, 3) arrays."""
    if len(hist) < 2:
        return 0.0, 0.0
    dn = _min_image(np.asarray(R) - hist[0], L).ravel()
    d1 = _min_image(hist[0] - hist[1], L).ravel()
    if len(hist) >= 3:
        d2 = _min_image(hist[1] - hist[2], L).ravel()
        A = np.array([[d1 @ d1, d1 @ d2], [d1 @ d2, d2 @ d2]])
        if np.linalg.det(A) > 1e-12 * A[0, 0] * A[1, 1]:
            a, b = np.linalg.solve(A, np.array([dn @ d1, dn @ d2]))
            return float(a), float(b)
    return float(dn @ d1 / (d1 @ d1)), 0.0


def extrapolated_density(rho_sad_new, deltas, alpha, beta, nelec, dV):
    """rho_sad_new: (nspin, ngrid) reference at the new positions; deltas: newest-first corrections."""
    g = np.array(rho_sad_new, float, copy=True)
    coef = [1.0 + alpha, beta - alpha, -beta]
    for c, d in zip(coef, deltas):
        g = g + c * d
    g = np.maximum(g, 0.0)
    return g * (nelec / (dV * g.sum()))
