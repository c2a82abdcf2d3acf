"""Kerker-preconditioned periodic Pulay mixing (test infrastructure: only tests/, the smoke check and
the benchmark's CPU baseline may use the oracle).

Sec. 2.1 accelerates the SCF with restarted periodic Pulay mixing and a real-space
preconditioner (the cited scheme of Kumar et al. 2019 is Kerker-type).  The preconditioner damps
the long-wavelength part of the density residual f, the charge sloshing that slows the SCF of
large cells:

    P f = (-L_h) (-L_h + k0^2)^-1 f,

L_h the order-12 periodic FD Laplacian of the grid.  On a plane wave of FD eigenvalue -lambda
(lambda >= 0) P multiplies by lambda / (lambda + k0^2): short waves pass almost unchanged, the
uniform component (lambda = 0) is removed for k0 > 0, and k0 = 0 is the identity.  Here P is
written by that definition through the FD symbol and FFTs; a GPU path solves the screened
Poisson equation (-L_h + k0^2) y = f in real space, and P f = f - k0^2 y.

Preconditioned Pulay: the linear part of every update becomes P(beta f):

    x_{k+1} = x_k + P(beta f_k) - (X_k + P(beta F_k)) gamma,   gamma = (F_k^T F_k)^-1 F_k^T f_k,

with X_k, F_k the last `hist` differences of inputs and residuals (Pulay steps every `period`-th
iteration, linear steps x_k + P(beta f_k) otherwise; `restart` clears the history after a Pulay
step).  Spin-polarised vectors [rho_up; rho_dn] are preconditioned channel by channel.

Pinned by tests/test_oracle_kerker.py: plane-wave factors against eigenvalues measured with the
real-space stencil, the removed uniform mode, the screened-Poisson identity checked with the
real-space Laplacian, and reduction to the plain Pulay mixer at k0 = 0.
"""
from __future__ import annotations

import numpy as np

from . import fd


def kerker(cell, f: np.ndarray, k0: float) -> np.ndarray:
    """P f for one grid vector or a stack of channels (..., ngrid), x fastest (n3, n2, n1 order)."""
    n1, n2, n3 = cell.n
    lam = -fd.laplacian_symbol(cell.n, cell.h)          # >= 0, zero for the uniform mode
    if k0 > 0.0:
        factor = lam / (lam + k0 * k0)
    else:
        factor = np.ones_like(lam)
    f = np.asarray(f, dtype=np.float64)
    lead = f.shape[:-1]
    g = f.reshape((-1, n3, n2, n1))
    out = np.empty_like(g)
    for c in range(g.shape[0]):
        out[c] = np.real(np.fft.ifftn(factor * np.fft.fftn(g[c])))
    return out.reshape(lead + (f.shape[-1],))


class KerkerPulayMixer:
    """Periodic Pulay mixing with the Kerker preconditioner on the linear part (see module
    docstring); `nchan` channels of `cell`'s grid are stacked in the mixed vector."""

    def __init__(self, cell, k0=0.8, beta=0.3, hist=7, period=1, restart=False, nchan=1):
        self.cell, self.k0, self.nchan = cell, k0, nchan
        self.beta, self.hist, self.period, self.restart = beta, hist, period, restart
        self.k = 0
        self.dx, self.df = [], []
        self.x_prev = self.f_prev = None

    def precondition(self, v):
        ng = self.cell.ngrid
        return kerker(self.cell, v.reshape(self.nchan, ng), self.k0).reshape(-1)

    def update(self, x_in, x_out):
        f = x_out - x_in
        if self.k > 0:
            self.dx.append(x_in - self.x_prev)
            self.df.append(f - self.f_prev)
            self.dx, self.df = self.dx[-self.hist:], self.df[-self.hist:]
        self.x_prev, self.f_prev = x_in.copy(), f.copy()
        pulay_step = self.k > 0 and len(self.df) > 0 and (self.k + 1) % self.period == 0
        if pulay_step:
            Fm = np.array(self.df).T
            Xm = np.array(self.dx).T
            gamma = np.linalg.solve(Fm.T @ Fm, Fm.T @ f)
            r = f - Fm @ gamma                              # optimal residual
            x_new = x_in - Xm @ gamma + self.precondition(self.beta * r)
            if self.restart:
                self.dx, self.df = [], []
        else:
            x_new = x_in + self.precondition(self.beta * f)
        self.k += 1
        return x_new
