"""Kohn-Sham operator, electrostatics, occupations and density (Eq. 1, Eq. 2, Sec. 2.1).

Orbital blocks are arrays of shape (nstates, ngrid): row n is orbital n on the flattened
grid (x fastest), Euclidean-normalised (sum_g |X_ng|^2 = 1), so the continuum orbital is
X / sqrt(dV) with dV = h1 h2 h3 (trapezoidal rule, Sec. 2.1).

  H X = -1/2 L_h X + V_eff * X + sum_a E_a dV beta_a (beta_a^H X)           (Eq. 1)
  rho(x) = sum_k w_k sum_n g_nk |X_nk(x)|^2 / dV                             (Eq. 2)
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np
import scipy.sparse as sp

from . import fd

_POOL = None


def _pool():
    global _POOL
    if _POOL is None:
        _POOL = cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1))
    return _POOL


def bloch_phases(kred):
    return tuple(np.exp(2j * np.pi * k) if k != 0 else 1.0 for k in kred)


def kinetic(cell, X, kred=(0.0, 0.0, 0.0)):
    """-1/2 L_h X for a block X (nstates, ngrid), orbitals processed in parallel chunks."""
    ns = X.shape[0]
    n1, n2, n3 = cell.n
    ph = bloch_phases(kred)

    dirichlet = getattr(cell, "boundary", "periodic") == "dirichlet"

    def work(lo, hi):
        u = X[lo:hi].reshape(hi - lo, n3, n2, n1)
        return lo, -0.5 * fd.laplacian(u, cell.h, ph, dirichlet=dirichlet).reshape(hi - lo, -1)

    out = np.empty(X.shape, dtype=np.result_type(X, complex) if any(k != 0 for k in kred) else X.dtype)
    chunk = max(1, -(-ns // (4 * (os.cpu_count() or 1))))
    futs = [_pool().submit(work, lo, min(ns, lo + chunk)) for lo in range(0, ns, chunk)]
    for f in futs:
        lo, v = f.result()
        out[lo:lo + v.shape[0]] = v
    return out


def nonlocal_apply(P, E, dV, X):
    """sum_a E_a dV beta_a (beta_a^H X): C = conj(P) X^T, then P^T (E dV C)."""
    C = (P.conj() @ X.T)                      # (natom, nstates)
    return (P.T @ ((E * dV)[:, None] * C)).T


def apply_h(cell, X, V, P, E, kred=(0.0, 0.0, 0.0)):
    """Matrix-free H X (Sec. 2.1: FD stencil + outer-product nonlocal operator)."""
    dV = float(np.prod(cell.h))
    return kinetic(cell, X, kred) + V[None, :] * X + nonlocal_apply(P, E, dV, X)


def dense_h(cell, V, P, E, kred=(0.0, 0.0, 0.0)):
    """H as an explicit ngrid x ngrid matrix, entry by entry from the stencil definition.
    Only for brute-force checks on tiny grids."""
    w = fd.fd_weights()
    p = fd.FD_RADIUS
    n1, n2, n3 = cell.n
    N = cell.ngrid
    ph = bloch_phases(kred)
    cplx = any(k != 0 for k in kred)
    dirichlet = getattr(cell, "boundary", "periodic") == "dirichlet"
    H = np.zeros((N, N), complex if cplx else float)
    for k in range(n3):
        for j in range(n2):
            for i in range(n1):
                g = i + n1 * (j + n2 * k)
                base = (i, j, k)
                for d in range(3):
                    inv_h2 = 1.0 / (cell.h[d] ** 2)
                    for r in range(-p, p + 1):
                        q = list(base)
                        q[d] = base[d] + r
                        wraps = q[d] // cell.n[d]
                        if dirichlet and wraps != 0:
                            continue          # zero outside an isolated cell
                        q[d] = q[d] % cell.n[d]
                        gq = q[0] + n1 * (q[1] + n2 * q[2])
                        H[g, gq] += -0.5 * w[abs(r)] * inv_h2 * (ph[d] ** wraps)
                H[g, g] += V[g]
    dV = float(np.prod(cell.h))
    B = P.toarray()
    H += (B.T * (E * dV)[None, :]) @ B.conj()
    return H


def poisson_exact(cell, f):
    """Solve -L_h phi = 4 pi (f - mean f) on the periodic grid with zero-mean phi, exactly:
    L_h is diagonal on discrete Fourier modes with the FD symbol (Sec. 2.1 electrostatics)."""
    n1, n2, n3 = cell.n
    F = np.fft.fftn((f - f.mean()).reshape(n3, n2, n1))
    sym = -fd.laplacian_symbol(cell.n, cell.h)   # eigenvalues of -L_h, >= 0
    sym[0, 0, 0] = 1.0
    phiF = 4.0 * np.pi * F / sym
    phiF[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(phiF)).reshape(-1)


def fermi_occupations(eigs, kw, nelec, kT, spin_factor):
    """Fermi-Dirac occupations g = f_s / (1 + exp((lambda - mu)/kT)) with mu from bisection on
    sum_{s,k} w_k sum_n g = N_e (Sec. 2: "occupations ... typically given by the Fermi-Dirac
    distribution").  eigs has shape (nspin, nk, nstates).  Returns (mu, g)."""
    eigs = np.asarray(eigs, float)
    wk = np.asarray(kw, float)[None, :, None]

    def occ(mu):
        x = (eigs - mu) / kT
        return spin_factor * 0.5 * (1.0 - np.tanh(0.5 * x))

    def count(mu):
        return float(np.sum(wk * occ(mu)))

    lo = eigs.min() - 50.0 * kT - 1.0
    hi = eigs.max() + 50.0 * kT + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if count(mid) < nelec:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-15 * max(1.0, abs(mid)):
            break
    mu = 0.5 * (lo + hi)
    return mu, occ(mu)


def entropy_term(g, kw, kT, spin_factor):
    """-TS = kT sum_{s,k} w_k f_s [f ln f + (1-f) ln(1-f)], f = g/f_s, 0 ln 0 = 0 (Mermin)."""
    f = np.asarray(g, float) / spin_factor
    wk = np.asarray(kw, float)[None, :, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(f > 0, f * np.log(f), 0.0) + np.where(f < 1, (1 - f) * np.log(1 - f), 0.0)
    return float(kT * spin_factor * np.sum(wk * t))


def density(blocks, g, kw, dV):
    """rho^s(x) = sum_k w_k sum_n g_snk |X_snk(x)|^2 / dV (Eq. 2).  blocks[s][k] is (nstates, ngrid)."""
    nspin = len(blocks)
    out = []
    for s in range(nspin):
        r = 0.0
        for k, X in enumerate(blocks[s]):
            r = r + kw[k] * np.einsum("n,ng->g", g[s, k], np.abs(X) ** 2)
        out.append(r / dV)
    return np.array(out)
