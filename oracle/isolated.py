"""Electrostatics of isolated systems: Dirichlet boundary values from a multipole expansion (test
infrastructure: only tests/, the smoke check and the benchmark's CPU baseline may use the oracle).

The paper treats isolated systems with Dirichlet boundary conditions, the electrostatic potential on
the boundary coming from a multipole expansion of the charge (Sec. 2 and 2.1).  Discrete form used
here (the paper gives neither the expansion order nor the centre; readings: l_max = 6, centre = the
middle of the grid box):

* grid points x_i = i h_d, i = 0..n_d-1, per axis; the order-12 Laplacian reaches 6 ghost layers
  beyond each face.  Orbitals are zero there; the potential there is
      phi(x) = sum_{l <= l_max} sum_m 4 pi / (2l + 1) q_lm Y_lm(x^) / r^(l+1),  x relative to the centre,
      q_lm   = dV sum_g f_g r_g^l Y_lm(x_g^)     (f = rho + b, Y_lm real orthonormal harmonics);
* inside, -L_h phi = 4 pi f with those ghost values, i.e. -L0 phi = 4 pi f + G, L0 the Laplacian with
  zero ghost layers and G the ghost values' share of the stencil.  The system is symmetric positive
  definite and is solved by conjugate gradients to a relative residual of 1e-13.

Pinned by tests/test_oracle_isolated.py: orthonormality of the harmonics, the multipole potential of
an off-centre Gaussian against Coulomb's law, the solution for a Gaussian charge against its closed-form
potential, and symmetry / definiteness of the Dirichlet Laplacian.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import sph_harm_y

from . import fd

LMAX = 6


def real_ylm(lmax, x, y, z):
    """Real orthonormal spherical harmonics of the directions (x, y, z): array (nlm, npts), index l^2 + l + m."""
    r = np.sqrt(x * x + y * y + z * z)
    rs = np.where(r > 0, r, 1.0)
    theta = np.arccos(np.clip(np.where(r > 0, z / rs, 1.0), -1.0, 1.0))
    phi = np.arctan2(y, x)
    out = np.zeros(((lmax + 1) ** 2,) + np.shape(x))
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                v = Y.real
            elif m > 0:
                v = np.sqrt(2.0) * (-1) ** m * Y.real
            else:
                v = np.sqrt(2.0) * (-1) ** m * Y.imag
            out[l * l + l + m] = v
    return out


def grid_coords(cell):
    z, y, x = np.meshgrid(*[np.arange(cell.n[d]) * cell.h[d] for d in (2, 1, 0)], indexing="ij")
    return x.reshape(-1), y.reshape(-1), z.reshape(-1)


def centre(cell):
    return np.array([0.5 * (cell.n[d] - 1) * cell.h[d] for d in range(3)])


def multipole_moments(cell, f, lmax=LMAX):
    x, y, z = grid_coords(cell)
    c = centre(cell)
    dx, dy, dz = x - c[0], y - c[1], z - c[2]
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    Y = real_ylm(lmax, dx, dy, dz)
    dV = float(np.prod(cell.h))
    q = np.zeros((lmax + 1) ** 2)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            k = l * l + l + m
            q[k] = dV * np.sum(f * r ** l * Y[k])
    return q


def multipole_potential(q, dx, dy, dz, lmax=LMAX):
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    Y = real_ylm(lmax, dx, dy, dz)
    v = np.zeros(np.shape(dx))
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            k = l * l + l + m
            v = v + 4.0 * np.pi / (2 * l + 1) * q[k] * Y[k] / r ** (l + 1)
    return v


def dirichlet_laplacian_matrix(cell):
    """L0: the order-12 Laplacian with zero values outside the grid, as a sparse matrix."""
    w = fd.fd_weights()
    n1, n2, n3 = cell.n
    N = cell.ngrid
    idx = np.arange(N).reshape(n3, n2, n1)
    rows, cols, vals = [idx.reshape(-1)], [idx.reshape(-1)], [np.full(N, sum(w[0] / cell.h[d] ** 2 for d in range(3)))]
    for d in range(3):
        ax = 2 - d
        n = cell.n[d]
        for r in range(1, fd.FD_RADIUS + 1):
            for sgn in (1, -1):
                src = [slice(None)] * 3
                dst = [slice(None)] * 3
                if sgn > 0:
                    src[ax], dst[ax] = slice(0, n - r), slice(r, n)
                else:
                    src[ax], dst[ax] = slice(r, n), slice(0, n - r)
                if n - r <= 0:
                    continue
                rows.append(idx[tuple(src)].reshape(-1))
                cols.append(idx[tuple(dst)].reshape(-1))
                vals.append(np.full(rows[-1].size, w[r] / cell.h[d] ** 2))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def ghost_term(cell, q, lmax=LMAX):
    """G: the share of the ghost-layer potential in L_h phi at every grid point."""
    w = fd.fd_weights()
    c = centre(cell)
    n1, n2, n3 = cell.n
    G = np.zeros((n3, n2, n1))
    kk, jj, ii = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    I = [ii, jj, kk]
    for d in range(3):
        for r in range(1, fd.FD_RADIUS + 1):
            for sgn in (1, -1):
                nb = [I[0].astype(float), I[1].astype(float), I[2].astype(float)]
                nb[d] = nb[d] + sgn * r
                outside = (nb[d] < 0) | (nb[d] > cell.n[d] - 1)
                if not np.any(outside):
                    continue
                dx = nb[0][outside] * cell.h[0] - c[0]
                dy = nb[1][outside] * cell.h[1] - c[1]
                dz = nb[2][outside] * cell.h[2] - c[2]
                G[outside] += w[r] / cell.h[d] ** 2 * multipole_potential(q, dx, dy, dz, lmax)
    return G.reshape(-1)


def poisson_isolated(cell, f, lmax=LMAX):
    """phi with -L_h phi = 4 pi f inside and the multipole potential of f in the ghost layers."""
    f = np.asarray(f, float)
    q = multipole_moments(cell, f, lmax)
    A = -dirichlet_laplacian_matrix(cell)
    b = 4.0 * np.pi * f + ghost_term(cell, q, lmax)
    phi, info = spla.cg(A, b, rtol=1e-13, atol=0.0, maxiter=20000)
    if info != 0:
        raise RuntimeError("isolated Poisson: CG did not converge")
    return phi
