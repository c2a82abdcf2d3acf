"""Pins of the isolated-system electrostatics oracle (oracle/isolated.py) and of the Dirichlet form of the
kinetic operator, against facts that do not come from its own formulas: quadrature orthonormality of the
harmonics, Coulomb's law for a distant charge, the closed-form potential of a Gaussian charge, and
the structure of the zero-padded stencil."""
import numpy as np
import pytest
from scipy.special import erf

import workloads
from oracle import fd, ham, isolated


def _box(n=24, L=9.6):
    c = workloads.small_cell(npts=n, L=L, natom=1, seed=1, nstates=4)
    c.boundary = "dirichlet"
    return c


def test_real_harmonics_are_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform phi integrates products up to degree 12 exactly
    xg, wg = np.polynomial.legendre.leggauss(16)
    ph = np.arange(32) * 2 * np.pi / 32
    ct, p = np.meshgrid(xg, ph, indexing="ij")
    w = np.outer(wg, np.full(32, 2 * np.pi / 32)).reshape(-1)
    st = np.sqrt(1 - ct ** 2)
    Y = isolated.real_ylm(isolated.LMAX, (st * np.cos(p)).reshape(-1), (st * np.sin(p)).reshape(-1), ct.reshape(-1))
    G = (Y * w) @ Y.T
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-12
    assert abs(Y[0, 0] - 0.5 / np.sqrt(np.pi)) < 1e-15


def test_multipole_potential_of_offcentre_gaussian_follows_coulomb():
    c = _box()
    x, y, z = isolated.grid_coords(c)
    q0, s = 1.7, 0.6
    a = isolated.centre(c) + np.array([0.9, -0.5, 0.4])
    f = q0 * (2 * np.pi * s * s) ** -1.5 * np.exp(-((x - a[0]) ** 2 + (y - a[1]) ** 2 + (z - a[2]) ** 2) / (2 * s * s))
    q = isolated.multipole_moments(c, f)
    assert abs(q[0] * 2 * np.sqrt(np.pi) - q0) < 1e-10        # monopole = total charge
    pts = np.array([[12.0, 4.0, 5.0], [-3.0, 4.5, 4.0], [4.8, -2.5, 14.0]]) - isolated.centre(c)
    v = isolated.multipole_potential(q, pts[:, 0], pts[:, 1], pts[:, 2])
    exact = q0 / np.linalg.norm(pts - (a - isolated.centre(c)), axis=1)
    # truncation after l = 6 at |a - centre| / r ~ 0.15: relative error ~ 0.15^7
    assert np.max(np.abs(v - exact) / exact) < 1e-5


def test_isolated_poisson_of_gaussian_matches_closed_form():
    # phi = Q erf(r / (sqrt 2 s)) / r for a Gaussian charge of total Q: order-12 differences at h = 0.4
    # reproduce it to ~1e-7, the l <= 6 boundary values of a centred charge are exact (monopole)
    # (with s = 0.9 in a 9.6 bohr box the charge left outside the grid is 2e-7 of Q)
    c = _box(n=24, L=9.6)
    x, y, z = isolated.grid_coords(c)
    cc = isolated.centre(c)
    r = np.sqrt((x - cc[0]) ** 2 + (y - cc[1]) ** 2 + (z - cc[2]) ** 2)
    Q, s = 2.0, 0.9
    f = Q * (2 * np.pi * s * s) ** -1.5 * np.exp(-r * r / (2 * s * s))
    phi = isolated.poisson_isolated(c, f)
    exact = Q * np.where(r > 1e-12, erf(r / (np.sqrt(2) * s)) / np.where(r > 1e-12, r, 1), np.sqrt(2 / np.pi) / s)
    assert np.max(np.abs(phi - exact)) < 2e-6 * np.max(exact)


def test_dirichlet_laplacian_is_symmetric_negative_definite_and_matches_zero_padding():
    c = _box(n=8, L=3.2)
    c.n = (8, 7, 6)
    c.L = (3.2, 2.8, 2.4)
    A = isolated.dirichlet_laplacian_matrix(c).toarray()
    assert np.max(np.abs(A - A.T)) < 1e-13
    assert np.max(np.linalg.eigvalsh(A)) < 0
    u = np.random.default_rng(2).normal(size=c.ngrid)
    Lu = fd.laplacian(u.reshape(c.n[::-1]), c.h, dirichlet=True).reshape(-1)
    assert np.max(np.abs(A @ u - Lu)) < 1e-10 * np.max(np.abs(Lu))
    # the kinetic operator of an isolated cell is the same zero-padded stencil (dense and matrix-free agree)
    c.pos = np.array([[1.6, 1.4, 1.2]])
    V = np.random.default_rng(3).normal(0, 0.2, c.ngrid)
    from oracle import model
    P, E = model.projectors(c), model.kb_energies(c)
    H = ham.dense_h(c, V, P, E)
    X = np.random.default_rng(4).normal(size=(2, c.ngrid))
    assert np.max(np.abs(X @ H.T - ham.apply_h(c, X, V, P, E))) < 1e-10
