"""Pins for oracle.scf: energy identities, forces vs finite differences, exact symmetries,
spin and k-point identities."""
import functools

import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import ham, model, scf


@functools.lru_cache(maxsize=None)
def _tight_two_atom():
    return scf.scf(workloads.two_atom_cell(), tol=1e-9, max_iter=200)


def _small(pos, n=12, L=4.5, nspin=1, nstates=6, r_cut_proj=3.0):
    c = workloads.small_cell(npts=n, L=L, natom=len(pos), nstates=nstates, degree=12)
    c.species = [workloads.Species(r_cut_proj=r_cut_proj)]
    c.pos = np.array(pos, float)
    c.types = np.zeros(len(pos), int)
    c.nspin = nspin
    return c


def test_two_atom_energy_forms_and_invariants():
    r = _tight_two_atom()
    c = workloads.two_atom_cell()
    dV = float(np.prod(c.h))
    assert r.converged
    # Harris-Foulkes and Kohn-Sham free energies coincide at self-consistency.
    assert abs(r.energy - r.energy_ks) < 1e-9
    assert abs(dV * r.rho.sum() - c.nelec) < 1e-10
    X = r.blocks[0][0]
    assert np.allclose(X @ X.T, np.eye(c.nstates), atol=1e-12)
    # Forces vanish by the inversion symmetry of the CsCl-like arrangement.
    f = scf.Problem(c).forces(r.blocks, r.occ, r.phi)
    assert np.max(np.abs(f)) < 1e-6


def test_variational_ks_energy_above_ground_state():
    # The Kohn-Sham (Mermin) free energy of the output of a non-self-consistent potential is
    # above the self-consistent minimum.
    c = workloads.two_atom_cell()
    F0 = _tight_two_atom().energy
    for it in (1, 3, 6):
        r = scf.scf(workloads.two_atom_cell(), max_iter=it, tol=1e-30)
        assert r.energy_ks >= F0 - 1e-9


def _converged(cell):
    return scf.scf(cell, tol=1e-10, max_iter=300, final_tol=1e-9, with_forces=True)


def test_forces_match_central_difference_of_free_energy():
    # The projector support is cut at r_c; at r_c = 5 r_p grid points entering or leaving the
    # sphere make F(R) jump by ~1e-9 Ha, which spoils a 1e-6 finite difference.  With
    # r_c = 7 r_p (chi(r_c)/chi(0) = e^-24.5) F is smooth to round-off and the analytic
    # Hellmann-Feynman force must match the central difference.
    pos = [[0.3, 0.2, 0.1], [2.4, 2.1, 2.6]]
    rc = 4.2
    r0 = _converged(_small(pos, r_cut_proj=rc))
    a, d, delta = 1, 0, 1e-3
    step = delta * np.eye(3)[d] * (np.arange(2) == a)[:, None]
    Fp = _converged(_small(np.array(pos) + step, r_cut_proj=rc)).energy
    Fm = _converged(_small(np.array(pos) - step, r_cut_proj=rc)).energy
    fd_force = -(Fp - Fm) / (2 * delta)
    assert abs(r0.forces[a, d]) > 1e-3          # a non-trivial component
    assert abs(r0.forces[a, d] - fd_force) < 1e-6
    # Newton's third law within the cell (translation invariance of the discrete energy is only
    # broken by the grid, so the sum is small but not zero): |sum F| << |F|.
    assert np.max(np.abs(r0.forces.sum(axis=0))) < 0.2 * np.max(np.abs(r0.forces))


def test_translation_by_grid_vector_leaves_energy_unchanged():
    pos = np.array([[0.3, 0.2, 0.1], [2.4, 2.1, 2.6]])
    c0 = _small(pos)
    shift = np.array([3, 1, 7]) * c0.h[0]
    r0 = scf.scf(c0, tol=1e-10, max_iter=300)
    r1 = scf.scf(_small(pos + shift), tol=1e-10, max_iter=300)
    assert abs(r0.energy - r1.energy) < 1e-9
    assert np.allclose(r0.eigs[0, 0, :3], r1.eigs[0, 0, :3], atol=1e-8)


def test_zero_moment_spin_polarized_equals_unpolarized():
    # Equal spin densities and equal starting blocks in both channels: the polarized SCF must
    # reproduce the unpolarized one (each channel holds half the electrons with f_s = 1).
    pos = [[0.3, 0.2, 0.1], [2.4, 2.1, 2.6]]
    c0 = _small(pos)
    X0 = scf.initial_blocks(c0)[0][0]
    rho = scf.initial_density(c0)[0]
    r0 = scf.scf(c0, tol=1e-10, max_iter=300, blocks=[[X0.copy()]])
    c1 = _small(pos, nspin=2)
    orig = scf.initial_density
    try:
        scf.initial_density = lambda cell, rho0=None, moment=0.0: np.stack([rho / 2, rho / 2])
        r1 = scf.scf(c1, tol=1e-10, max_iter=300, blocks=[[X0.copy()], [X0.copy()]])
    finally:
        scf.initial_density = orig
    assert abs(r0.energy - r1.energy) < 1e-9
    assert np.allclose(r0.eigs[0, 0, :3], r1.eigs[0, 0, :3], atol=1e-8)
    assert np.allclose(r0.eigs[0, 0, :3], r1.eigs[1, 0, :3], atol=1e-8)


def test_supercell_gamma_equals_primitive_k_grid():
    # A 1-atom primitive cell with the 2x2x2 Gamma-centred k-grid {0, 1/2}^3 has exactly the
    # Gamma-point spectrum of the 2x2x2 supercell with the same (tiled) potential.
    n, L = 6, 3.0
    prim = workloads.small_cell(npts=n, L=L, natom=1, seed=5)
    prim.pos = np.array([[0.7, 1.1, 0.4]])
    rng = np.random.default_rng(8)
    Vp = rng.normal(0, 0.3, prim.ngrid)
    E = model.kb_energies(prim)
    lam_k = []
    for kx in (0.0, 0.5):
        for ky in (0.0, 0.5):
            for kz in (0.0, 0.5):
                P = model.projectors(prim, (kx, ky, kz))
                lam_k.append(sla.eigvalsh(ham.dense_h(prim, Vp, P, E, (kx, ky, kz))))
    lam_k = np.sort(np.concatenate(lam_k))
    sup = workloads.small_cell(npts=2 * n, L=2 * L, natom=8, seed=5)
    sup.pos = np.array([prim.pos[0] + L * np.array([i, j, k]) for k in (0, 1) for j in (0, 1) for i in (0, 1)])
    Vs = np.tile(Vp.reshape(n, n, n), (2, 2, 2)).reshape(-1)
    lam_s = sla.eigvalsh(ham.dense_h(sup, Vs, model.projectors(sup), model.kb_energies(sup)))
    assert np.allclose(lam_s, lam_k, atol=1e-10)
