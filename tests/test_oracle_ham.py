"""Pins for oracle.model / oracle.ham / oracle.chefsi against brute force, closed forms and
exact invariants of the discrete operator."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import chefsi, fd, ham, model


def _tiny(n=10, L=4.0, natom=2, seed=3, kred=(0.0, 0.0, 0.0)):
    c = workloads.small_cell(npts=n, L=L, natom=natom, seed=seed)
    rng = np.random.default_rng(seed + 100)
    V = rng.normal(0.0, 0.5, c.ngrid)
    P = model.projectors(c, kred)
    E = model.kb_energies(c)
    return c, V, P, E


def test_pseudocharge_and_sad_integrals():
    c = workloads.two_atom_cell()
    dV = float(np.prod(c.h))
    b = model.pseudocharge(c)
    # A Gaussian sampled at h = 0.25 with width 0.5 sums to its integral up to exp(-2 pi^2 r_loc^2/h^2).
    assert abs(dV * b.sum() + c.nelec) < 1e-10
    rho = model.sad_density(c)
    assert abs(dV * rho.sum() - c.nelec) < 1e-10 and rho.min() > 0


def test_projector_continuum_norm():
    # integral of chi^2 = 1; the truncation at r_c = 5 r_p removes ~1e-10 of it.
    c = workloads.two_atom_cell()
    P = model.projectors(c)
    dV = float(np.prod(c.h))
    norms = dV * np.asarray(P.multiply(P).sum(axis=1)).ravel()
    assert np.allclose(norms, 1.0, atol=1e-8)


def test_self_energy_closed_form():
    # Coulomb self-energy of a Gaussian of charge Z, width s: Z^2 / (2 sqrt(pi) s) = 9.0270333 Ha for Z=4, s=0.5.
    c = workloads.two_atom_cell()
    assert abs(model.self_energy(c) / 2 - 9.027033336764101) < 1e-12


def test_overlap_correction_gradient_and_decay():
    c = workloads.small_cell(npts=8, L=5.0, natom=3, seed=11)
    E0, g = model.overlap_correction(c)
    for a in range(3):
        for d in range(3):
            cp = workloads.small_cell(npts=8, L=5.0, natom=3, seed=11)
            cm = workloads.small_cell(npts=8, L=5.0, natom=3, seed=11)
            cp.pos = c.pos.copy(); cm.pos = c.pos.copy()
            cp.pos[a, d] += 1e-5
            cm.pos[a, d] -= 1e-5
            fdv = (model.overlap_correction(cp)[0] - model.overlap_correction(cm)[0]) / 2e-5
            assert abs(fdv - g[a, d]) < 1e-6 * max(1.0, abs(g[a, d]))
    # Lattice cell with 5.13 bohr spacing: erfc(5.13) makes E_sc negligible.
    assert abs(model.overlap_correction(workloads.two_atom_cell())[0]) < 1e-10


@pytest.mark.parametrize("kred", [(0.0, 0.0, 0.0), (0.25, -0.5, 0.125)])
def test_apply_h_matches_dense_matrix(kred):
    c, V, P, E = _tiny(kred=kred)
    Hd = ham.dense_h(c, V, P, E, kred)
    assert np.allclose(Hd, Hd.conj().T, atol=1e-12)
    rng = np.random.default_rng(5)
    X = rng.normal(size=(5, c.ngrid))
    if any(kred):
        X = X + 1j * rng.normal(size=X.shape)
    HX = ham.apply_h(c, X, V, P, E, kred)
    ref = (Hd @ X.T).T
    assert np.max(np.abs(HX - ref)) < 1e-11 * np.max(np.abs(ref))


def test_translation_by_grid_vector_is_a_permutation():
    c = workloads.small_cell(npts=12, L=4.0, natom=2, seed=4)
    b0 = model.pseudocharge(c).reshape(12, 12, 12)
    P0 = model.projectors(c).toarray().reshape(2, 12, 12, 12)
    c.pos = c.pos + np.array([2, 0, 5]) * c.h[0]
    b1 = model.pseudocharge(c).reshape(12, 12, 12)
    P1 = model.projectors(c).toarray().reshape(2, 12, 12, 12)
    assert np.allclose(np.roll(b0, shift=(5, 0, 2), axis=(0, 1, 2)), b1, atol=1e-12)
    assert np.allclose(np.roll(P0, shift=(5, 0, 2), axis=(1, 2, 3)), P1, atol=1e-12)


def test_poisson_plane_wave_closed_form_and_stencil_residual():
    c = workloads.small_cell(npts=16, L=5.0, natom=1)
    x, y, z = [np.arange(16) * c.h[d] for d in range(3)]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    G = 2 * np.pi / 5.0
    f = np.cos(G * X + 2 * G * Z).reshape(-1)
    phi = ham.poisson_exact(c, f)
    # Plane wave: -L_h cos = lambda cos, lambda from the FD weights' cosine series.
    w = fd.fd_weights()
    lam = -sum((w[0] + 2 * sum(w[r] * np.cos(r * th) for r in range(1, 7))) / c.h[0] ** 2
               for th in (G * c.h[0], 0.0, 2 * G * c.h[0]))
    assert np.allclose(phi, 4 * np.pi * f / lam, atol=1e-12)
    # Independent check through the stencil: -L_h phi = 4 pi f for a zero-mean random f.
    rng = np.random.default_rng(2)
    f = rng.normal(size=c.ngrid)
    phi = ham.poisson_exact(c, f)
    res = -fd.laplacian(phi.reshape(16, 16, 16), c.h).reshape(-1) - 4 * np.pi * (f - f.mean())
    assert np.max(np.abs(res)) < 1e-10 * np.max(np.abs(f))
    assert abs(phi.mean()) < 1e-14


def test_fermi_counts_electrons_and_zero_temperature_limit():
    rng = np.random.default_rng(1)
    eigs = np.sort(rng.normal(size=(2, 3, 12)), axis=-1)
    kw = np.array([0.5, 0.25, 0.25])
    mu, g = ham.fermi_occupations(eigs, kw, 17.3, 0.01, 1.0)
    assert abs(np.sum(kw[None, :, None] * g) - 17.3) < 1e-12
    # gapped spectrum, tiny kT: integer occupations of the lowest states
    e = np.array([[[-1.0, -0.5, 0.0, 2.0, 3.0]]])
    mu, g = ham.fermi_occupations(e, np.ones(1), 6.0, 1e-3, 2.0)
    assert np.allclose(g[0, 0], [2, 2, 2, 0, 0], atol=1e-12) and -0.1 < mu < 2.0
    ts = ham.entropy_term(g, np.ones(1), 1e-3, 2.0)
    assert abs(ts) < 1e-12


def test_empty_lattice_eigenvalues_via_chefsi():
    # V = 0, no atoms: eigenvalues of -1/2 L_h on the two-atom cell's grid (L = 6, h = 0.25).
    # Continuum values 1/2 (2 pi/L)^2 |m|^2; the order-12 FD error here is below 1e-11 Ha.
    c = workloads.two_atom_cell()
    c.pos = np.zeros((0, 3))
    c.types = np.zeros(0, int)
    V = np.zeros(c.ngrid)
    apply = lambda X: ham.kinetic(c, X)
    X = workloads.initial_orbitals(1, c.ngrid, 19)   # 1 + 6 + 12: closed shells
    lo, up = chefsi.lanczos_bounds(apply, X[0], 25)
    a0, a = lo, lo + 0.1 * (up - lo)
    for _ in range(25):
        lam, X = chefsi.chefsi_pass(apply, X, 12, a, up, a0)
        a0, a = lam[0], lam[-1]
    e1 = 0.5 * (2 * np.pi / 6.0) ** 2
    assert abs(lam[0]) < 1e-10
    assert np.allclose(lam[1:7], e1, atol=1e-9)
    assert np.allclose(lam[7:], 2 * e1, atol=1e-2)   # the edge shell converges slowly by design
    assert abs(e1 - 0.548311355616075) < 1e-12
    # Lanczos upper bound is above the top of the discrete spectrum 3/(2h^2) * 7.07293891...
    w = fd.fd_weights()
    top = 1.5 / 0.25 ** 2 * -(w[0] + 2 * sum(w[r] * (-1) ** r for r in range(1, 7)))
    assert abs(top - 169.7505) < 1e-3 and up >= top - 1e-9


@pytest.mark.parametrize("kred", [(0.0, 0.0, 0.0), (0.5, 0.0, 0.25)])
def test_chefsi_matches_dense_eigensolver(kred):
    c, V, P, E = _tiny(n=10, kred=kred)
    Hd = ham.dense_h(c, V, P, E, kred)
    lam_ref = sla.eigh(Hd, eigvals_only=True)
    apply = lambda X: ham.apply_h(c, X, V, P, E, kred)
    ns = 9
    X = workloads.initial_orbitals(4, c.ngrid, ns, complex_valued=any(kred))
    lo, up = chefsi.lanczos_bounds(apply, X[0], 20)
    assert up >= lam_ref[-1] - 1e-9 and lo >= lam_ref[0] - 1e-9
    a0, a = lo, lo + 0.1 * (up - lo)
    for _ in range(60):
        lam, X = chefsi.chefsi_pass(apply, X, 10, a, up, a0)
        a0, a = lam[0], lam[-1]
    assert np.allclose(lam[:ns - 2], lam_ref[:ns - 2], atol=1e-9)
    assert np.allclose(X.conj() @ X.T, np.eye(ns), atol=1e-12)


def test_chebyshev_filter_matches_closed_form_polynomial():
    # p(lambda) = T_m((lambda - c)/e) / T_m((a0 - c)/e) with T_m = cos(m acos t) or cosh(m acosh |t|) sign^m.
    c, V, P, E = _tiny(n=8)
    Hd = ham.dense_h(c, V, P, E)
    lam, Q = sla.eigh(Hd)
    apply = lambda X: ham.apply_h(c, X, V, P, E)
    X = workloads.initial_orbitals(9, c.ngrid, 4)
    m, a, b = 9, lam[20], lam[-1] + 0.5
    a0 = lam[0]
    Y = chefsi.chebyshev_filter(apply, X, m, a, b, a0)

    def T(t):
        t = np.asarray(t, float)
        out = np.empty_like(t)
        inside = np.abs(t) <= 1
        out[inside] = np.cos(m * np.arccos(t[inside]))
        out[~inside] = np.sign(t[~inside]) ** m * np.cosh(m * np.arccosh(np.abs(t[~inside])))
        return out

    e, cc = (b - a) / 2, (b + a) / 2
    p = T((lam - cc) / e) / T(np.array([(a0 - cc) / e]))[0]
    ref = (Q @ (p[:, None] * (Q.T @ X.T))).T
    assert np.max(np.abs(Y - ref)) < 1e-10 * np.max(np.abs(ref))


def test_entropy_term_equals_grand_potential_identity_at_finite_temperature():
    # Fermi-Dirac occupations g = f_s f(x), x = (lambda - mu)/kT, satisfy, eigenvalue by eigenvalue,
    #   f ln f + (1 - f) ln(1 - f) = -ln(1 + e^-x) - f x,
    # so at fixed eigenvalues the Mermin term is
    #   -TS = -kT f_s sum_k w_k sum_n ln(1 + e^-x) - sum_k w_k sum_n g (lambda - mu)
    # (the grand potential of the occupied levels minus their band energy relative to mu).  This pins
    # the prefactor and sign of entropy_term at finite kT, where every candidate formula differs.
    rng = np.random.default_rng(5)
    for nspin, fs in ((1, 2.0), (2, 1.0)):
        eigs = np.sort(rng.normal(0.0, 0.05, size=(nspin, 3, 20)), axis=-1)
        kw = np.array([0.5, 0.3, 0.2])
        for kT in (0.002, 0.01, 0.03):
            nelec = 0.6 * fs * 20 * nspin / (2.0 if nspin == 1 else 1.0)
            mu, g = ham.fermi_occupations(eigs, kw, nelec, kT, fs)
            x = (eigs - mu) / kT
            wk = kw[None, :, None]
            ref = -kT * fs * np.sum(wk * np.logaddexp(0.0, -x)) - np.sum(wk * g * (eigs - mu))
            got = ham.entropy_term(g, kw, kT, fs)
            assert abs(got - ref) < 1e-13 * max(1.0, abs(ref)), (nspin, kT, got, ref)
            assert got < 0.0   # -TS is negative for fractional occupations
