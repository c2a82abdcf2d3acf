"""Self-consistent field loop, mixing, free energy and forces (Sec. 2.1).

* SCF: fixed point on the density; SAD initial guess; CheFSI partial diagonalisation with
  several filter passes in the first SCF iteration (Sec. 2.1).
* Mixing: periodic Pulay (A. S. Banerjee, P. Suryanarayana, J. E. Pask, Chem. Phys. Lett.
  647 (2016) 31) with optional restart (P. P. Pratapa, P. Suryanarayana, Chem. Phys. Lett.
  635 (2015) 69): Pulay extrapolation every `period`-th iteration, linear mixing otherwise.
  Spin-polarised runs mix the stacked vector [rho_up; rho_dn] (Sec. 2.1).
* Energy: Mermin free energy in the pseudocharge formulation; the per-iteration value is the
  Harris-Foulkes form at rho_in, the Kohn-Sham form at rho_out is reported at the end.
* Forces: Hellmann-Feynman derivative of the discrete free energy (Sec. 2.1, "Hellmann-Feynman
  atomic forces").
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

import workloads
from . import chefsi, gga, ham, isolated, model, xc


class PulayMixer:
    """x_{k+1} = x_k + beta f_k - (X_k + beta F_k) (F_k^T F_k)^{-1} F_k^T f_k on Pulay steps,
    x_{k+1} = x_k + beta f_k otherwise; f = x_out - x_in, X/F hold the last `hist` differences."""

    def __init__(self, beta=0.3, hist=7, period=1, restart=False):
        self.beta, self.hist, self.period, self.restart = beta, hist, period, restart
        self.k = 0
        self.dx, self.df = [], []
        self.x_prev = self.f_prev = None

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
            x_new = x_in + self.beta * f - (Xm + self.beta * Fm) @ gamma
            if self.restart:
                self.dx, self.df = [], []
        else:
            x_new = x_in + self.beta * f
        self.k += 1
        return x_new


@dataclasses.dataclass
class SCFResult:
    energy: float            # Harris-Foulkes free energy at the last iteration (Ha)
    energy_ks: float         # Kohn-Sham free energy at rho_out (Ha)
    eigs: np.ndarray         # (nspin, nk, nstates)
    occ: np.ndarray
    mu: float
    rho: np.ndarray          # (nspin, ngrid) output density
    phi: np.ndarray
    veff: np.ndarray
    blocks: list
    niter: int
    history: list            # per-iteration dicts
    converged: bool
    forces: np.ndarray = None


class Problem:
    """Geometry-dependent quantities of one cell (Sec. 2.1 setup)."""

    def __init__(self, cell):
        self.cell = cell
        self.dV = float(np.prod(cell.h))
        self.b = model.pseudocharge(cell)
        self.kpts, self.kw = cell.kpoints()
        self.P = [model.projectors(cell, tuple(k)) for k in self.kpts]
        self.E = model.kb_energies(cell)
        self.E_self = model.self_energy(cell)
        self.E_sc, self.dEsc = model.overlap_correction(cell)
        self.spin_factor = 2.0 if cell.nspin == 1 else 1.0

    def apply_h(self, V, ik):
        k = tuple(self.kpts[ik])
        return lambda X: ham.apply_h(self.cell, X, V, self.P[ik], self.E, k)

    def potentials(self, rho):
        """V_eff^s = phi + V_xc^s (Sec. 2.1); returns (veff (nspin, ngrid), phi, exc per electron)."""
        rho_tot = rho.sum(axis=0)
        if getattr(self.cell, "boundary", "periodic") == "dirichlet":
            phi = isolated.poisson_isolated(self.cell, rho_tot + self.b)
        else:
            phi = ham.poisson_exact(self.cell, rho_tot + self.b)
        if getattr(self.cell, "xc", "lda_pz") == "gga_pbe":
            if self.cell.nspin != 1:
                raise ValueError("the PBE oracle is spin-unpolarized")
            exc, vxc = gga.pbe_unpolarized(self.cell, rho_tot)
            vxc = vxc[None, :]
        elif self.cell.nspin == 1:
            exc, vxc = xc.lda_pz_unpolarized(rho_tot)
            vxc = vxc[None, :]
        else:
            exc, vu, vd = xc.lda_pz_polarized(rho[0], rho[1])
            vxc = np.stack([vu, vd])
        return phi[None, :] + vxc, phi, exc

    def electrostatic(self, rho_tot, phi):
        return 0.5 * self.dV * float(np.dot(rho_tot + self.b, phi))

    def free_energy_hf(self, eigs, occ, rho_in, veff, phi, exc, ts):
        """F_HF = sum w g lambda - dV sum V_eff rho_in + E_xc[rho_in] + 1/2 dV sum (rho_in+b) phi
        - E_self + E_sc - TS."""
        e_band = float(np.sum(self.kw[None, :, None] * occ * eigs))
        rho_tot = rho_in.sum(axis=0)
        return (e_band - self.dV * float(np.sum(veff * rho_in)) + self.dV * float(np.dot(exc, rho_tot))
                + self.electrostatic(rho_tot, phi) - self.E_self + self.E_sc + ts)

    def free_energy_ks(self, eigs, occ, rho_out, veff_in, ts):
        """Kohn-Sham form at rho_out: band energy minus the potential energy of V_eff^in gives
        the kinetic + nonlocal energy of the Ritz vectors; Hartree, local and XC at rho_out."""
        e_band = float(np.sum(self.kw[None, :, None] * occ * eigs))
        _, phi_o, exc_o = self.potentials(rho_out)
        rho_tot = rho_out.sum(axis=0)
        return (e_band - self.dV * float(np.sum(veff_in * rho_out)) + self.dV * float(np.dot(exc_o, rho_tot))
                + self.electrostatic(rho_tot, phi_o) - self.E_self + self.E_sc + ts)

    def forces(self, blocks, occ, phi):
        """F_a = -dV sum_x (d b/d R_a) phi - dE_sc/dR_a
                 - sum_{s,k,n} w_k g E_a dV 2 Re[conj(beta_a^H x) (d beta_a/dR_a)^H x]."""
        cell = self.cell
        F = -self.dEsc.copy()
        for a in range(cell.natom):
            db = model.pseudocharge_gradient(cell, a)
            F[a] -= self.dV * (db @ phi)
        for ik, k in enumerate(self.kpts):
            dP = model.projector_gradients(cell, tuple(k))
            for s in range(cell.nspin):
                X = blocks[s][ik]
                C = self.P[ik].conj() @ X.T              # (natom, nstates)
                for d in range(3):
                    D = dP[d].conj() @ X.T
                    t = 2.0 * np.real(np.conj(C) * D)    # (natom, nstates)
                    F[:, d] -= self.kw[ik] * self.dV * self.E * (t @ occ[s, ik])
        return F


def initial_blocks(cell, seed=None, nvec=None):
    """Starting orbitals for every (spin, k) problem from the shared counter-based generator
    (nvec rows, default nstates; the first nstates rows do not depend on nvec)."""
    kpts, _ = cell.kpoints()
    seed = cell.seed if seed is None else seed
    nvec = cell.nstates if nvec is None else nvec
    out = []
    for s in range(cell.nspin):
        row = []
        for ik in range(kpts.shape[0]):
            cplx = bool(np.any(kpts[ik] != 0))
            row.append(workloads.initial_orbitals(problem_seed(seed, s, ik, kpts.shape[0]),
                                                  cell.ngrid, nvec, cplx))
        out.append(row)
    return out


def problem_seed(seed, s, ik, nk):
    return int(seed) * 4099 + s * nk + ik


def initial_density(cell, rho0=None, moment=0.125):
    """SAD guess split into spins as rho (1 +- zeta0)/2 for spin-polarised runs."""
    rho = model.sad_density(cell) if rho0 is None else np.asarray(rho0, float).reshape(-1)
    if cell.nspin == 1:
        return rho[None, :]
    return np.stack([0.5 * rho * (1 + moment), 0.5 * rho * (1 - moment)])


def scf(cell, max_iter=100, tol=None, mix_beta=0.3, mix_hist=7, pulay_period=1, pulay_restart=False,
        first_passes=4, rho0=None, blocks=None, lanczos_steps=20, final_tol=None, final_max_passes=60,
        with_forces=False, verbose=False, ref_energy=None, nbuffer=0, degree=None, kerker_k0=None):
    """SCF fixed point on the density with CheFSI (Sec. 2.1).

    final_tol: if given, after density convergence keep doing CheFSI passes at the final
    V_eff until max |H x - lambda x| < final_tol (used for tight parity references).

    Solver choices that leave the fixed point unchanged (the self-consistent density built from
    the lowest nstates eigenpairs of H[rho] with Fermi-Dirac occupations over those nstates):
      nbuffer    extra filtered vectors that are never occupied.  The filter cutoff becomes the
                 top Ritz value of the larger block, so the partially occupied states at the top
                 of the nstates block are no longer next to the cutoff, where the Chebyshev
                 filter barely separates them (Zhou et al. 2006 use such buffer states too);
      degree     Chebyshev degree (default: the cell's);
      kerker_k0  if given, Kerker-preconditioned periodic Pulay mixing (oracle.kerker, Sec. 2.1
                 preconditioned mixing) with this screening wavevector instead of plain Pulay."""
    tol = cell.scf_tol if tol is None else tol
    pr = Problem(cell)
    nk = pr.kpts.shape[0]
    ns = cell.nstates
    degree = cell.cheb_degree if degree is None else int(degree)
    rho_in = initial_density(cell, rho0)
    blocks = initial_blocks(cell, nvec=ns + nbuffer) if blocks is None else blocks
    if kerker_k0 is None:
        mixer = PulayMixer(mix_beta, mix_hist, pulay_period, pulay_restart)
    else:
        from .kerker import KerkerPulayMixer
        mixer = KerkerPulayMixer(cell, kerker_k0, mix_beta, mix_hist, pulay_period, pulay_restart,
                                 nchan=cell.nspin)
    bounds = {}
    hist = []
    t0 = time.time()
    converged = False
    it = 0
    for it in range(max_iter):
        veff, phi, exc = pr.potentials(rho_in)
        eigs = np.zeros((cell.nspin, nk, cell.nstates))
        for s in range(cell.nspin):
            for ik in range(nk):
                H = pr.apply_h(veff[s], ik)
                if it == 0:
                    lo, up = chefsi.lanczos_bounds(H, blocks[s][ik][0], lanczos_steps)
                    bounds[s, ik] = [lo, lo + 0.1 * (up - lo), up]
                for _ in range(first_passes if it == 0 else 1):
                    a0, a, b = bounds[s, ik]
                    lam, blocks[s][ik] = chefsi.chefsi_pass(H, blocks[s][ik], degree, a, b, a0)
                    bounds[s, ik] = [lam[0], lam[-1], b]
                eigs[s, ik] = lam[:ns]
        mu, occ = ham.fermi_occupations(eigs, pr.kw, cell.nelec, cell.kT, pr.spin_factor)
        ts = ham.entropy_term(occ, pr.kw, cell.kT, pr.spin_factor)
        rho_out = ham.density(_lowest(blocks, ns), occ, pr.kw, pr.dV)
        F = pr.free_energy_hf(eigs, occ, rho_in, veff, phi, exc, ts)
        err = float(np.linalg.norm(rho_out - rho_in) / np.linalg.norm(rho_out))
        hist.append(dict(iter=it, energy=F, err=err, mu=mu, t=time.time() - t0))
        if verbose:
            print(f"scf {it:3d}  F={F:.12f}  err={err:.3e}  mu={mu:.8f}  t={time.time()-t0:.1f}s", flush=True)
        if err < tol:
            converged = True
            break
        rho_in = mixer.update(rho_in.reshape(-1), rho_out.reshape(-1)).reshape(rho_in.shape)
    if final_tol is not None:
        for _ in range(final_max_passes):
            worst = 0.0
            for s in range(cell.nspin):
                for ik in range(nk):
                    H = pr.apply_h(veff[s], ik)
                    a0, a, b = bounds[s, ik]
                    lam, blocks[s][ik] = chefsi.chefsi_pass(H, blocks[s][ik], degree, a, b, a0)
                    bounds[s, ik] = [lam[0], lam[-1], b]
                    eigs[s, ik] = lam[:ns]
                    nocc = int(np.sum(occ[s, ik] > 1e-12 * pr.spin_factor)) + 1
                    res = chefsi.residual_norms(H, blocks[s][ik][:nocc], lam[:nocc])
                    worst = max(worst, float(res.max()))
            if worst < final_tol:
                break
        mu, occ = ham.fermi_occupations(eigs, pr.kw, cell.nelec, cell.kT, pr.spin_factor)
        ts = ham.entropy_term(occ, pr.kw, cell.kT, pr.spin_factor)
        rho_out = ham.density(_lowest(blocks, ns), occ, pr.kw, pr.dV)
        F = pr.free_energy_hf(eigs, occ, rho_in, veff, phi, exc, ts)
    Fks = pr.free_energy_ks(eigs, occ, rho_out, veff, ts)
    blocks = _lowest(blocks, ns)
    res = SCFResult(F, Fks, eigs, occ, mu, rho_out, phi, veff, blocks, it + 1, hist, converged)
    if with_forces:
        res.forces = pr.forces(blocks, occ, phi)
    return res


def _lowest(blocks, ns):
    """The lowest ns Ritz vectors of every (spin, k) block (buffer vectors dropped)."""
    return [[X[:ns] for X in row] for row in blocks]
