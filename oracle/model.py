"""Synthetic pseudopotential model on the periodic grid (Sec. 2.1).

The paper uses the pseudopotential approximation with a local real-space electrostatics
formulation: the ionic charge is smeared into pseudocharges b(x) so that the electrostatic
potential phi (ionic + Hartree) solves one Poisson problem, -L phi = 4 pi (rho + b).  Its
ONCV psp8 files are not available, so every atom here carries

* a Gaussian pseudocharge  b_a(r) = -Z (2 pi r_loc^2)^(-3/2) exp(-r^2 / (2 r_loc^2)),
  whose potential is the Goedecker-Teter-Hutter-style local part -Z erf(r/(sqrt2 r_loc))/r;
* one s-channel Kleinman-Bylander projector
  chi(r) = (pi^(3/2) r_p^3)^(-1/2) exp(-r^2/(2 r_p^2)) for r < r_c  (continuum norm 1),
  giving V_nl = sum_a E_KB |beta_a><beta_a| ("outer product nature", Sec. 2.1);
* for the superposition-of-atomic-densities guess (Sec. 2.1), a Gaussian atomic density
  Z (2 pi s^2)^(-3/2) exp(-r^2/(2 s^2)).

Periodic images are summed explicitly; Bloch projectors carry the phase exp(i k.T) of the
image T they come from.  Grid point (i,j,k) sits at h*(i,j,k); flat index i + n1 (j + n2 k).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp
from scipy.special import erfc

B_CUTOFF_FACTOR = 10.0    # pseudocharge summed for r <= 10 r_loc
SAD_CUTOFF_FACTOR = 10.0  # SAD Gaussian summed for r <= 10 s


def grid_axes(cell):
    return [np.arange(cell.n[d]) * cell.h[d] for d in range(3)]


def _images(center, rcut, L):
    """Integer image vectors t (T = t*L) whose ball of radius rcut around center+T meets the cell."""
    rng = []
    for d in range(3):
        lo = math.floor((-rcut - center[d]) / L[d]) - 1
        hi = math.ceil((L[d] + rcut - center[d]) / L[d]) + 1
        rng.append(range(lo, hi + 1))
    return itertools.product(*rng)


def _cell_images(cell, center, rcut):
    """Periodic images of an atom-centred sum; an isolated (Dirichlet) cell has the atom itself only."""
    if getattr(cell, "boundary", "periodic") == "dirichlet":
        return [(0, 0, 0)]
    return _images(center, rcut, cell.L)


def _ball_points(cell, c, rcut, strict):
    """Grid points of the cell within rcut of the point c (no wrapping): returns
    (flat indices, displacement vectors x - c)."""
    sub = []
    for d in range(3):
        h = cell.h[d]
        lo = max(0, math.ceil((c[d] - rcut) / h))
        hi = min(cell.n[d] - 1, math.floor((c[d] + rcut) / h))
        if hi < lo:
            return None, None
        sub.append(np.arange(lo, hi + 1))
    dx = sub[0] * cell.h[0] - c[0]
    dy = sub[1] * cell.h[1] - c[1]
    dz = sub[2] * cell.h[2] - c[2]
    Z, Y, X = np.meshgrid(dz, dy, dx, indexing="ij")
    r2 = X * X + Y * Y + Z * Z
    mask = (r2 < rcut * rcut) if strict else (r2 <= rcut * rcut)
    kk, jj, ii = np.meshgrid(sub[2], sub[1], sub[0], indexing="ij")
    flat = ii + cell.n[0] * (jj + cell.n[1] * kk)
    disp = np.stack([X[mask], Y[mask], Z[mask]], axis=-1)
    return flat[mask], disp


def _sum_gaussians(cell, amp_of, width_of, cut_factor):
    """sum_a sum_T amp_a exp(-|x - R_a - T|^2 / (2 w_a^2)) over r <= cut_factor * w_a."""
    out = np.zeros(cell.ngrid)
    L = cell.L
    for a in range(cell.natom):
        w = width_of(a)
        rcut = cut_factor * w
        for t in _cell_images(cell, cell.pos[a], rcut):
            c = cell.pos[a] + np.array(t) * np.array(L)
            idx, disp = _ball_points(cell, c, rcut, strict=False)
            if idx is None or idx.size == 0:
                continue
            r2 = np.sum(disp * disp, axis=1)
            np.add.at(out, idx, amp_of(a) * np.exp(-r2 / (2.0 * w * w)))
    return out


def pseudocharge(cell) -> np.ndarray:
    """b(x) = sum_a sum_T b_a(x - R_a - T); integrates to -sum Z (Sec. 2.1 pseudocharges)."""
    sp_ = cell.species
    return _sum_gaussians(
        cell,
        lambda a: -sp_[cell.types[a]].Z * (2 * np.pi * sp_[cell.types[a]].r_loc ** 2) ** -1.5,
        lambda a: sp_[cell.types[a]].r_loc, B_CUTOFF_FACTOR)


def pseudocharge_gradient(cell, a: int) -> tuple:
    """d b / d R_a as three grid arrays: (x - R_a - T)/r_loc^2 * b_a(x - R_a - T)."""
    s = cell.species[cell.types[a]]
    amp = -s.Z * (2 * np.pi * s.r_loc ** 2) ** -1.5
    rcut = B_CUTOFF_FACTOR * s.r_loc
    out = np.zeros((3, cell.ngrid))
    for t in _cell_images(cell, cell.pos[a], rcut):
        c = cell.pos[a] + np.array(t) * np.array(cell.L)
        idx, disp = _ball_points(cell, c, rcut, strict=False)
        if idx is None or idx.size == 0:
            continue
        r2 = np.sum(disp * disp, axis=1)
        val = amp * np.exp(-r2 / (2 * s.r_loc ** 2))
        for d in range(3):
            np.add.at(out[d], idx, disp[:, d] / s.r_loc ** 2 * val)
    return out


def sad_density(cell) -> np.ndarray:
    """Superposition of atomic densities (Sec. 2.1), renormalised so that h^3 sum rho = N_e."""
    sp_ = cell.species
    rho = _sum_gaussians(
        cell,
        lambda a: sp_[cell.types[a]].Z * (2 * np.pi * sp_[cell.types[a]].sad_width ** 2) ** -1.5,
        lambda a: sp_[cell.types[a]].sad_width, SAD_CUTOFF_FACTOR)
    dV = float(np.prod(cell.h))
    return rho * (cell.nelec / (dV * rho.sum()))


def projector_value(r2: np.ndarray, rp: float) -> np.ndarray:
    return (np.pi ** 1.5 * rp ** 3) ** -0.5 * np.exp(-r2 / (2.0 * rp * rp))


def projectors(cell, kred=(0.0, 0.0, 0.0)) -> sp.csr_matrix:
    """Bloch KB projectors beta_a(x) = sum_T exp(i k.T) chi(x - R_a - T), r < r_c strictly,
    as a sparse (natom x ngrid) matrix (real for k = 0).  k.T = 2 pi kred.t."""
    rows, cols, vals = [], [], []
    cplx = any(abs(k) > 0 for k in kred)
    for a in range(cell.natom):
        s = cell.species[cell.types[a]]
        for t in _cell_images(cell, cell.pos[a], s.r_cut_proj):
            c = cell.pos[a] + np.array(t) * np.array(cell.L)
            idx, disp = _ball_points(cell, c, s.r_cut_proj, strict=True)
            if idx is None or idx.size == 0:
                continue
            v = projector_value(np.sum(disp * disp, axis=1), s.r_proj)
            if cplx:
                v = v * np.exp(2j * np.pi * np.dot(kred, t))
            rows.append(np.full(idx.size, a))
            cols.append(idx)
            vals.append(v)
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(cell.natom, cell.ngrid), dtype=complex if cplx else float)
    return P.tocsr()   # duplicates (a point reached from two images) are summed


def projector_gradients(cell, kred=(0.0, 0.0, 0.0)) -> list:
    """d beta_a / d R_a along each direction d: sum_T exp(ik.T) (x-R_a-T)_d / r_p^2 chi(...)."""
    mats = []
    cplx = any(abs(k) > 0 for k in kred)
    for d in range(3):
        rows, cols, vals = [], [], []
        for a in range(cell.natom):
            s = cell.species[cell.types[a]]
            for t in _cell_images(cell, cell.pos[a], s.r_cut_proj):
                c = cell.pos[a] + np.array(t) * np.array(cell.L)
                idx, disp = _ball_points(cell, c, s.r_cut_proj, strict=True)
                if idx is None or idx.size == 0:
                    continue
                v = disp[:, d] / s.r_proj ** 2 * projector_value(np.sum(disp * disp, axis=1), s.r_proj)
                if cplx:
                    v = v * np.exp(2j * np.pi * np.dot(kred, t))
                rows.append(np.full(idx.size, a))
                cols.append(idx)
                vals.append(v)
        mats.append(sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                  shape=(cell.natom, cell.ngrid),
                                  dtype=complex if cplx else float).tocsr())
    return mats


def kb_energies(cell) -> np.ndarray:
    return np.array([cell.species[cell.types[a]].E_kb for a in range(cell.natom)])


def self_energy(cell) -> float:
    """E_self = sum_a Z_a^2 / (2 sqrt(pi) r_loc): Coulomb self-energy of each Gaussian."""
    return float(sum(cell.species[t].Z ** 2 / (2 * np.sqrt(np.pi) * cell.species[t].r_loc)
                     for t in cell.types))


def _pair_images(cell, rmax):
    if getattr(cell, "boundary", "periodic") == "dirichlet":
        return [(0, 0, 0)]
    n = [int(math.ceil(rmax / cell.L[d])) + 1 for d in range(3)]
    return itertools.product(range(-n[0], n[0] + 1), range(-n[1], n[1] + 1), range(-n[2], n[2] + 1))


def overlap_correction(cell, rmax: float = 30.0) -> tuple:
    """E_sc = 1/2 sum_{(a,T) != (a',0)} Z_a Z_a' erfc(d / s) / d, s = sqrt(2 (r_a^2 + r_a'^2)),
    d = |R_a - R_a' - T|: point-ion minus Gaussian-Gaussian interaction.  Returns (E_sc, dE/dR)."""
    E = 0.0
    grad = np.zeros((cell.natom, 3))
    L = np.array(cell.L)
    for a in range(cell.natom):
        sa = cell.species[cell.types[a]]
        for b in range(cell.natom):
            sb = cell.species[cell.types[b]]
            s = np.sqrt(2.0 * (sa.r_loc ** 2 + sb.r_loc ** 2))
            for t in _pair_images(cell, rmax):
                if a == b and t == (0, 0, 0):
                    continue
                v = cell.pos[a] - cell.pos[b] - np.array(t) * L
                d = float(np.linalg.norm(v))
                if d > rmax:
                    continue
                E += 0.5 * sa.Z * sb.Z * erfc(d / s) / d
                if a != b:
                    dfd = sa.Z * sb.Z * (-2.0 / (s * np.sqrt(np.pi)) * np.exp(-(d / s) ** 2) / d
                                         - erfc(d / s) / d ** 2)
                    grad[a] += dfd * v / d
    return E, grad
