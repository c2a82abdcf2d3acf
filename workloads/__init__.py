"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds no arithmetic of the Kohn-Sham method itself: only cell/grid
sizes, atom positions and the counter-based random numbers that seed the
eigensolver.  Both sides receive what it produces as plain arrays.

Workload shapes follow the paper's illustrative systems: periodic cells of
O(100-500) atoms, Gamma point, LDA, mesh sizes of 0.2-0.55 bohr (Sec. 3, Sec. 4).
The paper's own structures and pseudopotential files are not available, so
synthetic cells of the same shape stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------
# splitmix64 (Steele, Lea & Flood 2014, as published by S. Vigna), used as a
# counter-based generator: value i of stream `seed` is mix(seed * 2^32 + i + GOLDEN).
# The CUDA library implements the same published definition for on-device
# generation; both sides then draw bit-identical numbers.
# ---------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 output for a uint64 counter array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_counter(seed: int, index: np.ndarray) -> np.ndarray:
    """Uniform doubles in [-0.5, 0.5): top 53 bits of splitmix64(seed*2^32 + index)."""
    base = np.uint64((int(seed) & 0xFFFFFFFF) << 32)
    z = splitmix64(base + index.astype(np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) - 0.5


def initial_orbitals(seed: int, ngrid: int, nstates: int, complex_valued: bool = False) -> np.ndarray:
    """Random starting block X0, shape (nstates, ngrid): orbital n occupies one row.

    Entry (n, g) is uniform_counter(seed, n*ngrid + g).  For a complex block the
    imaginary part uses stream seed+0x5bd1 with the same counter.
    """
    idx = np.arange(nstates * ngrid, dtype=np.uint64)
    re = uniform_counter(seed, idx).reshape(nstates, ngrid)
    if not complex_valued:
        return re
    im = uniform_counter(seed + 0x5BD1, idx).reshape(nstates, ngrid)
    return re + 1j * im


# ---------------------------------------------------------------------------
# Cells
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Species:
    """Synthetic pseudo-atom: Gaussian local part + one s-channel KB projector."""
    Z: float = 4.0          # valence charge
    r_loc: float = 0.5      # width of the Gaussian pseudocharge (bohr)
    r_proj: float = 0.6     # width of the Gaussian KB projector (bohr)
    E_kb: float = 1.0       # KB energy (Ha)
    r_cut_proj: float = 3.0  # projector support radius (bohr)
    sad_width: float = 1.0  # width of the atomic density used by the SAD guess (bohr)


@dataclasses.dataclass
class Cell:
    name: str
    L: tuple            # cell edges (bohr)
    n: tuple            # grid points per edge
    pos: np.ndarray     # (natom, 3) bohr
    types: np.ndarray   # (natom,) int
    species: list
    nstates: int
    cheb_degree: int
    kT: float = 0.01
    nspin: int = 1
    kpts: np.ndarray = None     # (nk, 3) reduced coordinates
    kw: np.ndarray = None       # (nk,) weights summing to 1
    scf_tol: float = 1e-6
    seed: int = 0
    xc: str = "lda_pz"          # exchange-correlation functional: "lda_pz" or "gga_pbe" (unpolarized)
    boundary: str = "periodic"  # "periodic", or "dirichlet" (isolated system: zero orbitals outside the grid,
                                # electrostatic boundary values from a multipole expansion)

    @property
    def natom(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nelec(self) -> float:
        return float(sum(self.species[t].Z for t in self.types))

    @property
    def ngrid(self) -> int:
        return int(np.prod(self.n))

    @property
    def h(self) -> tuple:
        return tuple(self.L[d] / self.n[d] for d in range(3))

    def kpoints(self):
        if self.kpts is None:
            return np.zeros((1, 3)), np.ones(1)
        return np.asarray(self.kpts, float), np.asarray(self.kw, float)


def nstates_rule(nelec: float) -> int:
    """Number of states: max(Ne/2 + 4, 1.2 Ne/2) rounded up to even."""
    v = max(nelec / 2 + 4, 1.2 * nelec / 2)
    n = int(math.ceil(v - 1e-9))
    return n + (n % 2)


def lattice_positions(ncell: int, spacing: float, sigma: float, seed: int) -> np.ndarray:
    """Simple-cubic lattice, atom (i,j,k) at spacing*(i,j,k) + spacing/2*(1,1,1) + delta,
    delta ~ N(0, sigma^2) per component from numpy's default_rng(seed)."""
    ijk = np.array([(i, j, k) for k in range(ncell) for j in range(ncell) for i in range(ncell)], float)
    pos = spacing * ijk + 0.5 * spacing
    if sigma > 0:
        pos = pos + np.random.default_rng(seed).normal(0.0, sigma, size=pos.shape)
    return pos


SPACING = 5.13
H_MESH = 0.2565


def two_atom_cell() -> Cell:
    """Edge 6.0 bohr, 24^3 grid (h = 0.25), atoms at (0,0,0) and (3,3,3), 8 states, degree 12."""
    return Cell("two_atom_24", (6.0, 6.0, 6.0), (24, 24, 24),
                np.array([[0.0, 0.0, 0.0], [3.0, 3.0, 3.0]]), np.zeros(2, int), [Species()],
                nstates=8, cheb_degree=12, scf_tol=1e-6, seed=0)


def lattice_cell(ncell: int, npts: int, sigma: float, seed: int, degree: int, name: str) -> Cell:
    pos = lattice_positions(ncell, SPACING, sigma, seed)
    L = ncell * SPACING
    nat = pos.shape[0]
    return Cell(name, (L, L, L), (npts, npts, npts), pos, np.zeros(nat, int), [Species()],
                nstates=nstates_rule(4.0 * nat), cheb_degree=degree, scf_tol=1e-6, seed=seed)


def lattice64_cell(seed: int = 0, sigma: float = 0.1) -> Cell:
    """64 atoms on a 4x4x4 lattice, edge 20.52 bohr, 80^3 grid, 154 states, degree 20."""
    return lattice_cell(4, 80, sigma, seed, 20, "lattice64_80")


def lattice216_cell(seed: int = 1, sigma: float = 0.1) -> Cell:
    """216 atoms on a 6x6x6 lattice, edge 30.78 bohr, 120^3 grid, 520 states, degree 24."""
    return lattice_cell(6, 120, sigma, seed, 24, "lattice216_120")


def small_cell(npts: int = 12, L: float = 4.0, natom: int = 1, seed: int = 7, nstates: int = 6,
               degree: int = 10) -> Cell:
    """Tiny cell for brute-force checks (dense diagonalisation is affordable)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, L, size=(natom, 3))
    return Cell(f"small_{npts}", (L, L, L), (npts, npts, npts), pos, np.zeros(natom, int),
                [Species()], nstates=nstates, cheb_degree=degree, seed=seed)


def isolated_pair_cell() -> Cell:
    """Isolated (Dirichlet) two-atom molecule: a 9.9 bohr box, 30^3 grid (h = 0.33), atoms 1.8 bohr apart
    around the box centre, 8 states, degree 14."""
    n, L = 30, 9.9
    ctr = 0.5 * (n - 1) * L / n
    pos = np.array([[ctr - 0.9, ctr + 0.1, ctr - 0.05], [ctr + 0.9, ctr - 0.1, ctr + 0.05]])
    return Cell("isolated_pair_30", (L, L, L), (n, n, n), pos, np.zeros(2, int), [Species()], nstates=8,
                cheb_degree=14, scf_tol=1e-6, seed=11, boundary="dirichlet")


def monkhorst_pack(nk: int) -> tuple:
    """nk^3 Monkhorst-Pack grid in reduced coordinates (2n - nk - 1)/(2 nk), equal weights."""
    g = (2.0 * np.arange(1, nk + 1) - nk - 1) / (2.0 * nk)
    k = np.array([(a, b, c) for c in g for b in g for a in g])
    return k, np.full(k.shape[0], 1.0 / k.shape[0])


def kpoint_cell(nk: int = 4, npts: int = 40) -> Cell:
    """8-atom undisplaced 2x2x2 lattice cell, edge 10.26, 40^3 grid, nk^3 MP k-grid, 2 spins."""
    pos = lattice_positions(2, SPACING, 0.0, 0)
    k, w = monkhorst_pack(nk)
    c = Cell("kpoint8_40", (2 * SPACING,) * 3, (npts,) * 3, pos, np.zeros(8, int), [Species()],
             nstates=nstates_rule(32.0), cheb_degree=20, nspin=2, kpts=k, kw=w)
    return c


def uneven_cells(count: int = 32, seed: int = 3) -> list:
    """Independent small cells: n_i uniform in [24, 48], edge n_i*0.2565,
    natom = clamp(round((L/5.13)^3), 2, 16), uniform positions with >= 3.0 bohr separation."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        n = int(rng.integers(24, 49))
        L = n * H_MESH
        nat = int(min(16, max(2, round((L / SPACING) ** 3))))
        pos = []
        while len(pos) < nat:
            p = rng.uniform(0.0, L, 3)
            ok = True
            for q in pos:
                d = p - q
                d -= L * np.round(d / L)
                if np.linalg.norm(d) < 3.0:
                    ok = False
                    break
            if ok:
                pos.append(p)
        out.append(Cell(f"uneven{c}_{n}", (L, L, L), (n, n, n), np.array(pos), np.zeros(nat, int),
                        [Species()], nstates=nstates_rule(4.0 * nat), cheb_degree=20, seed=seed))
    return out


# ---------------------------------------------------------------------------
# learned initial density: QMD-like configuration sequences and network initialisation
# ---------------------------------------------------------------------------
def qmd_lattice64_cell(seed: int, sigma: float = 0.15) -> Cell:
    """One configuration of the 64-atom sequence: the 4x4x4 lattice (edge 20.52, 80^3 grid,
    154 states, degree 20) with Gaussian displacements sigma = 0.15 bohr drawn with `seed`."""
    c = lattice_cell(4, 80, sigma, seed, 20, f"qmd64_{seed}")
    return c


def qmd_lattice8_cell(seed: int, sigma: float = 0.15) -> Cell:
    """Small member of the same family for tests: 2x2x2 lattice, edge 10.26 bohr, 40^3 grid
    (h = 0.2565), Gamma point, degree 16, displacements sigma = 0.15 bohr.  28 states: the
    states-count rule's 20 leaves partially occupied states (kT = 0.01 Ha) at the top of the
    subspace of this metallic cell, where the filter barely converges them."""
    c = lattice_cell(2, 40, sigma, seed, 16, f"qmd8_{seed}")
    c.nstates = 28
    return c


def qmd_trajectory(pos0: np.ndarray, nsteps: int, amplitude: float = 0.15, seed: int = 0,
                   steps_per_period: float = 24.0) -> list:
    """Smooth synthetic trajectory for QMD-style tests: atom a moves as
    R_a(t) = R_a(0) + A_a (sin(w_a t + p_a) - sin(p_a)), with amplitudes A_a ~ N(0, amplitude^2) per
    component, angular frequencies w_a = 2 pi / steps_per_period * u_a, u_a uniform in [0.8, 1.2], and
    phases p_a uniform in [0, 2 pi), all from numpy's default_rng(seed).  Returns nsteps (natom, 3) arrays."""
    rng = np.random.default_rng(seed)
    n = pos0.shape[0]
    amp = rng.normal(0.0, amplitude, size=(n, 3))
    w = 2.0 * np.pi / steps_per_period * rng.uniform(0.8, 1.2, size=(n, 3))
    ph = rng.uniform(0.0, 2.0 * np.pi, size=(n, 3))
    return [pos0 + amp * (np.sin(w * t + ph) - np.sin(ph)) for t in range(nsteps)]


MLP_NFEAT, MLP_HIDDEN = 32, 64
MLP_NPARAM = MLP_HIDDEN * MLP_NFEAT + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1


def mlp_init_params(seed: int) -> np.ndarray:
    """Flat FP32 parameter vector (W1 [64x32], b1, W2 [64x64], b2, w3, b3): weights uniform in
    +-sqrt(6/(fan_in+fan_out)) (Glorot) from uniform_counter(seed, i), biases zero."""
    sizes = [(MLP_HIDDEN, MLP_NFEAT), (MLP_HIDDEN,), (MLP_HIDDEN, MLP_HIDDEN), (MLP_HIDDEN,), (1, MLP_HIDDEN), (1,)]
    out, off = [], 0
    for shp in sizes:
        n = int(np.prod(shp))
        if len(shp) == 2:
            a = math.sqrt(6.0 / (shp[0] + shp[1]))
            out.append(2.0 * a * uniform_counter(seed, np.arange(off, off + n, dtype=np.uint64)))
        else:
            out.append(np.zeros(n))
        off += n
    return np.concatenate(out).astype(np.float32)


def kspin_small_cell() -> Cell:
    """Batched-CheFSI parity cell: 2 atoms in a 5.13 bohr cube, 20^3 grid, 2 spins, 2x2x2
    Monkhorst-Pack k-points (8 complex): 16 filter problems of 8 Bloch orbitals, degree 12."""
    rng_free_pos = np.array([[0.4, 0.3, 0.2], [2.9, 2.5, 2.8]])
    k, w = monkhorst_pack(2)
    return Cell("kspin_20", (5.13, 5.13, 5.13), (20, 20, 20), rng_free_pos, np.zeros(2, int), [Species()],
                nstates=8, cheb_degree=12, nspin=2, kpts=k, kw=w, seed=7)
