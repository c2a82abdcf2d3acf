"""Isolated systems (paper Sec. 2, 2.1: Dirichlet boundary conditions, multipole boundary values of the
electrostatic potential) on the GPU against the FP64 oracle (oracle/isolated.py and the Dirichlet forms
of oracle/ham.py and oracle/model.py): the Poisson solve and H X elementwise, and the SCF of an isolated
two-atom molecule against the oracle's converged reference (tests/golden/isolated_pair_30.json) at
the FP64 bounds."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import ham, isolated, model  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_10431_gb300 import build
    build.build()
    import paper_2005_10431_gb300 as m
    return m


def _box(n=(22, 20, 18), L=(8.8, 8.0, 7.2), pos=((3.9, 4.2, 3.4), (5.2, 3.5, 3.9))):
    c = workloads.small_cell(npts=12, L=4.0, natom=2, seed=1, nstates=6)
    c.n, c.L = n, L
    c.pos = np.array(pos)
    c.types = np.zeros(2, int)
    c.boundary = "dirichlet"
    return c


def _ctx(sd, cell):
    return sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                          dict(nstates=cell.nstates, precision=sd.SDFT_FP64, boundary=sd.SDFT_BC_DIRICHLET))


def test_isolated_poisson_matches_oracle(sd):
    cell = _box()
    ctx = _ctx(sd, cell)
    x, y, z = isolated.grid_coords(cell)
    f = np.zeros(cell.ngrid)
    for (a, q, s) in (((4.0, 3.7, 3.3), 1.3, 0.7), ((5.1, 4.4, 3.9), -0.8, 0.9), ((3.3, 4.9, 3.0), 0.4, 0.6)):
        f += q * (2 * np.pi * s * s) ** -1.5 * np.exp(-((x - a[0]) ** 2 + (y - a[1]) ** 2 + (z - a[2]) ** 2) / (2 * s * s))
    ref = isolated.poisson_isolated(cell, f)
    fd_ = torch.from_numpy(f.copy()).cuda()
    phi = torch.zeros_like(fd_)
    sd.sdft_poisson(ctx, fd_, phi, tol=1e-12, max_iter=20000)
    assert np.max(np.abs(phi.cpu().numpy() - ref)) < 1e-9 * np.max(np.abs(ref))


def test_isolated_apply_h_and_setup_fields_match_oracle(sd):
    cell = _box()
    ctx = _ctx(sd, cell)
    assert np.max(np.abs(sd.sdft_get_pseudocharge(ctx) - model.pseudocharge(cell))) < 1e-12 * 2.0
    assert np.max(np.abs(sd.sdft_get_sad_density(ctx) - model.sad_density(cell))) < 1e-12
    V = np.random.default_rng(3).normal(0, 0.3, cell.ngrid)
    sd.sdft_set_veff(ctx, 0, V)
    X = workloads.initial_orbitals(5, cell.ngrid, 6)
    x = sd.pack_block(X, sd.SDFT_FP64)
    y = torch.empty_like(x)
    sd.sdft_apply_h(ctx, 0, 0, sd.SDFT_FP64, x, y, 6)
    ref = ham.apply_h(cell, X, V, model.projectors(cell), model.kb_energies(cell))
    got = sd.unpack_block(y, sd.SDFT_FP64, False)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_isolated_molecule_scf_matches_oracle(sd):
    g = json.load(open(os.path.join(HERE, "golden", "isolated_pair_30.json")))
    cell = workloads.isolated_pair_cell()
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=cell.nstates, cheb_degree=cell.cheb_degree, precision=sd.SDFT_FP64,
                              scf_tol=1e-10, max_scf=300, kT=cell.kT, seed=cell.seed, boundary=sd.SDFT_BC_DIRICHLET))
    r = sd.sdft_scf(ctx)
    assert r["converged"]
    assert abs(r["energy"] - g["energy"]) / cell.natom < 1e-9
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-10))
    assert np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc])) < 1e-8
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < 1e-6


def test_dirichlet_needs_fp64_gamma(sd):
    cell = _box()
    with pytest.raises(sd.SdftError):
        sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                       dict(nstates=6, precision=sd.SDFT_MIXED, boundary=sd.SDFT_BC_DIRICHLET))
