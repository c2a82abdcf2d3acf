"""End-to-end SCF parity on the GPU against the FP64 CPU oracle.

FP64 path: converged free energy within 1e-9 Ha/atom and occupied eigenvalues within 1e-8 Ha
of the oracle (both sides converged to an SCF error of 1e-10).  Mixed path (FP32 filter): within
1e-5 Ha/atom, 1e-5 Ha eigenvalues and 1e-4 Ha/bohr forces.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import scf as oscf  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_10431_gb300 import build
    build.build()
    import paper_2005_10431_gb300 as m
    return m


def _run(sd, cell, precision, tol, final=0, max_scf=300, kpts=None, kw=None, **extra):
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=cell.nstates, cheb_degree=cell.cheb_degree, precision=precision,
                              scf_tol=tol, max_scf=max_scf, final_fp64_pass=final, nspin=cell.nspin,
                              kT=cell.kT, seed=cell.seed, **extra),
                         kpts=kpts, kw=kw)
    r = sd.sdft_scf(ctx)
    return ctx, r


def _gold(name):
    return json.load(open(os.path.join(HERE, "golden", name + ".json")))


def test_fp64_scf_two_atom_matches_oracle(sd):
    cell = workloads.two_atom_cell()
    g = _gold("two_atom_24")
    ctx, r = _run(sd, cell, sd.SDFT_FP64, 1e-10)
    assert r["converged"]
    assert abs(r["energy"] - g["energy"]) / cell.natom < 1e-9
    assert abs(r["energy_ks"] - g["energy_ks"]) / cell.natom < 1e-9
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-10))
    assert np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc])) < 1e-8
    f = sd.sdft_get_forces(ctx)
    assert np.max(np.abs(f - np.array(g["forces"]))) < 1e-6
    rho = sd.sdft_get_density(ctx)
    dV = float(np.prod(cell.h))
    assert abs(dV * rho.sum() - cell.nelec) < 1e-9
    log = sd.sdft_get_scf_log(ctx)
    assert len(log) == r["niter"] and log[-1]["scf_error"] < 1e-10


def test_mixed_scf_two_atom_matches_oracle(sd):
    cell = workloads.two_atom_cell()
    g = _gold("two_atom_24")
    ctx, r = _run(sd, cell, sd.SDFT_MIXED, 1e-6, final=1)
    assert r["converged"]
    assert abs(r["energy"] - g["energy"]) / cell.natom < 1e-5
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-10))
    assert np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc])) < 1e-5
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < 1e-4


def test_mixed_scf_lattice64_fp64_tail_matches_converged_oracle(sd):
    # the same cell finishing with FP64 passes instead: converged, and tighter against the oracle
    cell = workloads.lattice64_cell()
    g = _gold("lattice64_80")
    ctx, r = _run(sd, cell, sd.SDFT_MIXED, cell.scf_tol, max_scf=100, nbuffer=LATTICE64_NBUFFER,
                  fp64_switch_tol=LATTICE64_GEMM_SWITCH)
    assert r["converged"]
    assert abs(r["energy"] - g["energy"]) / cell.natom < 1e-8
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    assert np.max(np.abs(eig - np.array(g["eigs"])[0, 0])) < 1e-5
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < 1e-5


def test_mixed_scf_with_fp64_tail_reaches_the_fp64_fixed_point(sd):
    # the mixed run continues in FP64 below an SCF error of 1e-5 and then meets the FP64 bounds
    cell = workloads.two_atom_cell()
    g = _gold("two_atom_24")
    ctx, r = _run(sd, cell, sd.SDFT_MIXED, 1e-10, fp64_switch_tol=1e-5)
    assert r["converged"]
    log = sd.sdft_get_scf_log(ctx)
    assert any(rec["scf_error"] < 1e-5 for rec in log[:-3])      # the switch happened well before the end
    assert abs(r["energy"] - g["energy"]) / cell.natom < 1e-9
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-10))
    assert np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc])) < 1e-8
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < 1e-6


@pytest.mark.parametrize("nbuffer", [2, 6])
def test_fp64_scf_with_buffer_states_reaches_the_same_fixed_point(sd, nbuffer):
    # extra filtered, never occupied orbitals: the FP64 fixed point of the 8-state cell is unchanged
    cell = workloads.two_atom_cell()
    g = _gold("two_atom_24")
    ctx, r = _run(sd, cell, sd.SDFT_FP64, 1e-10, nbuffer=nbuffer)
    assert r["converged"]
    assert abs(r["energy"] - g["energy"]) / cell.natom < 1e-9
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    assert eig.shape == (cell.nstates,)
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-10))
    assert np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc])) < 1e-8
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < 1e-6
    x = torch.empty(cell.nstates, cell.ngrid, dtype=torch.float64, device="cuda")
    sd.sdft_get_orbitals(ctx, 0, 0, x)      # the lowest nstates Ritz vectors, orthonormal (X^T X = I)
    X = x.cpu().numpy()
    assert np.max(np.abs(X @ X.T - np.eye(cell.nstates))) < 1e-8


def _displaced_small():
    c = workloads.small_cell(npts=12, L=4.5, natom=2, nstates=6, degree=12)
    c.pos = np.array([[0.3, 0.2, 0.1], [2.4, 2.1, 2.6]])
    return c


def test_fp64_forces_match_oracle_on_displaced_cell(sd):
    cell = _displaced_small()
    ref = oscf.scf(_displaced_small(), tol=1e-10, max_iter=300, with_forces=True)
    ctx, r = _run(sd, cell, sd.SDFT_FP64, 1e-10)
    assert abs(r["energy"] - ref.energy) / cell.natom < 1e-9
    f = sd.sdft_get_forces(ctx)
    assert np.max(np.abs(f)) > 1e-3
    assert np.max(np.abs(f - ref.forces)) < 1e-7


def test_fp64_spin_kpoint_scf_matches_oracle(sd):
    # spin-polarised, two k-points (one complex), on a small cell
    cell = _displaced_small()
    cell.nspin = 2
    cell.kpts = np.array([[0.0, 0.0, 0.0], [0.25, 0.0, -0.25]])
    cell.kw = np.array([0.5, 0.5])
    # The spin-polarised run relaxes a soft spin mode slowly and its SCF error levels off near
    # 3e-9 (energy already converged to ~1e-10), so both sides stop at 1e-8 here.
    ref = oscf.scf(cell, tol=1e-8, max_iter=300)
    ctx, r = _run(sd, cell, sd.SDFT_FP64, 1e-8, kpts=cell.kpts, kw=cell.kw)
    assert r["converged"]
    assert abs(r["energy"] - ref.energy) / cell.natom < 1e-9
    eig = sd.sdft_get_eigenvalues(ctx)
    nocc = 4
    assert np.max(np.abs(eig[:, :, :nocc] - ref.eigs[:, :, :nocc])) < 1e-8


def test_not_converged_status_returns_partial_result(sd):
    cell = workloads.two_atom_cell()
    ctx, r = _run(sd, cell, sd.SDFT_FP64, 1e-12, max_scf=3)
    assert r["status"] == -4 and r["niter"] == 3 and not r["converged"]
    assert len(sd.sdft_get_scf_log(ctx)) == 3
    assert np.isfinite(r["energy"])


def _qmd8_72():
    c = workloads.qmd_lattice8_cell(2000)
    c.nstates = 72
    return c


@pytest.mark.parametrize("final", [0, 1])
def test_mixed_scf_through_tensor_core_gemms_and_refined_eigensolver_matches_oracle(sd, monkeypatch, final):
    # 8 atoms, 40^3, 72 real states: the blocks are wide enough for the tcgen05 BF16x3 Gram and
    # rotation (real FP32 blocks of >= 32 columns) and the refined eigensolver (64 < n <= 160), whose
    # device-side check sends a rejected solve to cuSOLVER; most solves must be the refined ones.  The
    # converged oracle reference is tests/golden/qmd8_72.json.  The BF16x3 rotation (about 17
    # significant bits) holds the mixed SCF's density residual near 3e-6, so the mixed run stops at
    # 1e-5; its energy, occupied eigenvalues and forces must still meet the mixed bounds (1e-5 Ha/atom,
    # 1e-5 Ha, 1e-4 Ha/bohr), and with the final FP64 pass the energy and eigenvalues tighten to 1e-7.
    cell = _qmd8_72()
    g = _gold("qmd8_72")
    assert g["converged"] and g["nstates"] == 72
    ctx, r = _run(sd, cell, sd.SDFT_MIXED, 1e-5, final=final, max_scf=150)
    accepted, rejected = sd.sdft_get_eig_stats(ctx)
    assert accepted >= 10 and rejected <= accepted // 4, (accepted, rejected)
    assert r["converged"], [f"{rec['scf_error']:.2e}" for rec in sd.sdft_get_scf_log(ctx)[-8:]]
    tol_e, tol_eig = (1e-5, 1e-5) if final == 0 else (1e-7, 1e-6)
    assert abs(r["energy"] - g["energy"]) / cell.natom < tol_e
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-6))
    assert nocc >= 16
    assert np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc])) < tol_eig
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < 1e-4


def test_fp64_scf_72_states_matches_oracle(sd):
    # the same cell on the FP64 path: the oracle's fixed point to the FP64 bounds
    cell = _qmd8_72()
    g = _gold("qmd8_72")
    ctx, r = _run(sd, cell, sd.SDFT_FP64, 1e-9, max_scf=150)
    assert r["converged"]
    assert abs(r["energy"] - g["energy"]) / cell.natom < 1e-9
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-6))
    assert np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc])) < 1e-8
    assert np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"]))) < 1e-6


# buffer states of the 64-atom cell (the oracle reference used 26), and the SCF error below which its
# mixed run takes FP32 CUDA-core Rayleigh-Ritz GEMMs (with the BF16x3 tensor-core products the mixed
# density residual levels off near 1.2e-6 there)
LATTICE64_NBUFFER = 26
LATTICE64_GEMM_SWITCH = 4e-6


def test_mixed_scf_lattice64_matches_converged_oracle(sd):
    # The benchmark cell (64 atoms, 80^3, 154 states) in the benchmark's configuration: mixed
    # precision, buffer states, FP32 CUDA-core GEMMs for the last iterations, the final FP64 pass, at
    # most 100 SCF iterations; it must reach the density tolerance.  The converged oracle reference (tests/golden/lattice64_80.json, SCF
    # error 5e-9) bounds the mixed path: free energy within 1e-5 Ha/atom, eigenvalues of all 154
    # states (the top ones partially occupied) within 1e-5 Ha, forces within 1e-4 Ha/bohr.  Without
    # buffer states the top four states sit at the filter cutoff and stay ~1e-3 Ha off.
    cell = workloads.lattice64_cell()
    g = _gold("lattice64_80")
    assert g["converged"] and g["nstates"] == cell.nstates
    ctx, r = _run(sd, cell, sd.SDFT_MIXED, cell.scf_tol, final=1, max_scf=100, nbuffer=LATTICE64_NBUFFER,
                  gemm_fp32_switch_tol=LATTICE64_GEMM_SWITCH)
    assert r["converged"], [f"{rec['scf_error']:.2e}" for rec in sd.sdft_get_scf_log(ctx)[-6:]]
    de = abs(r["energy"] - g["energy"]) / cell.natom
    eig = sd.sdft_get_eigenvalues(ctx)[0, 0]
    occ = np.array(g["occ"])[0, 0]
    nocc = int(np.sum(occ > 1e-6))
    deig = np.max(np.abs(eig[:nocc] - np.array(g["eigs"])[0, 0, :nocc]))
    df = np.max(np.abs(sd.sdft_get_forces(ctx) - np.array(g["forces"])))
    msg = f"dE/atom {de:.2e}, max d eig {deig:.2e} over {nocc} states, max d force {df:.2e}, niter {r['niter']}"
    assert de < 1e-5, msg
    assert deig < 1e-5, msg
    assert df < 1e-4, msg
