"""Batched CheFSI: the (spin, k-point) problems of a context filtered together (one grouped
stencil launch and one grouped KB projection per Chebyshev step for all problems, one batched
eigensolve) must give the same SCF as the problem-by-problem path, and match the FP64 oracle
to the mixed-precision tolerances (1e-5 Ha/atom energy, 1e-5 Ha eigenvalues).
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_10431_gb300 import build
    build.build()
    import paper_2005_10431_gb300 as m
    return m


def _gold(name):
    return json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name + ".json")))


def _run(sd, cell, batch, tol, graphs=1, max_scf=200):
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=cell.nstates, cheb_degree=cell.cheb_degree, precision=sd.SDFT_MIXED,
                              scf_tol=tol, max_scf=max_scf, nspin=cell.nspin, kT=cell.kT, seed=cell.seed,
                              batch_problems=batch, use_graphs=graphs),
                         kpts=cell.kpts, kw=cell.kw)
    n0 = sd.sdft_launch_count(ctx)
    r = sd.sdft_scf(ctx)
    return ctx, r, sd.sdft_launch_count(ctx) - n0


def test_batched_chefsi_matches_problem_by_problem_and_oracle(sd):
    cell = workloads.kspin_small_cell()   # 2 spins x 8 complex k-points = 16 problems
    ref = _gold("kspin_20")
    cb, rb, lb = _run(sd, cell, 1, 1e-6)
    cs, rs, ls = _run(sd, cell, 0, 1e-6)
    assert rb["converged"] and rs["converged"]
    # the grouped launches ran (a row tile fits the 20^3 complex blocks)
    idx, name = sd.sdft_get_stencil_variant(cb, True)
    assert name.startswith("row")
    assert abs(rb["energy"] - rs["energy"]) / cell.natom < 1e-6
    assert abs(rb["energy"] - ref["energy"]) / cell.natom < 1e-5
    eb = sd.sdft_get_eigenvalues(cb)
    nocc = 3
    assert np.max(np.abs(eb[:, :, :nocc] - np.array(ref["eigs"])[:, :, :nocc])) < 1e-5
    # fewer launches per SCF iteration than one problem at a time
    assert lb / rb["niter"] < 0.5 * ls / rs["niter"]


def test_graph_replay_of_the_grouped_filter_is_exact(sd):
    """The CUDA graph replays the same launches with the same tables: the SCF history is bitwise the
    one of the directly launched batched filter."""
    cell = workloads.kspin_small_cell()
    cg, rg, lg = _run(sd, cell, 1, 1e-12, graphs=1, max_scf=8)
    cd, rd, ld = _run(sd, cell, 1, 1e-12, graphs=0, max_scf=8)
    eg = [r["energy"] for r in sd.sdft_get_scf_log(cg)]
    ed = [r["energy"] for r in sd.sdft_get_scf_log(cd)]
    assert len(eg) == len(ed) == 8
    assert eg == ed
    assert np.array_equal(sd.sdft_get_density(cg), sd.sdft_get_density(cd))
    assert lg == ld      # replayed graph launches are counted like direct ones


def test_batched_chefsi_with_buffer_states_matches_oracle(sd):
    # buffer states change the filtered block width (grouped launches, batched eigensolve over
    # nstates + nbuffer) but not the fixed point: the oracle's occupied eigenvalues and energy hold
    cell = workloads.kspin_small_cell()
    ref = _gold("kspin_20")
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=cell.nstates, nbuffer=4, cheb_degree=cell.cheb_degree, precision=sd.SDFT_MIXED,
                              scf_tol=1e-6, max_scf=200, nspin=cell.nspin, kT=cell.kT, seed=cell.seed,
                              batch_problems=1),
                         kpts=cell.kpts, kw=cell.kw)
    r = sd.sdft_scf(ctx)
    assert r["converged"]
    assert abs(r["energy"] - ref["energy"]) / cell.natom < 1e-5
    e = sd.sdft_get_eigenvalues(ctx)
    assert e.shape == (cell.nspin, len(cell.kpts), cell.nstates)
    assert np.max(np.abs(e[:, :, :3] - np.array(ref["eigs"])[:, :, :3])) < 1e-5
