"""Several independent cells of uneven grid size filtered together: one column-tile stencil launch
per Chebyshev step covers every cell.  Each cell's result must be bitwise the one of filtering it
alone with the same tile, and the smallest cell is checked against the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import chefsi, ham, model  # noqa: E402


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_10431_gb300 import build
    build.build()
    import paper_2005_10431_gb300 as m
    return m


def test_multi_cell_filter_matches_single_cells_and_oracle(sd, monkeypatch):
    monkeypatch.setenv("SDFT_STENCIL_VARIANT", "0")   # the column tile the multi-cell launch uses
    cells = workloads.uneven_cells(count=6, seed=3)
    ctxs, xs, ys, Vs, Xs = [], [], [], [], []
    a, b, a0 = [], [], []
    for i, c in enumerate(cells):
        ctx = sd.sdft_create(c.L, c.n, c.pos, c.types, c.species, dict(nstates=c.nstates, precision=sd.SDFT_MIXED))
        V = np.random.default_rng(i).normal(0, 0.3, c.ngrid)
        sd.sdft_set_veff(ctx, 0, V)
        X = workloads.initial_orbitals(50 + i, c.ngrid, c.nstates)
        ctxs.append(ctx)
        Vs.append(V)
        Xs.append(X)
        xs.append(sd.pack_block(X, sd.SDFT_MIXED))
        ys.append(torch.empty_like(xs[-1]))
        a.append(2.0 + 0.1 * i)
        b.append(90.0 + i)
        a0.append(-1.0 - 0.05 * i)
    deg = 6
    sd.sdft_chebyshev_filter_multi(ctxs, xs, ys, deg, a, b, a0)
    for i, c in enumerate(cells):
        y1 = torch.empty_like(xs[i])
        sd.sdft_chebyshev_filter(ctxs[i], 0, 0, sd.SDFT_MIXED, xs[i], y1, c.nstates, deg, a[i], b[i], a0[i])
        assert torch.equal(ys[i], y1), f"cell {i} ({c.n}) differs from its single-cell filter"
    # the smallest cell against the FP64 oracle (FP32 filter tolerance 3e-5 per step)
    i = int(np.argmin([c.ngrid for c in cells]))
    c = cells[i]
    P = model.projectors(c)
    E = model.kb_energies(c)
    ref = chefsi.chebyshev_filter(lambda Z: ham.apply_h(c, Z, Vs[i], P, E), Xs[i], deg, a[i], b[i], a0[i])
    got = sd.unpack_block(ys[i], sd.SDFT_MIXED, False)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 3e-5 * deg


def test_multi_cell_filter_rejects_complex_and_fp64(sd):
    c = workloads.uneven_cells(count=1, seed=3)[0]
    ctx = sd.sdft_create(c.L, c.n, c.pos, c.types, c.species, dict(nstates=c.nstates, precision=sd.SDFT_FP64))
    x = torch.zeros((c.nstates, c.ngrid), dtype=torch.float64, device="cuda")
    with pytest.raises(sd.SdftError):
        sd.sdft_chebyshev_filter_multi([ctx], [x], [torch.empty_like(x)], 4, [2.0], [90.0], [-1.0])


def test_batch_scf_matches_cell_by_cell(sd, monkeypatch):
    """sdft_batch_scf over four uneven cells (multi-cell filter) and one FP64 context (filtered on
    its own inside the lockstep): every context's SCF is bitwise the one it runs alone with the
    same stencil tile -- same iteration count, energies and eigenvalues."""
    monkeypatch.setenv("SDFT_STENCIL_VARIANT", "0")   # the column tile the multi-cell launch uses
    cells = workloads.uneven_cells(count=4, seed=5)
    specs = [(c, sd.SDFT_MIXED) for c in cells] + [(cells[0], sd.SDFT_FP64)]

    def make(c, prec):
        return sd.sdft_create(c.L, c.n, c.pos, c.types, c.species,
                              dict(nstates=c.nstates, precision=prec, scf_tol=1e-6, max_scf=30))

    alone = []
    for c, prec in specs:
        ctx = make(c, prec)
        r = sd.sdft_scf(ctx)
        alone.append((r, sd.sdft_get_eigenvalues(ctx), sd.sdft_get_forces(ctx)))
        sd.sdft_destroy(ctx)
    ctxs = [make(c, prec) for c, prec in specs]
    rs = sd.sdft_batch_scf(ctxs)
    for i, (r, eig, frc) in enumerate(alone):
        assert rs[i]["niter"] == r["niter"]
        assert rs[i]["converged"] == r["converged"]
        assert rs[i]["energy"] == r["energy"]
        assert rs[i]["energy_ks"] == r["energy_ks"]
        assert np.array_equal(sd.sdft_get_eigenvalues(ctxs[i]), eig)
        assert np.array_equal(sd.sdft_get_forces(ctxs[i]), frc)
    for ctx in ctxs:
        sd.sdft_destroy(ctx)


def test_batch_scf_rejects_repeated_context(sd):
    c = workloads.uneven_cells(count=1, seed=5)[0]
    ctx = sd.sdft_create(c.L, c.n, c.pos, c.types, c.species, dict(nstates=c.nstates, precision=sd.SDFT_MIXED))
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_batch_scf([ctx, ctx])
    assert e.value.code == -1
    sd.sdft_destroy(ctx)


def test_batch_scf_of_uneven_cells_converges_with_buffer_states(sd):
    """The uneven cells of the batching workload reach the density tolerance 1e-6 within 100 SCF
    iterations in the lockstep batch when their filtered blocks carry buffer states and the last
    iterations take FP32 Rayleigh-Ritz GEMMs (without them several cells stop at the cap)."""
    cells = workloads.uneven_cells(count=8, seed=3)
    stream = torch.cuda.Stream()
    ctxs = [sd.sdft_create(c.L, c.n, c.pos, c.types, c.species,
                           dict(nstates=c.nstates, nbuffer=4, cheb_degree=c.cheb_degree, precision=sd.SDFT_MIXED,
                                scf_tol=1e-6, max_scf=100, kT=c.kT, seed=c.seed, gemm_fp32_switch_tol=4e-6),
                           stream=stream) for c in cells]
    rs = sd.sdft_batch_scf(ctxs)
    assert all(r["converged"] for r in rs), [r["niter"] for r in rs]
    for ctx, c in zip(ctxs, cells):
        # the orbital norms carry FP32 rounding: the density integrates to nelec to ~1e-7 relative
        rho = sd.sdft_get_density(ctx)
        assert abs(float(np.prod(c.h)) * rho.sum() - c.nelec) < 1e-6 * c.nelec
        sd.sdft_destroy(ctx)
