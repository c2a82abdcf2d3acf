"""GPU parity of each hot-path step against the FP64 CPU oracle, elementwise, through the C ABI.

Tolerances: FP64 kernels agree with the oracle to round-off (1e-12 relative for one H X,
growing linearly with the number of recurrence steps).  FP32 (SDFT_MIXED) kernels: one H X
has relative error ~ (37 terms) * 2^-24 * |stencil sum| / |H X| -> 2e-5 of max|H X| is used;
the degree-m filter accumulates ~m such errors -> 3e-5 * m relative to max|Y|.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads  # noqa: E402
from oracle import chefsi, ham, model, xc  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_10431_gb300 import build
    build.build()
    import paper_2005_10431_gb300 as m
    return m


def _ctx(sd, cell, precision, nstates, kpts=None, nspin=1):
    return sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                          dict(nstates=nstates, precision=precision, nspin=nspin), kpts=kpts)


def _ragged_cell():
    # 9 x 10 x 11 grid (ragged against the 32 x 8 stencil tile), orthorhombic, 3 atoms
    c = workloads.small_cell(npts=10, L=4.0, natom=3, seed=21, nstates=6)
    c.n = (9, 10, 11)
    c.L = (3.6, 4.0, 4.4)
    return c


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_setup_fields_match_oracle(sd):
    for cell in (workloads.two_atom_cell(), _ragged_cell()):
        ctx = _ctx(sd, cell, sd.SDFT_FP64, 6)
        b = sd.sdft_get_pseudocharge(ctx)
        sad = sd.sdft_get_sad_density(ctx)
        assert _relerr(b, model.pseudocharge(cell)) < 1e-12
        assert _relerr(sad, model.sad_density(cell)) < 1e-12


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kred", [(0.0, 0.0, 0.0), (0.25, -0.375, 0.5)])
def test_apply_h_matches_oracle(sd, precision, kred):
    cell = _ragged_cell()
    cplx = any(kred)
    ns = 6
    ctx = _ctx(sd, cell, precision, ns, kpts=[kred] if cplx else None)
    V = np.random.default_rng(1).normal(0, 0.4, cell.ngrid)
    sd.sdft_set_veff(ctx, 0, V)
    X = workloads.initial_orbitals(3, cell.ngrid, ns, complex_valued=cplx)
    x = sd.pack_block(X, precision)
    y = torch.empty_like(x)
    sd.sdft_apply_h(ctx, 0, 0, precision, x, y, ns)
    P = model.projectors(cell, kred)
    ref = ham.apply_h(cell, X, V, P, model.kb_energies(cell), kred)
    got = sd.unpack_block(y, precision, cplx)
    tol = 1e-12 if precision == sd.SDFT_FP64 else 2e-5
    assert _relerr(got, ref) < tol


# FP32 tile variants compiled for each storage kind: (name, grid that the variant fits).
# Row tiles need an even n1, TY | n2 and (n1/2)*TY threads in [64, max]; the grids below give
# each row variant a shape it accepts (and several z chunks, ragged against the queue length).
REAL_VARIANTS = [("col32x8", (9, 10, 11)), ("col32x8pf3", (9, 10, 11)), ("col32x16", (9, 10, 11)),
                 ("col32x4", (9, 10, 11)), ("col32x8occ3", (9, 10, 11)), ("col32x8occ4", (9, 10, 11)),
                 ("col32x4occ6", (9, 10, 11)), ("row4", (40, 40, 29)), ("row8", (40, 40, 29)),
                 ("row5", (40, 40, 29)), ("row6", (24, 36, 31))]
CPLX_VARIANTS = [("col32x8", (9, 10, 11)), ("col32x8pf3", (9, 10, 11)), ("row4", (40, 40, 29)),
                 ("row8", (40, 40, 29)), ("row10", (40, 40, 29))]


def _variant_cell(n):
    c = workloads.small_cell(npts=10, L=4.0, natom=3, seed=21, nstates=6)
    c.n = n
    c.L = tuple(0.3 * k + 0.6 for k in n) if n[0] > 12 else (3.6, 4.0, 4.4)
    rng = np.random.default_rng(5)
    c.pos = rng.uniform(0, 1, (3, 3)) * np.array(c.L)
    return c


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("variant", range(11))
def test_every_stencil_tile_variant_matches_oracle(sd, variant, cplx, monkeypatch):
    # The autotuner may pick any compiled tile shape; each one must give the same filter output.
    # 6 real states = 3 orbital pairs, so the two-column variants also run a ragged tail.
    table = CPLX_VARIANTS if cplx else REAL_VARIANTS
    if variant >= len(table):
        pytest.skip("no such variant for this storage kind")
    name, n = table[variant]
    kred = (0.25, 0.125, -0.5) if cplx else (0.0, 0.0, 0.0)
    monkeypatch.setenv("SDFT_STENCIL_VARIANT", str(variant))
    cell = _variant_cell(n)
    ns = 6
    ctx = _ctx(sd, cell, sd.SDFT_MIXED, ns, kpts=[kred] if cplx else None)
    V = np.random.default_rng(11).normal(0, 0.4, cell.ngrid)
    sd.sdft_set_veff(ctx, 0, V)
    X = workloads.initial_orbitals(13, cell.ngrid, ns, complex_valued=cplx)
    x = sd.pack_block(X, sd.SDFT_MIXED)
    y = torch.empty_like(x)
    sd.sdft_chebyshev_filter(ctx, 0, 0, sd.SDFT_MIXED, x, y, ns, 4, 3.0, 90.0, -1.5)
    assert sd.sdft_get_stencil_variant(ctx, cplx) == (variant, name)
    P = model.projectors(cell, kred)
    ref = chefsi.chebyshev_filter(lambda Z: ham.apply_h(cell, Z, V, P, model.kb_energies(cell), kred), X, 4,
                                  3.0, 90.0, -1.5)
    assert _relerr(sd.unpack_block(y, sd.SDFT_MIXED, cplx), ref) < 3e-5 * 4


# TMA-fed slab tiles (real FP32 blocks): variant index in the real table, grid, and a cell whose KB
# spheres overlap in pairs but never three at a point (the tile stages two KB slots per point).
# n2 = 24 gives slabs at the lower periodic y boundary, in the interior and at the upper boundary;
# n3 = 40 gives several z chunks with a ragged last one; 6 states = 3 pairs, a ragged pair group.
SLAB_VARIANTS = [(11, "slab80", (80, 24, 40)), (12, "slab80np1", (80, 24, 40)), (13, "slab120", (120, 24, 30)),
                 (14, "slab40", (40, 24, 40)), (15, "slab80ry2", (80, 24, 40))]


def _slab_cell(n):
    h = 0.3
    c = workloads.small_cell(npts=10, L=4.0, natom=3, seed=21, nstates=6)
    c.n = n
    c.L = tuple(h * k for k in n)
    c.pos = np.array([[3.0, 2.0, 1.5], [6.5, 4.5, 4.0], [9.5, 5.5, 5.0]]) if n[0] == 40 else \
        np.array([[3.0, 2.0, 1.5], [6.5, 4.5, 4.0], [16.0, 3.0, 3.0]])
    c.types = np.zeros(3, int)
    return c


@pytest.mark.parametrize("variant,name,n", SLAB_VARIANTS)
def test_slab_stencil_variants_match_oracle(sd, variant, name, n, monkeypatch):
    monkeypatch.setenv("SDFT_STENCIL_VARIANT", str(variant))
    cell = _slab_cell(n)
    ns = 6
    ctx = _ctx(sd, cell, sd.SDFT_MIXED, ns)
    V = np.random.default_rng(17).normal(0, 0.4, cell.ngrid)
    sd.sdft_set_veff(ctx, 0, V)
    X = workloads.initial_orbitals(19, cell.ngrid, ns)
    x = sd.pack_block(X, sd.SDFT_MIXED)
    y = torch.empty_like(x)
    P = model.projectors(cell)
    E = model.kb_energies(cell)
    # one H X (no recurrence term), then a degree-4 filter (with the Yprev term)
    sd.sdft_apply_h(ctx, 0, 0, sd.SDFT_MIXED, x, y, ns)
    assert sd.sdft_get_stencil_variant(ctx, False) == (variant, name)
    ref = ham.apply_h(cell, X, V, P, E)
    assert _relerr(sd.unpack_block(y, sd.SDFT_MIXED, False), ref) < 2e-5
    sd.sdft_chebyshev_filter(ctx, 0, 0, sd.SDFT_MIXED, x, y, ns, 4, 3.0, 90.0, -1.5)
    assert sd.sdft_get_stencil_variant(ctx, False) == (variant, name)
    ref = chefsi.chebyshev_filter(lambda Z: ham.apply_h(cell, Z, V, P, E), X, 4, 3.0, 90.0, -1.5)
    assert _relerr(sd.unpack_block(y, sd.SDFT_MIXED, False), ref) < 3e-5 * 4


# the step that also sums its output's KB coefficients (slab tiles with one row per thread) against
# the separate projection pass, on the 64-atom cell (two KB slots per point, 64 projector spheres):
# the same filter to FP32 rounding, and only the first step's projection is a separate launch
@pytest.mark.parametrize("variant", [11, 12])
def test_fused_kb_projection_matches_separate_pass(sd, variant, monkeypatch):
    cell = workloads.lattice64_cell()
    ns, m = cell.nstates, 8
    monkeypatch.setenv("SDFT_STENCIL_VARIANT", str(variant))
    X = workloads.initial_orbitals(3, cell.ngrid, ns)
    V = np.random.default_rng(5).normal(-0.3, 0.2, cell.ngrid)
    out, nproj = {}, {}
    for fuse in ("1", "0"):
        monkeypatch.setenv("SDFT_FUSE_KB", fuse)
        ctx = _ctx(sd, cell, sd.SDFT_MIXED, ns)
        sd.sdft_set_veff(ctx, 0, V)
        x = sd.pack_block(X, sd.SDFT_MIXED)
        y = torch.empty_like(x)
        sd.sdft_set_timing(ctx, True)
        sd.sdft_chebyshev_filter(ctx, 0, 0, sd.SDFT_MIXED, x, y, ns, m, 3.0, 90.0, -1.5)
        torch.cuda.synchronize()
        assert sd.sdft_get_stencil_variant(ctx, False)[0] == variant
        nproj[fuse] = sd.sdft_get_kernel_stats(ctx)["kb_project"]["launches"]
        out[fuse] = sd.unpack_block(y, sd.SDFT_MIXED, False)
        sd.sdft_destroy(ctx)
    assert nproj == {"1": 1, "0": m}
    assert np.max(np.abs(out["1"] - out["0"])) < 2e-5 * np.max(np.abs(out["0"]))


def test_full_size_block_matches_oracle_on_sampled_orbitals(sd):
    # the 64-atom cell at full size -- 80^3 points, 154 states + 26 buffer states, the block the
    # benchmark filters, with the stencil tile the autotuner picks for it as in the benchmark: a
    # degree-20 Chebyshev filter and H X of the whole block on the GPU against the oracle applied
    # to three sampled orbitals (the columns are independent), at every grid point
    cell = workloads.lattice64_cell()
    ns = cell.nstates + 26
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                         dict(nstates=cell.nstates, nbuffer=26, precision=sd.SDFT_MIXED))
    V = np.random.default_rng(5).normal(-0.3, 0.2, cell.ngrid)
    sd.sdft_set_veff(ctx, 0, V)
    X = workloads.initial_orbitals(7, cell.ngrid, ns)
    x = sd.pack_block(X, sd.SDFT_MIXED)
    y = torch.empty_like(x)
    P, E = model.projectors(cell), model.kb_energies(cell)
    cols = [0, 77, ns - 1]
    sd.sdft_chebyshev_filter(ctx, 0, 0, sd.SDFT_MIXED, x, y, ns, 20, 1.0, 250.0, -1.5)
    ref = chefsi.chebyshev_filter(lambda Z: ham.apply_h(cell, Z, V, P, E), X[cols], 20, 1.0, 250.0, -1.5)
    assert _relerr(sd.unpack_block(y, sd.SDFT_MIXED, False)[cols], ref) < 3e-5 * 20
    sd.sdft_apply_h(ctx, 0, 0, sd.SDFT_MIXED, x, y, ns)
    assert _relerr(sd.unpack_block(y, sd.SDFT_MIXED, False)[cols], ham.apply_h(cell, X[cols], V, P, E)) < 2e-5
    sd.sdft_destroy(ctx)


def test_slab_cell_has_at_most_two_kb_slots():
    # the slab test cells must stay within the tile's two staged KB slots per point
    for _, _, n in SLAB_VARIANTS:
        cell = _slab_cell(n)
        P = model.projectors(cell)
        per_point = np.asarray((P != 0).sum(axis=0)).ravel()
        assert per_point.max() <= 2


@pytest.mark.parametrize("precision", [0, 1])
def test_chebyshev_filter_matches_oracle(sd, precision):
    cell = _ragged_cell()
    ns, m = 6, 10
    ctx = _ctx(sd, cell, precision, ns)
    V = np.random.default_rng(2).normal(0, 0.4, cell.ngrid)
    sd.sdft_set_veff(ctx, 0, V)
    X = workloads.initial_orbitals(4, cell.ngrid, ns)
    a, b, a0 = 3.0, 90.0, -1.5
    x = sd.pack_block(X, precision)
    y = torch.empty_like(x)
    sd.sdft_chebyshev_filter(ctx, 0, 0, precision, x, y, ns, m, a, b, a0)
    P = model.projectors(cell)
    ref = chefsi.chebyshev_filter(lambda Z: ham.apply_h(cell, Z, V, P, model.kb_energies(cell)), X, m, a, b, a0)
    tol = 1e-11 if precision == sd.SDFT_FP64 else 3e-5 * m
    assert _relerr(sd.unpack_block(y, precision, False), ref) < tol


@pytest.mark.parametrize("kred", [(0.0, 0.0, 0.0), (0.5, 0.25, 0.0)])
def test_rayleigh_ritz_fp64_matches_oracle(sd, kred):
    cell = _ragged_cell()
    cplx = any(kred)
    ns = 6
    ctx = _ctx(sd, cell, sd.SDFT_FP64, ns, kpts=[kred] if cplx else None)
    V = np.random.default_rng(3).normal(0, 0.4, cell.ngrid)
    sd.sdft_set_veff(ctx, 0, V)
    P = model.projectors(cell, kred)
    apply = lambda Z: ham.apply_h(cell, Z, V, P, model.kb_energies(cell), kred)
    Y = chefsi.chebyshev_filter(apply, workloads.initial_orbitals(6, cell.ngrid, ns, cplx), 8, 5.0, 80.0, -2.0)
    lam_ref, X_ref = chefsi.rayleigh_ritz(apply, Y)
    y = sd.pack_block(Y, sd.SDFT_FP64)
    x = torch.empty_like(y)
    eig = torch.empty(ns, dtype=torch.float64, device="cuda")
    sd.sdft_rayleigh_ritz(ctx, 0, 0, sd.SDFT_FP64, y, x, eig, ns)
    assert np.allclose(eig.cpu().numpy(), lam_ref, rtol=0, atol=1e-10 * np.max(np.abs(lam_ref)))
    X = sd.unpack_block(x, sd.SDFT_FP64, cplx)
    # eigenvectors are unique up to a phase per (non-degenerate) column: compare projectors
    for n in range(ns):
        ov = abs(np.vdot(X_ref[n], X[n]))
        assert abs(ov - 1.0) < 1e-9


def test_subspace_matrices_and_rotation_mixed(sd):
    cell = _ragged_cell()
    ns = 6
    ctx = _ctx(sd, cell, sd.SDFT_MIXED, ns)
    rng = np.random.default_rng(7)
    Y = rng.normal(size=(ns, cell.ngrid))
    HY = rng.normal(size=(ns, cell.ngrid))
    Y32 = Y.astype(np.float32).astype(np.float64)
    HY32 = HY.astype(np.float32).astype(np.float64)
    m = torch.empty(ns, ns, dtype=torch.float64, device="cuda")
    h = torch.empty_like(m)
    sd.sdft_subspace_matrices(ctx, 0, sd.SDFT_MIXED, sd.pack_block(Y, 1), sd.pack_block(HY, 1), m, h, ns)
    M_ref = Y32 @ Y32.T
    H_ref = Y32 @ HY32.T
    H_ref = 0.5 * (H_ref + H_ref.T)
    scale = np.sqrt(np.outer(np.diag(M_ref), np.diag(M_ref)))
    # column-major result: element (i, j) at i + j*ns -> tensor [j, i]
    assert np.max(np.abs(m.cpu().numpy().T - M_ref) / scale) < 1e-5
    Hs = h.cpu().numpy().T
    # the library mirrors the upper triangle of Y^T HY
    upper = np.triu(Y32 @ HY32.T)
    H_lib_ref = upper + np.triu(upper, 1).T
    assert np.max(np.abs(Hs - H_lib_ref) / scale) < 1e-5
    Q = rng.normal(size=(ns, ns))
    q = torch.from_numpy(np.ascontiguousarray(Q.T)).cuda()   # column-major Q
    x = torch.empty_like(sd.pack_block(Y, 1))
    sd.sdft_rotate(ctx, 0, sd.SDFT_MIXED, sd.pack_block(Y, 1), q, x, ns)
    ref = (Y32.T @ Q.astype(np.float32).astype(np.float64)).T
    assert _relerr(sd.unpack_block(x, 1, False), ref) < 1e-5


# (orbitals, grid): 154 = two 128-row tiles with a ragged 26-row one; 40 = one narrow tile; 258 and
# 520 = three and five tiles (the rotation in two and three 144/176-column blocks); grids with a
# ragged last 32-point stage and 128-point tile; an odd point count (no TMA copies of the paired
# layout: the CUDA-core path) must give the same result
GEMM_CASES = [(154, (9, 10, 11)), (154, (9, 11, 14)), (154, (40, 40, 40)), (40, (9, 10, 11)),
              (258, (9, 10, 11)), (520, (12, 12, 10)), (154, (9, 11, 13))]


@pytest.mark.parametrize("ns,n", GEMM_CASES)
def test_gram_tcgen05_bf16x3_matches_fp64(sd, ns, n):
    # The tensor-core BF16x3 path.  The split product drops lo*lo and the bf16 remainders: ~2^-16
    # relative per product, far less after summation; 2e-5 of sqrt(M_ii M_jj) is the bar.
    cell = workloads.small_cell(npts=10, L=4.0, natom=2, seed=5, nstates=ns)
    cell.n = n
    cell.L = tuple(0.4 * x for x in n)
    ng = int(np.prod(n))
    ctx = _ctx(sd, cell, sd.SDFT_MIXED, ns)
    rng = np.random.default_rng(17)
    Y = rng.normal(size=(ns, ng)).astype(np.float32).astype(np.float64)
    HY = rng.normal(size=(ns, ng)).astype(np.float32).astype(np.float64)
    m = torch.empty(ns, ns, dtype=torch.float64, device="cuda")
    h = torch.empty_like(m)
    sd.sdft_subspace_matrices(ctx, 0, sd.SDFT_MIXED, sd.pack_block(Y, 1), sd.pack_block(HY, 1), m, h, ns)
    M_ref = Y @ Y.T
    upper = np.triu(Y @ HY.T)
    H_ref = upper + np.triu(upper, 1).T
    scale = np.sqrt(np.outer(np.diag(M_ref), np.diag(M_ref)))
    assert np.max(np.abs(m.cpu().numpy().T - M_ref) / scale) < 2e-5
    assert np.max(np.abs(h.cpu().numpy().T - H_ref) / scale) < 2e-5


@pytest.mark.parametrize("ns,n", GEMM_CASES)
def test_rotation_tcgen05_bf16x3_matches_fp64(sd, ns, n):
    # X = Y Q on the tensor cores (32-orbital K stages with a ragged last one, a ragged last grid
    # tile): BF16x3 of FP32 operands, error ~2^-16 of |Y||Q| per term.
    cell = workloads.small_cell(npts=10, L=4.0, natom=2, seed=5, nstates=ns)
    cell.n = n
    cell.L = tuple(0.4 * x for x in n)
    ng = int(np.prod(n))
    ctx = _ctx(sd, cell, sd.SDFT_MIXED, ns)
    rng = np.random.default_rng(23)
    Y = rng.normal(size=(ns, ng)).astype(np.float32).astype(np.float64)
    Q = np.linalg.qr(rng.normal(size=(ns, ns)))[0]
    q = torch.from_numpy(np.ascontiguousarray(Q.T)).cuda()   # column-major Q
    y = sd.pack_block(Y, 1)
    x = torch.empty_like(y)
    sd.sdft_rotate(ctx, 0, sd.SDFT_MIXED, y, q, x, ns)
    ref = (Y.T @ Q.astype(np.float32).astype(np.float64)).T
    err = np.abs(sd.unpack_block(x, 1, False) - ref)
    assert np.max(err) < 2e-5 * np.max(np.abs(Y)) * np.sqrt(ns)


def test_poisson_aar_matches_exact_solve(sd):
    cell = workloads.two_atom_cell()
    ctx = _ctx(sd, cell, sd.SDFT_FP64, 8)
    f = model.sad_density(cell) + model.pseudocharge(cell)
    ref = ham.poisson_exact(cell, f)
    ft = torch.from_numpy(f).cuda()
    phi = torch.zeros_like(ft)
    it = sd.sdft_poisson(ctx, ft, phi, 1e-12, 3000)
    assert it > 0
    assert _relerr(phi.cpu().numpy(), ref) < 1e-9


def test_poisson_mixed_refinement_matches_exact_solve(sd):
    # FP32 AAR corrections inside FP64 residual refinement still reach FP64-level accuracy
    cell = workloads.two_atom_cell()
    ctx = _ctx(sd, cell, sd.SDFT_MIXED, 8)
    f = model.sad_density(cell) + model.pseudocharge(cell)
    ref = ham.poisson_exact(cell, f)
    ft = torch.from_numpy(f).cuda()
    phi = torch.zeros_like(ft)
    it = sd.sdft_poisson(ctx, ft, phi, 1e-11, 4000)
    assert it > 0
    assert _relerr(phi.cpu().numpy(), ref) < 1e-9


# grids: 24^3 coarsens to 6^3 (multigrid), 40 x 24 x 30 stops at an odd 20 x 12 x 15 coarsest grid,
# 25^3 does not coarsen (Jacobi-scaled AAR in the persistent kernel)
@pytest.mark.parametrize("n", [(24, 24, 24), (40, 24, 30), (25, 25, 25)])
def test_poisson_mixed_multigrid_matches_exact_solve(sd, n, monkeypatch):
    cell = workloads.two_atom_cell()
    h = cell.L[0] / cell.n[0]
    cell.n = n
    cell.L = tuple(h * k for k in n)
    f = model.sad_density(cell) + model.pseudocharge(cell)
    ref = ham.poisson_exact(cell, f)
    its = {}
    for mg in ("1", "0"):
        monkeypatch.setenv("SDFT_AAR_MG", mg)
        ctx = _ctx(sd, cell, sd.SDFT_MIXED, 8)
        ft = torch.from_numpy(f).cuda()
        phi = torch.zeros_like(ft)
        its[mg] = sd.sdft_poisson(ctx, ft, phi, 1e-11, 4000)
        assert its[mg] > 0
        assert _relerr(phi.cpu().numpy(), ref) < 1e-9
        sd.sdft_destroy(ctx)
    if n != (25, 25, 25):   # the V-cycle preconditioner cuts the FP32 AAR iterations several-fold
        assert 4 * its["1"] < its["0"], its
    else:
        assert its["1"] == its["0"], its


@pytest.mark.parametrize("nspin", [1, 2])
def test_lda_matches_oracle(sd, nspin):
    cell = workloads.two_atom_cell()
    ctx = _ctx(sd, cell, sd.SDFT_FP64, 8)
    rng = np.random.default_rng(4)
    n = 5000
    rho = 10 ** rng.uniform(-6, 1.5, (nspin, n))
    exc = torch.empty(n, dtype=torch.float64, device="cuda")
    vxc = torch.empty(nspin * n, dtype=torch.float64, device="cuda")
    sd.sdft_lda(ctx, nspin, torch.from_numpy(rho.reshape(-1)).cuda(), exc, vxc, n)
    if nspin == 1:
        e_ref, v_ref = xc.lda_pz_unpolarized(rho[0])
        v_ref = v_ref[None]
    else:
        e_ref, vu, vd = xc.lda_pz_polarized(rho[0], rho[1])
        v_ref = np.stack([vu, vd])
    assert np.max(np.abs(exc.cpu().numpy() - e_ref) / np.abs(e_ref)) < 1e-13
    assert np.max(np.abs(vxc.cpu().numpy().reshape(nspin, n) - v_ref) / np.abs(v_ref)) < 1e-13


def test_fermi_matches_oracle(sd):
    cell = workloads.two_atom_cell()
    ctx = _ctx(sd, cell, sd.SDFT_FP64, 8)
    eigs = np.sort(np.random.default_rng(5).normal(0, 0.3, (1, 1, 8)), axis=-1)
    e = torch.from_numpy(eigs.reshape(-1)).cuda()
    occ = torch.empty_like(e)
    mu, ts = sd.sdft_fermi(ctx, e, occ)
    mu_ref, g_ref = ham.fermi_occupations(eigs, np.ones(1), cell.nelec, cell.kT, 2.0)
    assert abs(mu - mu_ref) < 1e-12
    assert np.max(np.abs(occ.cpu().numpy() - g_ref.reshape(-1))) < 1e-12
    assert abs(ts - ham.entropy_term(g_ref, np.ones(1), cell.kT, 2.0)) < 1e-13


def test_lanczos_bounds_match_oracle(sd):
    cell = workloads.two_atom_cell()
    ctx = _ctx(sd, cell, sd.SDFT_FP64, 8)
    V = model.sad_density(cell) * 0.1 - 0.5
    sd.sdft_set_veff(ctx, 0, V)
    lo, up = sd.sdft_lanczos_bounds(ctx, 0, 0, 20)
    P = model.projectors(cell)
    v0 = workloads.initial_orbitals(0 * 4099, cell.ngrid, 1)[0]
    lo_r, up_r = chefsi.lanczos_bounds(lambda Z: ham.apply_h(cell, Z, V, P, model.kb_energies(cell)), v0, 20)
    assert abs(lo - lo_r) < 1e-8 and abs(up - up_r) < 1e-8


def test_invalid_arguments_are_rejected(sd):
    cell = workloads.two_atom_cell()
    pos = cell.pos.copy()
    pos[0, 0] = np.nan
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_create(cell.L, cell.n, pos, cell.types, cell.species, dict(nstates=8))
    assert e.value.code == -7
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, dict(nstates=7, precision=1))
    assert e.value.code == -1
    ctx = _ctx(sd, cell, sd.SDFT_FP64, 8)
    with pytest.raises(sd.SdftError):
        sd.sdft_get_eigenvalues(ctx)          # no SCF yet
    bad = np.full(cell.ngrid, np.inf)
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_set_veff(ctx, 0, bad)
    assert e.value.code == -7


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 7, 24, 64, 65])
def test_subspace_eig_matches_lapack(sd, n, cplx, monkeypatch):
    """Generalized eigensolve Hs q = lambda M q: the one-CTA Jacobi solver (n <= 64) and cuSOLVER
    (n = 65) against LAPACK, with M shaped like a filtered block's overlap (condition ~1e4)."""
    import scipy.linalg as sla
    rng = np.random.default_rng(n + 100 * cplx)
    B = rng.normal(size=(3 * n, n)) * np.logspace(0, -2, n)
    G = rng.normal(size=(3 * n, 3 * n))
    if cplx:
        B = B + 1j * rng.normal(size=(3 * n, n)) * np.logspace(0, -2, n)
        G = G + 1j * rng.normal(size=(3 * n, 3 * n))
    M = B.conj().T @ B
    H = B.conj().T @ ((G + G.conj().T) / 2) @ B
    lam_ref, Q_ref = sla.eigh(H, M)
    cell = workloads.small_cell(npts=6, L=3.0, natom=1, seed=1, nstates=n + 1)
    ctx = _ctx(sd, cell, sd.SDFT_FP64, n + 1, kpts=[(0.25, 0.0, 0.0)] if cplx else None)

    def dev(A):
        a = np.asfortranarray(A)
        if cplx:
            a = np.stack([a.real, a.imag], axis=-1)   # (n, n, 2) in Fortran order of (i, j)
            return torch.from_numpy(np.ascontiguousarray(a.transpose(1, 0, 2))).cuda()
        return torch.from_numpy(np.ascontiguousarray(A.T)).cuda()

    m, h = dev(M), dev(H)
    eig = torch.zeros(n, dtype=torch.float64, device="cuda")
    sd.sdft_subspace_eig(ctx, cplx, m, h, eig, n)
    lam = eig.cpu().numpy()
    q = h.cpu().numpy()
    Q = (q[..., 0] + 1j * q[..., 1]).T if cplx else q.T
    scale = np.max(np.abs(lam_ref))
    assert np.max(np.abs(lam - lam_ref)) < 1e-11 * scale
    assert np.max(np.abs(Q.conj().T @ M @ Q - np.eye(n))) < 1e-10
    assert np.max(np.abs(H @ Q - M @ Q * lam[None, :])) < 1e-9 * scale * np.max(np.abs(M))


def test_subspace_eig_rejects_indefinite_overlap(sd):
    cell = workloads.small_cell(npts=6, L=3.0, natom=1, seed=1, nstates=4)
    ctx = _ctx(sd, cell, sd.SDFT_FP64, 4)
    M = np.diag([1.0, -1.0, 2.0])
    m = torch.from_numpy(M.copy()).cuda()
    h = torch.from_numpy(np.eye(3)).cuda()
    eig = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_subspace_eig(ctx, False, m, h, eig, 3)
    assert e.value.code == -5
