"""The allocation-free subspace Gram entry point, for callers that may not allocate device
memory (inside a global-mode graph capture, under a host-owned memory pool, or in loops that
cannot afford an allocation's synchronisation).  It must give M = Y^H Y and Hs = Y^H (H Y) to the
accuracy of its storage kind, checked against an FP64 numpy product of the stored values, and agree
with the context-based sdft_subspace_matrices call after call, although every call reuses the same
fixed scratch array inside the library.  (For real SDFT_MIXED blocks with ncol >= 32 the context
path runs the BF16x3 tensor-core Gram and this entry point the FP32 CUDA-core Gram: the same result
to FP32 tolerance, not the same kernels.)

This file is named so that pytest collects it last; it also passes when run on its own.
"""
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


def _blocks(sd, precision, cplx, ns, ng, seed):
    """Random Y, HY, rounded to the storage type, as FP64/complex128 numpy plus the device blocks."""
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=(ns, ng))
    HY = rng.normal(size=(ns, ng))
    if cplx:
        Y = Y + 1j * rng.normal(size=(ns, ng))
        HY = HY + 1j * rng.normal(size=(ns, ng))
    if precision != sd.SDFT_FP64:
        rnd = (lambda a: a.astype(np.complex64).astype(np.complex128)) if cplx else \
              (lambda a: a.astype(np.float32).astype(np.float64))
        Y, HY = rnd(Y), rnd(HY)
    return Y, HY, sd.pack_block(Y, precision), sd.pack_block(HY, precision)


def _fp64_reference(Y, HY):
    """M[i, j] = <Y_i, Y_j>; Hs from the upper triangle of <Y_i, HY_j> mirrored Hermitian with a real
    diagonal, as the library returns it (for a Hermitian H the dropped parts are rounding)."""
    M = np.conj(Y) @ Y.T
    upper = np.triu(np.conj(Y) @ HY.T)
    H = upper + np.conj(np.triu(upper, 1).T)
    np.fill_diagonal(H, np.real(np.diag(H)))
    np.fill_diagonal(M, np.real(np.diag(M)))
    return M, H


def _as_matrix(t, cplx):
    # column-major ncol x ncol (double2 if complex): element (i, j) sits at tensor [j, i]
    a = t.cpu().numpy()
    if cplx:
        a = a[..., 0] + 1j * a[..., 1]
    return a.T


def _noalloc(sd, precision, cplx, y, hy, ns, ng):
    shape = (ns, ns, 2) if cplx else (ns, ns)
    # poison the outputs so that a call that writes nothing cannot pass
    m = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    h = torch.full_like(m, float("nan"))
    sd.sdft_subspace_matrices_noalloc(precision, cplx, y, hy, ng, ns, m, h)
    torch.cuda.synchronize()
    return _as_matrix(m, cplx), _as_matrix(h, cplx)


def _tol(sd, precision):
    # FP32 blocks accumulate in FP32 within each split-K chunk: ~1e-6 relative to |Y_i||Y_j| at
    # these lengths; the BF16x3 tensor-core Gram of the context path drops lo*lo terms (~2^-16).
    return 1e-12 if precision == sd.SDFT_FP64 else 2e-5


def _check(M_ref, H_ref, m, h, tol):
    scale = np.sqrt(np.outer(np.real(np.diag(M_ref)), np.real(np.diag(M_ref))))
    assert np.all(np.isfinite(m)) and np.all(np.isfinite(h))
    assert np.max(np.abs(m - M_ref) / scale) < tol
    assert np.max(np.abs(h - H_ref) / scale) < tol


def _compare_with_context(sd, ctx, precision, ns, ng, seed):
    Y, HY, y, hy = _blocks(sd, precision, False, ns, ng, seed)
    m_ref = torch.empty((ns, ns), dtype=torch.float64, device="cuda")
    h_ref = torch.empty_like(m_ref)
    sd.sdft_subspace_matrices(ctx, 0, precision, y, hy, m_ref, h_ref, ns)
    m, h = _noalloc(sd, precision, False, y, hy, ns, ng)
    M64, H64 = _fp64_reference(Y, HY)
    tol = _tol(sd, precision)
    _check(M64, H64, m, h, tol)                                                        # vs FP64 numpy
    _check(M64, H64, _as_matrix(m_ref, False), _as_matrix(h_ref, False), tol)         # context path too
    _check(_as_matrix(m_ref, False), _as_matrix(h_ref, False), m, h, tol)             # and each other


def test_noalloc_gram_matches_fp64_and_context_gram_on_consecutive_calls(sd):
    cell = workloads.small_cell(npts=10, L=4.0, natom=2, seed=5, nstates=40)
    cell.n = (9, 10, 11)
    ng = int(np.prod(cell.n))
    ctx_mixed = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                               dict(nstates=40, precision=sd.SDFT_MIXED))
    # first call: FP32 paired real block; second call: a different size and data in FP64
    _compare_with_context(sd, ctx_mixed, sd.SDFT_MIXED, 8, ng, seed=1)
    ctx64 = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                           dict(nstates=6, precision=sd.SDFT_FP64))
    _compare_with_context(sd, ctx64, sd.SDFT_FP64, 6, ng, seed=2)
    # ncol >= 32 mixed real: the context path takes the tensor-core Gram, this entry point does not
    _compare_with_context(sd, ctx_mixed, sd.SDFT_MIXED, 40, ng, seed=4)
    # and once more on the first configuration, after the scratch held the other calls' data
    _compare_with_context(sd, ctx_mixed, sd.SDFT_MIXED, 8, ng, seed=3)


@pytest.mark.parametrize("precision_name,ns", [("SDFT_FP64", 6), ("SDFT_MIXED", 12), ("SDFT_MIXED", 37)])
def test_noalloc_gram_complex_blocks_match_fp64(sd, precision_name, ns):
    precision = getattr(sd, precision_name)
    ng = 9 * 10 * 11
    Y, HY, y, hy = _blocks(sd, precision, True, ns, ng, seed=10 + ns)
    m, h = _noalloc(sd, precision, True, y, hy, ns, ng)
    M64, H64 = _fp64_reference(Y, HY)
    _check(M64, H64, m, h, _tol(sd, precision))
    assert np.max(np.abs(np.imag(np.diag(m)))) == 0.0 and np.max(np.abs(np.imag(np.diag(h)))) == 0.0


def test_noalloc_gram_rejects_sizes_beyond_its_scratch(sd):
    y = torch.zeros(2, dtype=torch.float64, device="cuda")
    m = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_subspace_matrices_noalloc(sd.SDFT_FP64, False, y, y, 1, 1449, m, m)
    assert e.value.code == -1 and "scratch" in str(e.value)
