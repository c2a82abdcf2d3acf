"""The allocation-free subspace Gram entry point, for callers that may not allocate device
memory (inside a global-mode graph capture, under a host-owned memory pool, or in loops that
cannot afford an allocation's synchronisation).  It must give the same M = Y^H Y and
Hs = Y^H (H Y) as the context-based sdft_subspace_matrices, call after call, although every call
reuses the same fixed scratch array inside the library.

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


def _pair(sd, precision, cplx, ns, ng, seed):
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=(ns, ng))
    HY = rng.normal(size=(ns, ng))
    if cplx:
        Y = Y + 1j * rng.normal(size=(ns, ng))
        HY = HY + 1j * rng.normal(size=(ns, ng))
    return sd.pack_block(Y, precision), sd.pack_block(HY, precision)


def _compare(sd, ctx, precision, cplx, ns, ng, seed):
    y, hy = _pair(sd, precision, cplx, ns, ng, seed)
    shape = (ns, ns, 2) if cplx else (ns, ns)
    m_ref = torch.empty(shape, dtype=torch.float64, device="cuda")
    h_ref = torch.empty_like(m_ref)
    sd.sdft_subspace_matrices(ctx, 1 if cplx else 0, precision, y, hy, m_ref, h_ref, ns)
    # poison the outputs so that a call that writes nothing cannot pass
    m = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    h = torch.full_like(m, float("nan"))
    sd.sdft_subspace_matrices_noalloc(precision, cplx, y, hy, ng, ns, m, h)
    torch.cuda.synchronize()
    m_ref, h_ref, m, h = (t.cpu().numpy() for t in (m_ref, h_ref, m, h))
    # FP32 blocks accumulate in FP32 within each split-K chunk, so a different chunking changes
    # the rounding: compare relative to |y_i||y_j| with the FP32 Gram tolerance of the parity tests.
    diag = np.diagonal(m_ref[..., 0] if cplx else m_ref)
    scale = np.sqrt(np.outer(diag, diag))
    if cplx:
        scale = scale[..., None]
    tol = 1e-12 if precision == sd.SDFT_FP64 else 1e-5
    assert np.all(np.isfinite(m)) and np.all(np.isfinite(h))
    assert np.max(np.abs(m - m_ref) / scale) < tol
    assert np.max(np.abs(h - h_ref) / scale) < tol


def test_noalloc_gram_matches_context_gram_on_consecutive_calls(sd):
    cell = workloads.small_cell(npts=10, L=4.0, natom=2, seed=5, nstates=8)
    cell.n = (9, 10, 11)
    ng = int(np.prod(cell.n))
    ctx_mixed = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                               dict(nstates=8, precision=sd.SDFT_MIXED))
    # first call: FP32 paired real block; second call: a different size and data in FP64
    _compare(sd, ctx_mixed, sd.SDFT_MIXED, False, 8, ng, seed=1)
    ctx64 = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species,
                           dict(nstates=6, precision=sd.SDFT_FP64))
    _compare(sd, ctx64, sd.SDFT_FP64, False, 6, ng, seed=2)
    # and once more on the first configuration, after the scratch held the other call's data
    _compare(sd, ctx_mixed, sd.SDFT_MIXED, False, 8, ng, seed=3)


def test_noalloc_gram_rejects_sizes_beyond_its_scratch(sd):
    y = torch.zeros(2, dtype=torch.float64, device="cuda")
    m = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(sd.SdftError) as e:
        sd.sdft_subspace_matrices_noalloc(sd.SDFT_FP64, False, y, y, 1, 1449, m, m)
    assert e.value.code == -1 and "scratch" in str(e.value)
