"""Python binding of libsdft: real-space Kohn-Sham DFT with CheFSI on one GB300 GPU.

Thin marshalling over the C ABI in include/sdft.h: every function here has the name of the
C entry point it calls, converts arguments (numpy / torch tensors, structs) and raises
SdftError on a non-zero status.  All computation happens in the CUDA library; PyTorch only
provides device memory (through the allocator callbacks) and the stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (SDFT_FP64, SDFT_MIXED, SDFT_GUESS_SAD, SDFT_GUESS_USER, SDFT_XC_LDA_PZ, SDFT_XC_GGA_PBE, SDFT_BC_PERIODIC, SDFT_BC_DIRICHLET, sdft_options,  # noqa: F401
                   sdft_iter_record, sdft_result, SDFT_MLP_NFEAT, SDFT_MLP_NPARAM)

__all__ = [
    "SdftError", "Context", "SDFT_FP64", "SDFT_MIXED", "sdft_default_options", "sdft_create", "sdft_destroy",
    "sdft_scf", "sdft_batch_scf", "sdft_reset", "sdft_get_eigenvalues", "sdft_get_occupations", "sdft_get_density",
    "sdft_set_density", "sdft_get_forces", "sdft_get_scf_log", "sdft_get_pseudocharge", "sdft_get_sad_density",
    "sdft_set_orbitals", "sdft_get_orbitals", "sdft_set_veff", "sdft_apply_h", "sdft_chebyshev_filter",
    "sdft_rayleigh_ritz", "sdft_subspace_matrices", "sdft_subspace_matrices_noalloc", "sdft_subspace_eig", "sdft_chebyshev_filter_multi", "sdft_rotate", "sdft_poisson", "sdft_lda", "sdft_fermi",
    "sdft_lanczos_bounds", "sdft_kerker", "sdft_mix_step", "sdft_move_atoms", "sdft_get_input_density", "sdft_get_eig_stats", "sdft_launch_count", "sdft_get_stencil_variant", "sdft_set_timing", "sdft_get_kernel_stats",
    "sdft_reset_kernel_stats", "pack_block", "unpack_block", "block_shape",
    "SDFT_MLP_NFEAT", "SDFT_MLP_NPARAM", "sdft_mlp_dataset", "sdft_mlp_loss_grad", "sdft_mlp_adam",
    "sdft_mlp_train", "sdft_mlp_forward", "sdft_mlp_predict",
]


class SdftError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_lib.ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(code: int, handle=None):
    if code != _lib.SDFT_OK:
        msg = _lib.lib().sdft_last_error(handle)
        raise SdftError(code, msg.decode() if msg else "")
    return code


def _ptr(t) -> int:
    """Device or host address of a torch tensor / numpy array (contiguous)."""
    if hasattr(t, "data_ptr"):
        assert t.is_contiguous()
        return t.data_ptr()
    assert t.flags["C_CONTIGUOUS"]
    return t.ctypes.data


class Context:
    """Owns an sdft_ctx* plus the ctypes callbacks and host arrays it references."""

    def __init__(self, handle, keep, nspin, nkpt, nstates, ngrid, natom, precision, cplx):
        self.handle = handle
        self._keep = keep
        self.nspin, self.nkpt, self.nstates, self.ngrid, self.natom = nspin, nkpt, nstates, ngrid, natom
        self.precision = precision
        self.cplx = cplx          # per k-point: complex (Bloch) storage

    def __del__(self):
        try:
            sdft_destroy(self)
        except Exception:
            pass


def sdft_default_options(**overrides) -> sdft_options:
    o = sdft_options()
    _lib.lib().sdft_default_options(C.byref(o))
    for k, v in overrides.items():
        if k in ("kpts", "kw"):
            continue
        setattr(o, k, v)
    return o


def _torch_allocator(device):
    import torch

    def alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=device)
        except Exception:
            return None

    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    return _lib.ALLOC_FN(alloc), _lib.FREE_FN(free)


def sdft_create(L, n, pos, types, species, options: dict | None = None, kpts=None, kw=None, stream=None,
                torch_allocator: bool = True) -> Context:
    """Create a context.  L: 3 edges (bohr); n: 3 grid sizes; pos: (natom, 3); types: (natom,);
    species: list of objects/dicts with Z, r_loc, r_proj, E_kb, r_cut_proj, sad_width;
    options: fields of sdft_options; kpts (nk, 3) reduced, kw (nk,).  stream: torch.cuda.Stream
    or raw handle (None = current torch stream)."""
    L_ = _lib.lib()
    options = dict(options or {})
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    types = np.ascontiguousarray(np.asarray(types, dtype=np.int32).reshape(-1))
    cell = _lib.sdft_cell((C.c_double * 3)(*[float(x) for x in L]))
    grid = _lib.sdft_grid((C.c_int * 3)(*[int(x) for x in n]), 12)
    atoms = _lib.sdft_atoms(pos.shape[0], pos.ctypes.data_as(C.POINTER(C.c_double)),
                            types.ctypes.data_as(C.POINTER(C.c_int)))
    sp = (_lib.sdft_pseudo * len(species))()
    for i, s in enumerate(species):
        g = (lambda k: s[k]) if isinstance(s, dict) else (lambda k: getattr(s, k))
        sp[i] = _lib.sdft_pseudo(g("Z"), g("r_loc"), g("r_proj"), g("E_kb"), g("r_cut_proj"), g("sad_width"))
    o = sdft_default_options(**options)
    keep = [pos, types]
    if kpts is not None:
        k = np.ascontiguousarray(np.asarray(kpts, float).reshape(-1, 3))
        w = np.ascontiguousarray(np.asarray(kw if kw is not None else np.full(k.shape[0], 1.0 / k.shape[0]), float))
        o.nkpt = k.shape[0]
        o.kpts = k.ctypes.data_as(C.POINTER(C.c_double))
        o.kw = w.ctypes.data_as(C.POINTER(C.c_double))
        keep += [k, w]
    else:
        k = np.zeros((o.nkpt, 3))
    import torch
    if stream is None:
        stream_handle = torch.cuda.current_stream().cuda_stream
    else:
        stream_handle = getattr(stream, "cuda_stream", stream)
    if torch_allocator:
        af, ff = _torch_allocator(torch.cuda.current_device())
    else:
        af, ff = _lib.ALLOC_FN(), _lib.FREE_FN()
    keep += [af, ff]
    h = C.c_void_p()
    code = L_.sdft_create(C.byref(cell), C.byref(grid), C.byref(atoms), len(species), sp, C.byref(o), af, ff, None,
                          C.c_void_p(stream_handle), C.byref(h))
    _check(code, None)
    cplx = [bool(np.any(k[i] != 0)) for i in range(o.nkpt)]
    return Context(h, keep, o.nspin, o.nkpt, o.nstates, int(np.prod(n)), pos.shape[0], o.precision, cplx)


def sdft_destroy(ctx: Context):
    if ctx.handle:
        _lib.lib().sdft_destroy(ctx.handle)
        ctx.handle = None


def sdft_scf(ctx: Context, raise_not_converged: bool = False) -> dict:
    r = sdft_result()
    code = _lib.lib().sdft_scf(ctx.handle, C.byref(r))
    if code != _lib.SDFT_ERR_NOT_CONVERGED or raise_not_converged:
        _check(code, ctx.handle)
    out = {name: getattr(r, name) for name, _ in sdft_result._fields_}
    out["status"] = code
    return out


def sdft_batch_scf(ctxs, raise_not_converged: bool = False) -> list:
    """The SCFs of several contexts in lockstep (cells that qualify share the multi-cell filter);
    one result dict per context, as sdft_scf returns."""
    n = len(ctxs)
    handles = (C.c_void_p * n)(*[c.handle for c in ctxs])
    res = (sdft_result * n)()
    code = _lib.lib().sdft_batch_scf(handles, n, res)
    if code != _lib.SDFT_ERR_NOT_CONVERGED or raise_not_converged:
        _check(code, ctxs[0].handle if n else None)
    out = []
    for r in res:
        d = {name: getattr(r, name) for name, _ in sdft_result._fields_}
        d["status"] = code
        out.append(d)
    return out


def sdft_reset(ctx: Context):
    _check(_lib.lib().sdft_reset(ctx.handle), ctx.handle)


def _host_vec(ctx, fn, n):
    a = np.empty(n, dtype=np.float64)
    _check(fn(ctx.handle, a.ctypes.data, a.size), ctx.handle)
    return a


def sdft_get_eigenvalues(ctx: Context) -> np.ndarray:
    n = ctx.nspin * ctx.nkpt * ctx.nstates
    return _host_vec(ctx, _lib.lib().sdft_get_eigenvalues, n).reshape(ctx.nspin, ctx.nkpt, ctx.nstates)


def sdft_get_occupations(ctx: Context) -> np.ndarray:
    n = ctx.nspin * ctx.nkpt * ctx.nstates
    return _host_vec(ctx, _lib.lib().sdft_get_occupations, n).reshape(ctx.nspin, ctx.nkpt, ctx.nstates)


def sdft_get_forces(ctx: Context) -> np.ndarray:
    return _host_vec(ctx, _lib.lib().sdft_get_forces, 3 * ctx.natom).reshape(ctx.natom, 3)


def _field(ctx, fn, count, out=None):
    if out is None:
        a = np.empty(count, dtype=np.float64)
        _check(fn(ctx.handle, a.ctypes.data, a.size, 0), ctx.handle)
        return a
    _check(fn(ctx.handle, _ptr(out), out.numel(), 1), ctx.handle)
    return out


def sdft_get_density(ctx: Context, out=None):
    r = _field(ctx, _lib.lib().sdft_get_density, ctx.nspin * ctx.ngrid, out)
    return r.reshape(ctx.nspin, ctx.ngrid) if out is None else r


def sdft_get_pseudocharge(ctx: Context, out=None):
    return _field(ctx, _lib.lib().sdft_get_pseudocharge, ctx.ngrid, out)


def sdft_get_sad_density(ctx: Context, out=None):
    return _field(ctx, _lib.lib().sdft_get_sad_density, ctx.ngrid, out)


def sdft_set_density(ctx: Context, rho):
    on_dev = hasattr(rho, "is_cuda") and rho.is_cuda
    if not on_dev:
        rho = np.ascontiguousarray(np.asarray(rho, np.float64).reshape(-1))
    n = rho.numel() if on_dev else rho.size
    _check(_lib.lib().sdft_set_density(ctx.handle, _ptr(rho), n, 1 if on_dev else 0), ctx.handle)


def sdft_get_scf_log(ctx: Context) -> list:
    cnt = C.c_size_t(0)
    _check(_lib.lib().sdft_get_scf_log(ctx.handle, None, 0, C.byref(cnt)), ctx.handle)
    recs = (sdft_iter_record * max(1, cnt.value))()
    _check(_lib.lib().sdft_get_scf_log(ctx.handle, recs, cnt.value, C.byref(cnt)), ctx.handle)
    return [{name: getattr(recs[i], name) for name, _ in sdft_iter_record._fields_} for i in range(cnt.value)]


def sdft_set_orbitals(ctx: Context, spin: int, kpt: int, block):
    _check(_lib.lib().sdft_set_orbitals(ctx.handle, spin, kpt, _ptr(block), block.numel() * block.element_size()),
           ctx.handle)


def sdft_get_orbitals(ctx: Context, spin: int, kpt: int, block):
    _check(_lib.lib().sdft_get_orbitals(ctx.handle, spin, kpt, _ptr(block), block.numel() * block.element_size()),
           ctx.handle)
    return block


def sdft_set_veff(ctx: Context, spin: int, v):
    on_dev = hasattr(v, "is_cuda") and v.is_cuda
    if not on_dev:
        v = np.ascontiguousarray(np.asarray(v, np.float64).reshape(-1))
    _check(_lib.lib().sdft_set_veff(ctx.handle, spin, _ptr(v), 1 if on_dev else 0), ctx.handle)


def sdft_apply_h(ctx: Context, spin: int, kpt: int, precision: int, x, y, ncol: int):
    _check(_lib.lib().sdft_apply_h(ctx.handle, spin, kpt, precision, _ptr(x), _ptr(y), ncol), ctx.handle)
    return y


def sdft_chebyshev_filter(ctx: Context, spin: int, kpt: int, precision: int, x, y, ncol: int, degree: int,
                          a: float, b: float, a0: float):
    _check(_lib.lib().sdft_chebyshev_filter(ctx.handle, spin, kpt, precision, _ptr(x), _ptr(y), ncol, degree,
                                            a, b, a0), ctx.handle)
    return y


def sdft_rayleigh_ritz(ctx: Context, spin: int, kpt: int, precision: int, y, x, eig, ncol: int):
    _check(_lib.lib().sdft_rayleigh_ritz(ctx.handle, spin, kpt, precision, _ptr(y), _ptr(x), _ptr(eig), ncol),
           ctx.handle)
    return x, eig


def sdft_subspace_matrices(ctx: Context, kpt: int, precision: int, y, hy, m, hs, ncol: int):
    _check(_lib.lib().sdft_subspace_matrices(ctx.handle, kpt, precision, _ptr(y), _ptr(hy), _ptr(m), _ptr(hs),
                                             ncol), ctx.handle)
    return m, hs


def sdft_subspace_matrices_noalloc(precision: int, is_complex: bool, y, hy, ngrid: int, ncol: int, m, hs,
                                   stream=None):
    """Allocation-free M = Y^H Y, Hs = Y^H HY (no context; fixed library scratch, see sdft.h)."""
    import torch
    s = torch.cuda.current_stream().cuda_stream if stream is None else getattr(stream, "cuda_stream", stream)
    _check(_lib.lib().sdft_subspace_matrices_noalloc(precision, 1 if is_complex else 0, _ptr(y), _ptr(hy), ngrid,
                                                     ncol, _ptr(m), _ptr(hs), C.c_void_p(s)), None)
    return m, hs


def sdft_chebyshev_filter_multi(ctxs, xs, ys, degree: int, a, b, a0):
    """One filter of degree `degree` on several cells (contexts) with one stencil launch per step."""
    n = len(ctxs)
    P = C.c_void_p * n
    D = C.c_double * n
    hv = [c.handle.value if hasattr(c.handle, "value") else c.handle for c in ctxs]
    _check(_lib.lib().sdft_chebyshev_filter_multi(P(*hv), n, P(*[_ptr(x) for x in xs]),
                                                  P(*[_ptr(y) for y in ys]), degree, D(*a), D(*b), D(*a0)),
           ctxs[0].handle)
    return ys


def sdft_subspace_eig(ctx: Context, is_complex: bool, m, hs, eig, ncol: int):
    """Hs q = lambda M q on device FP64 matrices; Hs <- Q, eig ascending, M overwritten."""
    _check(_lib.lib().sdft_subspace_eig(ctx.handle, 1 if is_complex else 0, _ptr(m), _ptr(hs), _ptr(eig), ncol),
           ctx.handle)
    return hs, eig


def sdft_rotate(ctx: Context, kpt: int, precision: int, y, q, x, ncol: int):
    _check(_lib.lib().sdft_rotate(ctx.handle, kpt, precision, _ptr(y), _ptr(q), _ptr(x), ncol), ctx.handle)
    return x


def sdft_kerker(ctx: Context, f, out, nchan: int = 1, k0: float = 0.8, tol: float = 1e-10, max_iter: int = 2000):
    """out = (-L)(-L + k0^2)^-1 f per channel (device FP64 [nchan][ngrid]); see include/sdft.h."""
    _check(_lib.lib().sdft_kerker(ctx.handle, _ptr(f), _ptr(out), nchan, k0, tol, max_iter), ctx.handle)
    return out


def sdft_mix_step(ctx: Context, x_in, x_out, x_next):
    """One step of the context's density mixer (plain or Kerker-preconditioned Pulay); device FP64."""
    _check(_lib.lib().sdft_mix_step(ctx.handle, _ptr(x_in), _ptr(x_out), _ptr(x_next)), ctx.handle)
    return x_next


def sdft_move_atoms(ctx: Context, pos, guess: int = 1):
    """Move the atoms (natom x 3 bohr) and prepare the next SCF (0: SAD + seeded orbitals, 1: extrapolated
    density + kept orbitals); returns the extrapolation coefficients (alpha, beta)."""
    p = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1))
    coef = np.zeros(2)
    _check(_lib.lib().sdft_move_atoms(ctx.handle, p.ctypes.data, guess, coef.ctypes.data), ctx.handle)
    return float(coef[0]), float(coef[1])


def sdft_get_eig_stats(ctx: Context):
    """(accepted, rejected) refined subspace eigensolves on this context."""
    a, r = C.c_int(0), C.c_int(0)
    _check(_lib.lib().sdft_get_eig_stats(ctx.handle, C.byref(a), C.byref(r)), ctx.handle)
    return a.value, r.value


def sdft_get_input_density(ctx: Context) -> np.ndarray:
    """The density [nspin][ngrid] the next sdft_scf starts from (host copy)."""
    out = np.empty((ctx.nspin, ctx.ngrid))
    _check(_lib.lib().sdft_get_input_density(ctx.handle, out.ctypes.data, out.size, 0), ctx.handle)
    return out


def sdft_poisson(ctx: Context, f, phi, tol: float = 1e-10, max_iter: int = 2000) -> int:
    it = C.c_int(0)
    _check(_lib.lib().sdft_poisson(ctx.handle, _ptr(f), _ptr(phi), tol, max_iter, C.byref(it)), ctx.handle)
    return it.value


def sdft_lda(ctx: Context, nspin: int, rho, exc, vxc, n: int):
    _check(_lib.lib().sdft_lda(ctx.handle, nspin, _ptr(rho), _ptr(exc), _ptr(vxc), n), ctx.handle)
    return exc, vxc


def sdft_fermi(ctx: Context, eig, occ):
    mu, ts = C.c_double(0), C.c_double(0)
    _check(_lib.lib().sdft_fermi(ctx.handle, _ptr(eig), _ptr(occ), C.byref(mu), C.byref(ts)), ctx.handle)
    return mu.value, ts.value


def sdft_lanczos_bounds(ctx: Context, spin: int, kpt: int, steps: int = 20):
    lo, up = C.c_double(0), C.c_double(0)
    _check(_lib.lib().sdft_lanczos_bounds(ctx.handle, spin, kpt, steps, C.byref(lo), C.byref(up)), ctx.handle)
    return lo.value, up.value


def sdft_launch_count(ctx: Context) -> int:
    n = C.c_uint64(0)
    _check(_lib.lib().sdft_launch_count(ctx.handle, C.byref(n)), ctx.handle)
    return n.value


def sdft_get_stencil_variant(ctx: Context, is_complex: bool = False):
    """(index, name) of the FP32 stencil tile variant used by the last filter step (-1, '' if none)."""
    idx = C.c_int(-1)
    buf = C.create_string_buffer(64)
    _check(_lib.lib().sdft_get_stencil_variant(ctx.handle, 1 if is_complex else 0, C.byref(idx), buf, 64),
           ctx.handle)
    return idx.value, buf.value.decode()


def sdft_set_timing(ctx: Context, on: bool = True):
    _check(_lib.lib().sdft_set_timing(ctx.handle, 1 if on else 0), ctx.handle)


def sdft_get_kernel_stats(ctx: Context) -> dict:
    """{family name: {launches, seconds, bytes, flops}} for every kernel family."""
    out = {}
    for i, name in enumerate(_lib.KERNEL_FAMILIES):
        st = _lib.sdft_kernel_stats()
        _check(_lib.lib().sdft_get_kernel_stats(ctx.handle, i, C.byref(st)), ctx.handle)
        out[name] = {f: getattr(st, f) for f, _ in _lib.sdft_kernel_stats._fields_}
    return out


def sdft_reset_kernel_stats(ctx: Context):
    _check(_lib.lib().sdft_reset_kernel_stats(ctx.handle), ctx.handle)


# ---- learned initial density (see include/sdft.h) -----------------------------------------
def _stream(stream):
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None
                      else getattr(stream, "cuda_stream", stream))


def sdft_mlp_dataset(ctx: Context, feat, target=None):
    """feat: device int16/uint16 tensor [ngrid, 32] (BF16 bits); target: device float32 [ngrid] or None."""
    _check(_lib.lib().sdft_mlp_dataset(ctx.handle, _ptr(feat), None if target is None else _ptr(target)),
           ctx.handle)
    return feat, target


def sdft_mlp_loss_grad(feat, target, npts: int, batch: int, start: int, params, grad, loss, stream=None):
    _check(_lib.lib().sdft_mlp_loss_grad(_ptr(feat), _ptr(target), npts, batch, start, _ptr(params), _ptr(grad),
                                         _ptr(loss), _stream(stream)), None)
    return grad, loss


def sdft_mlp_adam(params, grad, m, v, step: int, lr: float, stream=None):
    _check(_lib.lib().sdft_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr, _stream(stream)), None)
    return params


def sdft_mlp_train(feat, target, npts: int, batch: int, params, grad, m, v, first_step: int, nsteps: int,
                   lr: float, loss, stream=None):
    _check(_lib.lib().sdft_mlp_train(_ptr(feat), _ptr(target), npts, batch, _ptr(params), _ptr(grad), _ptr(m),
                                     _ptr(v), first_step, nsteps, lr, _ptr(loss), _stream(stream)), None)
    return loss


def sdft_mlp_forward(feat, npts: int, params, y, stream=None):
    _check(_lib.lib().sdft_mlp_forward(_ptr(feat), npts, _ptr(params), _ptr(y), _stream(stream)), None)
    return y


def sdft_mlp_predict(ctx: Context, params):
    _check(_lib.lib().sdft_mlp_predict(ctx.handle, _ptr(params)), ctx.handle)


# ---- block storage marshalling (see the storage kinds in include/sdft.h) -----------------
def block_shape(precision: int, cplx: bool, nstates: int, ngrid: int):
    """torch dtype and shape of a device block in the library's storage kind."""
    import torch
    if precision == SDFT_FP64:
        return (torch.float64, (nstates, ngrid, 2)) if cplx else (torch.float64, (nstates, ngrid))
    return (torch.float32, (nstates, ngrid, 2)) if cplx else (torch.float32, (nstates // 2, ngrid, 2))


def pack_block(X: np.ndarray, precision: int, device="cuda"):
    """(nstates, ngrid) numpy block (row n = orbital n) -> device tensor in storage layout."""
    import torch
    cplx = np.iscomplexobj(X)
    dt = np.float64 if precision == SDFT_FP64 else np.float32
    if cplx:
        host = np.stack([X.real, X.imag], axis=-1).astype(dt)
    elif precision == SDFT_FP64:
        host = X.astype(dt)
    else:
        ns, ng = X.shape
        host = X.reshape(ns // 2, 2, ng).transpose(0, 2, 1).astype(dt)
    return torch.from_numpy(np.ascontiguousarray(host)).to(device)


def unpack_block(T, precision: int, cplx: bool) -> np.ndarray:
    """Inverse of pack_block: device tensor -> (nstates, ngrid) numpy (float64 / complex128)."""
    a = T.detach().cpu().numpy().astype(np.float64)
    if cplx:
        return a[..., 0] + 1j * a[..., 1]
    if precision == SDFT_FP64:
        return a
    p, ng, _ = a.shape
    return a.transpose(0, 2, 1).reshape(2 * p, ng)
