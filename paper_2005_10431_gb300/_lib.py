"""ctypes declarations of the C ABI in include/sdft.h and the loader of libsdft.so.

There is no fallback: if the in-tree library has not been built (``build.build()``) or cannot be
loaded, importing a function from here raises.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

SDFT_OK = 0
SDFT_ERR_INVALID_ARG = -1
SDFT_ERR_OOM = -2
SDFT_ERR_CUDA = -3
SDFT_ERR_NOT_CONVERGED = -4
SDFT_ERR_CHOLESKY = -5
SDFT_ERR_DEVICE_TIMEOUT = -6
SDFT_ERR_NONFINITE = -7
SDFT_FP64 = 0
SDFT_MIXED = 1
SDFT_GUESS_SAD = 0
SDFT_GUESS_USER = 1
SDFT_XC_LDA_PZ = 0
SDFT_XC_GGA_PBE = 1
SDFT_BC_PERIODIC = 0
SDFT_BC_DIRICHLET = 1

ERROR_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED", -5: "CHOLESKY",
               -6: "DEVICE_TIMEOUT", -7: "NONFINITE"}


class sdft_cell(C.Structure):
    _fields_ = [("L", C.c_double * 3)]


class sdft_grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("fd_order", C.c_int)]


class sdft_atoms(C.Structure):
    _fields_ = [("natom", C.c_int), ("pos", C.POINTER(C.c_double)), ("type", C.POINTER(C.c_int))]


class sdft_pseudo(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("Z", "r_loc", "r_proj", "E_kb", "r_cut_proj", "sad_width")]


class sdft_options(C.Structure):
    _fields_ = [
        ("nspin", C.c_int), ("nkpt", C.c_int), ("kpts", C.POINTER(C.c_double)), ("kw", C.POINTER(C.c_double)),
        ("nstates", C.c_int), ("cheb_degree", C.c_int), ("first_scf_filter_passes", C.c_int),
        ("lanczos_steps", C.c_int), ("kT", C.c_double), ("mix_hist", C.c_int), ("mix_beta", C.c_double),
        ("pulay_period", C.c_int), ("pulay_restart", C.c_int), ("scf_tol", C.c_double), ("max_scf", C.c_int),
        ("precision", C.c_int), ("final_fp64_pass", C.c_int), ("poisson_tol", C.c_double),
        ("init_guess", C.c_int), ("initial_moment", C.c_double), ("seed", C.c_uint64),
        ("batch_problems", C.c_int), ("use_graphs", C.c_int), ("kerker_k0", C.c_double),
        ("xc", C.c_int), ("boundary", C.c_int), ("nbuffer", C.c_int), ("fp64_switch_tol", C.c_double),
        ("gemm_fp32_switch_tol", C.c_double),
    ]


class sdft_iter_record(C.Structure):
    _fields_ = [("iter", C.c_int), ("energy", C.c_double), ("scf_error", C.c_double), ("mu", C.c_double),
                ("seconds", C.c_double), ("lower", C.c_double), ("cutoff", C.c_double), ("upper", C.c_double),
                ("poisson_iters", C.c_int), ("poisson_tol", C.c_double)]


class sdft_result(C.Structure):
    _fields_ = [("energy", C.c_double), ("energy_ks", C.c_double), ("mu", C.c_double),
                ("entropy_term", C.c_double), ("niter", C.c_int), ("converged", C.c_int),
                ("t_total", C.c_double), ("t_filter", C.c_double), ("t_rr", C.c_double),
                ("t_poisson", C.c_double), ("t_other", C.c_double)]


class sdft_kernel_stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("seconds", C.c_double), ("bytes", C.c_double), ("flops", C.c_double)]


SDFT_K_STENCIL, SDFT_K_KB_PROJECT, SDFT_K_GRAM, SDFT_K_EIGEN, SDFT_K_ROTATE, SDFT_K_POISSON, SDFT_K_DENSITY = range(7)
KERNEL_FAMILIES = ["stencil", "kb_project", "gram", "eigen", "rotate", "poisson", "density", "stencil_fp64"]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_LIB = None

# name -> (restype, argtypes); every function in include/sdft.h
SIGNATURES = {
    "sdft_default_options": (None, [C.POINTER(sdft_options)]),
    "sdft_create": (C.c_int, [C.POINTER(sdft_cell), C.POINTER(sdft_grid), C.POINTER(sdft_atoms), C.c_int,
                              C.POINTER(sdft_pseudo), C.POINTER(sdft_options), ALLOC_FN, FREE_FN, C.c_void_p,
                              C.c_void_p, C.POINTER(C.c_void_p)]),
    "sdft_destroy": (None, [C.c_void_p]),
    "sdft_last_error": (C.c_char_p, [C.c_void_p]),
    "sdft_scf": (C.c_int, [C.c_void_p, C.POINTER(sdft_result)]),
    "sdft_batch_scf": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(sdft_result)]),
    "sdft_reset": (C.c_int, [C.c_void_p]),
    "sdft_get_eigenvalues": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sdft_get_occupations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sdft_get_density": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "sdft_set_density": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "sdft_get_forces": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sdft_get_scf_log": (C.c_int, [C.c_void_p, C.POINTER(sdft_iter_record), C.c_size_t, C.POINTER(C.c_size_t)]),
    "sdft_get_pseudocharge": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "sdft_get_sad_density": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "sdft_set_orbitals": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t]),
    "sdft_get_orbitals": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t]),
    "sdft_set_veff": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "sdft_apply_h": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "sdft_chebyshev_filter": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                        C.c_int, C.c_double, C.c_double, C.c_double]),
    "sdft_rayleigh_ritz": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int]),
    "sdft_subspace_matrices": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_int]),
    "sdft_subspace_matrices_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int,
                                                 C.c_void_p, C.c_void_p, C.c_void_p]),
    "sdft_rotate": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "sdft_poisson": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "sdft_lda": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t]),
    "sdft_fermi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sdft_kerker": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int]),
    "sdft_mix_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sdft_move_atoms": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sdft_get_eig_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sdft_get_input_density": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "sdft_lanczos_bounds": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]),
    "sdft_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "sdft_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "sdft_get_kernel_stats": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(sdft_kernel_stats)]),
    "sdft_reset_kernel_stats": (C.c_int, [C.c_void_p]),
    "sdft_chebyshev_filter_multi": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p),
                                              C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_double),
                                              C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sdft_subspace_eig": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "sdft_get_stencil_variant": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_char_p, C.c_size_t]),
    "sdft_mlp_dataset": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sdft_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p]),
    "sdft_mlp_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p]),
    "sdft_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    "sdft_mlp_forward": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sdft_mlp_predict": (C.c_int, [C.c_void_p, C.c_void_p]),
}
SDFT_MLP_NFEAT = 32
SDFT_MLP_NPARAM = 6337


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libsdft.so (raises OSError if it is missing or does not load)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise OSError(f"libsdft.so is not built ({path}); run paper_2005_10431_gb300.build.build()")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB
