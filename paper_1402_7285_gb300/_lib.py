"""ctypes declarations of the tbgf C ABI (include/tbgf.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libtbgf.so")

TB_OK = 0
TB_ERR_ARG, TB_ERR_CUDA, TB_ERR_ALLOC, TB_ERR_UNSUPPORTED, TB_ERR_SIZE, TB_ERR_STRUCTURE = -1, -2, -3, -4, -5, -6
TB_WARN_MAX_ITER, TB_WARN_BREAKDOWN, TB_WARN_NONFINITE = 1, 2, 4
TB_COL_CONVERGED, TB_COL_MAX_ITER, TB_COL_BREAKDOWN, TB_COL_NONFINITE = 0, 1, 2, 3
TB_PREC_FP64, TB_PREC_MIXED, TB_PREC_DF64 = 0, 1, 2
TB_SOLVER_COCG, TB_SOLVER_QMR = 0, 1
TB_LATTICE_SC_PERIODIC, TB_LATTICE_FCC_CLUSTER = 0, 1
TB_ONSITE_UNIFORM, TB_ONSITE_DIAG_NORMAL = 0, 1
TB_HOP_CONST, TB_HOP_NORMAL = 0, 1
TB_S_IDENTITY, TB_S_NORMAL, TB_S_CONST = 0, 1, 2
TB_REDUCE_STATIC_MAX_ENTRIES = 524288


class TbSystemSpec(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32), ("L", ctypes.c_int32), ("n_sites", ctypes.c_int64),
        ("bdim", ctypes.c_int32), ("onsite_mode", ctypes.c_int32),
        ("onsite_lo", ctypes.c_double), ("onsite_hi", ctypes.c_double), ("onsite_sigma", ctypes.c_double),
        ("onsite_diag", ctypes.c_double * 16),
        ("hop_mode", ctypes.c_int32), ("hop_t", ctypes.c_double), ("hop_sigma", ctypes.c_double),
        ("s_mode", ctypes.c_int32), ("s_param", ctypes.c_double),
        ("vacancy_frac", ctypes.c_double), ("slab", ctypes.c_int32),
        ("subst_frac", ctypes.c_double), ("subst_shift", ctypes.c_double),
    ]


class TbBsr(ctypes.Structure):
    _fields_ = [
        ("n_brows", ctypes.c_int64), ("bdim", ctypes.c_int32), ("nnzb", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
    ]


class TbSolveOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("panel_w", ctypes.c_int32), ("seed_shift", ctypes.c_int32), ("inner_tol", ctypes.c_double),
        ("inner_max", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("stream", ctypes.c_void_p),
        ("solver", ctypes.c_int32), ("stats", ctypes.c_void_p),
    ]


P = ctypes.c_void_p
PS = ctypes.POINTER(TbSystemSpec)
PB = ctypes.POINTER(TbBsr)
PO = ctypes.POINTER(TbSolveOpts)

# name -> (restype, argtypes); every function include/tbgf.h declares
SIGNATURES = {
    "tb_ctx_create": (ctypes.c_int, [ctypes.POINTER(P)]),
    "tb_ctx_destroy": (ctypes.c_int, [P]),
    "tb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tb_last_error": (ctypes.c_char_p, [P]),
    "tb_version": (ctypes.c_int, []),
    "tb_build_bsr": (ctypes.c_int, [PS, ctypes.c_uint64, PB, PB, ctypes.POINTER(ctypes.c_uint64)]),
    "tb_build_csr": (ctypes.c_int, [PS, ctypes.c_uint64, PB, PB, ctypes.POINTER(ctypes.c_uint64)]),
    "tb_bsr_spmm": (ctypes.c_int, [P, PB, P, ctypes.c_int32, P, ctypes.c_int32, P]),
    "tb_bsr_spmm_profile": (ctypes.c_int, [P, PB, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P,
                                           ctypes.POINTER(ctypes.c_double)]),
    "tb_solve_opts_default": (None, [PO]),
    "shifted_cocg_solve": (ctypes.c_int, [P, PB, PB, P, ctypes.c_int32, P, ctypes.c_int64, P, P, PO, P, P, P,
                                          P]),
    "shifted_cocg_profile": (ctypes.c_int, [P, PB, PB, P, ctypes.c_int32, P, ctypes.c_int64, P, P, PO,
                                            ctypes.c_int32, P]),
    "tb_local_subspaces": (ctypes.c_int, [PB, P, P, ctypes.c_int64, P, P]),
    "shifted_cocg_solve_local": (ctypes.c_int, [P, PB, PB, P, ctypes.c_int32, P, ctypes.c_int64, P, P, P, P, P,
                                                PO, P, P, P, P]),
    "tb_descriptors": (ctypes.c_int, [P, PB, PB, P, P, ctypes.c_int64, P, P, P, P]),
    "mlp_param_count": (ctypes.c_int, []),
    "mlp_grad": (ctypes.c_int, [P, P, P, P, ctypes.c_int64, P, P, P]),
    "mlp_train": (ctypes.c_int, [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, P, P,
                                 P]),
    "mlp_predict": (ctypes.c_int, [P, P, P, ctypes.c_int64, P, P]),
    "gf_reduce_ldos_dm_static": (ctypes.c_int, [P, P, ctypes.c_int32, P, P, ctypes.c_double, ctypes.c_double,
                                                P, ctypes.c_int64, P, ctypes.c_int64, P, PB, P, P, P]),
    "gf_reduce_ldos_dm": (ctypes.c_int, [P, P, ctypes.c_int32, P, P, ctypes.c_double, ctypes.c_double, P,
                                         ctypes.c_int64, P, P, PB, P, P, P]),
}

_LIB = None


def load() -> ctypes.CDLL:
    """Load libtbgf.so; raises if it has not been built (there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB
