"""GB300 shifted-COCG Green's-function library: Python binding of libtbgf.

The work runs in the C-ABI library (include/tbgf.h, CUDA kernels for sm_103a);
this module only marshals arguments.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); outputs are allocated like the matrix H: torch
CUDA tensors when H is on the GPU, numpy arrays otherwise.  If the library has
not been built, every call raises: there is no CPU fallback.

  build_system(spec, seed)            synthetic H, S                   (tb_build_bsr)
  bsr_spmm(ctx, A, X)                 Y = A X, complex panel           (tb_bsr_spmm)
  spmm_profile(ctx, A, ncols, prec)   ms per product kernel launch     (tb_bsr_spmm_profile)
  solve(ctx, H, S, z, rhs, optr, orows, ...)
                                      G_ij(z) = e_i^T (zS-H)^{-1} e_j  (shifted_cocg_solve)
  reduce_ldos_dm(ctx, G, z, ...)      LDOS and DM elements              (gf_reduce_ldos_dm)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Any, Optional

import numpy as np

from . import _lib
from ._lib import (TB_COL_BREAKDOWN, TB_COL_CONVERGED, TB_COL_MAX_ITER, TB_COL_NONFINITE, TB_ERR_ARG,
                   TB_ERR_SIZE, TB_ERR_STRUCTURE, TB_ERR_UNSUPPORTED, TB_PREC_DF64, TB_PREC_FP64, TB_PREC_MIXED, TB_SOLVER_COCG,
                   TB_SOLVER_QMR, TB_WARN_BREAKDOWN, TB_WARN_MAX_ITER, TB_WARN_NONFINITE)

__all__ = ["Context", "Bsr", "TbError", "build_system", "bsr_spmm", "spmm_profile", "solve", "profile", "reduce_ldos_dm",
           "spec_to_c", "local_subspaces", "solve_local", "descriptors", "mlp_grad", "mlp_train", "mlp_predict",
           "mlp_param_count",
           "TB_PREC_FP64", "TB_PREC_MIXED", "TB_PREC_DF64", "TB_COL_CONVERGED", "TB_COL_MAX_ITER", "TB_COL_BREAKDOWN",
           "TB_COL_NONFINITE", "TB_WARN_MAX_ITER", "TB_WARN_BREAKDOWN", "TB_WARN_NONFINITE", "TB_ERR_ARG",
           "TB_ERR_SIZE", "TB_ERR_STRUCTURE", "TB_ERR_UNSUPPORTED", "TB_SOLVER_COCG", "TB_SOLVER_QMR"]


class TbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tbgf error {code}: {msg}")
        self.code = code


def _torch():
    import torch
    return torch


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return x.ctypes.data


def _on_cuda(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _as(x, np_dtype, torch_dtype=None, like=None):
    """x as a contiguous array of the given dtype, in the memory space of `like`."""
    if x is None:
        return None
    if like is not None and _on_cuda(like):
        torch = _torch()
        td = torch_dtype or getattr(torch, np.dtype(np_dtype).name)
        if _is_torch(x):
            return x.to(device=like.device, dtype=td).contiguous()
        return torch.as_tensor(np.ascontiguousarray(x, dtype=np_dtype), device=like.device)
    if _is_torch(x):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=np_dtype)


def _empty(shape, np_dtype, like):
    if _on_cuda(like):
        torch = _torch()
        return torch.empty(shape, dtype=getattr(torch, np.dtype(np_dtype).name), device=like.device)
    return np.empty(shape, dtype=np_dtype)


def _stream_of(like):
    if _on_cuda(like):
        return _torch().cuda.current_stream(like.device).cuda_stream
    return None


class Context:
    """Owns a tb_ctx (device workspace) on the current CUDA device."""

    def __init__(self):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        rc = self.lib.tb_ctx_create(ctypes.byref(h))
        if rc != 0:
            raise TbError(rc, "tb_ctx_create failed")
        self.h = h

    def check(self, rc: int, what: str) -> int:
        if rc < 0:
            msg = self.lib.tb_last_error(self.h).decode()
            raise TbError(rc, f"{what}: {self.lib.tb_status_string(rc).decode()}: {msg}")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.tb_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


@dataclass
class Bsr:
    """BSR matrix: row_ptr int64[n+1], col_idx int32[nnzb], val float64[nnzb, b, b]."""
    n_brows: int
    bdim: int
    row_ptr: Any
    col_idx: Any
    val: Any

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n_rows(self) -> int:
        return self.n_brows * self.bdim

    def c_struct(self) -> _lib.TbBsr:
        return _lib.TbBsr(self.n_brows, self.bdim, self.nnzb, _ptr(self.row_ptr), _ptr(self.col_idx),
                          _ptr(self.val))

    def to(self, device) -> "Bsr":
        torch = _torch()
        conv = lambda a, dt: torch.as_tensor(a if not _is_torch(a) else a.cpu().numpy()).to(device=device,
                                                                                            dtype=dt).contiguous()
        return Bsr(self.n_brows, self.bdim, conv(self.row_ptr, torch.int64), conv(self.col_idx, torch.int32),
                   conv(self.val, torch.float64))

    def numpy(self) -> "Bsr":
        f = lambda a: a.cpu().numpy() if _is_torch(a) else a
        return Bsr(self.n_brows, self.bdim, f(self.row_ptr), f(self.col_idx), f(self.val))


_LAT = {"sc_periodic": _lib.TB_LATTICE_SC_PERIODIC, "fcc_cluster": _lib.TB_LATTICE_FCC_CLUSTER}
_ONS = {"uniform": _lib.TB_ONSITE_UNIFORM, "diag_normal": _lib.TB_ONSITE_DIAG_NORMAL}
_HOP = {"const": _lib.TB_HOP_CONST, "normal": _lib.TB_HOP_NORMAL}
_SMODE = {"identity": _lib.TB_S_IDENTITY, "normal": _lib.TB_S_NORMAL, "const": _lib.TB_S_CONST}


def spec_to_c(spec) -> _lib.TbSystemSpec:
    """workloads.SystemSpec -> tb_system_spec."""
    c = _lib.TbSystemSpec()
    c.lattice = _LAT[spec.lattice]
    c.L = spec.L
    c.n_sites = spec.n_sites
    c.bdim = spec.bdim
    c.onsite_mode = _ONS[spec.onsite_mode]
    c.onsite_lo, c.onsite_hi, c.onsite_sigma = spec.onsite_lo, spec.onsite_hi, spec.onsite_sigma
    for i, v in enumerate(spec.onsite_diag):
        c.onsite_diag[i] = v
    c.hop_mode = _HOP[spec.hop_mode]
    c.hop_t, c.hop_sigma = spec.hop_t, spec.hop_sigma
    c.s_mode = _SMODE[spec.s_mode]
    c.s_param = spec.s_param
    c.vacancy_frac = spec.vacancy_frac
    c.slab = 1 if spec.slab else 0
    c.subst_frac, c.subst_shift = spec.subst_frac, spec.subst_shift
    return c


def build_system(spec, seed: int):
    """(H, S or None, overlap_seed) on the host via tb_build_bsr."""
    lib = _lib.load()
    cs = spec_to_c(spec)
    H, S = _lib.TbBsr(), _lib.TbBsr()
    want_s = spec.s_mode != "identity"
    rc = lib.tb_build_bsr(ctypes.byref(cs), seed, ctypes.byref(H), ctypes.byref(S) if want_s else None, None)
    if rc != 0:
        raise TbError(rc, "tb_build_bsr (sizes)")
    b, n, nnzb = H.bdim, H.n_brows, H.nnzb

    def alloc():
        return Bsr(n, b, np.empty(n + 1, np.int64), np.empty(nnzb, np.int32), np.empty((nnzb, b, b), np.float64))

    h = alloc()
    s = alloc() if want_s else None
    Hc = h.c_struct()
    Sc = s.c_struct() if s is not None else None
    oseed = ctypes.c_uint64(0)
    rc = lib.tb_build_bsr(ctypes.byref(cs), seed, ctypes.byref(Hc), ctypes.byref(Sc) if Sc is not None else None,
                          ctypes.byref(oseed))
    if rc != 0:
        raise TbError(rc, "tb_build_bsr")
    return h, s, int(oseed.value)


def bsr_spmm(ctx: Context, A: Bsr, X, precision: int = TB_PREC_FP64):
    """Y = A X for a complex panel X [n_rows, ncols] (complex128)."""
    Xc = _as(X, np.complex128, like=A.val)
    ncols = int(Xc.shape[1])
    Y = _empty(tuple(Xc.shape), np.complex128, A.val)
    Ac = A.c_struct()
    rc = ctx.lib.tb_bsr_spmm(ctx.h, ctypes.byref(Ac), _ptr(Xc), ncols, _ptr(Y), precision, _stream_of(A.val))
    ctx.check(rc, "tb_bsr_spmm")
    return Y


def spmm_profile(ctx: Context, A: Bsr, ncols: int, precision: int = TB_PREC_FP64, reps: int = 20) -> float:
    """Average milliseconds of one product kernel launch (tb_bsr_spmm_profile)."""
    ms = ctypes.c_double(0.0)
    Ac = A.c_struct()
    rc = ctx.lib.tb_bsr_spmm_profile(ctx.h, ctypes.byref(Ac), int(ncols), int(precision), int(reps),
                                     _stream_of(A.val), ctypes.byref(ms))
    ctx.check(rc, "tb_bsr_spmm_profile")
    return float(ms.value)


@dataclass
class SolveResult:
    G: Any        # complex128 [n_out, n_z]
    iters: Any    # int32 [n_rhs]
    resid: Any    # float64 [n_rhs, n_z]
    status: Any   # int32 [n_rhs]
    rc: int       # 0 or OR of TB_WARN_*
    outer_iters: int = 0   # outer iterations summed over panels
    inner_iters: int = 0   # inner CG iterations summed over panels (S != I; df64: FP32 sweep steps)
    refinements: int = 0   # refinement passes of the df64 inner solve
    light_refinements: int = 0   # of those, passes that took S c in FP32


def solve(ctx: Context, H: Bsr, S: Optional[Bsr], z, rhs_rows, out_row_ptr, out_rows, *, tol=1e-10,
          max_iter=100000, precision=TB_PREC_FP64, panel_w=0, seed_shift=-1, inner_tol=0.0, inner_max=0,
          outputs_like=None, ctas_per_sm=0, solver=TB_SOLVER_COCG) -> SolveResult:
    """G[(out_row_ptr[c] + k), m] = e_i^T (z_m S - H)^{-1} e_j, i = out_rows[...], j = rhs_rows[c]
    (solver: TB_SOLVER_COCG or TB_SOLVER_QMR)."""
    like = H.val if outputs_like is None else outputs_like
    zc = _as(z, np.complex128, like=like)
    rhs = _as(rhs_rows, np.int64, like=like)
    optr = _as(out_row_ptr, np.int64, like=like)
    orows = _as(out_rows, np.int64, like=like)
    n_rhs = int(rhs.shape[0])
    n_z = int(zc.shape[0])
    n_out = int(optr[-1])
    G = _empty((n_out, n_z), np.complex128, like)
    iters = _empty((n_rhs,), np.int32, like)
    resid = _empty((n_rhs, n_z), np.float64, like)
    status = _empty((n_rhs,), np.int32, like)
    stats = np.zeros(4, np.int64)
    opts = _opts(ctx, tol, max_iter, precision, panel_w, seed_shift, inner_tol, inner_max, _stream_of(like), stats,
                 ctas_per_sm, solver)
    Hc = H.c_struct()
    Sc = S.c_struct() if S is not None else None
    rc = ctx.lib.shifted_cocg_solve(ctx.h, ctypes.byref(Hc), ctypes.byref(Sc) if Sc is not None else None,
                                    _ptr(zc), n_z, _ptr(rhs), n_rhs, _ptr(optr), _ptr(orows), ctypes.byref(opts),
                                    _ptr(G), _ptr(iters), _ptr(resid), _ptr(status))
    ctx.check(rc, "shifted_cocg_solve")
    return SolveResult(G, iters, resid, status, rc, int(stats[0]), int(stats[1]), int(stats[2]), int(stats[3]))


def _opts(ctx, tol, max_iter, precision, panel_w, seed_shift, inner_tol, inner_max, stream, stats, ctas_per_sm=0,
          solver=TB_SOLVER_COCG):
    opts = _lib.TbSolveOpts()
    ctx.lib.tb_solve_opts_default(ctypes.byref(opts))
    opts.ctas_per_sm = ctas_per_sm
    opts.solver = solver
    opts.tol, opts.max_iter, opts.precision, opts.panel_w = tol, max_iter, precision, panel_w
    opts.seed_shift, opts.inner_tol, opts.inner_max = seed_shift, inner_tol, inner_max
    opts.stream = stream
    opts.stats = stats.ctypes.data if stats is not None else None
    return opts


PROFILE_KERNELS = ("A_outer_H_product", "B_update", "IC_A_inner_S_product", "IC_B_inner_update", "C_rho",
                   "R_refine", "R_refine_fp32")


def profile(ctx: Context, H: Bsr, S: Optional[Bsr], z, rhs_rows, out_row_ptr, out_rows, *, reps=20,
            precision=TB_PREC_FP64, panel_w=0, seed_shift=-1, tol=1e-10, ctas_per_sm=0) -> dict:
    """Average ms per launch of each solver kernel (CUDA events; shifted_cocg_profile)."""
    like = H.val
    zc = _as(z, np.complex128, like=like)
    rhs = _as(rhs_rows, np.int64, like=like)
    optr = _as(out_row_ptr, np.int64, like=like)
    orows = _as(out_rows, np.int64, like=like)
    opts = _opts(ctx, tol, 100000, precision, panel_w, seed_shift, 0.0, 0, _stream_of(like), None, ctas_per_sm)
    ms = np.zeros(8, np.float64)
    Hc = H.c_struct()
    Sc = S.c_struct() if S is not None else None
    rc = ctx.lib.shifted_cocg_profile(ctx.h, ctypes.byref(Hc), ctypes.byref(Sc) if Sc is not None else None,
                                      _ptr(zc), int(zc.shape[0]), _ptr(rhs), int(rhs.shape[0]), _ptr(optr),
                                      _ptr(orows), ctypes.byref(opts), reps, ms.ctypes.data)
    ctx.check(rc, "shifted_cocg_profile")
    return {k: float(ms[i]) for i, k in enumerate(PROFILE_KERNELS)}


def local_subspaces(H: Bsr, rhs_rows, radii):
    """(sub_ptr int64[n+1], sub_atoms int32[...]) hop-shell subspaces (host; tb_local_subspaces)."""
    lib = _lib.load()
    Hn = H.numpy()
    rhs = np.ascontiguousarray(rhs_rows, np.int64)
    rad = np.ascontiguousarray(radii, np.int32)
    n = int(rhs.shape[0])
    ptr = np.zeros(n + 1, np.int64)
    Hc = Hn.c_struct()
    rc = lib.tb_local_subspaces(ctypes.byref(Hc), _ptr(rhs), _ptr(rad), n, _ptr(ptr), None)
    if rc != 0:
        raise TbError(rc, "tb_local_subspaces (sizes)")
    atoms = np.empty(int(ptr[-1]), np.int32)
    rc = lib.tb_local_subspaces(ctypes.byref(Hc), _ptr(rhs), _ptr(rad), n, _ptr(ptr), _ptr(atoms))
    if rc != 0:
        raise TbError(rc, "tb_local_subspaces")
    return ptr, atoms


def solve_local(ctx: Context, H: Bsr, S: Optional[Bsr], z, rhs_rows, sub_ptr, sub_atoms, out_row_ptr, out_rows,
                *, order=None, tol=1e-10, max_iter=100000, precision=TB_PREC_FP64, seed_shift=-1, inner_tol=0.0,
                inner_max=0, solver=TB_SOLVER_COCG) -> SolveResult:
    """Truncated-subspace solves, one CTA per column (shifted_cocg_solve_local)."""
    like = H.val
    zc = _as(z, np.complex128, like=like)
    rhs = _as(rhs_rows, np.int64, like=like)
    sptr = _as(sub_ptr, np.int64, like=like)
    satoms = _as(sub_atoms, np.int32, like=like)
    optr = _as(out_row_ptr, np.int64, like=like)
    orows = _as(out_rows, np.int64, like=like)
    ordr = _as(order, np.int64, like=like) if order is not None else None
    n_rhs, n_z, n_out = int(rhs.shape[0]), int(zc.shape[0]), int(optr[-1])
    G = _empty((n_out, n_z), np.complex128, like)
    iters = _empty((n_rhs,), np.int32, like)
    resid = _empty((n_rhs, n_z), np.float64, like)
    status = _empty((n_rhs,), np.int32, like)
    stats = np.zeros(4, np.int64)
    opts = _opts(ctx, tol, max_iter, precision, 0, seed_shift, inner_tol, inner_max, _stream_of(like), stats,
                 solver=solver)
    Hc = H.c_struct()
    Sc = S.c_struct() if S is not None else None
    rc = ctx.lib.shifted_cocg_solve_local(ctx.h, ctypes.byref(Hc), ctypes.byref(Sc) if Sc is not None else None,
                                          _ptr(zc), n_z, _ptr(rhs), n_rhs, _ptr(sptr), _ptr(satoms), _ptr(optr),
                                          _ptr(orows), _ptr(ordr), ctypes.byref(opts), _ptr(G), _ptr(iters),
                                          _ptr(resid), _ptr(status))
    ctx.check(rc, "shifted_cocg_solve_local")
    return SolveResult(G, iters, resid, status, rc, int(stats[0]), int(stats[1]))


def descriptors(ctx: Context, H: Bsr, S: Optional[Bsr], rhs_rows, radii, sub_ptr, sub_atoms):
    """float32 [n, 32] local-environment descriptors (tb_descriptors)."""
    like = H.val
    rhs = _as(rhs_rows, np.int64, like=like)
    rad = _as(radii, np.int32, like=like)
    sptr = _as(sub_ptr, np.int64, like=like)
    satoms = _as(sub_atoms, np.int32, like=like)
    n = int(rhs.shape[0])
    out = _empty((n, 32), np.float32, like)
    Hc = H.c_struct()
    Sc = S.c_struct() if S is not None else None
    rc = ctx.lib.tb_descriptors(ctx.h, ctypes.byref(Hc), ctypes.byref(Sc) if Sc is not None else None, _ptr(rhs),
                                _ptr(rad), n, _ptr(sptr), _ptr(satoms), _ptr(out), _stream_of(like))
    ctx.check(rc, "tb_descriptors")
    return out


def mlp_param_count() -> int:
    return int(_lib.load().mlp_param_count())


def mlp_grad(ctx: Context, params, X, y):
    """(grad float32[n_param], loss) of the mean squared error at params (host arrays)."""
    p = np.ascontiguousarray(params, np.float32)
    Xc = np.ascontiguousarray(X, np.float32)
    yc = np.ascontiguousarray(y, np.float32)
    g = np.empty_like(p)
    loss = ctypes.c_double(0.0)
    rc = ctx.lib.mlp_grad(ctx.h, _ptr(p), _ptr(Xc), _ptr(yc), int(Xc.shape[0]), _ptr(g), ctypes.byref(loss), None)
    ctx.check(rc, "mlp_grad")
    return g, float(loss.value)


def mlp_train(ctx: Context, X, y, *, epochs, batch, lr, params):
    """(trained float32 params, per-epoch loss) via mlp_train (host arrays)."""
    p = np.array(params, np.float32, copy=True)
    Xc = np.ascontiguousarray(X, np.float32)
    yc = np.ascontiguousarray(y, np.float32)
    hist = np.zeros(max(epochs, 1), np.float64)
    rc = ctx.lib.mlp_train(ctx.h, _ptr(Xc), _ptr(yc), int(Xc.shape[0]), int(epochs), int(batch), float(lr), _ptr(p),
                           _ptr(hist), None)
    ctx.check(rc, "mlp_train")
    return p, hist[:epochs]


def mlp_predict(ctx: Context, params, X):
    p = np.ascontiguousarray(params, np.float32)
    Xc = _as(X, np.float32, like=X)
    out = _empty((int(Xc.shape[0]),), np.float32, Xc)
    rc = ctx.lib.mlp_predict(ctx.h, _ptr(p), _ptr(Xc), int(Xc.shape[0]), _ptr(out), _stream_of(Xc))
    ctx.check(rc, "mlp_predict")
    return out


def reduce_ldos_dm(ctx: Context, G, z, w, mu: float, kT: float, rhs_rows, out_row_ptr, out_rows,
                   S: Optional[Bsr] = None, ldos=True, dm=True):
    """(ldos [n_rhs, n_z] or None, dm [n_out] or None) from shifted_cocg_solve's G."""
    like = G
    zc = _as(z, np.complex128, like=like)
    wc = _as(w, np.float64, like=like) if w is not None else None
    rhs = _as(rhs_rows, np.int64, like=like)
    optr = _as(out_row_ptr, np.int64, like=like)
    orows = _as(out_rows, np.int64, like=like)
    n_rhs, n_z = int(rhs.shape[0]), int(zc.shape[0])
    n_out = int(optr[-1])
    L = _empty((n_rhs, n_z), np.float64, like) if ldos else None
    D = _empty((n_out,), np.float64, like) if dm else None
    Sc = S.c_struct() if S is not None else None
    rc = ctx.lib.gf_reduce_ldos_dm(ctx.h, _ptr(G), n_z, _ptr(zc), _ptr(wc), mu, kT, _ptr(rhs), n_rhs, _ptr(optr),
                                   _ptr(orows), ctypes.byref(Sc) if Sc is not None else None, _ptr(L), _ptr(D),
                                   _stream_of(like))
    ctx.check(rc, "gf_reduce_ldos_dm")
    return L, D
