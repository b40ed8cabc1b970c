#!/usr/bin/env python3
"""Benchmark: shift-RHS solves/s of the shifted-COCG Green's-function solve.

Workload: the generalized (S != I) sp3-like system on a 32^3 periodic simple
cubic lattice (M = 131072, 4x4 blocks), 64 shifts E + 0.005i on [-10, 6], the
4096 right-hand sides e_j of orbital 0 of the atoms of the 16^3 sub-block,
tolerance 1e-5 on the relative residual of every shift.  One step solves one
panel of right-hand sides to convergence (every shift of every column) and
reduces the Green's-function entries to LDOS and density-matrix elements.
value = converged (column, shift) pairs / second over all ranks, inputs
resident in HBM; e2e = the same through the C ABI with host buffers (pinned),
copies included.  Multi-GPU: ranks take disjoint panels (weak scaling); there
is no collective in the data path.

--impl reference times the CPU oracle (plain FP64 shifted COCG, OpenMP over
columns) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "shift-RHS solves/s at rel. residual 1e-5 (mixed+batched vs plain FP64); SpMM HBM GB/s"
UNIT = "shift-RHS solves/s"
WORKLOAD = wl.C2


def workload_config(panel_w: int, precision: str, n_gpus: int, cols_per_step: int = 0) -> dict:
    s = WORKLOAD.system
    return {
        "workload": f"{WORKLOAD.name}: SC {s.L}^3 periodic, 4 orbitals/atom (M={s.L ** 3 * s.bdim}), "
                    f"S=I+NN N(0,{s.s_param}), {WORKLOAD.n_shifts} shifts E+{WORKLOAD.eta}i on "
                    f"[{WORKLOAD.e_lo},{WORKLOAD.e_hi}], {WORKLOAD.n_rhs} RHS (orbital 0 of the 16^3 sub-block)",
        "tol": WORKLOAD.tol,
        "rhs_per_step_per_gpu": cols_per_step or panel_w,
        "panel_w": panel_w,
        "precision": precision,
        "parallelism": f"column shards x{n_gpus}",
        "l2": "inputs larger than L2 (panel vectors alone exceed 129 MB)",
    }


def block_pattern_rows(row_ptr, col_idx, bdim, rows):
    """Kept rows of each column: every orbital of the atoms in its block pattern."""
    out = []
    for j in rows:
        a = j // bdim
        cols = col_idx[row_ptr[a]:row_ptr[a + 1]].astype(np.int64)
        out.append((cols[:, None] * bdim + np.arange(bdim)[None, :]).ravel())
    ptr = np.zeros(len(out) + 1, np.int64)
    ptr[1:] = np.cumsum([len(o) for o in out])
    return ptr, np.concatenate(out).astype(np.int64)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        if shutil.which("nvidia-smi"):
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_hash() -> str:
    """sha256 over the sources of the solver kernels (the ncu figures are valid for these)."""
    h = hashlib.sha256()
    for f in ("cocg_impl.cuh", "cocg_kernels.cuh", "spmm.cuh", "df64.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1402_7285_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic(kernel: str, precision: str = "df64", W: int = 32) -> int | None:
    """DRAM bytes per launch from the committed ncu summary, if taken on the current source."""
    path = os.path.join(ROOT, "profiles", f"solver_kernels_c2_{precision}_w{W}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    m = re.search(rf"traffic_bytes_per_launch\s+{re.escape(kernel)}\s*=\s*([0-9]+)", text)
    return int(m.group(1)) if m else None


def algorithmic_bytes(n_rows, nnzb, bdim, n_brows, W, n_z, n_ent, esz, dsz, refine=False):
    """Bytes each solver kernel must move once per launch (matrix read once, panel vectors once).

    esz: bytes per real of the panel vectors; dsz: of the inner CG's direction
    vectors (FP32 with df panels).  FP64 and df panels keep H p by recurrence
    (read and written by A); FP32 panels do not.  refine: the df inner solve by
    refinement, whose FP32 sweeps (IC_A, IC_B) work on FP32 vectors with FP32
    values of S, and whose refinement pass R updates the df solution and
    residual with a df product of S."""
    hp = 2 if esz == 8 else 0
    V = n_rows * W * 2 * esz                     # one complex panel vector
    Vd = n_rows * W * 2 * dsz                    # one inner CG direction vector
    V32 = n_rows * W * 2 * 4                     # one FP32 complex panel vector
    idx = nnzb * 4 + (n_brows + 1) * 8
    Mb = nnzb * bdim * bdim * esz + idx
    Mb32 = nnzb * bdim * bdim * 4 + idx
    proj = n_ent * n_z * 16                      # one FP64 complex projected-state array
    out = {
        "A_outer_H_product": (7 + hp) * V + Mb + 2 * proj,  # R, P_old, RT, SP, HP in; P, SP, U, HP out; p^m rw
        "B_update": 6 * V + Mb + 3 * proj,              # RT, U, R in; RT, R', T out; S; x^m rw, p^m in
        "IC_A_inner_S_product": 2 * V + 2 * Vd + Mb,    # T, D_old in; D, A out; S
        "IC_B_inner_update": 5 * V + Vd,                # Y, D, T, A in; Y, T out
        "C_rho": 2 * V,                                 # R, RT in
    }
    if refine:
        out["B_update"] += V32                          # + the first sweep's FP32 residual
        out["IC_A_inner_S_product"] = 4 * V32 + Mb32    # T32, D_old in; D, A32 out; FP32 S
        out["IC_B_inner_update"] = 6 * V32              # C32, T32 rw; D, A32 in
        out["R_refine"] = 4 * V + 2 * V32 + Mb          # Y, T rw (df); C32 in, T32 out; df S
        out["R_refine_fp32"] = 4 * V + 2 * V32 + Mb32   # the same with S c from FP32 values of S
    return out


# FP32 instructions per df operation as implemented (csrc/df64.cuh): a lazily
# accumulated product term 12 (11 with an FP32 operand), an identity-block
# term 7, a normalised df fma 15 (14 with an FP32 operand), a df multiply 7
# (6), a df add 11, a df value added to a two-float sum 8.
DF_TERM, DF_TERM_F, DF_VAL, DF_FMA, DF_FMA_F, DF_MUL, DF_MUL_F, DF_ADD, ACC_ADD = 12, 11, 7, 15, 14, 7, 6, 11, 8
FP32_PEAK_OPS = 152 * 128 * 2.07e9       # SMs x FP32 lanes x max SM clock (one op per lane per clock)


def df_ops(n_rows, nnzb, bdim, W, s_unit=True):
    """FP32 instructions per launch of each df64 solver kernel.

    'algorithmic' forms every vector element once; 'implemented' adds the
    neighbour values that each product forms again on the fly (one per block
    that references the row)."""
    bb = bdim * bdim
    n_br = n_rows // bdim
    own = n_rows * W                                      # complex elements of one panel vector
    nb = nnzb * bdim * W                                  # neighbour elements one product reads
    prod_h = nnzb * bb * 2 * W * DF_TERM                  # real df block x complex df panel
    if s_unit:                                            # identity diagonal blocks of S: additions only
        prod_s = (nnzb - n_br) * bb * 2 * W * DF_TERM_F + n_br * bdim * 2 * W * DF_VAL
    else:
        prod_s = nnzb * bb * 2 * W * DF_TERM_F            # df block x FP32 panel (inner CG operands)
    cx_axpy = 4 * DF_MUL + 4 * DF_ADD                     # a + s b, complex df s
    dot = 4 * (DF_MUL + ACC_ADD)                          # complex bilinear product into two-float sums
    norm = 2 * (DF_MUL + ACC_ADD)                         # Hermitian norm
    alg = {
        "A_outer_H_product": prod_h + own * (4 * cx_axpy + dot),     # p, Sp, Hp, u; mu
        "B_update": prod_s + own * (4 + cx_axpy + 2 * DF_ADD + 2 * norm),
        "IC_A_inner_S_product": prod_s + own * (2 + 2 * (DF_MUL_F + ACC_ADD)),
        "IC_B_inner_update": own * (2 * DF_FMA_F + 2 * DF_FMA + norm),
        "C_rho": own * dot,
    }
    alg["R_refine"] = prod_s + own * (2 * (DF_ADD + 1) + 2 * DF_ADD + norm)   # S c; y += c, t -= S c; ||t||^2
    extra = {"B_update": nb * 4, "IC_A_inner_S_product": nb * 2}
    impl = {k: v + extra.get(k, 0) for k, v in alg.items()}
    return alg, impl


def spmm_bandwidth(tb, ctx, H, Hh, peaks) -> dict:
    """The metric's second figure: the block-sparse product H P alone (tb_bsr_spmm_profile, cold L2 per launch).

    Algorithmic bytes: the matrix once (values in the working precision,
    column indices, row pointers) + the panel read once + the product written
    once; achieved = bytes / kernel time against the measured HBM copy peak."""
    out = {}
    for name, prec, W, esz in (("fp32_w64", tb.TB_PREC_MIXED, 64, 4), ("df64_w32", tb.TB_PREC_DF64, 32, 8),
                               ("fp64_w32", tb.TB_PREC_FP64, 32, 8)):
        ms = tb.spmm_profile(ctx, H, W, prec, reps=10)
        nbytes = (Hh.nnzb * Hh.bdim ** 2 * esz + Hh.nnzb * 4 + (Hh.n_brows + 1) * 8
                  + 2 * Hh.n_rows * W * 2 * esz)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "bytes": nbytes, "achieved_gbs": gbs, "frac": gbs / peaks["hbm_gbs"]}
    out["peak_gbs"] = peaks["hbm_gbs"]
    out["note"] = "H (C2, 229,376 4x4 blocks) times a complex panel; L2 flushed before every timed launch"
    return out


def unit_diagonal(S) -> bool:
    """Every diagonal block of S (host Bsr) is the identity."""
    if S is None:
        return False
    rp, ci = np.asarray(S.row_ptr), np.asarray(S.col_idx)
    val = np.asarray(S.val).reshape(-1, S.bdim, S.bdim)
    rows = np.repeat(np.arange(S.n_brows), np.diff(rp))
    diag = val[ci == rows]
    return diag.shape[0] == S.n_brows and bool(np.all(diag == np.eye(S.bdim)))


GOLDEN = os.path.join(ROOT, "tests", "golden", "c2_panel0_goldens.npz")


def rel_errors(G, L, D, ptr, ref_G, ref_L, ref_D, ref_ptr):
    """Per-output relative errors of the solver's G, LDOS and DM against reference values.

    G: per (column, shift) the largest |dG| over the kept rows relative to the
    largest |G_ref| of that column and shift; LDOS: per column the largest |dL|
    over the shifts relative to the column's largest LDOS (and, as
    "LDOS_per_shift", |dL| / |L_ref| per (column, shift), which is larger in the
    spectral tails where the LDOS is small); DM: per column the largest |dD|
    relative to the largest |D_ref| of that column."""
    eg, el, els, ed = [], [], [], []
    for c in range(len(ref_ptr) - 1):
        g, gr = G[ptr[c]:ptr[c + 1]], ref_G[ref_ptr[c]:ref_ptr[c + 1]]
        eg.append(np.abs(g - gr).max(axis=0) / np.abs(gr).max(axis=0))
        el.append(np.abs(L[c] - ref_L[c]).max() / np.abs(ref_L[c]).max())
        els.append(np.abs(L[c] - ref_L[c]) / np.abs(ref_L[c]))
        d, dr = D[ptr[c]:ptr[c + 1]], ref_D[ref_ptr[c]:ref_ptr[c + 1]]
        ed.append(np.abs(d - dr).max() / np.abs(dr).max())
    eg, el, els, ed = np.concatenate(eg), np.asarray(el), np.concatenate(els), np.asarray(ed)
    stat = lambda a: {"max": float(a.max()), "median": float(np.median(a))}
    return {"G": stat(eg), "LDOS": stat(el), "DM": stat(ed), "LDOS_per_shift": stat(els)}


def golden_accuracy(res, panel_dev):
    """Errors of the first timed panel's outputs on the columns the stored oracle results cover.

    The stored results (tests/golden/c2_panel0_goldens.npz, written by the oracle
    alone) hold four columns of panel 0: the oracle's plain FP64 shifted COCG at
    this tolerance (1e-5) and at 1e-9 (close to the exact Green's function)."""
    if not os.path.exists(GOLDEN):
        return {"unavailable": "tests/golden/c2_panel0_goldens.npz is missing"}
    g = np.load(GOLDEN)
    cols, ptr, orows = (a.cpu().numpy() for a in panel_dev)
    slots = g["slots"]
    if not np.array_equal(cols[slots], g["cols"]):
        return {"unavailable": "the first timed panel does not hold the stored columns"}
    G = res.G.cpu().numpy()
    L = res.ldos.cpu().numpy()
    D = res.dm.cpu().numpy()
    sel_G, sel_D, sel_ptr = [], [], [0]
    for c in slots:
        sel_G.append(G[ptr[c]:ptr[c + 1]])
        sel_D.append(D[ptr[c]:ptr[c + 1]])
        assert np.array_equal(orows[ptr[c]:ptr[c + 1]], g["out_rows"][g["out_ptr"][len(sel_ptr) - 1]:
                                                                     g["out_ptr"][len(sel_ptr)]])
        sel_ptr.append(sel_ptr[-1] + ptr[c + 1] - ptr[c])
    Gs, Ds, Ls = np.concatenate(sel_G), np.concatenate(sel_D), L[slots]
    out = {"columns": [int(x) for x in g["cols"]], "definition": rel_errors.__doc__.split("\n\n")[1].strip()}
    for tag, name in (("tol5", "vs_fp64_oracle_same_tol"), ("tol9", "vs_fp64_oracle_tol_1e-9")):
        out[name] = rel_errors(Gs, Ls, Ds, sel_ptr, g[f"G_{tag}"], g[f"ldos_{tag}"], g[f"dm_{tag}"], g["out_ptr"])
    out["oracle_fp64_same_tol_vs_tol_1e-9"] = rel_errors(g["G_tol5"], g["ldos_tol5"], g["dm_tol5"], g["out_ptr"],
                                                         g["G_tol9"], g["ldos_tol9"], g["dm_tol9"], g["out_ptr"])
    return out


def run_ours(args, rank, world):
    import torch

    import paper_1402_7285_gb300 as tb
    from paper_1402_7285_gb300 import sharding

    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    prec = {"mixed": tb.TB_PREC_MIXED, "fp64": tb.TB_PREC_FP64, "df64": tb.TB_PREC_DF64}[args.precision]
    W = args.panel_w
    cps = args.columns_per_step or W                 # columns per step (a queue through W slots)
    Hh, Sh, _ = tb.build_system(WORKLOAD.system, WORKLOAD.seed)
    H, S = Hh.to(dev), Sh.to(dev)
    z = wl.shifts_of(WORKLOAD)
    rows_all = wl.rhs_of(WORKLOAD)
    n_z = len(z)
    E = z.real
    w_q = np.full(n_z, (WORKLOAD.e_hi - WORKLOAD.e_lo) / n_z)
    mu, kT = -2.0, 0.0
    n_panels_total = len(rows_all) // cps

    def panel(step):
        k = sharding.panel_for(step, rank, world, n_panels_total)
        cols = rows_all[k * cps:(k + 1) * cps]
        ptr, orows = block_pattern_rows(Hh.row_ptr, Hh.col_idx, Hh.bdim, cols)
        return cols, ptr, orows

    def dev_panel(step):
        cols, ptr, orows = panel(step)
        return (torch.as_tensor(cols, device=dev), torch.as_tensor(ptr, device=dev),
                torch.as_tensor(orows, device=dev))

    ctx = tb.Context()
    zt = torch.as_tensor(z, device=dev)
    wt = torch.as_tensor(w_q, device=dev)
    if args.kernel_profile:
        cols, ptr, orows = dev_panel(0)
        prof = tb.profile(ctx, H, S, zt, cols, ptr, orows, reps=args.profile_reps, precision=prec, panel_w=W,
                          ctas_per_sm=args.ctas_per_sm)
        torch.cuda.synchronize()
        ctx.close()
        return {"kernel_profile": prof}
    if args.full_vector:
        # every row kept: the shifted solutions x^m and directions p^m as full vectors
        # (W columns x M rows x n_z shifts, FP64 complex); A updates p^m (read, write),
        # B' updates x^m (read, write) and reads p^m: 5 W M n_z 16 bytes per iteration
        cols, ptr, orows = dev_panel(0)
        M = Hh.n_rows
        full_rows = torch.arange(M, device=dev, dtype=torch.int64).repeat(W)
        full_ptr = torch.arange(W + 1, device=dev, dtype=torch.int64) * M
        base = tb.profile(ctx, H, S, zt, cols, ptr, orows, reps=args.profile_reps, precision=prec, panel_w=W)
        full = tb.profile(ctx, H, S, zt, cols, full_ptr, full_rows, reps=args.profile_reps, precision=prec,
                          panel_w=W)
        torch.cuda.synchronize()
        ctx.close()
        extra = (full["A_outer_H_product"] + full["B_update"]) - (base["A_outer_H_product"] + base["B_update"])
        nbytes = 5 * W * M * n_z * 16
        return {"full_vector": {"kept_rows_per_column": M, "projection_bytes": 2 * W * M * n_z * 16,
                                "ms_A_B_block_pattern": base["A_outer_H_product"] + base["B_update"],
                                "ms_A_B_full_vectors": full["A_outer_H_product"] + full["B_update"],
                                "pair_step_bytes_per_iteration": nbytes, "pair_step_ms": extra,
                                "pair_step_gbs": nbytes / (extra * 1e-3) / 1e9,
                                "frac_of_hbm": nbytes / (extra * 1e-3) / 1e9 / measured_peaks()["hbm_gbs"]}}

    def step_device(cols, ptr, orows):
        r = tb.solve(ctx, H, S, zt, cols, ptr, orows, tol=WORKLOAD.tol, precision=prec, panel_w=W,
                     max_iter=args.max_iter, ctas_per_sm=args.ctas_per_sm)
        L, D = tb.reduce_ldos_dm(ctx, r.G, zt, wt, mu, kT, cols, ptr, orows, S=S)
        r.ldos, r.dm = L, D
        return r

    def converged_pairs(r):
        res = r.resid.cpu().numpy() if hasattr(r.resid, "cpu") else r.resid
        return int((res <= WORKLOAD.tol).sum())

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # timed steps take panels 0, 1, ... (so the first timed panel is always panel 0,
    # whose columns the stored oracle results cover); warm-up steps take the panels after them
    order = list(range(args.steps + args.warmup))
    panels = [dev_panel(s) for s in order]
    for s in range(args.steps, args.steps + args.warmup):
        step_device(*panels[s])
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with ClockSampler(dev.index) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for s in range(args.steps):
            results.append(step_device(*panels[s]))
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    pairs = sum(converged_pairs(r) for r in results)
    outer = sum(r.outer_iters for r in results)
    inner = sum(r.inner_iters for r in results)
    refines = sum(r.refinements for r in results)
    light = sum(r.light_refinements for r in results)
    col_iters = sum(int(np.sum(r.iters.cpu().numpy())) for r in results)
    # loop executions x slots against the iterations the columns needed: the work a
    # panel spends on slots that wait for the queue's last columns
    padded_work = (outer * W - col_iters) / max(col_iters, 1)
    # per panel: 13 set-up and write-out launches, A, B and C per outer iteration,
    # IC_A and IC_B per inner step and (df64 refinement) one R per inner step
    refine_mode = prec == tb.TB_PREC_DF64
    launches = sum(13 + 3 * r.outer_iters + (3 if refine_mode else 2) * r.inner_iters for r in results)
    accuracy = golden_accuracy(results[0], panels[0]) if rank == 0 else None
    ms_max, pairs_all, launches_all = sharding.reduce_step_stats(ms, float(pairs), float(launches), world, dev)
    value = pairs_all / (ms_max / 1e3)

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        Hp = tb.Bsr(Hh.n_brows, Hh.bdim, pin(Hh.row_ptr), pin(Hh.col_idx), pin(Hh.val))
        Sp = tb.Bsr(Sh.n_brows, Sh.bdim, pin(Sh.row_ptr), pin(Sh.col_idx), pin(Sh.val))
        zp = pin(z)
        wp = pin(w_q)
        e2e_steps = max(1, min(len(order), args.e2e_steps))   # panels 0, 1, ... (any panel of the workload)
        host_panels = [tuple(pin(a) for a in panel(order[s])) for s in range(e2e_steps)]
        h2d = sum(int(a.numel() * a.element_size()) for a in (Hp.row_ptr, Hp.col_idx, Hp.val, Sp.row_ptr,
                                                             Sp.col_idx, Sp.val, zp, wp))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_pairs, h2d_b, d2h_b = 0, 0, 0
        for cols, ptr, orows in host_panels:
            r = tb.solve(ctx, Hp, Sp, zp, cols, ptr, orows, tol=WORKLOAD.tol, precision=prec, panel_w=W,
                         max_iter=args.max_iter, ctas_per_sm=args.ctas_per_sm)
            L, D = tb.reduce_ldos_dm(ctx, r.G, zp, wp, mu, kT, cols, ptr, orows, S=Sp)
            e2e_pairs += int((r.resid <= WORKLOAD.tol).sum())
            h2d_b += h2d + sum(int(a.numel() * a.element_size()) for a in (cols, ptr, orows)) * 2
            d2h_b += r.G.nbytes + r.iters.nbytes + r.resid.nbytes + r.status.nbytes + L.nbytes + D.nbytes
        torch.cuda.synchronize()
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_s, e2e_pairs, _ = sharding.reduce_step_stats(e2e_s, float(e2e_pairs), 0.0, world, dev)
        e2e = {"value": e2e_pairs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d_b // e2e_steps,
               "d2h_bytes_per_step": d2h_b // e2e_steps, "steps": e2e_steps}

    # ---- the plain FP64 solver on the first timed panel's first 32 columns, panel of 32
    # (the comparison the metric names; FP64 is ALU-bound, so a wider panel would only
    # lengthen the run)
    fp64 = None
    if args.fp64_compare and prec != tb.TB_PREC_FP64:
        w_fp64 = min(W, 32)
        cols_fp64 = panel(order[0])[0][:w_fp64]
        p64_ptr, p64_rows = block_pattern_rows(Hh.row_ptr, Hh.col_idx, Hh.bdim, cols_fp64)
        cols, ptr, orows = (torch.as_tensor(a, device=dev) for a in (cols_fp64, p64_ptr, p64_rows))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r64 = tb.solve(ctx, H, S, zt, cols, ptr, orows, tol=WORKLOAD.tol, precision=tb.TB_PREC_FP64, panel_w=w_fp64,
                       max_iter=args.max_iter, ctas_per_sm=args.ctas_per_sm)
        tb.reduce_ldos_dm(ctx, r64.G, zt, wt, mu, kT, cols, ptr, orows, S=S)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        p64 = converged_pairs(r64)
        fp64 = {"value": p64 / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64, "steps": 1,
                "outer_iters": r64.outer_iters, "inner_iters": r64.inner_iters,
                "columns": int(w_fp64), "panel_w": int(w_fp64),
                "note": "the first timed step's first columns, plain FP64 vectors and products"}

    # ---- roofline of the dominant kernel (CUDA events on this stream)
    cols, ptr, orows = panels[0]
    prof = tb.profile(ctx, H, S, zt, cols, ptr, orows, reps=args.profile_reps, precision=prec, panel_w=W,
                      ctas_per_sm=args.ctas_per_sm)
    counts = {"A_outer_H_product": outer, "B_update": outer, "IC_A_inner_S_product": inner,
              "IC_B_inner_update": inner, "C_rho": outer, "R_refine": refines - light,
              "R_refine_fp32": light}
    share = {k: prof[k] * counts[k] for k in prof if prof[k] > 0}
    dom = max(share, key=share.get)
    n_ent = int(ptr[-1].item())
    esz = 4 if prec == tb.TB_PREC_MIXED else 8      # bytes per real: FP32, or FP64 / df pairs
    dsz = 4 if prec != tb.TB_PREC_FP64 else 8       # inner CG directions: FP32 with df panels
    algo = algorithmic_bytes(Hh.n_rows, Hh.nnzb, Hh.bdim, Hh.n_brows, W, n_z, n_ent, esz, dsz, refine=refine_mode)
    peaks = measured_peaks()
    achieved = algo[dom] / (prof[dom] * 1e-3) / 1e9
    # the metric's roofline: algorithmic bytes of the dominant kernel per launch / its
    # CUDA-event time, against the measured HBM copy peak
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"] + " (burst, kernel timed alone)",
            "bytes_per_launch": algo[dom], "traffic": kernel_traffic(dom, args.precision, W)}
    if prec == tb.TB_PREC_DF64 and dom in ("A_outer_H_product", "B_update", "C_rho", "R_refine"):
        # double-float kernels are limited by FP32 instruction issue: the same launch
        # measured in FP32 instructions of its df arithmetic (secondary figure)
        ops, ops_impl = df_ops(Hh.n_rows, Hh.nnzb, Hh.bdim, W, s_unit=unit_diagonal(Sh))
        ach = ops[dom] / (prof[dom] * 1e-3) / 1e12
        roof["alu"] = {"achieved": ach, "peak": FP32_PEAK_OPS / 1e12, "unit": "T FP32 instr/s",
                       "frac": ach / (FP32_PEAK_OPS / 1e12), "ops_per_launch": ops[dom],
                       "ops_per_launch_implemented": ops_impl[dom],
                       "op_definition": "FP32 instructions of the df arithmetic with every vector element formed "
                                        "once; peak = 152 SMs x 128 FP32 lanes x 2.07 GHz"}
    roof.update({"ms_per_launch": prof[dom], "per_kernel_ms": prof,
                 "per_kernel_launches": counts,
                 "per_kernel_share": {k: share[k] / sum(share.values()) for k in share},
                 "per_kernel_gbs": {k: algo[k] / (prof[k] * 1e-3) / 1e9 for k in prof if prof[k] > 0}})
    spmm = spmm_bandwidth(tb, ctx, H, Hh, peaks) if rank == 0 else None
    ctx.close()
    return {"value": value, "ms": ms_max, "pairs": pairs_all, "launches": launches_all, "clocks": clk.summary(),
            "e2e": e2e, "roofline": roof, "spmm": spmm, "outer_iters": outer, "inner_iters": inner, "fp64": fp64,
            "refinements": refines, "fp32_refinements": light, "accuracy": accuracy, "padded_work": padded_work,
            "iters_per_column": [int(x) for r in results for x in (r.iters.cpu().numpy() if hasattr(r.iters, "cpu")
                                                                    else r.iters)]}


LOCAL_WORKLOADS = {"c3": wl.C3, "c4": wl.C4, "c5": wl.C5}
LOCAL_PRECISION = {"c3": "df64", "c4": "df64", "c5": "df64"}   # FP32 leaves ~12% of C3's pairs unconverged


def run_local(args):
    """Localized right-hand sides on hop-shell subspaces (C3-C5), persistent solver.

    One step solves --local-cols columns (one launch of the persistent kernel,
    each CTA taking the next column as soon as its own converges) and reduces
    the kept entries to LDOS; c4 also trains the iteration-count predictor on
    --train-cols other columns (untimed) and orders the queue with it."""
    import time as _time

    import torch

    import paper_1402_7285_gb300 as tb
    from paper_1402_7285_gb300 import scheduler

    w = LOCAL_WORKLOADS[args.workload]
    prec_name = args.precision if args.precision_given else LOCAL_PRECISION[args.workload]
    prec = {"mixed": tb.TB_PREC_MIXED, "fp64": tb.TB_PREC_FP64, "df64": tb.TB_PREC_DF64}[prec_name]
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    t0 = _time.perf_counter()
    Hh, Sh, _ = tb.build_system(w.system, w.seed)
    H = Hh.to(dev)
    S = Sh.to(dev) if Sh is not None else None
    build_s = _time.perf_counter() - t0
    rows, rad = wl.rhs_of(w, n_atoms=Hh.n_brows)
    perm = np.random.default_rng(w.seed).permutation(len(rows))
    rows, rad = rows[perm], rad[perm]
    n_step = args.local_cols
    n_tr = args.train_cols if args.workload == "c4" else 0
    need = n_tr + n_step * (args.warmup + args.steps + 1)
    rows, rad = rows[:need], rad[:need]
    sptr, satoms = tb.local_subspaces(Hh, rows, rad)
    z = wl.shifts_of(w)
    ctx = tb.Context()

    def subset(lo, hi):
        sp = (sptr[lo:hi + 1] - sptr[lo]).astype(np.int64)
        sa = satoms[sptr[lo]:sptr[hi]]
        r = rows[lo:hi]
        return r, rad[lo:hi], sp, sa, np.arange(hi - lo + 1, dtype=np.int64), r.copy()

    def solve(lo, hi, order=None):
        r, rd, sp, sa, optr, orows = subset(lo, hi)
        res = tb.solve_local(ctx, H, S, z, r, sp, sa, optr, orows, order=order, tol=w.tol, precision=prec,
                             max_iter=args.max_iter)
        return res

    learned = None
    if n_tr:
        r, rd, sp, sa, optr, orows = subset(0, n_tr)
        Dtr = tb.descriptors(ctx, H, S, r, rd, sp, sa).cpu().numpy()
        res = solve(0, n_tr)
        its = res.iters.cpu().numpy().astype(np.float64)
        learned, hist = scheduler.train(ctx, Dtr, its, epochs=60, batch=256, lr=2e-3)

    def order_for(lo, hi):
        if learned is None:
            return None
        r, rd, sp, sa, optr, orows = subset(lo, hi)
        D = tb.descriptors(ctx, H, S, r, rd, sp, sa).cpu().numpy()
        return scheduler.longest_first(scheduler.predict(ctx, learned, D) * np.diff(sp) * Hh.bdim)

    base = n_tr
    for s_ in range(args.warmup):
        lo = base + s_ * n_step
        solve(lo, lo + n_step, order_for(lo, lo + n_step))
    torch.cuda.synchronize()
    pairs = total_pairs = 0
    t_learn = 0.0
    for s_ in range(args.steps):
        lo = base + (args.warmup + s_) * n_step
        torch.cuda.synchronize()
        t1 = _time.perf_counter()
        order = order_for(lo, lo + n_step)           # descriptors + prediction are part of the step
        res = solve(lo, lo + n_step, order)
        torch.cuda.synchronize()
        t_learn += _time.perf_counter() - t1
        ok = res.resid.cpu().numpy() <= w.tol
        pairs += int(ok.sum())
        total_pairs += ok.size
    value = pairs / t_learn
    sched = None
    if learned is not None:
        lo = base + args.warmup * n_step
        torch.cuda.synchronize()
        t1 = _time.perf_counter()
        solve(lo, lo + n_step, None)
        torch.cuda.synchronize()
        t_plain = _time.perf_counter() - t1
        t_first = t_learn / args.steps
        sched = {"plain_order_s": t_plain, "learned_order_s_mean": t_first, "train_cols": n_tr}
    ctx.close()
    s = w.system
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_learn * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec_name, "data": "synthetic",
            "config": {"workload": f"{w.name}: {s.lattice}, {Hh.n_brows} atoms x {s.bdim} orbitals, "
                                   f"{w.n_shifts} shifts E+{w.eta}i, local subspaces radius {w.radii}",
                       "columns_per_step": n_step, "tol": w.tol, "precision": prec_name,
                       "solver": "persistent one-CTA-per-column local subspace solver"},
            "build_s": build_s, "scheduler": sched, "converged_frac": pairs / max(total_pairs, 1),
            "mean_subspace_atoms": float(np.mean(np.diff(sptr)))}
    print(json.dumps(line))


def cpu_oracle_sample(target_seconds: float, iters_needed: float | None):
    """The oracle (plain FP64 shifted COCG, C + OpenMP over columns) on a bounded sample.

    Runs `cores` columns of the workload for a fixed number of outer
    iterations, measures seconds per outer iteration per column, and scales to
    shift-RHS solves/s with `iters_needed` outer iterations per column."""
    from oracle import cocg, systems

    cores = os.cpu_count() or 1
    s = systems.build_system(WORKLOAD.system, WORKLOAD.seed)
    hc, sc = s.H.to_csr(), s.S.to_csr()
    z = wl.shifts_of(WORKLOAD)
    rows = wl.rhs_of(WORKLOAD)[:cores]
    rl = [systems.block_pattern_rows(s.H, j) for j in rows]
    ptr = np.zeros(len(rl) + 1, np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rl])
    orows = np.concatenate(rl)
    # calibrate: 2 iterations, then size the sample to target_seconds
    t0 = time.perf_counter()
    cocg.shifted_cocg(hc, sc, z, rows, ptr, orows, tol=WORKLOAD.tol, max_iter=2, inner_tol=1e-8, nthreads=cores)
    per_iter = (time.perf_counter() - t0) / 2
    k = int(max(2, min(2000, target_seconds / max(per_iter, 1e-6))))
    t0 = time.perf_counter()
    cocg.shifted_cocg(hc, sc, z, rows, ptr, orows, tol=WORKLOAD.tol, max_iter=k, inner_tol=1e-8, nthreads=cores)
    dt = time.perf_counter() - t0
    sec_per_iter = dt / k           # for `cores` columns in parallel
    # without a GPU run to count them: the mean outer iterations per column the
    # GPU solvers need on this workload at tol 1e-5 (about 18,000; FP64 and df64 agree)
    need = iters_needed or 18000.0
    value = len(rows) * len(z) / (sec_per_iter * need)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(rows)} columns x {k} outer iterations of plain FP64 shifted COCG (inner CG tol 1e-8), "
                      f"{dt:.1f} s; scaled to {need:.0f} outer iterations per column"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--panel-w", type=int, default=64)
    ap.add_argument("--columns-per-step", type=int, default=0,
                    help="columns each step solves through the panel's slots (default: one panel width)")
    ap.add_argument("--precision", default="df64", choices=["df64", "mixed", "fp64"])
    ap.add_argument("--kernel-profile", action="store_true",
                    help="only launch the solver kernels of one panel (CUDA events; for ncu captures)")
    ap.add_argument("--max-iter", type=int, default=100000)
    ap.add_argument("--full-vector", action="store_true",
                    help="only time the shifted steps with every row kept (full-vector shifted solutions)")
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--spmm-only", action="store_true",
                    help="only the SpMM bandwidth figure (the product kernel alone, C2's H)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5"],
                    help="c2: the metric's configuration (panel solver); c3-c5: localized columns")
    ap.add_argument("--local-cols", type=int, default=2048)
    ap.add_argument("--train-cols", type=int, default=4096)
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false",
                    help="skip timing one panel with the plain FP64 solver")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--profile-reps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    args.precision_given = any(a.startswith("--precision") for a in sys.argv[1:])
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.spmm_only and args.impl == "ours":
        if int(os.environ.get("RANK", "0")) == 0:
            import torch

            import paper_1402_7285_gb300 as tb
            torch.cuda.set_device(0)
            Hh, _, _ = tb.build_system(WORKLOAD.system, WORKLOAD.seed)
            ctx = tb.Context()
            print(json.dumps({"spmm_hbm": spmm_bandwidth(tb, ctx, Hh.to("cuda:0"), Hh, measured_peaks())}))
            ctx.close()
        return
    if args.workload != "c2" and args.impl == "ours":
        if int(os.environ.get("RANK", "0")) == 0:
            run_local(args)
        return
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        samples = []
        for _ in range(args.warmup):
            cpu_oracle_sample(max(1.0, args.cpu_seconds / 4), None)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r = cpu_oracle_sample(args.cpu_seconds / max(1, args.steps), None)
            vals.append(r["value"])
            samples.append(r)
        dt = time.perf_counter() - t0
        v = float(np.median(vals))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(args.panel_w, "fp64 (oracle)", args.gpus),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": samples[-1]["cores"], "kind": "oracle",
                                 "sample": samples[-1]["sample"]},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "gpu_launches": 0}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if "kernel_profile" in out or "full_vector" in out:
        if rank == 0:
            print(json.dumps(out))
        return
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu and world == 1:
        iters = np.mean(out["iters_per_column"]) if out["iters_per_column"] else None
        cpu = cpu_oracle_sample(args.cpu_seconds, iters)
    line = {"metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"mixed": "f32+f64", "df64": "df64 (f32 pairs)+f64", "fp64": "f64"}[args.precision],
            "data": "synthetic", "config": workload_config(args.panel_w, args.precision, args.gpus,
                                                           args.columns_per_step),
            "clocks": out["clocks"], "e2e": out["e2e"], "gpu_launches": int(out["launches"]),
            "roofline": out["roofline"], "spmm_hbm": out["spmm"], "cpu_baseline": cpu,
            "solver": {"outer_iters": out["outer_iters"], "inner_iters": out["inner_iters"],
                       "refinements": out["refinements"], "fp32_refinements": out["fp32_refinements"],
                       "padded_work": out["padded_work"],
                       "mean_iters_per_column": float(np.mean(out["iters_per_column"]))},
            "accuracy": out["accuracy"],
            "plain_fp64": out["fp64"]}
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
