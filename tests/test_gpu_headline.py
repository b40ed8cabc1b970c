"""Per-output parity at the benchmark's own configuration, converged.

The generalized (S != I) system on the 32^3 periodic simple cubic lattice
(M = 131072, 4x4 blocks), 64 shifts E + 0.005i on [-10, 6], panel 0 of the
right-hand sides (64 columns of orbital 0 of the 16^3 sub-block), solved
exactly as the benchmark's step solves it: df64, panel of 64, tolerance 1e-5
on every shift's relative residual, default inner solve and restart rule,
then reduced to LDOS and density-matrix elements (midpoint weights,
chemical potential -2, kT = 0).

Four of its first 32 columns are compared with stored results the CPU oracle alone
wrote (tests/golden/make_c2_panel_goldens.py): its plain FP64 shifted COCG at
the same tolerance, and at 1e-9.  Relative errors, per output:
  G     per (column, shift): max over kept rows |dG| / max |G_ref|;
  LDOS  per column: max over shifts |dL| / max |L_ref|;
  DM    per column: max over kept rows |dD| / max |D_ref|.
Bound 1e-5 for each against the FP64 oracle at the same tolerance (the
mixed-precision target), and for G also against the tol-1e-9 result.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1402_7285_gb300 as tb
import workloads as wl

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_panel0_goldens.npz")
PANEL_W = 64


def _errors(G, L, D, ptr, rG, rL, rD, rptr):
    eg, el, ed = [], [], []
    for c in range(len(rptr) - 1):
        g, gr = G[ptr[c]:ptr[c + 1]], rG[rptr[c]:rptr[c + 1]]
        eg.append((np.abs(g - gr).max(axis=0) / np.abs(gr).max(axis=0)).max())
        el.append(np.abs(L[c] - rL[c]).max() / np.abs(rL[c]).max())
        d, dr = D[ptr[c]:ptr[c + 1]], rD[rptr[c]:rptr[c + 1]]
        ed.append(np.abs(d - dr).max() / np.abs(dr).max())
    return max(eg), max(el), max(ed)


def test_c2_bench_panel_converged_matches_fp64_oracle_per_output():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = np.load(GOLDEN)
    w = wl.C2
    Hh, Sh, _ = tb.build_system(w.system, w.seed)
    H, S = Hh.to(DEV), Sh.to(DEV)
    cols = wl.rhs_of(w)[:PANEL_W]
    assert np.array_equal(cols[g["slots"]], g["cols"])
    # kept rows: every orbital of the atoms in each column's block pattern
    rl = []
    for j in cols:
        a = j // 4
        blk = Hh.col_idx[Hh.row_ptr[a]:Hh.row_ptr[a + 1]].astype(np.int64)
        rl.append((blk[:, None] * 4 + np.arange(4)[None, :]).ravel())
    ptr = np.zeros(PANEL_W + 1, np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rl])
    rows = np.concatenate(rl)
    z = wl.shifts_of(w)
    with tb.Context() as ctx:
        res = tb.solve(ctx, H, S, z, cols, ptr, rows, tol=w.tol, precision=tb.TB_PREC_DF64, panel_w=PANEL_W)
        assert res.rc == 0 and np.all(res.status.cpu().numpy() == tb.TB_COL_CONVERGED)
        assert np.all(res.resid.cpu().numpy() <= w.tol)
        L, D = tb.reduce_ldos_dm(ctx, res.G, z, g["w"], float(g["mu"]), float(g["kT"]), cols, ptr, rows, S=S)
        torch.cuda.synchronize()
        G, L, D = res.G.cpu().numpy(), L.cpu().numpy(), D.cpu().numpy()
    sel_ptr = [0]
    sG, sD = [], []
    for i, c in enumerate(g["slots"]):
        assert np.array_equal(rows[ptr[c]:ptr[c + 1]], g["out_rows"][g["out_ptr"][i]:g["out_ptr"][i + 1]])
        sG.append(G[ptr[c]:ptr[c + 1]])
        sD.append(D[ptr[c]:ptr[c + 1]])
        sel_ptr.append(sel_ptr[-1] + ptr[c + 1] - ptr[c])
    sG, sD, sL = np.concatenate(sG), np.concatenate(sD), L[g["slots"]]
    eG, eL, eD = _errors(sG, sL, sD, sel_ptr, g["G_tol5"], g["ldos_tol5"], g["dm_tol5"], g["out_ptr"])
    print(f"vs FP64 oracle at 1e-5: G {eG:.2e} LDOS {eL:.2e} DM {eD:.2e}")
    assert eG <= 1e-5 and eL <= 1e-5 and eD <= 1e-5, (eG, eL, eD)
    eG9, eL9, eD9 = _errors(sG, sL, sD, sel_ptr, g["G_tol9"], g["ldos_tol9"], g["dm_tol9"], g["out_ptr"])
    print(f"vs FP64 oracle at 1e-9: G {eG9:.2e} LDOS {eL9:.2e} DM {eD9:.2e}")
    assert eG9 <= 1e-5, eG9
