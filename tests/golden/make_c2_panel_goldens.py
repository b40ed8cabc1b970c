#!/usr/bin/env python3
"""Write the stored C2 Green's-function goldens (calls only the CPU oracle).

Workload: the generalized (S != I) sp3-like system on the 32^3 periodic simple
cubic lattice (M = 131072, 4x4 blocks), 64 shifts E + 0.005i on [-10, 6], the
right-hand sides e_j of orbital 0 of the 16^3 sub-block.  The columns are four
of the first panel of 32 that the benchmark times (slots 0, 7, 16, 31).

For each column the oracle's plain FP64 shifted COCG (Eq. 2, Sec. 3) solves
(z_m S - H) x = e_j twice:
  * at the benchmark's stopping rule, relative residual 1e-5 for every shift
    (inner CG on S to 1e-12), the FP64 result the faster precisions must
    reproduce;
  * at relative residual 1e-9 (inner CG to 1e-13), close to the exact
    Green's function, which states the error the 1e-5 stopping rule itself
    leaves.
Kept rows: every orbital of the atoms in column j's block pattern.  LDOS and
density-matrix elements are the oracle's reductions (Sec. 2) with midpoint
weights (E_hi - E_lo) / n_z, chemical potential -2 and kT = 0, the reduction
the benchmark applies.

Runtime: about an hour on 8 cores (one column per thread, ~18,000 outer
iterations at 1e-5 and ~30,000 at 1e-9, each with ~10 sparse products).
Output: tests/golden/c2_panel0_goldens.npz.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import cocg, gf, systems  # noqa: E402

SLOTS = (0, 7, 16, 31)     # slots of the first panel of 32 columns
PANEL_W = 32
MU, KT = -2.0, 0.0
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_panel0_goldens.npz")


def s_column(S: systems.Bsr, j: int, rows: np.ndarray) -> np.ndarray:
    """S_ij for the kept rows i of column j (rows are orbitals of atoms in j's block pattern)."""
    b = S.bdim
    a = j // b
    k0, k1 = int(S.row_ptr[a]), int(S.row_ptr[a + 1])
    blk = {int(S.col_idx[k]): k for k in range(k0, k1)}
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        out[t] = S.val[blk[int(i) // b], j % b, int(i) % b]   # S_ji = S_ij (symmetric)
    return out


def main():
    w = wl.C2
    t0 = time.time()
    o = systems.build_system(w.system, w.seed)
    hc, sc = o.H.to_csr(), o.S.to_csr()
    z = wl.shifts_of(w)
    cols = wl.rhs_of(w)[list(SLOTS)]
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr = np.zeros(len(rl) + 1, np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rl])
    rows = np.concatenate(rl).astype(np.int64)
    # both tolerances at once: one thread per (column, tolerance)
    import threading
    res = {}

    def run(tag, tol, inner_tol):
        res[tag] = cocg.shifted_cocg(hc, sc, z, cols, ptr, rows, tol=tol, max_iter=200000,
                                     inner_tol=inner_tol, inner_max=1000, nthreads=len(cols))

    th = [threading.Thread(target=run, args=("tol5", w.tol, 1e-12)),
          threading.Thread(target=run, args=("tol9", 1e-9, 1e-13))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    wq = np.full(len(z), (w.e_hi - w.e_lo) / len(z))
    out = {"cols": cols, "slots": np.array(SLOTS, np.int64), "out_ptr": ptr, "out_rows": rows, "z": z,
           "w": wq, "mu": np.float64(MU), "kT": np.float64(KT)}
    for tag, r in res.items():
        L = np.stack([gf.ldos(r.G[ptr[c]:ptr[c + 1]], s_column(o.S, int(j), rl[c]), None)
                      for c, j in enumerate(cols)])
        D = np.concatenate([gf.density_matrix(r.G[ptr[c]:ptr[c + 1]], z.real, wq, MU, KT)
                            for c in range(len(cols))])
        out[f"G_{tag}"] = r.G
        out[f"ldos_{tag}"] = L
        out[f"dm_{tag}"] = D
        out[f"iters_{tag}"] = r.iters
        out[f"status_{tag}"] = r.status
        out[f"resid_{tag}"] = r.resid
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s; iterations "
          f"{res['tol5'].iters.tolist()} (1e-5), {res['tol9'].iters.tolist()} (1e-9)")


if __name__ == "__main__":
    main()
