"""Parity at the benchmark's full sizes.

C1 (SC 16^3, M = 4096, 32 shifts, 256 columns) is compared in full with the
exact Green's function from the generalized eigen-decomposition (Eq. 1 route).
C2 (SC 32^3 with overlap, M = 131072) in the benchmark's launch configuration
(df64, panel of 32) is compared on sampled columns with the oracle's plain
FP64 shifted COCG after the same fixed number of outer iterations; both follow
the same recurrence, so their iterates agree to rounding.  The converged
comparison of the same panel with stored oracle results (an hour of CPU per
column) is test_gpu_headline.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1402_7285_gb300 as tb
from oracle import cocg, dense, systems
from tests.helpers import out_layout, rel_err_per_shift
import workloads as wl

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tb.Context()
    yield c
    c.close()


def _np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else x


def test_c1_full_size_all_columns_vs_exact(ctx):
    w = wl.C1
    o = systems.build_system(w.system, w.seed)
    z = wl.shifts_of(w)
    cols = wl.rhs_of(w)
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    H = tb.Bsr(o.H.n_brows, o.H.bdim, o.H.row_ptr, o.H.col_idx, o.H.val).to(DEV)
    res = tb.solve(ctx, H, None, z, cols, ptr, rows, tol=1e-12, precision=tb.TB_PREC_FP64, panel_w=32)
    assert res.rc == 0 and np.all(_np(res.status) == tb.TB_COL_CONVERGED)
    G = _np(res.G)
    lam, Y = dense.eigenpairs(o.H.to_dense(), None)
    inv = 1.0 / (z[None, :] - lam[:, None])
    worst = 0.0
    for c, j in enumerate(cols):
        ex = np.einsum("ik,k,km->im", Y[rl[c], :], Y[j, :], inv)
        worst = max(worst, rel_err_per_shift(G[ptr[c]:ptr[c + 1]], ex).max())
    assert worst < 1e-9, worst
    # df64 on the same workload at the configured tolerance
    rd = tb.solve(ctx, H, None, z, cols[:64], ptr[:65], rows[:ptr[64]], tol=w.tol, precision=tb.TB_PREC_DF64,
                  panel_w=32)
    assert np.all(_np(rd.status) == tb.TB_COL_CONVERGED)
    Gd = _np(rd.G)
    for c in range(64):
        ex = np.einsum("ik,k,km->im", Y[rl[c], :], Y[cols[c], :], inv)
        assert rel_err_per_shift(Gd[ptr[c]:ptr[c + 1]], ex).max() < 1e-7


def test_c2_full_size_bench_configuration_vs_oracle_truncated(ctx):
    w = wl.C2
    Hh, Sh, _ = tb.build_system(w.system, w.seed)         # product builder (checked against the oracle's elsewhere)
    o = systems.build_system(w.system, w.seed)           # oracle's own matrices for the oracle side
    z = wl.shifts_of(w)
    cols = wl.rhs_of(w)[:32]                             # the first panel the bench times
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    n_it = 40
    # a tolerance no shift reaches in 40 iterations: both sides run the same 40 steps
    res = tb.solve(ctx, Hh.to(DEV), Sh.to(DEV), z, cols, ptr, rows, tol=1e-30, precision=tb.TB_PREC_DF64,
                   panel_w=32, max_iter=n_it, inner_tol=1e-12)
    assert np.all(_np(res.iters) == n_it) and np.all(_np(res.status) == tb.TB_COL_MAX_ITER)
    G = _np(res.G)
    sample = [0, 5, 11, 31]                              # oracle columns, one thread each
    ref = cocg.shifted_cocg(o.H.to_csr(), o.S.to_csr(), z, cols[sample],
                            np.concatenate([[0], np.cumsum([len(rl[c]) for c in sample])]),
                            np.concatenate([rl[c] for c in sample]), tol=1e-30, max_iter=n_it, inner_tol=1e-13)
    off = 0
    for i, c in enumerate(sample):
        n = len(rl[c])
        err = rel_err_per_shift(G[ptr[c]:ptr[c + 1]], ref.G[off:off + n])
        off += n
        assert err.max() < 1e-8, (c, err.max())
