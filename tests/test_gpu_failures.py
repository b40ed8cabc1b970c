"""Failure detection of the solver, each failure made on the host.

A NaN in H reaches the recurrence scalars and the column reports
TB_COL_NONFINITE; a malformed block structure (a column index out of range, a
row pointer that decreases, an unsorted block row) is rejected by the device
validation with TB_ERR_STRUCTURE before any solver kernel runs (the validator
bounds its own reads); an overlap S that is not positive definite is met by
the inner CG on S (a direction with d^H S d <= 0) and the column reports
TB_COL_BREAKDOWN.  None of these faults the GPU: every loop of the solver is
bounded and reports a status.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1402_7285_gb300 as tb
from oracle import systems
from tests.helpers import out_layout
from workloads import C1_SYSTEM, C2_SYSTEM, midpoint_shifts, scaled

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tb.Context()
    yield c
    c.close()


def _case(spec):
    o = systems.build_system(spec, 1234)
    M = o.n_rows
    cols = np.array([0, M // 2, M - 1], np.int64)
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    return o, cols, ptr, rows, midpoint_shifts(6, -6.0, 6.0, 0.05)


def _bsr(rp, ci, val, n_brows, bdim):
    return tb.Bsr(n_brows, bdim, rp, ci, val).to(DEV)


@pytest.mark.parametrize("prec", [tb.TB_PREC_FP64, tb.TB_PREC_DF64, tb.TB_PREC_MIXED], ids=["fp64", "df64", "mixed"])
def test_nan_in_H_gives_nonfinite_status(ctx, prec):
    o, cols, ptr, rows, z = _case(scaled(C2_SYSTEM, L=4))
    val = o.H.val.copy()
    a = int(cols[1]) // 4
    val[o.H.row_ptr[a] + 1, 2, 3] = np.nan          # a block in the row of column 1's atom
    H = _bsr(o.H.row_ptr, o.H.col_idx, val, o.H.n_brows, 4)
    S = _bsr(o.S.row_ptr, o.S.col_idx, o.S.val, o.S.n_brows, 4)
    res = tb.solve(ctx, H, S, z, cols, ptr, rows, tol=1e-8, precision=prec, panel_w=8, max_iter=200)
    st = res.status.cpu().numpy()
    assert res.rc & tb.TB_WARN_NONFINITE
    assert np.all(st == tb.TB_COL_NONFINITE), st   # the NaN spreads to every column within a few products


@pytest.mark.parametrize("fault", ["col_out_of_range", "row_ptr_decreasing", "row_unsorted"])
def test_malformed_structure_is_rejected(ctx, fault):
    o, cols, ptr, rows, z = _case(scaled(C1_SYSTEM, L=5))
    rp, ci = o.H.row_ptr.copy(), o.H.col_idx.copy()
    if fault == "col_out_of_range":
        ci[17] = o.H.n_brows + 5
    elif fault == "row_ptr_decreasing":
        rp[10] = rp[12] + 1
    else:
        k = rp[7]
        ci[k], ci[k + 1] = ci[k + 1], ci[k]
    H = _bsr(rp, ci, o.H.val, o.H.n_brows, 1)
    with pytest.raises(tb.TbError) as e:
        tb.solve(ctx, H, None, z, cols, ptr, rows, tol=1e-8, panel_w=8)
    assert e.value.code == tb.TB_ERR_STRUCTURE
    # the context stays usable: the same call on the well-formed matrix converges
    Hok = _bsr(o.H.row_ptr, o.H.col_idx, o.H.val, o.H.n_brows, 1)
    ok = tb.solve(ctx, Hok, None, z, cols, ptr, rows, tol=1e-8, panel_w=8)
    assert ok.rc == 0


@pytest.mark.parametrize("prec", [tb.TB_PREC_FP64, tb.TB_PREC_DF64], ids=["fp64", "df64"])
def test_overlap_not_positive_definite_gives_breakdown(ctx, prec):
    o, cols, ptr, rows, z = _case(scaled(C2_SYSTEM, L=4))
    # S = -I on H's diagonal blocks: d^H S d < 0 for every inner direction
    n = o.H.n_brows
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    sval = np.broadcast_to(-np.eye(4), (n, 4, 4)).copy()
    H = _bsr(o.H.row_ptr, o.H.col_idx, o.H.val, n, 4)
    S = _bsr(rp, ci, sval, n, 4)
    res = tb.solve(ctx, H, S, z, cols, ptr, rows, tol=1e-8, precision=prec, panel_w=8, max_iter=50)
    st = res.status.cpu().numpy()
    assert res.rc & tb.TB_WARN_BREAKDOWN
    assert np.all(st == tb.TB_COL_BREAKDOWN), st
