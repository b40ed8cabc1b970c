"""gsQMR (the generalized shifted QMR of Sec. 3) on the GPU against the CPU oracle.

The library obtains the QMR iterates by QMR smoothing of its gsCOCG iterates;
the oracle (oracle/qmr.py) runs QMR directly on the unconjugated Lanczos
process with a Givens QR of every shift's tridiagonal.  The two agree in exact
arithmetic; here they must agree to the tolerance, and both with dense LU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1402_7285_gb300 as tb
from oracle import dense, qmr, systems
from tests.helpers import out_layout, rel_err_per_shift
from workloads import C1_SYSTEM, C2_SYSTEM, C5_SYSTEM, midpoint_shifts, scaled

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tb.Context()
    yield c
    c.close()


def _bsr(b):
    return tb.Bsr(b.n_brows, b.bdim, b.row_ptr, b.col_idx, b.val).to(DEV)


@pytest.mark.parametrize("spec,prec,tol,bound", [
    (scaled(C1_SYSTEM, L=6), tb.TB_PREC_FP64, 1e-10, 1e-8),
    (scaled(C2_SYSTEM, L=4), tb.TB_PREC_FP64, 1e-10, 1e-8),
    (scaled(C2_SYSTEM, L=4), tb.TB_PREC_DF64, 1e-9, 1e-7),
    (scaled(C5_SYSTEM, L=4), tb.TB_PREC_FP64, 1e-10, 1e-8),
], ids=["c1_fp64", "c2_fp64", "c2_df64", "c5_fp64"])
def test_gsqmr_matches_oracle_qmr_and_exact(ctx, spec, prec, tol, bound):
    o = systems.build_system(spec, 1234)
    M = o.n_rows
    cols = np.unique(np.linspace(0, M - 1, 12).astype(np.int64))
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    z = midpoint_shifts(10, -9.0, 7.0, 0.05)
    S = None if o.S is None else _bsr(o.S)
    res = tb.solve(ctx, _bsr(o.H), S, z, cols, ptr, rows, tol=tol, precision=prec, panel_w=8,
                   solver=tb.TB_SOLVER_QMR)
    assert res.rc == 0 and np.all(res.status.cpu().numpy() == tb.TB_COL_CONVERGED)
    assert np.all(res.resid.cpu().numpy() <= tol)
    G = res.G.cpu().numpy()
    ref = qmr.shifted_qmr(o.H.to_csr(), None if o.S is None else o.S.to_csr(), z, cols, ptr, rows, tol=tol)
    ex = dense.green_lu(o.H.to_dense(), None if o.S is None else o.S.to_dense(), z, cols)
    for c in range(len(cols)):
        assert rel_err_per_shift(G[ptr[c]:ptr[c + 1]], ref.G[ptr[c]:ptr[c + 1]]).max() < bound, c
        assert rel_err_per_shift(G[ptr[c]:ptr[c + 1]], ex[rl[c], c, :]).max() < bound, c
    # the smoothed iterates stop near where the Lanczos-based QMR does (finite precision moves it a little)
    its, ref_its = res.iters.cpu().numpy(), ref.iters
    assert np.all(np.abs(its - ref_its) <= 0.15 * ref_its + 3), (its, ref_its)


def test_gsqmr_quasi_residual_smooths_the_cocg_residual(ctx):
    """On the same problem and tolerance the QMR iterates stop no later than
    gsCOCG's (their quasi-residual is never above the COCG quasi-norm), and both
    give the same Green's function to the tolerance."""
    o = systems.build_system(scaled(C2_SYSTEM, L=4), 7)
    cols = np.array([0, 100, 255], np.int64)
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    z = midpoint_shifts(12, -9.0, 7.0, 0.02)
    H, S = _bsr(o.H), _bsr(o.S)
    q = tb.solve(ctx, H, S, z, cols, ptr, rows, tol=1e-8, panel_w=8, solver=tb.TB_SOLVER_QMR)
    c = tb.solve(ctx, H, S, z, cols, ptr, rows, tol=1e-8, panel_w=8)
    assert q.rc == 0 and c.rc == 0
    Gq, Gc = q.G.cpu().numpy(), c.G.cpu().numpy()
    for k in range(len(cols)):
        assert rel_err_per_shift(Gq[ptr[k]:ptr[k + 1]], Gc[ptr[k]:ptr[k + 1]]).max() < 1e-6


def test_local_solver_rejects_gsqmr(ctx):
    o = systems.build_system(scaled(C5_SYSTEM, L=6), 3)
    Hh = tb.Bsr(o.H.n_brows, o.H.bdim, o.H.row_ptr, o.H.col_idx, o.H.val)
    rows = np.array([0, 40], np.int64)
    sptr, sat = tb.local_subspaces(Hh, rows, np.array([1, 1], np.int32))
    with pytest.raises(tb.TbError) as e:
        tb.solve_local(ctx, Hh.to(DEV), _bsr(o.S), midpoint_shifts(4, -5, 5, 0.1), rows, sptr, sat,
                       np.arange(3, dtype=np.int64), rows, solver=tb.TB_SOLVER_QMR)
    assert e.value.code == tb.TB_ERR_UNSUPPORTED
