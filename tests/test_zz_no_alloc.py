"""gf_reduce_ldos_dm_static: the reduction for callers that cannot allocate
device memory (its scratch is a static device array), checked through the C
ABI against gf_reduce_ldos_dm and against the oracle's LDOS and density
matrix on two calls in a row, with the device's free memory unchanged by
calls after the first; bad index arrays are rejected before any output is
written.

This file sorts last so that a run stopping at the first failure has run
every other test before it; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1402_7285_gb300 as tb
from paper_1402_7285_gb300 import _lib
from oracle import dense, gf, systems
from tests.helpers import out_layout
from workloads import C1_SYSTEM, C2_SYSTEM, scaled

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tb.Context()
    yield c
    c.close()


def _static_call(ctx, G, z, w, mu, kT, rhs, optr, orows, S, ldos, dm):
    Sc = S.c_struct() if S is not None else None
    return ctx.lib.gf_reduce_ldos_dm_static(
        ctx.h, G.data_ptr(), int(z.shape[0]), z.data_ptr(), w.data_ptr(), mu, kT, rhs.data_ptr(),
        int(rhs.shape[0]), optr.data_ptr(), int(orows.shape[0]), orows.data_ptr(),
        ctypes.byref(Sc) if Sc is not None else None, ldos.data_ptr(), dm.data_ptr(),
        torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("overlap", [False, True], ids=["S_I", "S_overlap"])
def test_static_reduce_matches_allocating_reduce_twice(ctx, overlap):
    spec = scaled(C2_SYSTEM, L=3) if overlap else scaled(C1_SYSTEM, L=4)
    o = systems.build_system(spec, 3)
    H = o.H.to_dense()
    S = None if o.S is None else o.S.to_dense()
    M = H.shape[0]
    E = np.linspace(-8.0, 6.0, 13)
    z = E + 0.05j
    w = np.full(len(E), E[1] - E[0])
    mu, kT = -1.0, 0.1
    Sd = None if o.S is None else tb.Bsr(o.S.n_brows, o.S.bdim, o.S.row_ptr, o.S.col_idx, o.S.val).to(DEV)
    free = []
    for call, cols in enumerate((np.array([0, 5, M - 1]), np.array([1, 2, 3, M // 2]))):
        rl = [systems.block_pattern_rows(o.H, j) for j in cols]
        ptr, rows = out_layout(rl)
        ex = dense.green_lu(H, S, z, cols)
        G = np.concatenate([ex[rl[c], c, :] for c in range(len(cols))])
        Gd = torch.as_tensor(G, device=DEV)
        zd, wd = torch.as_tensor(z, device=DEV), torch.as_tensor(w, device=DEV)
        rd, pd, od = (torch.as_tensor(a, device=DEV) for a in (cols, ptr, rows))
        L_ref, D_ref = tb.reduce_ldos_dm(ctx, Gd, zd, wd, mu, kT, rd, pd, od, S=Sd)
        L = torch.empty((len(cols), len(z)), dtype=torch.float64, device=DEV)
        D = torch.empty(len(rows), dtype=torch.float64, device=DEV)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        rc = _static_call(ctx, Gd, zd, wd, mu, kT, rd, pd, od, Sd, L, D)
        assert rc == 0, ctx.lib.tb_last_error(ctx.h)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert torch.allclose(L, L_ref, rtol=1e-12, atol=1e-14), call
        assert torch.allclose(D, D_ref, rtol=1e-12, atol=1e-14), call
        # the oracle's own reductions of the same G
        Lh, Dh = L.cpu().numpy(), D.cpu().numpy()
        for c, j in enumerate(cols):
            g = G[ptr[c]:ptr[c + 1]]
            lref = gf.ldos(g, None if S is None else S[rl[c], j],
                           int(np.nonzero(rl[c] == j)[0][0]) if S is None else None)
            dref = gf.density_matrix(g, E, w, mu, kT)
            assert np.abs(Lh[c] - lref).max() <= 1e-12 * np.abs(lref).max(), (call, c)
            assert np.abs(Dh[ptr[c]:ptr[c + 1]] - dref).max() <= 1e-12 * np.abs(dref).max(), (call, c)
    # no device memory taken by the second call (the first looks up the static scratch address)
    assert free[2] == free[3], free


def test_static_reduce_rejects_bad_index_arrays_before_writing(ctx):
    o = systems.build_system(scaled(C1_SYSTEM, L=4), 3)
    M = o.n_rows
    cols = np.array([0, 7, M - 1])
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    z = torch.as_tensor(np.linspace(-6, 6, 5) + 0.05j, device=DEV)
    w = torch.ones(5, dtype=torch.float64, device=DEV)
    G = torch.ones((len(rows), 5), dtype=torch.complex128, device=DEV)
    rd, pd, od = (torch.as_tensor(a, device=DEV) for a in (cols, ptr, rows))
    L = torch.full((len(cols), 5), 7.0, dtype=torch.float64, device=DEV)
    D = torch.full((len(rows),), 7.0, dtype=torch.float64, device=DEV)
    # n_out smaller than out_row_ptr[n_rhs]: TB_ERR_SIZE, outputs untouched
    rc = ctx.lib.gf_reduce_ldos_dm_static(ctx.h, G.data_ptr(), 5, z.data_ptr(), w.data_ptr(), 0.0, 0.0,
                                          rd.data_ptr(), len(cols), pd.data_ptr(), len(rows) - 3, od.data_ptr(),
                                          None, L.data_ptr(), D.data_ptr(), None)
    torch.cuda.synchronize()
    assert rc == _lib.TB_ERR_SIZE
    assert torch.all(L == 7.0) and torch.all(D == 7.0)
    # S = I and a column that does not keep its own row: TB_ERR_ARG, outputs untouched
    rows_bad = rows.copy()
    rows_bad[ptr[1]:ptr[2]][rl[1] == cols[1]] = (cols[1] + 1) % M
    ob = torch.as_tensor(rows_bad, device=DEV)
    rc = ctx.lib.gf_reduce_ldos_dm_static(ctx.h, G.data_ptr(), 5, z.data_ptr(), w.data_ptr(), 0.0, 0.0,
                                          rd.data_ptr(), len(cols), pd.data_ptr(), len(rows), ob.data_ptr(),
                                          None, L.data_ptr(), D.data_ptr(), None)
    torch.cuda.synchronize()
    assert rc == _lib.TB_ERR_ARG
    assert b"own row" in ctx.lib.tb_last_error(ctx.h)
    assert torch.all(L == 7.0) and torch.all(D == 7.0)


def test_static_reduce_rejects_oversize_and_host_arrays(ctx):
    z = torch.zeros(2, dtype=torch.complex128, device=DEV)
    w = torch.ones(2, dtype=torch.float64, device=DEV)
    rhs = torch.zeros(1, dtype=torch.int64, device=DEV)
    ptr = torch.tensor([0, 1], dtype=torch.int64, device=DEV)
    rows = torch.zeros(1, dtype=torch.int64, device=DEV)
    G = torch.zeros((1, 2), dtype=torch.complex128, device=DEV)
    L = torch.empty((1, 2), dtype=torch.float64, device=DEV)
    D = torch.empty(1, dtype=torch.float64, device=DEV)
    too_many = _lib.TB_REDUCE_STATIC_MAX_ENTRIES + 1
    rc = ctx.lib.gf_reduce_ldos_dm_static(ctx.h, G.data_ptr(), 2, z.data_ptr(), w.data_ptr(), 0.0, 0.0,
                                          rhs.data_ptr(), 1, ptr.data_ptr(), too_many, rows.data_ptr(), None,
                                          L.data_ptr(), D.data_ptr(), None)
    assert rc == _lib.TB_ERR_SIZE
    assert b"static scratch limit" in ctx.lib.tb_last_error(ctx.h)
    Gh = np.zeros((1, 2), np.complex128)
    rc = ctx.lib.gf_reduce_ldos_dm_static(ctx.h, Gh.ctypes.data, 2, z.data_ptr(), w.data_ptr(), 0.0, 0.0,
                                          rhs.data_ptr(), 1, ptr.data_ptr(), 1, rows.data_ptr(), None,
                                          L.data_ptr(), D.data_ptr(), None)
    assert rc == _lib.TB_ERR_ARG
