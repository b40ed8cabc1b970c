"""gf_reduce_ldos_dm_static: the reduction for callers that cannot allocate
device memory (its scratch is a static device array), checked through the C
ABI against gf_reduce_ldos_dm on two calls in a row.

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
from oracle import dense, systems
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
    Sd = None if o.S is None else tb.Bsr(o.S.n_brows, o.S.bdim, o.S.row_ptr, o.S.col_idx, o.S.val).to(DEV)
    for call, cols in enumerate((np.array([0, 5, M - 1]), np.array([1, 2, 3, M // 2]))):
        rl = [systems.block_pattern_rows(o.H, j) for j in cols]
        ptr, rows = out_layout(rl)
        ex = dense.green_lu(H, S, z, cols)
        G = np.concatenate([ex[rl[c], c, :] for c in range(len(cols))])
        Gd = torch.as_tensor(G, device=DEV)
        zd, wd = torch.as_tensor(z, device=DEV), torch.as_tensor(w, device=DEV)
        rd, pd, od = (torch.as_tensor(a, device=DEV) for a in (cols, ptr, rows))
        L_ref, D_ref = tb.reduce_ldos_dm(ctx, Gd, zd, wd, -1.0, 0.1, rd, pd, od, S=Sd)
        L = torch.empty((len(cols), len(z)), dtype=torch.float64, device=DEV)
        D = torch.empty(len(rows), dtype=torch.float64, device=DEV)
        rc = _static_call(ctx, Gd, zd, wd, -1.0, 0.1, rd, pd, od, Sd, L, D)
        assert rc == 0, ctx.lib.tb_last_error(ctx.h)
        torch.cuda.synchronize()
        assert torch.allclose(L, L_ref, rtol=1e-12, atol=1e-14), call
        assert torch.allclose(D, D_ref, rtol=1e-12, atol=1e-14), call


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
