"""Users' own matrices from Matrix Market files, and the point-given internal
eigenvalue problem (Sec. 7, type I) answered from the Green's function.

The first test writes H and S of a synthetic system to Matrix Market files
(the format of the matrix collection of Sec. 6), reads them back with the
package's reader and solves on the GPU; the Green's function must match the
oracle's FP64 shifted COCG and dense LU of the original matrices.

The second finds the level nearest a given energy a (Sec. 7, type I) from
the density of states the library computes: DOS(E) = sum over all orbitals of
the Mulliken LDOS -(1/pi) Im [G(E + i eta) S]_jj is a sum of Lorentzians
(eta/pi) / ((E - lambda_k)^2 + eta^2), one per generalized eigenvalue.  Near
an isolated level 1/DOS is a parabola in E with its vertex at the level, so
the vertex of the parabola through 1/DOS at the grid maximum and its two
neighbours locates it; the result is checked against the generalized
eigenvalues of the oracle's dense routine.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1402_7285_gb300 as tb
from paper_1402_7285_gb300 import io
from oracle import cocg, dense, systems
from tests.helpers import out_layout, rel_err_per_shift
from workloads import C2_SYSTEM, C4_SYSTEM, midpoint_shifts, scaled

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tb.Context()
    yield c
    c.close()


@pytest.mark.parametrize("prec,tol,bound", [(tb.TB_PREC_FP64, 1e-11, 1e-9), (tb.TB_PREC_DF64, 1e-10, 1e-8)],
                         ids=["fp64", "df64"])
def test_solve_from_matrix_market_files(ctx, tmp_path, prec, tol, bound):
    o = systems.build_system(scaled(C4_SYSTEM, n_sites=400), 1234)
    hp, sp_ = str(tmp_path / "H.mtx"), str(tmp_path / "S.mtx")
    io.write_matrix_market(hp, o.H)
    io.write_matrix_market(sp_, o.S)
    H = io.read_matrix_market(hp, o.H.bdim).to(DEV)
    S = io.read_matrix_market(sp_, o.S.bdim).to(DEV)
    M = o.n_rows
    cols = np.unique(np.linspace(0, M - 1, 10).astype(np.int64))
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    z = midpoint_shifts(9, -8.0, 8.0, 0.05)
    res = tb.solve(ctx, H, S, z, cols, ptr, rows, tol=tol, precision=prec, panel_w=8)
    assert res.rc == 0
    G = res.G.cpu().numpy()
    ref = cocg.shifted_cocg(o.H.to_csr(), o.S.to_csr(), z, cols, ptr, rows, tol=tol, inner_tol=1e-13)
    ex = dense.green_lu(o.H.to_dense(), o.S.to_dense(), z, cols)
    for c in range(len(cols)):
        assert rel_err_per_shift(G[ptr[c]:ptr[c + 1]], ref.G[ptr[c]:ptr[c + 1]]).max() < bound
        assert rel_err_per_shift(G[ptr[c]:ptr[c + 1]], ex[rl[c], c, :]).max() < bound


def test_point_given_level_from_the_density_of_states(ctx):
    o = systems.build_system(scaled(C2_SYSTEM, L=3), 21)
    Hd, Sd = o.H.to_dense(), o.S.to_dense()
    lam, _ = dense.eigenpairs(Hd, Sd)
    # a point between levels, next to a level whose neighbours are far (in units of eta)
    gaps = np.minimum(np.diff(lam)[:-1], np.diff(lam)[1:])
    k = int(np.argmax(gaps)) + 1
    eta = 2e-3
    a = lam[k] + 0.3 * gaps[k - 1]
    # DOS on a grid around a, every orbital a column, kept rows its block pattern (Mulliken LDOS)
    M = o.n_rows
    cols = np.arange(M, dtype=np.int64)
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    E = a + np.linspace(-0.6, 0.6, 121) * gaps[k - 1]
    z = E + 1j * eta
    H = tb.Bsr(o.H.n_brows, o.H.bdim, o.H.row_ptr, o.H.col_idx, o.H.val).to(DEV)
    S = tb.Bsr(o.S.n_brows, o.S.bdim, o.S.row_ptr, o.S.col_idx, o.S.val).to(DEV)
    res = tb.solve(ctx, H, S, z, cols, ptr, rows, tol=1e-11, precision=tb.TB_PREC_FP64, panel_w=32)
    assert res.rc == 0
    L, _ = tb.reduce_ldos_dm(ctx, res.G, z, None, 0.0, 0.0, cols, ptr, rows, S=S, dm=False)
    dos = L.cpu().numpy().sum(axis=0)
    # the Lorentzian sum the DOS must equal (a check of the reduction as well)
    ref = (eta / np.pi / ((E[:, None] - lam[None, :]) ** 2 + eta ** 2)).sum(axis=1)
    assert np.abs(dos - ref).max() < 1e-8 * ref.max()
    i = int(np.argmax(dos))
    assert 0 < i < len(E) - 1
    y = 1.0 / dos[i - 1:i + 2]
    x = E[i - 1:i + 2]
    c2, c1, _ = np.polyfit(x, y, 2)
    level = -c1 / (2 * c2)
    nearest = lam[np.argmin(np.abs(lam - a))]
    assert nearest == lam[k]
    assert abs(level - nearest) < 0.05 * eta, (level, nearest)
