"""GPU parity of the local-subspace path: hop-shell subspaces (bit-exact) and the
truncated-problem shifted COCG (one CTA per column) against the oracle's plain
BFS, principal submatrices and FP64 shifted COCG / dense LU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1402_7285_gb300 as tb
from oracle import cocg, dense, subspace, systems
from tests.helpers import out_layout, rel_err_per_shift
from workloads import shifts_of as wl_shifts
from workloads import C3_SYSTEM, C4_SYSTEM, C5_SYSTEM, midpoint_shifts, sample_local_rhs, scaled

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


def _bsr(b, device=DEV):
    return tb.Bsr(b.n_brows, b.bdim, b.row_ptr, b.col_idx, b.val).to(device)


@pytest.mark.parametrize("spec", [scaled(C3_SYSTEM, n_sites=2000, bdim=9), scaled(C4_SYSTEM, n_sites=6000),
                                  scaled(C5_SYSTEM, L=14)], ids=["fcc_b9", "fcc_vac_slab", "sc_b4"])
def test_subspaces_match_oracle_bfs(spec):
    o = systems.build_system(spec, 1234)
    rows, rad = sample_local_rhs(o.n_atoms, spec.bdim, 200, (2, 3, 4, 5), 1234)
    H = tb.Bsr(o.H.n_brows, o.H.bdim, o.H.row_ptr, o.H.col_idx, o.H.val)
    ptr, atoms = tb.local_subspaces(H, rows, rad)
    for c in range(len(rows)):
        ref = subspace.subspace_atoms(o.nbr_ptr, o.nbr, rows[c] // spec.bdim, int(rad[c]))
        assert np.array_equal(atoms[ptr[c]:ptr[c + 1]], ref)


def _local_case(spec, n_rhs, radii, seed=1234, kept="pattern"):
    o = systems.build_system(spec, seed)
    rows, rad = sample_local_rhs(o.n_atoms, spec.bdim, n_rhs, radii, seed)
    H = tb.Bsr(o.H.n_brows, o.H.bdim, o.H.row_ptr, o.H.col_idx, o.H.val)
    sptr, satoms = tb.local_subspaces(H, rows, rad)
    if kept == "pattern":
        rl = [systems.block_pattern_rows(o.H, j) for j in rows]
    else:
        rl = [np.array([j]) for j in rows]
    optr, orows = out_layout(rl)
    return o, rows, rad, sptr, satoms, rl, optr, orows


def _oracle_local(o, rows, sptr, satoms, rl, z, tol):
    """Principal submatrix per column, oracle COCG and dense LU there."""
    b = o.spec.bdim
    out_cocg, out_lu = [], []
    for c, j in enumerate(rows):
        atoms = satoms[sptr[c]:sptr[c + 1]].astype(np.int64)
        Hs = subspace.principal_submatrix(o.H, atoms)
        Ss = None if o.S is None else subspace.principal_submatrix(o.S, atoms)
        lrow = {int(a): i for i, a in enumerate(atoms)}
        jl = lrow[int(j // b)] * b + int(j % b)
        keep = [lrow[int(r // b)] * b + int(r % b) if int(r // b) in lrow else -1 for r in rl[c]]
        kl = np.array([k if k >= 0 else 0 for k in keep])
        res = cocg.shifted_cocg(Hs.to_csr(), None if Ss is None else Ss.to_csr(), z, [jl], [0, len(kl)], kl,
                                tol=tol)
        g = res.G.copy()
        ex = dense.green_lu(Hs.to_dense(), None if Ss is None else Ss.to_dense(), z, [jl])[kl, 0, :]
        for i, k in enumerate(keep):
            if k < 0:
                g[i] = 0
                ex[i] = 0
        out_cocg.append(g)
        out_lu.append(ex)
    return out_cocg, out_lu


@pytest.mark.parametrize("spec,radii", [
    (scaled(C3_SYSTEM, n_sites=1500, bdim=9), (1, 2)),      # S = I, b = 9
    (scaled(C4_SYSTEM, n_sites=4000), (1, 2, 3)),           # S = I + 0.02 I, vacancies, slab
    (scaled(C5_SYSTEM, L=12), (2, 3, 4)),                   # SC b = 4, S != I
], ids=["fcc_b9", "fcc_overlap", "sc_overlap"])
def test_local_fp64_matches_oracle(ctx, spec, radii):
    o, rows, rad, sptr, satoms, rl, optr, orows = _local_case(spec, 24, radii)
    z = midpoint_shifts(10, -8.0, 8.0, 0.05)
    Hd = _bsr(o.H)
    Sd = None if o.S is None else _bsr(o.S)
    order = np.argsort(-np.diff(sptr), kind="stable")
    res = tb.solve_local(ctx, Hd, Sd, z, rows, sptr, satoms, optr, orows, order=order, tol=1e-12)
    assert res.rc == 0 and np.all(_np(res.status) == tb.TB_COL_CONVERGED)
    G = _np(res.G)
    ref_cocg, ref_lu = _oracle_local(o, rows, sptr, satoms, rl, z, 1e-12)
    for c in range(len(rows)):
        g = G[optr[c]:optr[c + 1]]
        assert rel_err_per_shift(g, ref_cocg[c]).max() < 1e-10
        assert rel_err_per_shift(g, ref_lu[c]).max() < 1e-10


def test_local_df64_matches_oracle(ctx):
    o, rows, rad, sptr, satoms, rl, optr, orows = _local_case(scaled(C5_SYSTEM, L=12), 16, (2, 3))
    z = midpoint_shifts(10, -8.0, 8.0, 0.05)
    res = tb.solve_local(ctx, _bsr(o.H), _bsr(o.S), z, rows, sptr, satoms, optr, orows, tol=1e-11,
                         precision=tb.TB_PREC_DF64)
    assert np.all(_np(res.status) == tb.TB_COL_CONVERGED)
    G = _np(res.G)
    _, ref_lu = _oracle_local(o, rows, sptr, satoms, rl, z, 1e-12)
    for c in range(len(rows)):
        assert rel_err_per_shift(G[optr[c]:optr[c + 1]], ref_lu[c]).max() < 1e-9


@pytest.mark.parametrize("spec,radii,precision", [
    (scaled(C3_SYSTEM, n_sites=20000, bdim=9), (5,), tb.TB_PREC_DF64),   # 3 vectors x 560 atoms x 9 x 16 B
    (scaled(C5_SYSTEM, L=16), (7,), tb.TB_PREC_FP64),                   # 8 vectors x 575 atoms x 4 x 16 B
], ids=["fcc_b9_r5_df64", "sc_r7_overlap_fp64"])
def test_local_vectors_beyond_shared_memory(ctx, spec, radii, precision):
    """Subspaces whose vectors exceed one CTA's shared memory run with the
    vectors in a global workspace; results as the oracle's COCG."""
    o, rows, rad, sptr, satoms, rl, optr, orows = _local_case(spec, 3, radii, kept="diag")
    b = spec.bdim
    nv = 3 if o.S is None else 8
    assert nv * np.diff(sptr).max() * b * 16 > 232448          # does not fit 227 KB
    z = midpoint_shifts(4, -6.0, 6.0, 0.1)
    res = tb.solve_local(ctx, _bsr(o.H), None if o.S is None else _bsr(o.S), z, rows, sptr, satoms, optr, orows,
                         tol=1e-11, precision=precision)
    assert res.rc == 0 and np.all(_np(res.status) == tb.TB_COL_CONVERGED)
    G = _np(res.G)
    for c, j in enumerate(rows):
        atoms = satoms[sptr[c]:sptr[c + 1]].astype(np.int64)
        Hs = subspace.principal_submatrix(o.H, atoms)
        Ss = None if o.S is None else subspace.principal_submatrix(o.S, atoms)
        jl = int(np.searchsorted(atoms, j // b)) * b + int(j % b)
        ref = cocg.shifted_cocg(Hs.to_csr(), None if Ss is None else Ss.to_csr(), z, [jl], [0, 1], [jl], tol=1e-12)
        assert rel_err_per_shift(G[optr[c]:optr[c + 1]], ref.G).max() < 1e-9


def test_local_df64_restarts_for_shifts_harder_than_the_seed(ctx):
    """C5-like columns at tol 1e-5 with the C5 shift grid: some shifts (near
    the p-orbital onsite level) need the seed residual far below what df64
    carries; the column restarts with the worst shift as its seed.  Every
    column converges and agrees with the oracle's FP64 COCG."""
    from workloads import C5
    spec = scaled(C5_SYSTEM, L=12)
    o, rows, rad, sptr, satoms, rl, optr, orows = _local_case(spec, 48, (4, 5), kept="diag")
    z = wl_shifts(C5)
    res = tb.solve_local(ctx, _bsr(o.H), _bsr(o.S), z, rows, sptr, satoms, optr, orows, tol=1e-5,
                         precision=tb.TB_PREC_DF64, max_iter=30000)
    assert np.all(_np(res.status) == tb.TB_COL_CONVERGED)
    assert np.all(_np(res.resid) <= 1e-5)
    G = _np(res.G)
    b = spec.bdim
    for c in range(0, len(rows), 12):
        atoms = satoms[sptr[c]:sptr[c + 1]].astype(np.int64)
        Hs = subspace.principal_submatrix(o.H, atoms)
        Ss = subspace.principal_submatrix(o.S, atoms)
        jl = int(np.searchsorted(atoms, rows[c] // b)) * b + int(rows[c] % b)
        ex = dense.green_lu(Hs.to_dense(), Ss.to_dense(), z, [jl])[[jl], 0, :]
        # the FP64 oracle at tol 1e-5 is up to 6.9e-6 from dense LU on these columns
        assert rel_err_per_shift(G[optr[c]:optr[c + 1]], ex).max() < 1e-5


def test_local_order_does_not_change_results(ctx):
    o, rows, rad, sptr, satoms, rl, optr, orows = _local_case(scaled(C5_SYSTEM, L=10), 30, (1, 2, 3))
    z = midpoint_shifts(6, -8.0, 6.0, 0.1)
    Hd, Sd = _bsr(o.H), _bsr(o.S)
    a = tb.solve_local(ctx, Hd, Sd, z, rows, sptr, satoms, optr, orows, tol=1e-11)
    rng = np.random.default_rng(0)
    b = tb.solve_local(ctx, Hd, Sd, z, rows, sptr, satoms, optr, orows, order=rng.permutation(len(rows)), tol=1e-11)
    assert np.array_equal(_np(a.G), _np(b.G))
    assert np.array_equal(_np(a.iters), _np(b.iters))


def test_local_mixed_precision_error(ctx):
    o, rows, rad, sptr, satoms, rl, optr, orows = _local_case(scaled(C3_SYSTEM, n_sites=1500, bdim=9), 16, (1, 2),
                                                              kept="diag")
    z = midpoint_shifts(16, -8.0, 8.0, 0.02)
    res = tb.solve_local(ctx, _bsr(o.H), None, z, rows, sptr, satoms, optr, orows, tol=1e-5,
                         precision=tb.TB_PREC_MIXED)
    assert np.all(_np(res.status) == tb.TB_COL_CONVERGED)
    G = _np(res.G)
    _, ref_lu = _oracle_local(o, rows, sptr, satoms, rl, z, 1e-12)
    errs = np.concatenate([rel_err_per_shift(G[optr[c]:optr[c + 1]], ref_lu[c]) for c in range(len(rows))])
    assert errs.max() < 1e-3 and np.median(errs) < 2e-4


def test_local_rejects_bad_subspace(ctx):
    o, rows, rad, sptr, satoms, rl, optr, orows = _local_case(scaled(C5_SYSTEM, L=6), 4, (1,))
    bad = satoms.copy()
    bad[sptr[1]:sptr[2]] = bad[sptr[1]:sptr[2]][::-1]       # not ascending
    with pytest.raises(tb.TbError):
        tb.solve_local(ctx, _bsr(o.H), _bsr(o.S), midpoint_shifts(4, -5, 5, 0.1), rows, sptr, bad, optr, orows)
    with pytest.raises(tb.TbError):
        tb.solve_local(ctx, _bsr(o.H), _bsr(o.S), midpoint_shifts(4, -5, 5, 0.1), rows, sptr, satoms, optr, orows,
                       order=np.zeros(len(rows), np.int64))
