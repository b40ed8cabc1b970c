"""GPU parity of the learned scheduler's parts: descriptors (K10) and the MLP
forward/backward/Adam kernels (K9) against the FP64 oracle, and the gain of
ordering the local-solver work queue by the trained predictor."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1402_7285_gb300 as tb
from oracle import descriptors, mlp, systems
from workloads import C3_SYSTEM, C4_SYSTEM, C5_SYSTEM, sample_local_rhs, scaled

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


def _flat(p):
    return np.concatenate([p[k].ravel() for k in mlp.PARAM_NAMES]).astype(np.float32)


def _unflat(v):
    v = v.astype(np.float64)
    out, o = {}, 0
    for k, shape in (("W1", (64, 32)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("w3", (64,)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[k] = v[o:o + n].reshape(shape)
        o += n
    return out


def _half(v):
    return v.astype(np.float16).astype(np.float64)


@pytest.mark.parametrize("spec,radii", [(scaled(C3_SYSTEM, n_sites=3000, bdim=9), (2, 3, 4)),
                                        (scaled(C4_SYSTEM, n_sites=8000), (2, 3, 4, 5)),
                                        (scaled(C5_SYSTEM, L=14), (2, 3, 4, 5))],
                         ids=["fcc_b9", "fcc_vac", "sc_b4"])
def test_descriptors_match_oracle(ctx, spec, radii):
    o = systems.build_system(spec, 1234)
    rows, rad = sample_local_rhs(o.n_atoms, spec.bdim, 40, radii, 1234)
    H = tb.Bsr(o.H.n_brows, o.H.bdim, o.H.row_ptr, o.H.col_idx, o.H.val)
    S = None if o.S is None else tb.Bsr(o.S.n_brows, o.S.bdim, o.S.row_ptr, o.S.col_idx, o.S.val)
    sptr, satoms = tb.local_subspaces(H, rows, rad)
    D = _np(tb.descriptors(ctx, H.to(DEV), None if S is None else S.to(DEV), rows, rad, sptr, satoms))
    for c in range(len(rows)):
        ref = descriptors.descriptor(o, int(rows[c]), int(rad[c]))
        assert np.allclose(D[c], ref, rtol=2e-5, atol=2e-6), (c, D[c], ref)


def test_mlp_gradient_matches_oracle(ctx):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((777, 32)).astype(np.float32)
    y = rng.standard_normal(777).astype(np.float32)
    p = mlp.init_params(11)
    flat = _flat(p)
    g, loss = tb.mlp_grad(ctx, flat, X, y)
    # oracle at the FP16-rounded weights the forward pass uses
    ph = {k: _half(v) for k, v in _unflat(flat).items()}
    gref = mlp.backward(ph, X.astype(np.float64), y.astype(np.float64))
    gref_flat = np.concatenate([gref[k].ravel() for k in mlp.PARAM_NAMES])
    assert np.linalg.norm(g - gref_flat) <= 2e-5 * np.linalg.norm(gref_flat)
    assert abs(loss - mlp.loss(ph, X.astype(np.float64), y.astype(np.float64))) <= 1e-5 * loss


def test_mlp_predict_and_train_track_oracle(ctx):
    rng = np.random.default_rng(6)
    X = rng.standard_normal((2048, 32)).astype(np.float32)
    t = (np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.1 * X[:, 7]).astype(np.float32)
    p0 = _flat(mlp.init_params(0))
    pred = tb.mlp_predict(ctx, p0, X)
    ref, _ = mlp.forward({k: _half(v) for k, v in _unflat(p0).items()}, X.astype(np.float64))
    assert np.abs(pred - ref).max() < 1e-5 * max(1.0, np.abs(ref).max())
    params, hist = tb.mlp_train(ctx, X, t, epochs=20, batch=128, lr=3e-3, params=p0)
    assert hist[-1] < 0.1 * hist[0]
    # the oracle trained on the same minibatch sequence lands close by
    po = _unflat(p0)
    opt = mlp.Adam(lr=3e-3)
    for _ in range(20):
        for s in range(0, 2048, 128):
            opt.step(po, mlp.backward(po, X[s:s + 128].astype(np.float64), t[s:s + 128].astype(np.float64)))
    lo = mlp.loss(po, X.astype(np.float64), t.astype(np.float64))
    assert abs(hist[-1] - lo) < 0.25 * lo + 1e-3


def test_learned_order_gains_over_plain_order(ctx):
    """Train the predictor on solver-generated (descriptor, iterations) pairs of
    one set of columns, order a held-out set longest-predicted-first, and
    compare the list-scheduling makespan over the solver's CTAs with the plain
    (given) order, using the measured per-column costs."""
    import time
    from paper_1402_7285_gb300 import scheduler
    from workloads import midpoint_shifts
    spec = scaled(C4_SYSTEM, n_sites=40000)
    Hh, Sh, _ = tb.build_system(spec, 1234)
    Hd, Sd = Hh.to(DEV), Sh.to(DEV)
    rows, rad = sample_local_rhs(Hh.n_brows, spec.bdim, 2400, (1, 2, 3, 4), 99)
    perm = np.random.default_rng(5).permutation(len(rows))     # plain order is arbitrary w.r.t. cost
    rows, rad = rows[perm], rad[perm]
    sptr, satoms = tb.local_subspaces(Hh, rows, rad)
    D = _np(tb.descriptors(ctx, Hd, Sd, rows, rad, sptr, satoms))
    optr = np.arange(len(rows) + 1, dtype=np.int64)
    z = midpoint_shifts(16, -8.0, 8.0, 0.01)
    res = tb.solve_local(ctx, Hd, Sd, z, rows, sptr, satoms, optr, rows, tol=1e-6, precision=tb.TB_PREC_DF64)
    assert np.all(_np(res.status) == tb.TB_COL_CONVERGED)
    iters = _np(res.iters).astype(np.float64)
    n_tr = 1600
    pred_model, hist = scheduler.train(ctx, D[:n_tr], iters[:n_tr], epochs=80, batch=128, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    test = slice(n_tr, len(rows))
    p_it = scheduler.predict(ctx, pred_model, D[test])
    true_it = iters[test]
    # rank correlation between predicted and true iteration counts
    rk = lambda a: np.argsort(np.argsort(a))
    rho = np.corrcoef(rk(p_it), rk(true_it))[0, 1]
    assert rho > 0.6, rho
    size = np.diff(sptr)[test] * spec.bdim
    cost = true_it * size                   # work per column ~ iterations x subspace rows
    workers = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    plain = scheduler.greedy_makespan(cost, np.arange(len(cost)), workers)
    learned = scheduler.greedy_makespan(cost, scheduler.longest_first(p_it * size), workers)
    best = scheduler.greedy_makespan(cost, scheduler.longest_first(cost), workers)
    # measured: modeled makespan gain 1.096 (equal to the exact order), rank correlation 0.997
    assert learned <= 0.98 * plain, (learned, plain)
    assert learned <= 1.02 * best, (learned, best)
    print(f"makespan plain {plain:.3e} learned {learned:.3e} exact-order {best:.3e} "
          f"(gain {plain / learned:.3f}); rank corr {rho:.3f}")
    # the same comparison on the GPU: solve the held-out columns in both orders
    sub = lambda a: a[test]
    tp = np.concatenate([[0], np.cumsum(np.diff(sptr)[test])]).astype(np.int64)
    ta = np.concatenate([satoms[sptr[c]:sptr[c + 1]] for c in range(n_tr, len(rows))])
    op = np.arange(len(true_it) + 1, dtype=np.int64)
    times = {}
    for name, order in (("plain", None), ("learned", scheduler.longest_first(p_it * size))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = tb.solve_local(ctx, Hd, Sd, z, sub(rows), tp, ta, op, sub(rows), order=order, tol=1e-6,
                           precision=tb.TB_PREC_DF64)
        torch.cuda.synchronize()
        times[name] = time.perf_counter() - t0
        assert np.array_equal(_np(r.iters), true_it.astype(np.int32))
    print(f"GPU time plain {times['plain']:.3f}s learned {times['learned']:.3f}s")
    # measured: 0.417 s against 0.636 s (1.53x)
    assert times["learned"] <= 0.9 * times["plain"], times
