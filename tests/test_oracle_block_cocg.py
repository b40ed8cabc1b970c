"""Pins of the oracle's shifted block COCG (oracle/block_cocg.py), on the CPU.

* One column per block: every block matrix is a scalar and the method is the
  scalar shifted COCG, so after the same number of iterations its iterates
  equal those of the oracle's scalar C implementation (oracle/cocg.c), a code
  that shares nothing with it.
* Blocks of several columns (and a ragged last block): the Green's function
  of Eq. 2 at every shift matches dense LU of z S - H.
* Finite termination: with S = I on a 27-site system, a block of 9 columns
  spans the whole space after 3 steps, so a few steps give the exact answer.
"""
import numpy as np
import pytest

from oracle import block_cocg, cocg, dense, systems
from tests.helpers import out_layout
from workloads import C1_SYSTEM, C2_SYSTEM, midpoint_shifts, scaled


def _case(spec, cols_idx, nz=8, eta=0.05):
    o = systems.build_system(spec, 1234)
    cols = np.asarray(cols_idx, np.int64)
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    z = midpoint_shifts(nz, -6.0, 6.0, eta)
    return o, cols, rl, ptr, rows, z


def test_single_column_blocks_reproduce_the_scalar_oracle_iterates():
    o, cols, rl, ptr, rows, z = _case(scaled(C2_SYSTEM, L=3), [0, 17, 50])
    hs, ss = o.H.to_csr(), o.S.to_csr()
    k = 12                                   # a fixed number of steps, far from convergence
    ref = cocg.shifted_cocg(hs, ss, z, cols, ptr, rows, tol=1e-300, max_iter=k, inner_tol=1e-15)
    got = block_cocg.shifted_block_cocg(hs, ss, z, cols, ptr, rows, tol=1e-300, block=1, max_iter=k)
    assert np.all(ref.iters == k) and np.all(got.iters == k)
    scale = np.abs(ref.G).max(axis=0)
    assert (np.abs(got.G - ref.G).max(axis=0) / scale).max() < 1e-9


@pytest.mark.parametrize("block", [2, 4, 3])
def test_blocks_match_dense_lu(block):
    o, cols, rl, ptr, rows, z = _case(scaled(C2_SYSTEM, L=4), [0, 9, 33, 64, 100, 171, 202, 255])
    hs, ss = o.H.to_csr(), o.S.to_csr()
    res = block_cocg.shifted_block_cocg(hs, ss, z, cols, ptr, rows, tol=1e-11, block=block)
    assert np.all(res.status == 0)
    ex = dense.green_lu(o.H.to_dense(), o.S.to_dense(), z, cols)
    for c in range(len(cols)):
        g, e = res.G[ptr[c]:ptr[c + 1]], ex[rl[c], c, :]
        assert (np.abs(g - e).max(axis=0) / np.abs(e).max(axis=0)).max() < 1e-8


def test_a_block_spanning_the_space_terminates():
    o, cols, rl, ptr, rows, z = _case(scaled(C1_SYSTEM, L=3), [0, 3, 7, 11, 13, 17, 20, 22, 26], nz=4, eta=0.2)
    res = block_cocg.shifted_block_cocg(o.H.to_csr(), None, z, cols, ptr, rows, tol=1e-10, block=9, max_iter=8)
    assert np.all(res.status == 0) and res.iters.max() <= 5
    ex = dense.green_lu(o.H.to_dense(), np.eye(o.n_rows), z, cols)
    for c in range(len(cols)):
        g, e = res.G[ptr[c]:ptr[c + 1]], ex[rl[c], c, :]
        assert np.abs(g - e).max() < 1e-9 * np.abs(e).max()


def test_fewer_block_steps_than_single_column_steps():
    o, cols, rl, ptr, rows, z = _case(scaled(C2_SYSTEM, L=4), [0, 9, 33, 64], nz=8, eta=0.02)
    hs, ss = o.H.to_csr(), o.S.to_csr()
    one = block_cocg.shifted_block_cocg(hs, ss, z, cols, ptr, rows, tol=1e-8, block=1)
    four = block_cocg.shifted_block_cocg(hs, ss, z, cols, ptr, rows, tol=1e-8, block=4)
    assert np.all(one.status == 0) and np.all(four.status == 0)
    assert four.iters.max() < one.iters.max()


_MUTATIONS = {
    "dropped e_n term": ("T = T - Ph @ np.linalg.solve(Php, e_n @ ainv @ Ph)", "T = T"),
    "wrong shift sign": ("T = c_n @ ainv @ Ph + sigma[m] * Ph", "T = c_n @ ainv @ Ph - sigma[m] * Ph"),
    "tau not transposed": ("P = Q1 + P @ tau1.T", "P = Q1 + P @ tau1"),
    "beta^s factors swapped": ("b_s = np.linalg.solve(a_s.T, (a_prev[m] @ g_s).T).T",
                               "b_s = a_prev[m] @ np.linalg.solve(a_s, g_s)"),
}


@pytest.mark.parametrize("name", sorted(_MUTATIONS))
def test_planted_mistakes_fail_a_pin(name, monkeypatch):
    """A plausible slip in the recurrences (a dropped term, a sign, a transposed
    or reordered factor), planted in a copy of the oracle, fails a pin above."""
    import types
    src = open(block_cocg.__file__).read()
    old, new = _MUTATIONS[name]
    assert old in src
    mod = types.ModuleType("mutated_block_cocg")
    exec(compile(src.replace(old, new), "mutated_block_cocg", "exec"), mod.__dict__)
    monkeypatch.setattr(__import__(__name__, fromlist=["x"]), "block_cocg", mod)
    caught = 0
    for pin, args in ((test_blocks_match_dense_lu, (4,)), (test_a_block_spanning_the_space_terminates, ())):
        try:
            pin(*args)
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError):
            caught += 1     # a failed pin, or a breakdown the mistake causes
    assert caught > 0, name
