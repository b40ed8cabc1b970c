"""Pins of the oracle's shifted QMR (oracle/qmr.py), CPU only.

* Real symmetric H, S = I and real shifts: the Lanczos vectors are
  orthonormal and the quasi-residual |tau_{k+1}| equals the 2-norm of the true
  residual e_j - (z - H) x_k at every step (the method is MINRES there);
  checked at each step against the explicitly computed residual.
* The quasi-residual never increases (complex shifts, S != I).
* Converged results equal the exact Green's function (dense LU) with S != I.
* With n_rows steps the Krylov space is the whole space: the result is exact.
* Planted mistakes (a dropped conjugate in a rotation, a wrong sign of the
  sub-diagonal, the previous rotation applied with the wrong cosine) fail them.
"""
import inspect

import numpy as np
import pytest

from oracle import dense, qmr, systems
from tests.helpers import out_layout, rel_err_per_shift
from workloads import C1_SYSTEM, C2_SYSTEM, midpoint_shifts, scaled


def _minres_pin(fn) -> bool:
    o = systems.build_system(scaled(C1_SYSTEM, L=4), 3)
    Hd = o.H.to_dense()
    n = Hd.shape[0]
    z = np.array([-6.7, -0.37, 0.0123, 5.9])               # real shifts (indefinite z - H for most)
    j = 5
    r = fn(o.H.to_csr(), None, z, [j], [0, n], np.arange(n), tol=1e-13, max_iter=40, keep_full=True)
    hist = r.history[0]
    b = np.zeros(n)
    b[j] = 1.0
    # replay: the k-step iterate is not stored, so compare the final step and recompute the
    # step-by-step residual norms with fresh runs of fixed length
    for steps in (1, 2, 5, 9, 17):
        rs = fn(o.H.to_csr(), None, z, [j], [0, n], np.arange(n), tol=0.0, max_iter=steps, keep_full=True)
        x = rs.x_full[0]
        for m in range(len(z)):
            true = np.linalg.norm(b - (z[m] * np.eye(n) - Hd) @ x[:, m])
            if not abs(true - rs.resid[0, m]) <= 1e-10 * max(true, 1e-300) + 1e-14:
                return False
            if not abs(rs.history[0][-1, m] - hist[steps - 1, m]) <= 1e-12:
                return False
    return True


def test_real_symmetric_quasi_residual_is_the_true_residual():
    assert _minres_pin(qmr.shifted_qmr)


def _case_overlap():
    o = systems.build_system(scaled(C2_SYSTEM, L=3), 11)
    cols = np.array([0, 37, o.n_rows - 1])
    rl = [systems.block_pattern_rows(o.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    return o, cols, rl, ptr, rows, midpoint_shifts(7, -9.0, 7.0, 0.05)


def _monotone_and_exact_pin(fn) -> bool:
    o, cols, rl, ptr, rows, z = _case_overlap()
    r = fn(o.H.to_csr(), o.S.to_csr(), z, cols, ptr, rows, tol=1e-12, max_iter=2000)
    if np.any(r.status != 0):
        return False
    for h in r.history:
        if np.any(np.diff(h, axis=0) > 1e-14 * h[:-1]):
            return False
    ex = dense.green_lu(o.H.to_dense(), o.S.to_dense(), z, cols)
    for c in range(len(cols)):
        if rel_err_per_shift(r.G[ptr[c]:ptr[c + 1]], ex[rl[c], c, :]).max() > 1e-9:
            return False
    return True


def test_quasi_residual_monotone_and_converged_result_exact():
    assert _monotone_and_exact_pin(qmr.shifted_qmr)


def test_full_krylov_space_gives_the_exact_solution():
    """n steps on an n-dimensional system (random symmetric H, random SPD S,
    distinct eigenvalues): the Krylov space is the whole space."""
    rng = np.random.default_rng(8)
    n = 10
    A = rng.standard_normal((n, n))
    Hd = (A + A.T) / 2
    B = rng.standard_normal((n, n)) * 0.1
    Sd = np.eye(n) + (B + B.T) / 2
    import scipy.sparse as sp
    def csr(m):
        c = sp.csr_matrix(m)
        return c.indptr.astype(np.int64), c.indices.astype(np.int32), c.data
    z = np.array([-1.3 + 0.2j, 0.4 + 0.05j, 2.2 + 0.5j])
    r = qmr.shifted_qmr(csr(Hd), csr(Sd), z, [3], [0, n], np.arange(n), tol=0.0, max_iter=n)
    ex = dense.green_lu(Hd, Sd, z, [3])[:, 0, :]
    assert rel_err_per_shift(r.G, ex).max() < 1e-9


MUTATIONS = {
    "rotation_without_conjugate": ("a = -np.conj(s1[m]) * theta + c1[m] * a_in", "a = -s1[m] * theta + c1[m] * a_in"),
    "subdiagonal_sign": ("bsub = -beta_next", "bsub = beta_next"),
    "second_rotation_cosine": ("theta = c2[m] * (-beta)", "theta = c1[m] * (-beta)"),
    "rhs_rotation_conjugate": ("tau[m] = -np.conj(sk) * tau[m]", "tau[m] = -sk * tau[m]"),
}


@pytest.mark.parametrize("mut", sorted(MUTATIONS))
def test_pins_catch_planted_mistakes(mut):
    old, new = MUTATIONS[mut]
    src = inspect.getsource(qmr.shifted_qmr)
    assert src.count(old) == 1
    ns = dict(vars(qmr))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    f = ns["shifted_qmr"]
    try:
        ok = _minres_pin(f) and _monotone_and_exact_pin(f)
    except Exception:
        ok = False
    assert not ok, mut
