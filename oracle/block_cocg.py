"""Oracle: shifted block COCG for (z_m S - H) X = [e_j1 ... e_jW] (seed sharing across columns).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

Eq. 2 (Sec. 3) for a block of W unit right-hand sides solved together: one
block Krylov space of the seed operator serves every column and every shift.
The paper names the generalized shifted COCG and prints no recurrences; this
file restates block CG (O'Leary 1980) for the complex-symmetric S-bilinear
form <U, V> = U^T S V (unconjugated), with the residual block kept
S-orthonormal at every step (the stabilisation of Dubrulle 2001), and derives
the shifted systems from the block three-term recurrence.  All matrices below
are W x W and act from the right; A = S^-1 (z_s S - H) is the seed operator,
self-adjoint in the S-form.

  seed:  R_0 = S^-1 B = Q_0 xi_0,  Q^T S Q = I (xi_0 from the unconjugated
         Cholesky factor of R_0^T S R_0),  P_0 = Q_0
         alpha_n = (P_n^T S A P_n)^-1 = (P_n^T U_n)^-1,  U_n = z_s S P_n - H P_n
         Q~ = Q_n - A P_n alpha_n = Q_{n+1} tau_{n+1}   (S-orthonormalised)
         P_{n+1} = Q_{n+1} + P_n tau_{n+1}^T,  xi_{n+1} = tau_{n+1} xi_n
         (seed residual R_n = Q_n xi_n)
  three-term form:  A Q_n = [Q_n c_n - Q_{n+1} tau_{n+1} - Q_{n-1} e_n] alpha_n^-1,
         e_n = alpha_{n-1}^-1 tau_n^T alpha_n,  c_n = I + tau_n e_n  (e_0 = 0)
  shift sigma = z_m - z_s, residual R^s_n = Q_n Phi_n (Phi_0 = xi_0): matching
  the coefficients of Q_{n+1}, Q_n, Q_{n-1} in the shifted block COCG's own
  three-term recurrence gives
         alpha^s_n = [c_n alpha_n^-1 Phi_n + sigma Phi_n - Phi_n Phi_{n-1}^-1 e_n alpha_n^-1 Phi_n]^-1 Phi_n
         K = alpha_n^-1 Phi_n alpha^s_n,  Phi_{n+1} = tau_{n+1} K,  gamma^s_n = Phi_{n-1}^-1 e_n K
         beta^s_{n-1} = alpha^s_{n-1} gamma^s_n (alpha^s_n)^-1
         P^s_n = R^s_n + P^s_{n-1} beta^s_{n-1},  X^s_{n+1} = X^s_n + P^s_n alpha^s_n
  With W = 1 every matrix is a scalar and the recurrences are those of the
  scalar shifted COCG (Phi_n = 1 / pi_n up to the seed's scaling).

Convergence: column c of shift m stops (its solution is frozen) when
||S R^s_n e_c|| = ||S Q_n Phi_n e_c|| <= tol ||b_c|| (the residual of the
original equation; ||b_c|| = 1); a block is done when every column of every
shift is.  S^-1 is applied exactly (a sparse LU of S); S = None means S = I.
Plain numpy, FP64, one block at a time: a reference, not a fast code.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


@dataclass
class BlockResult:
    G: np.ndarray          # complex [out_total, nz]
    iters: np.ndarray      # int [ncols] outer iterations of the column's block
    status: np.ndarray     # int [ncols] 0 converged, 1 max_iter


def _csr(m):
    if m is None:
        return None
    rp, ci, v = m
    n = len(rp) - 1
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def sym_cholesky(G: np.ndarray) -> np.ndarray:
    """Lower-triangular L with G = L L^T for a complex symmetric G (unconjugated)."""
    n = G.shape[0]
    L = np.zeros_like(G, dtype=np.complex128)
    for j in range(n):
        L[j, j] = np.sqrt(G[j, j] - L[j, :j] @ L[j, :j])
        for i in range(j + 1, n):
            L[i, j] = (G[i, j] - L[i, :j] @ L[j, :j]) / L[j, j]
    return L


def s_orthonormalise(Y: np.ndarray, SY: np.ndarray):
    """Y = Q tau with Q^T S Q = I; returns (Q, S Q, tau), tau upper triangular."""
    tau = sym_cholesky(Y.T @ SY).T
    Q = np.linalg.solve(tau.T, Y.T).T
    SQ = np.linalg.solve(tau.T, SY.T).T
    return Q, SQ, tau


def shifted_block_cocg(csr_h, csr_s, z, cols, out_ptr, out_rows, tol, block, seed=None,
                       max_iter=100000) -> BlockResult:
    """G[out_ptr[c] + k, m] = x^{(m)}_c at row out_rows[out_ptr[c] + k], columns solved in
    consecutive blocks of `block` (the last block may be smaller); seed = median Re z."""
    H = _csr(csr_h)
    S = _csr(csr_s)
    n = H.shape[0]
    z = np.asarray(z, np.complex128)
    nz = z.size
    if seed is None:
        seed = int(np.argsort(z.real, kind="stable")[nz // 2])
    zs = z[seed]
    sigma = z - zs
    if S is None:
        s_mul = lambda X: X
        s_solve = lambda X: X.copy()
    else:
        lu = spl.splu(sp.csc_matrix(S))
        s_mul = lambda X: S @ X
        s_solve = lambda X: lu.solve(X.real) + 1j * lu.solve(X.imag)
    cols = np.asarray(cols, np.int64)
    G = np.zeros((int(out_ptr[-1]), nz), np.complex128)
    iters = np.zeros(cols.size, np.int64)
    status = np.zeros(cols.size, np.int64)
    for g0 in range(0, cols.size, block):
        bc = cols[g0:g0 + block]
        w = bc.size
        I = np.eye(w)
        Bb = np.zeros((n, w), np.complex128)
        Bb[bc, np.arange(w)] = 1.0
        Q, SQ, xi = s_orthonormalise(s_solve(Bb), Bb)
        P, SP = Q.copy(), SQ.copy()
        Phi = np.stack([xi] * nz)
        Phi_prev = Phi.copy()
        Ps = np.zeros((nz, n, w), np.complex128)
        X = np.zeros((nz, n, w), np.complex128)
        a_prev = np.stack([I] * nz).astype(np.complex128)
        done = np.zeros((nz, w), bool)
        alpha_prev = None
        tau_n = np.zeros((w, w), np.complex128)
        it = 0
        while it < max_iter and not done.all():
            U = zs * SP - H @ P
            alpha = np.linalg.inv(P.T @ U)
            ainv = np.linalg.inv(alpha)
            if it == 0:
                e_n = np.zeros((w, w), np.complex128)
            else:
                e_n = np.linalg.solve(alpha_prev, tau_n.T @ alpha)
            c_n = I + tau_n @ e_n
            SQ_t = SQ - U @ alpha                       # S (Q_n - A P_n alpha_n)
            Q1, SQ1, tau1 = s_orthonormalise(s_solve(SQ_t), SQ_t)
            for m in range(nz):
                if done[m].all():
                    continue
                Ph, Php = Phi[m], Phi_prev[m]
                T = c_n @ ainv @ Ph + sigma[m] * Ph
                if it > 0:
                    T = T - Ph @ np.linalg.solve(Php, e_n @ ainv @ Ph)
                a_s = np.linalg.solve(T, Ph)
                K = ainv @ Ph @ a_s
                if it > 0:
                    g_s = np.linalg.solve(Php, e_n @ K)
                    b_s = np.linalg.solve(a_s.T, (a_prev[m] @ g_s).T).T
                else:
                    b_s = np.zeros((w, w), np.complex128)
                Ps[m] = Q @ Ph + Ps[m] @ b_s
                upd = Ps[m] @ a_s
                upd[:, done[m]] = 0.0
                X[m] += upd
                a_prev[m] = a_s
                Phi_prev[m] = Ph
                Phi[m] = tau1 @ K
                done[m] |= np.linalg.norm(SQ1 @ Phi[m], axis=0) <= tol
            P = Q1 + P @ tau1.T
            SP = SQ1 + SP @ tau1.T
            Q, SQ = Q1, SQ1
            alpha_prev, tau_n = alpha, tau1
            it += 1
        for i, c in enumerate(range(g0, g0 + w)):
            rows = np.asarray(out_rows[out_ptr[c]:out_ptr[c + 1]], np.int64)
            G[out_ptr[c]:out_ptr[c + 1]] = X[:, rows, i].T
            iters[c] = it
            status[c] = 0 if done[:, i].all() else 1
    return BlockResult(G, iters, status)
