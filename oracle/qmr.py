"""Oracle: shifted QMR for (z_m S - H) x = e_j (the gsQMR solver of Sec. 3).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

Sec. 3 names the generalized shifted QMR method for Eq. 2 and prints no
recurrences; this file restates the quasi-minimal residual method for complex
symmetric systems (the QMR of the unconjugated Lanczos process) in the
S-bilinear form <u, v> = u^T S v, step by step:

  Lanczos on A = S^{-1} H, self-adjoint in <.,.>:
    r_0 = S^{-1} b,  rho_1 = sqrt(r_0^T S r_0) = sqrt(r_0^T b)   (complex root)
    v_1 = r_0 / rho_1,  vt_1 = S v_1 = b / rho_1
    k = 1, 2, ...:  u = H v_k,  alpha_k = v_k^T u
                    vt_w = u - alpha_k vt_k - beta_k vt_{k-1}    ( = S w )
                    w = S^{-1} vt_w,  beta_{k+1} = sqrt(w^T vt_w)
                    v_{k+1} = w / beta_{k+1},  vt_{k+1} = vt_w / beta_{k+1}
  so that (z I - A) V_k = V_{k+1} Tz_k with Tz_k the (k+1) x k tridiagonal of
  z I - T: diagonal z - alpha_k, both off-diagonals -beta_{k+1}.
  Every shift z_m minimises || rho_1 e_1 - Tz_k y ||_2 over y (x_k = V_k y):
  the k-th column of Tz_k, (-beta_k, z - alpha_k, -beta_{k+1}) in rows
  k-1, k, k+1, is reduced by the two previous Givens rotations G_{k-2},
  G_{k-1}, then a new rotation G_k = [[c, s], [-conj(s), c]] (c real)
  annihilates its subdiagonal entry:
    eps_k = s_{k-2} (-beta_k),  theta = c_{k-2} (-beta_k)
    theta_k = c_{k-1} theta + s_{k-1} (z - alpha_k)
    a       = -conj(s_{k-1}) theta + c_{k-1} (z - alpha_k)
    nu = sqrt(|a|^2 + |beta_{k+1}|^2),  c_k = |a| / nu,
    s_k = (a / |a|) conj(-beta_{k+1}) / nu,  delta_k = (a / |a|) nu
  the right-hand side rho_1 e_1 is rotated alike: g_k = c_k tau_k,
  tau_{k+1} = -conj(s_k) tau_k (tau_1 = rho_1), and with R_k^{-1}'s direction
  vectors p_k = (v_k - theta_k p_{k-1} - eps_k p_{k-2}) / delta_k the iterate is
  x_k = x_{k-1} + g_k p_k.  |tau_{k+1}| is the quasi-residual; a shift stops
  when |tau_{k+1}| / |rho_1| <= tol (for real symmetric H, S = I and a real
  shift the Lanczos vectors are orthonormal and |tau_{k+1}| is the 2-norm of the
  residual b - (z - H) x_k: the method is then MINRES).
S^{-1} is applied exactly (a sparse LU of S), S = None means S = I.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl


@dataclass
class QmrResult:
    G: np.ndarray          # complex [out_total, nz]
    iters: np.ndarray      # int [ncols] Lanczos steps run
    resid: np.ndarray      # float [ncols, nz] relative quasi-residual at exit
    status: np.ndarray     # int [ncols] 0 converged, 1 max_iter
    history: list          # per column: float [steps, nz] relative quasi-residuals
    x_full: list           # per column (keep_full): complex [n, nz] iterates


def _csr(m):
    if m is None:
        return None
    rp, ci, v = m
    n = len(rp) - 1
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def shifted_qmr(csr_h, csr_s, z, cols, out_ptr, out_rows, tol, max_iter=100000, keep_full=False):
    """G[out_ptr[c] + k, m] = (x^{(m)})_{out_rows[...]} for b = e_{cols[c]}.

    csr_h, csr_s: (row_ptr, col, val) scalar CSR (csr_s None: S = I)."""
    H = _csr(csr_h)
    S = _csr(csr_s)
    n = H.shape[0]
    z = np.asarray(z, dtype=np.complex128)
    nz = z.size
    if S is None:
        solve_s = lambda v: v.copy()
    else:
        lu = spl.splu(sp.csc_matrix(S))
        solve_s = lambda v: lu.solve(v.real) + 1j * lu.solve(v.imag)
    G = np.zeros((int(out_ptr[-1]), nz), np.complex128)
    iters = np.zeros(len(cols), np.int64)
    resid = np.zeros((len(cols), nz))
    status = np.zeros(len(cols), np.int64)
    hist, fulls = [], []
    for c, j in enumerate(cols):
        rows = np.asarray(out_rows[out_ptr[c]:out_ptr[c + 1]], dtype=np.int64)
        b = np.zeros(n, np.complex128)
        b[j] = 1.0
        r0 = solve_s(b)
        rho1 = np.sqrt(r0 @ b)
        v, vt = r0 / rho1, b / rho1
        v_prev = np.zeros(n, np.complex128)
        vt_prev = np.zeros(n, np.complex128)
        beta = 0.0 + 0.0j
        # per shift: the two previous rotations, tau, the two previous directions, the iterate
        c1 = np.ones(nz)
        s1 = np.zeros(nz, np.complex128)
        c2 = np.ones(nz)
        s2 = np.zeros(nz, np.complex128)
        tau = np.full(nz, rho1, np.complex128)
        p1 = np.zeros((n, nz), np.complex128)
        p2 = np.zeros((n, nz), np.complex128)
        x = np.zeros((n, nz), np.complex128)
        active = np.ones(nz, bool)
        h = []
        k = 0
        while k < max_iter and active.any():
            k += 1
            u = H @ v
            alpha = v @ u
            vt_w = u - alpha * vt - beta * vt_prev
            w = solve_s(vt_w)
            beta_next = np.sqrt(w @ vt_w)
            for m in np.nonzero(active)[0]:
                eps = s2[m] * (-beta)
                theta = c2[m] * (-beta)
                a_in = z[m] - alpha
                theta_k = c1[m] * theta + s1[m] * a_in
                a = -np.conj(s1[m]) * theta + c1[m] * a_in
                bsub = -beta_next
                nu = np.sqrt(abs(a) ** 2 + abs(bsub) ** 2)
                if abs(a) == 0.0:
                    ck, sk, delta = 0.0, 1.0 + 0.0j, bsub
                else:
                    ph = a / abs(a)
                    ck, sk, delta = abs(a) / nu, ph * np.conj(bsub) / nu, ph * nu
                g = ck * tau[m]
                tau[m] = -np.conj(sk) * tau[m]
                p = (v - theta_k * p1[:, m] - eps * p2[:, m]) / delta
                x[:, m] += g * p
                p2[:, m], p1[:, m] = p1[:, m], p
                c2[m], s2[m], c1[m], s1[m] = c1[m], s1[m], ck, sk
            rel = np.abs(tau) / abs(rho1)
            h.append(rel.copy())
            active &= ~(rel <= tol)
            if beta_next == 0:
                break
            v_prev, vt_prev = v, vt
            v, vt = w / beta_next, vt_w / beta_next
            beta = beta_next
        G[out_ptr[c]:out_ptr[c + 1]] = x[rows]
        iters[c] = k
        resid[c] = np.abs(tau) / abs(rho1)
        status[c] = 0 if not active.any() else 1
        hist.append(np.array(h))
        fulls.append(x if keep_full else None)
    return QmrResult(G, iters, resid, status, hist, fulls)
