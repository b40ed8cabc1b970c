"""Exact Green's functions for small systems (oracle route O1) and closed forms.

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

G_ij(z) = e_i^T (z S - H)^{-1} e_j is the exact solution of Eq. 2 (Sec. 3)
with b = e_j.  Two independent library routes compute it:
  * LU: a dense complex solve of (z S - H) X = E for each shift;
  * eigen: H Y = S Y diag(lambda), Y^T S Y = I (Eq. 1, Sec. 2), then
    G_ij(z) = sum_k Y_ik Y_jk / (z - lambda_k).
Closed forms for clean periodic lattices (finite Fourier sums) pin both.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def green_lu(H: np.ndarray, S: np.ndarray | None, z: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """G[:, c, m] = (z_m S - H)^{-1} e_{cols[c]} (full columns), complex128 [M, ncols, nz]."""
    M = H.shape[0]
    Smat = np.eye(M) if S is None else S
    E = np.zeros((M, len(cols)))
    E[np.asarray(cols), np.arange(len(cols))] = 1.0
    out = np.empty((M, len(cols), len(z)), np.complex128)
    for m, zm in enumerate(z):
        out[:, :, m] = sla.solve(zm * Smat - H, E)
    return out


def green_eig(H: np.ndarray, S: np.ndarray | None, z: np.ndarray, cols: np.ndarray):
    """Same as green_lu via the generalized eigen-decomposition."""
    lam, Y = sla.eigh(H) if S is None else sla.eigh(H, S)
    Yc = Y[np.asarray(cols), :]                         # [ncols, K]
    inv = 1.0 / (np.asarray(z)[None, :] - lam[:, None])  # [K, nz]
    return np.einsum("ik,ck,km->icm", Y, Yc, inv)


def eigenpairs(H: np.ndarray, S: np.ndarray | None):
    return sla.eigh(H) if S is None else sla.eigh(H, S)


def chain_green(L: int, eps0: float, t: float, z: complex, i: int, j: int) -> complex:
    """Clean periodic chain: G_ij(z) = (1/L) sum_k e^{ik(i-j)} / (z - eps0 - 2 t cos k)."""
    k = 2.0 * np.pi * np.arange(L) / L
    return complex(np.sum(np.exp(1j * k * (i - j)) / (z - eps0 - 2.0 * t * np.cos(k))) / L)


def sc_green(L: int, eps0: float, t: float, z: complex, ri, rj) -> complex:
    """Clean periodic SC lattice (one orbital): Fourier sum over the L^3 Bloch vectors."""
    k = 2.0 * np.pi * np.arange(L) / L
    kx, ky, kz = np.meshgrid(k, k, k, indexing="ij")
    e = eps0 + 2.0 * t * (np.cos(kx) + np.cos(ky) + np.cos(kz))
    d = np.asarray(ri) - np.asarray(rj)
    phase = np.exp(1j * (kx * d[0] + ky * d[1] + kz * d[2]))
    return complex(np.sum(phase / (z - e)) / L ** 3)


def infinite_chain_g00(eps0: float, t: float, z: complex) -> complex:
    """Infinite 1D chain: G_00 = 1/sqrt((z-eps0)^2 - 4 t^2), branch with Im G < 0 for Im z > 0."""
    w = z - eps0
    g = 1.0 / np.sqrt(w * w - 4.0 * t * t + 0j)
    if g.imag > 0:
        g = -g
    return complex(g)
