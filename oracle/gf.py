"""Reductions of Green's-function entries to LDOS and density-matrix elements.

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

Sec. 2 names the density of states and a Green's-function based population
analysis as the physical quantities taken from G; it gives no formula, so the
standard ones are used:
  LDOS  d_j(E_m) = -(1/pi) Im [G(z_m) S]_jj = -(1/pi) Im sum_i G_ji(z_m) S_ij
        (S = I: -(1/pi) Im G_jj(z_m)), z_m = E_m + i eta
  DM    rho_ij   = -(1/pi) Im sum_m w_m f(E_m) G_ij(z_m),
        f the Fermi-Dirac occupation at chemical potential mu and temperature
        kT (kT = 0: step with f(mu) = 1/2), w_m the quadrature weights.
G is complex symmetric (G_ij = G_ji), so the rows kept for column j serve both.
"""
from __future__ import annotations

import numpy as np


def fermi(E: np.ndarray, mu: float, kT: float) -> np.ndarray:
    E = np.asarray(E, dtype=np.float64)
    if kT == 0.0:
        return np.where(E < mu, 1.0, np.where(E > mu, 0.0, 0.5))
    x = (E - mu) / kT
    out = np.empty_like(x)
    pos = x > 0
    ex = np.exp(-x[pos])
    out[pos] = ex / (1.0 + ex)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def ldos(G_rows: np.ndarray, s_row: np.ndarray | None, diag_pos: int | None) -> np.ndarray:
    """LDOS of one column over all shifts.

    G_rows: complex [n_rows_j, nz] = G_ij(z_m) for the kept rows i of column j.
    s_row:  float [n_rows_j] = S_ij for those rows (None: S = I, use the diagonal row).
    diag_pos: index of row j within the kept rows (used when s_row is None).
    """
    if s_row is None:
        return -np.imag(G_rows[diag_pos, :]) / np.pi
    return -np.imag(np.sum(G_rows * np.asarray(s_row)[:, None], axis=0)) / np.pi


def density_matrix(G_rows: np.ndarray, E: np.ndarray, w: np.ndarray, mu: float, kT: float):
    """rho_ij for the kept rows i of one column: -(1/pi) Im sum_m w_m f(E_m) G_ij(z_m)."""
    occ = np.asarray(w) * fermi(E, mu, kT)
    return -np.imag(G_rows @ occ) / np.pi
