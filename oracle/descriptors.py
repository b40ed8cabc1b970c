"""Per-column local-environment descriptors (oracle side).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

The paper has no learned component; these 32 numbers describe the local
problem of a right-hand side e_j (row j, atom a, orbital o) on its hop-shell
subspace O of radius R, for the iteration-count predictor of the scheduler.
Definition (index: value):
  0      R / 5
  1      log(number of atoms in O) / log(1000)
  2..6   number of atoms at hop distance 1..5 from a inside O, / 100
  7      number of nearest neighbours of a (whole lattice), / 12
  8      H_jj
  9..16  k = 2..9: m_k = e_j^T (H_OO - H_jj I)^k e_j, reported as
         sign(m_k) |m_k|^(1/k)   (normalized spectral moments of the local
         density of states of e_j; they set the spectral width and shape that
         decide how many Krylov iterations a shift needs)
  17     sum_{i != j} S_ij^2 over the row j of S_OO (0 when S = I)
  18     mean of H_ii over all rows of O
  19     standard deviation of H_ii over all rows of O
  20     min of H_ii over O
  21     max of H_ii over O
  22     sum_{i != j} H_ij^2 over row j of H_OO
  23     mean over the in-subspace neighbour blocks of a of their Frobenius norm
  24     rows of O / 1000
  25     fraction of atoms of O at the largest hop distance (surface of O)
  26..31 0 (reserved)
Moments use plain repeated products v <- (H_OO - H_jj I) v from v = e_j in FP64.
"""
from __future__ import annotations

import numpy as np

from .subspace import hop_distances, principal_submatrix

N_DESC = 32


def descriptor(system, j: int, radius: int) -> np.ndarray:
    b = system.spec.bdim
    a = j // b
    dist = hop_distances(system.nbr_ptr, system.nbr, a, radius)
    atoms = np.array(sorted(dist), dtype=np.int64)
    local = {int(x): i for i, x in enumerate(atoms)}
    Hs = principal_submatrix(system.H, atoms).to_dense()
    jl = local[a] * b + j % b
    d = np.zeros(N_DESC)
    d[0] = radius / 5.0
    d[1] = np.log(len(atoms)) / np.log(1000.0)
    for s in range(1, 6):
        d[1 + s] = sum(1 for v in dist.values() if v == s) / 100.0
    d[7] = (system.nbr_ptr[a + 1] - system.nbr_ptr[a]) / 12.0
    hjj = Hs[jl, jl]
    d[8] = hjj
    A = Hs - hjj * np.eye(Hs.shape[0])
    v = np.zeros(Hs.shape[0])
    v[jl] = 1.0
    powers = [v]
    for k in range(1, 10):
        powers.append(A @ powers[-1])
    for k in range(2, 10):
        # m_k = e_j^T A^k e_j = (A^p e_j)^T (A^q e_j) with p + q = k
        p_, q_ = k // 2, k - k // 2
        m = float(powers[p_] @ powers[q_])
        d[9 + k - 2] = np.sign(m) * abs(m) ** (1.0 / k)
    if system.S is not None:
        Ss = principal_submatrix(system.S, atoms).to_dense()
        row = Ss[jl].copy()
        row[jl] = 0.0
        d[17] = float(row @ row)
    diag = np.diag(Hs)
    d[18], d[19], d[20], d[21] = diag.mean(), diag.std(), diag.min(), diag.max()
    row = Hs[jl].copy()
    row[jl] = 0.0
    d[22] = float(row @ row)
    norms = []
    la = local[a]
    for c in system.nbr[system.nbr_ptr[a]:system.nbr_ptr[a + 1]]:
        if int(c) in local:
            lc = local[int(c)]
            norms.append(np.linalg.norm(Hs[la * b:(la + 1) * b, lc * b:(lc + 1) * b]))
    d[23] = float(np.mean(norms)) if norms else 0.0
    d[24] = Hs.shape[0] / 1000.0
    dmax = max(dist.values())
    d[25] = sum(1 for v in dist.values() if v == dmax) / len(atoms)
    return d
