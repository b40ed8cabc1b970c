"""Hop-shell local subspaces and principal submatrices (oracle side).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

The order-N principle (Sec. 2) rests on locality: the Green's-function column
of an atom is computed on the atoms near it.  A subspace of hop radius R
around atom a is every atom whose breadth-first hop distance from a in the
nearest-neighbour graph is at most R; its rows are all orbitals of those
atoms.  The truncated problem is the principal submatrix of H (and S) on those
rows, solved for the same unit right-hand side.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from .systems import Bsr


def hop_distances(nbr_ptr: np.ndarray, nbr: np.ndarray, start: int, radius: int) -> dict:
    """{atom: hop distance} for every atom within `radius` hops of `start` (plain BFS)."""
    dist = {int(start): 0}
    queue = deque([int(start)])
    while queue:
        a = queue.popleft()
        if dist[a] == radius:
            continue
        for c in nbr[nbr_ptr[a]:nbr_ptr[a + 1]]:
            c = int(c)
            if c not in dist:
                dist[c] = dist[a] + 1
                queue.append(c)
    return dist


def subspace_atoms(nbr_ptr, nbr, start: int, radius: int) -> np.ndarray:
    """Atoms within `radius` hops of `start`, ascending."""
    return np.array(sorted(hop_distances(nbr_ptr, nbr, start, radius)), dtype=np.int64)


def subspace_rows(atoms: np.ndarray, bdim: int) -> np.ndarray:
    return (np.asarray(atoms, dtype=np.int64)[:, None] * bdim + np.arange(bdim)[None, :]).ravel()


def principal_submatrix(A: Bsr, atoms: np.ndarray) -> Bsr:
    """BSR of A restricted to the block rows/columns `atoms` (ascending), renumbered 0.."""
    atoms = np.asarray(atoms, dtype=np.int64)
    local = {int(a): i for i, a in enumerate(atoms)}
    row_ptr = [0]
    cols, vals = [], []
    for a in atoms:
        for k in range(A.row_ptr[a], A.row_ptr[a + 1]):
            c = int(A.col_idx[k])
            if c in local:
                cols.append(local[c])
                vals.append(A.val[k])
        row_ptr.append(len(cols))
    b = A.bdim
    val = np.asarray(vals).reshape(-1, b, b) if vals else np.zeros((0, b, b))
    return Bsr(len(atoms), b, np.asarray(row_ptr, np.int64), np.asarray(cols, np.int32), val)
