"""Matrix Market input for users' own H and S (host side).

Sec. 6 describes a sparse matrix collection distributed as Matrix Market
files.  read_matrix_market() turns such a file (real, general or symmetric,
coordinate format) into the library's BSR layout with a given block edge:
block-column indices ascending within each block row and every diagonal block
present (explicit zeros where the file has none), values in FP64.
"""
from __future__ import annotations

import numpy as np

from . import Bsr


def read_matrix_market(path: str, bdim: int = 1) -> Bsr:
    import scipy.io
    import scipy.sparse as sp

    A = scipy.io.mmread(path)
    if not sp.issparse(A):
        A = sp.coo_matrix(A)
    A = sp.csr_matrix(A, dtype=np.float64)
    n = A.shape[0]
    if A.shape[0] != A.shape[1]:
        raise ValueError("matrix must be square")
    if n % bdim:
        raise ValueError(f"order {n} is not a multiple of the block edge {bdim}")
    if np.iscomplexobj(A.data):
        raise ValueError("H and S are real symmetric; complex files are not accepted")
    # make every diagonal block present: add an explicit structural diagonal
    A = (A + sp.eye(n, format="csr") * 0.0).tocsr()
    A.sum_duplicates()
    B = sp.bsr_matrix(A, blocksize=(bdim, bdim))
    # keep the diagonal blocks even where the file stores no entry in them
    nb = n // bdim
    pattern = sp.csr_matrix((np.ones(B.indices.size), B.indices, B.indptr), shape=(nb, nb))
    pattern = (pattern + sp.eye(nb, format="csr")).tocsr()
    pattern.sort_indices()
    row_ptr = pattern.indptr.astype(np.int64)
    col_idx = pattern.indices.astype(np.int32)
    val = np.zeros((col_idx.size, bdim, bdim))
    B.sort_indices()
    for a in range(nb):
        have = {int(c): k for k, c in enumerate(B.indices[B.indptr[a]:B.indptr[a + 1]])}
        for k in range(row_ptr[a], row_ptr[a + 1]):
            j = have.get(int(col_idx[k]))
            if j is not None:
                val[k] = B.data[B.indptr[a] + j]
    return Bsr(nb, bdim, row_ptr, col_idx, val)


def write_matrix_market(path: str, A: Bsr, symmetric: bool = True) -> None:
    """Write a BSR matrix as a real coordinate Matrix Market file."""
    import scipy.io
    import scipy.sparse as sp

    b = A.bdim
    blocks = sp.bsr_matrix((np.asarray(A.val), np.asarray(A.col_idx), np.asarray(A.row_ptr)),
                           shape=(A.n_brows * b, A.n_brows * b))
    scipy.io.mmwrite(path, sp.coo_matrix(blocks), symmetry="symmetric" if symmetric else "general")
