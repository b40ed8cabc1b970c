"""Shared test helpers: small systems and output-row layouts (no method arithmetic)."""
import numpy as np


def out_layout(row_lists):
    """CSR-style (out_ptr, out_rows) from a list of row arrays."""
    ptr = np.zeros(len(row_lists) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(r) for r in row_lists])
    rows = np.concatenate([np.asarray(r, dtype=np.int64) for r in row_lists]) if row_lists else \
        np.zeros(0, np.int64)
    return ptr, rows


def rel_err_per_shift(G, Gref):
    """max_k |G_k - Gref_k| / max_k |Gref_k| per shift (last axis)."""
    num = np.abs(G - Gref).max(axis=0)
    den = np.abs(Gref).max(axis=0)
    return num / den
