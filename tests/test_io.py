"""Matrix Market round trip of the builder's matrices (CPU only)."""
import numpy as np

from oracle import systems
from paper_1402_7285_gb300 import io
from workloads import C2_SYSTEM, C3_SYSTEM, scaled


def test_matrix_market_round_trip(tmp_path):
    for spec in (scaled(C2_SYSTEM, L=3), scaled(C3_SYSTEM, n_sites=80, bdim=9)):
        s = systems.build_system(spec, 5)
        p = str(tmp_path / "h.mtx")
        io.write_matrix_market(p, s.H)
        back = io.read_matrix_market(p, spec.bdim)
        assert np.array_equal(back.row_ptr, s.H.row_ptr)
        assert np.array_equal(back.col_idx, s.H.col_idx)
        assert np.abs(back.val - s.H.val).max() < 1e-15 * np.abs(s.H.val).max() + 1e-300


def test_missing_diagonal_blocks_are_added(tmp_path):
    import scipy.io
    import scipy.sparse as sp
    A = sp.coo_matrix(([1.0, 1.0], ([0, 1], [1, 0])), shape=(4, 4))
    p = str(tmp_path / "a.mtx")
    scipy.io.mmwrite(p, A)
    B = io.read_matrix_market(p, 1)
    for a in range(4):
        assert a in B.col_idx[B.row_ptr[a]:B.row_ptr[a + 1]]
