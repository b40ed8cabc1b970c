"""Pins of the oracle's generator and builder (CPU only).

The generator is pinned by the published Philox known-answer outputs; the
lattices by brute-force distance searches and by the closed-form hop-shell
counts of the SC and FCC lattices; the matrices by the structural facts of
Sec. 8 (H, S real symmetric, S_ii = 1, |S_ij| < 1, S positive definite) and by
the moments of the stated distributions.
"""
import numpy as np
import pytest

from oracle import philox, subspace, systems
from workloads import (C1_SYSTEM, C2_SYSTEM, C3_SYSTEM, C4_SYSTEM, C5_SYSTEM, FCC_CLUSTER,
                       SC_PERIODIC, scaled)


def _golden_philox():
    rows = []
    with open(__file__.replace("test_oracle_systems.py", "golden/philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    return rows


def test_philox_known_answers():
    rows = _golden_philox()
    assert len(rows) == 3
    for r in rows:
        ctr, key, expect = r[0:4], r[4:6], r[6:10]
        out = philox.philox4x32_10(*ctr, *key)
        assert [int(v) for v in out] == expect


def test_uniform_and_normal_moments():
    idx = np.arange(200_000)
    u = philox.uniform(99, 3, idx)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    g = philox.normal(99, 3, idx)
    assert abs(g.mean()) < 1e-2 and abs(g.std() - 1.0) < 1e-2
    # fourth moment of a standard normal is 3
    assert abs((g ** 4).mean() - 3.0) < 0.1
    # streams and seeds are independent sequences
    assert not np.allclose(philox.uniform(99, 4, idx[:100]), u[:100])
    assert not np.allclose(philox.uniform(98, 3, idx[:100]), u[:100])


@pytest.mark.parametrize("L", [3, 4, 5])
def test_sc_neighbours_brute_force(L):
    sites, lists = systems.neighbours_sc(L)
    n = L ** 3
    for a in range(n):
        d = np.minimum(np.abs(sites - sites[a]), L - np.abs(sites - sites[a]))
        nn = np.nonzero((d ** 2).sum(axis=1) == 1)[0]
        assert [e[0] for e in lists[a]] == sorted(nn.tolist())
        assert len(nn) == 6


def test_fcc_sites_and_neighbours_brute_force():
    n = 400
    sites = systems.fcc_candidate_sites(n)
    # brute force: all even-sum integer points in a box, ordered by (r^2, x, y, z)
    g = np.arange(-8, 9)
    pts = np.array([(x, y, z) for x in g for y in g for z in g if (x + y + z) % 2 == 0])
    key = sorted(map(tuple, pts), key=lambda p: (p[0] ** 2 + p[1] ** 2 + p[2] ** 2, p[0], p[1], p[2]))
    assert [tuple(s) for s in sites.tolist()] == key[:n]
    spec = scaled(C3_SYSTEM, n_sites=n, bdim=1)
    raster = systems.fcc_sites(spec, 1)
    lists = systems.neighbours_fcc(raster)
    for a in range(raster.shape[0]):
        d2 = ((raster - raster[a]) ** 2).sum(axis=1)
        assert [e[0] for e in lists[a]] == np.nonzero(d2 == 2)[0].tolist()
    # the origin of a 400-site ball is a bulk site: 12 neighbours
    origin = int(np.nonzero((raster == 0).all(axis=1))[0][0])
    assert len(lists[origin]) == 12


def test_hop_shell_counts_closed_forms():
    # FCC: centred cuboctahedral numbers (2n+1)(5n^2+5n+3)/3; SC: octahedral (2n+1)(2n^2+2n+3)/3
    fcc = systems.build_system(scaled(C3_SYSTEM, n_sites=9000, bdim=1), 5)
    origin = int(np.nonzero((fcc.coords == 0).all(axis=1))[0][0])
    sc = systems.build_system(scaled(C1_SYSTEM, L=13), 5)
    for R in range(6):
        fcc_count = (2 * R + 1) * (5 * R * R + 5 * R + 3) // 3
        sc_count = (2 * R + 1) * (2 * R * R + 2 * R + 3) // 3
        assert subspace.subspace_atoms(fcc.nbr_ptr, fcc.nbr, origin, R).size == fcc_count
        assert subspace.subspace_atoms(sc.nbr_ptr, sc.nbr, 0, R).size == sc_count
    assert [(2 * R + 1) * (5 * R * R + 5 * R + 3) // 3 for R in range(6)] == [1, 13, 55, 147, 309, 561]


@pytest.mark.parametrize("spec", [
    scaled(C1_SYSTEM, L=4),
    scaled(C2_SYSTEM, L=3),
    scaled(C3_SYSTEM, n_sites=300, bdim=3),
    scaled(C4_SYSTEM, n_sites=600),
    scaled(C5_SYSTEM, L=4),
], ids=["c1", "c2", "c3", "c4", "c5"])
def test_matrix_structure_facts(spec):
    s = systems.build_system(spec, 1234)
    H = s.H.to_dense()
    assert np.array_equal(H, H.T)
    # block rows: ascending, diagonal present
    for a in range(s.H.n_brows):
        cols = s.H.col_idx[s.H.row_ptr[a]:s.H.row_ptr[a + 1]]
        assert np.all(np.diff(cols) > 0) and a in cols
    if spec.has_overlap:
        S = s.S.to_dense()
        assert np.array_equal(S, S.T)
        assert np.all(np.diag(S) == 1.0)
        off = S - np.diag(np.diag(S))
        assert np.abs(off).max() < 1.0
        np.linalg.cholesky(S)
        assert np.array_equal(s.S.row_ptr, s.H.row_ptr) and np.array_equal(s.S.col_idx, s.H.col_idx)
    else:
        assert s.S is None


def test_distribution_moments_c2():
    s = systems.build_system(scaled(C2_SYSTEM, L=8), 1234)
    H, S = s.H, s.S
    rows = np.repeat(np.arange(H.n_brows), np.diff(H.row_ptr))
    off = H.col_idx != rows
    hop = H.val[off]
    assert abs(hop.mean()) < 0.02 and abs(hop.std() - 0.5) < 0.02
    on = H.val[~off]
    assert np.allclose(on.mean(axis=0).diagonal(), [-5, 1, 1, 1], atol=0.02)
    # symmetrised N(0, 0.1): off-diagonal entries (N_kl + N_lk)/2 have std 0.1/sqrt(2)
    od = on[:, 0, 1]
    assert abs(od.std() - 0.1 / np.sqrt(2)) < 0.01
    sv = S.val[off]
    assert abs(sv.std() - 0.02) < 0.002


def test_vacancies_slab_and_substitution():
    spec = scaled(C4_SYSTEM, n_sites=20000)
    kept = systems.fcc_sites(spec, 1234)
    cand = systems.fcc_candidate_sites(spec.n_sites)
    zmin, zmax = cand[:, 2].min(), cand[:, 2].max()
    # slab: everything above a cut in the upper third is removed
    assert kept[:, 2].max() >= zmin + (zmax - zmin) * 2.0 / 3.0 - 1
    below = (cand[:, 2] <= kept[:, 2].max()).sum()
    assert abs(kept.shape[0] / below - 0.7) < 0.02
    s = systems.build_system(scaled(C5_SYSTEM, L=10), 1234)
    on = s.H.val[s.H.col_idx == np.repeat(np.arange(s.H.n_brows), np.diff(s.H.row_ptr))]
    shifted = np.isclose(on[:, 0, 0], -3.5)
    assert abs(shifted.mean() - 0.1) < 0.02
    assert np.allclose(on[~shifted, 0, 0], -5.0)


def test_builder_is_deterministic():
    a = systems.build_system(scaled(C2_SYSTEM, L=3), 77)
    b = systems.build_system(scaled(C2_SYSTEM, L=3), 77)
    c = systems.build_system(scaled(C2_SYSTEM, L=3), 78)
    assert np.array_equal(a.H.val, b.H.val) and np.array_equal(a.S.val, b.S.val)
    assert not np.array_equal(a.H.val, c.H.val)
