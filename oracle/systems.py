"""Oracle builder of the synthetic tight-binding matrices H and S.

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

Sec. 2 (Eq. 1) and Sec. 8 fix what the matrices are: M x M sparse real
symmetric H (Hamiltonian) and S (overlap) in an atom-orbital (LCAO) basis,
S positive definite with S_ii = 1 and |S_ij| < 1, M proportional to the
number of atoms.  Everything else (lattices, distributions) is the synthetic
workload definition in `workloads`.  This file builds them plainly:

* SC periodic: atom a = x + L (y + L z), the 6 nearest neighbours wrap.
* FCC cluster: integer coordinates in units of half the cubic lattice
  constant with x + y + z even; keep the n sites closest to the origin,
  ordered by (r^2, x, y, z); optional vacancies and a slab cut; the kept
  atoms are numbered in (z, y, x) raster order; 12 neighbour vectors
  (+-1, +-1, 0) and permutations.
* Every random value comes from Philox4x32-10 (`oracle.philox`) keyed by the
  seed, counter (index, stream).  Streams: 1 onsite, 2 hopping, 3 overlap,
  4 vacancy, 5 slab, 6 substitution.  A nearest-neighbour pair (a, a + d)
  with d one of the "positive" directions draws block entry (k, l) at index
  (a * n_pos + d) * b^2 + k * b + l; the block seen from the other atom is
  its transpose, so H and S are exactly symmetric.

The BSR layout: row_ptr int64[n+1], col_idx int32[nnzb] ascending per block
row with the diagonal block included, val float64[nnzb, b, b] row-major.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from workloads import (FCC_CLUSTER, HOP_CONST, HOP_NORMAL, ONSITE_DIAG_NORMAL, ONSITE_UNIFORM,
                       S_CONST, S_IDENTITY, S_NORMAL, SC_PERIODIC, SystemSpec)
from . import philox

STREAM_ONSITE, STREAM_HOP, STREAM_OVERLAP, STREAM_VACANCY, STREAM_SLAB, STREAM_SUBST = 1, 2, 3, 4, 5, 6

SC_POS_DIRS = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.int64)
FCC_POS_DIRS = np.array([[1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1]],
                        dtype=np.int64)


@dataclass
class Bsr:
    n_brows: int
    bdim: int
    row_ptr: np.ndarray   # int64 [n+1]
    col_idx: np.ndarray   # int32 [nnzb]
    val: np.ndarray       # float64 [nnzb, b, b]

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.size)

    def to_dense(self) -> np.ndarray:
        b, n = self.bdim, self.n_brows
        out = np.zeros((n * b, n * b))
        for a in range(n):
            for k in range(self.row_ptr[a], self.row_ptr[a + 1]):
                c = self.col_idx[k]
                out[a * b:(a + 1) * b, c * b:(c + 1) * b] = self.val[k]
        return out

    def to_csr(self):
        """Scalar CSR (row_ptr int64, col int32, val float64) of the same matrix."""
        b, n = self.bdim, self.n_brows
        nnz_row = np.diff(self.row_ptr) * b
        rows_nnz = np.repeat(nnz_row, b)
        row_ptr = np.zeros(n * b + 1, dtype=np.int64)
        np.cumsum(rows_nnz, out=row_ptr[1:])
        col = np.empty(row_ptr[-1], dtype=np.int32)
        val = np.empty(row_ptr[-1], dtype=np.float64)
        for a in range(n):
            k0, k1 = self.row_ptr[a], self.row_ptr[a + 1]
            cols = self.col_idx[k0:k1].astype(np.int64)
            for i in range(b):
                r = a * b + i
                dst = slice(row_ptr[r], row_ptr[r + 1])
                col[dst] = (cols[:, None] * b + np.arange(b)[None, :]).ravel()
                val[dst] = self.val[k0:k1, i, :].ravel()
        return row_ptr, col, val


@dataclass
class System:
    spec: SystemSpec
    seed: int
    coords: np.ndarray     # int64 [n_atoms, 3]
    nbr_ptr: np.ndarray    # int64 [n_atoms+1]  neighbour lists without self, ascending
    nbr: np.ndarray        # int64 [...]
    H: Bsr
    S: Bsr | None
    overlap_seed: int      # seed actually used for the overlap draws

    @property
    def n_atoms(self) -> int:
        return self.coords.shape[0]

    @property
    def n_rows(self) -> int:
        return self.n_atoms * self.spec.bdim


# ---------------------------------------------------------------- lattices

def sc_sites(L: int) -> np.ndarray:
    a = np.arange(L ** 3, dtype=np.int64)
    return np.stack([a % L, (a // L) % L, a // (L * L)], axis=1)


def fcc_candidate_sites(n_sites: int) -> np.ndarray:
    """The n_sites FCC sites closest to the origin, ordered by (r^2, x, y, z)."""
    R = int(np.ceil((3.0 * n_sites / (2.0 * np.pi)) ** (1.0 / 3.0))) + 3
    while True:
        g = np.arange(-R, R + 1, dtype=np.int64)
        x, y, z = np.meshgrid(g, g, g, indexing="ij")
        x, y, z = x.ravel(), y.ravel(), z.ravel()
        keep = ((x + y + z) % 2) == 0
        x, y, z = x[keep], y[keep], z[keep]
        r2 = x * x + y * y + z * z
        order = np.lexsort((z, y, x, r2))
        if order.size >= n_sites and r2[order[n_sites - 1]] < R * R:
            sel = order[:n_sites]
            return np.stack([x[sel], y[sel], z[sel]], axis=1)
        R += 4


def fcc_sites(spec: SystemSpec, seed: int) -> np.ndarray:
    cand = fcc_candidate_sites(spec.n_sites)
    # raster order (z, y, x)
    order = np.lexsort((cand[:, 0], cand[:, 1], cand[:, 2]))
    sites = cand[order]
    keep = np.ones(sites.shape[0], dtype=bool)
    if spec.vacancy_frac > 0.0:
        u = philox.uniform(seed, STREAM_VACANCY, np.arange(sites.shape[0]))
        keep &= ~(u < spec.vacancy_frac)
    if spec.slab:
        zmin, zmax = sites[:, 2].min(), sites[:, 2].max()
        u = philox.uniform(seed, STREAM_SLAB, np.array([0]))[0]
        zcut = zmin + (zmax - zmin) * (2.0 / 3.0 + u / 3.0)
        keep &= ~(sites[:, 2] > zcut)
    return sites[keep]


# ------------------------------------------------------------ neighbours

def neighbours_sc(L: int):
    """Per atom: sorted neighbour atoms, and for each the (owner, dir, transposed) of its pair."""
    if L < 3:
        raise ValueError("periodic SC needs L >= 3")
    sites = sc_sites(L)
    n = sites.shape[0]
    lists = []
    for a in range(n):
        x, y, z = sites[a]
        entries = []
        for d, v in enumerate(SC_POS_DIRS):
            for sgn in (1, -1):
                cx, cy, cz = (x + sgn * v[0]) % L, (y + sgn * v[1]) % L, (z + sgn * v[2]) % L
                c = cx + L * (cy + L * cz)
                owner = a if sgn == 1 else c
                entries.append((c, owner, d, sgn == -1))
        entries.sort()
        lists.append(entries)
    return sites, lists


def neighbours_fcc(sites: np.ndarray):
    index = {tuple(s): i for i, s in enumerate(sites.tolist())}
    lists = []
    for a, s in enumerate(sites.tolist()):
        entries = []
        for d, v in enumerate(FCC_POS_DIRS.tolist()):
            for sgn in (1, -1):
                t = (s[0] + sgn * v[0], s[1] + sgn * v[1], s[2] + sgn * v[2])
                c = index.get(t)
                if c is None:
                    continue
                owner = a if sgn == 1 else c
                entries.append((c, owner, d, sgn == -1))
        entries.sort()
        lists.append(entries)
    return lists


# ------------------------------------------------------------ values

def _pair_blocks(seed, stream, owners, dirs, n_pos, b, sigma):
    """sigma * N(0,1) blocks for the pairs (owner, dir): array [n_pairs, b, b]."""
    base = (owners.astype(np.uint64) * np.uint64(n_pos) + dirs.astype(np.uint64)) * np.uint64(b * b)
    idx = base[:, None] + np.arange(b * b, dtype=np.uint64)[None, :]
    return sigma * philox.normal(seed, stream, idx).reshape(-1, b, b)


def _assemble(spec, lists, n_atoms, n_pos, onsite, pair_block_fn):
    """Build a Bsr from neighbour lists, an onsite array and a pair-block function."""
    b = spec.bdim
    row_ptr = np.zeros(n_atoms + 1, dtype=np.int64)
    cols, blocks = [], []
    owners, dirs, trans = [], [], []
    for a in range(n_atoms):
        entries = lists[a] + [(a, -1, -1, False)]
        entries.sort()
        row_ptr[a + 1] = row_ptr[a] + len(entries)
        for (c, owner, d, t) in entries:
            cols.append(c)
            owners.append(owner)
            dirs.append(d)
            trans.append(t)
    cols = np.asarray(cols, dtype=np.int64)
    owners = np.asarray(owners, dtype=np.int64)
    dirs = np.asarray(dirs, dtype=np.int64)
    trans = np.asarray(trans, dtype=bool)
    val = np.zeros((cols.size, b, b))
    diag = dirs < 0
    rows = np.repeat(np.arange(n_atoms), np.diff(row_ptr))
    val[diag] = onsite[rows[diag]]
    off = ~diag
    pb = pair_block_fn(owners[off], dirs[off])
    pb = np.where(trans[off][:, None, None], np.transpose(pb, (0, 2, 1)), pb)
    val[off] = pb
    return Bsr(n_atoms, b, row_ptr, cols.astype(np.int32), val)


def _onsite_h(spec: SystemSpec, seed: int, n_atoms: int) -> np.ndarray:
    b = spec.bdim
    a = np.arange(n_atoms, dtype=np.uint64)
    if spec.onsite_mode == ONSITE_UNIFORM:
        u = philox.uniform(seed, STREAM_ONSITE, a)
        e = spec.onsite_lo + (spec.onsite_hi - spec.onsite_lo) * u
        on = e[:, None, None] * np.eye(b)[None]
    elif spec.onsite_mode == ONSITE_DIAG_NORMAL:
        idx = a[:, None] * np.uint64(b * b) + np.arange(b * b, dtype=np.uint64)[None, :]
        N = spec.onsite_sigma * philox.normal(seed, STREAM_ONSITE, idx).reshape(-1, b, b)
        on = 0.5 * (N + np.transpose(N, (0, 2, 1))) + np.diag(np.asarray(spec.onsite_diag))[None]
    else:
        raise ValueError(spec.onsite_mode)
    if spec.subst_frac > 0.0:
        u = philox.uniform(seed, STREAM_SUBST, a)
        on = on + np.where(u < spec.subst_frac, spec.subst_shift, 0.0)[:, None, None] * np.eye(b)[None]
    return on


def build_system(spec: SystemSpec, seed: int) -> System:
    b = spec.bdim
    if spec.lattice == SC_PERIODIC:
        if spec.vacancy_frac or spec.slab:
            raise ValueError("vacancies and slabs are defined for the FCC cluster only")
        sites, lists = neighbours_sc(spec.L)
        n_pos = 3
    elif spec.lattice == FCC_CLUSTER:
        sites = fcc_sites(spec, seed)
        lists = neighbours_fcc(sites)
        n_pos = 6
    else:
        raise ValueError(spec.lattice)
    n = sites.shape[0]
    nbr_ptr = np.zeros(n + 1, dtype=np.int64)
    nbr_ptr[1:] = np.cumsum([len(l) for l in lists])
    nbr = np.asarray([e[0] for l in lists for e in l], dtype=np.int64)

    onsite = _onsite_h(spec, seed, n)
    if spec.hop_mode == HOP_CONST:
        hop = lambda owners, dirs: np.broadcast_to(spec.hop_t * np.eye(b), (owners.size, b, b)).copy()
    elif spec.hop_mode == HOP_NORMAL:
        hop = lambda owners, dirs: _pair_blocks(seed, STREAM_HOP, owners, dirs, n_pos, b, spec.hop_sigma)
    else:
        raise ValueError(spec.hop_mode)
    H = _assemble(spec, lists, n, n_pos, onsite, hop)

    S, s_seed = None, seed
    eye = np.broadcast_to(np.eye(b), (n, b, b))
    if spec.s_mode == S_CONST:
        S = _assemble(spec, lists, n, n_pos, eye,
                      lambda owners, dirs: np.broadcast_to(spec.s_param * np.eye(b), (owners.size, b, b)).copy())
    elif spec.s_mode == S_NORMAL:
        for attempt in range(64):
            s_seed = seed + attempt
            S = _assemble(spec, lists, n, n_pos, eye,
                          lambda owners, dirs: _pair_blocks(s_seed, STREAM_OVERLAP, owners, dirs, n_pos, b,
                                                            spec.s_param))
            if gershgorin_offdiag_max(S) < 1.0:
                break
        else:
            raise RuntimeError("no diagonally dominant overlap in 64 draws")
    elif spec.s_mode != S_IDENTITY:
        raise ValueError(spec.s_mode)
    return System(spec, seed, sites, nbr_ptr, nbr, H, S, s_seed)


def gershgorin_offdiag_max(S: Bsr) -> float:
    """max_i sum_{j != i} |S_ij| (the diagonal of S is exactly one by construction)."""
    b = S.bdim
    rows = np.repeat(np.arange(S.n_brows), np.diff(S.row_ptr))
    absval = np.abs(S.val)
    diag = S.col_idx.astype(np.int64) == rows
    absval[diag] = np.abs(S.val[diag] - np.eye(b)[None])
    row_sums = np.zeros((S.n_brows, b))
    np.add.at(row_sums, rows, absval.sum(axis=2))
    return float(row_sums.max()) if row_sums.size else 0.0


def block_pattern_rows(H: Bsr, row: int) -> np.ndarray:
    """All orbital rows of the atoms in the block pattern of the atom owning `row`."""
    b = H.bdim
    a = row // b
    cols = H.col_idx[H.row_ptr[a]:H.row_ptr[a + 1]].astype(np.int64)
    return (cols[:, None] * b + np.arange(b)[None, :]).ravel()
