"""Pins of the oracle's principal submatrices and descriptor entries 17-25 (CPU only).

principal_submatrix is checked against plain dense slicing A[O, O] of the
whole matrix on SC and FCC systems (with vacancies and a slab), for hop-shell
subspaces and for arbitrary atom subsets.  Descriptor entries 17-25 are
checked on a hand-built three-atom chain whose values are worked out below by
hand.  Each function is then re-run with one planted mistake (a dropped
block, a swapped renumbering, an off-by-one shell, a wrong normalisation):
every mutant must fail the same checks that the unmodified code passes.
"""
import inspect

import numpy as np
import pytest

from oracle import descriptors, subspace, systems
from workloads import C2_SYSTEM, C4_SYSTEM, SystemSpec, scaled


# ----------------------------------------------------------------- helpers
def _mutant(module, func, old, new):
    """`func` of `module` with one source substring replaced (must occur once)."""
    src = inspect.getsource(func)
    assert src.count(old) == 1, (func.__name__, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant {func.__name__}>", "exec"), ns)
    return ns[func.__name__]


def _principal_ok(sub_fn, system, atom_sets) -> bool:
    b = system.spec.bdim
    for A in (system.H, system.S):
        if A is None:
            continue
        dense = A.to_dense()
        for atoms in atom_sets:
            rows = subspace.subspace_rows(atoms, b)
            got = sub_fn(A, atoms)
            if got.n_brows != len(atoms) or got.bdim != b:
                return False
            if not np.array_equal(got.to_dense(), dense[np.ix_(rows, rows)]):
                return False
            # structure: ascending block columns with the diagonal present, as every BSR here
            for a in range(got.n_brows):
                c = got.col_idx[got.row_ptr[a]:got.row_ptr[a + 1]]
                if not (np.all(np.diff(c) > 0) and a in c):
                    return False
    return True


def _atom_sets(system, seed):
    rng = np.random.default_rng(seed)
    n = system.n_atoms
    sets = []
    for start, radius in ((0, 1), (n // 2, 2), (n - 1, 3)):
        sets.append(subspace.subspace_atoms(system.nbr_ptr, system.nbr, start, radius))
    sets.append(np.sort(rng.choice(n, size=min(n, 17), replace=False)))   # not a connected set
    sets.append(np.arange(n))                                              # the whole system
    return sets


SYSTEMS = {
    "sc_overlap": lambda: systems.build_system(scaled(C2_SYSTEM, L=4), 9),
    "fcc_vacancy_slab": lambda: systems.build_system(scaled(C4_SYSTEM, n_sites=400), 9),
}


# ----------------------------------------------------------- principal submatrix
@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_principal_submatrix_is_dense_slicing(name):
    s = SYSTEMS[name]()
    assert _principal_ok(subspace.principal_submatrix, s, _atom_sets(s, 1))


PRINCIPAL_MUTATIONS = {
    "drops_neighbour_blocks": ("if c in local:", "if c in local and c <= int(a):"),
    "renumbering_reversed": ("local = {int(a): i for i, a in enumerate(atoms)}",
                             "local = {int(a): len(atoms) - 1 - i for i, a in enumerate(atoms)}"),
    "block_transposed": ("vals.append(A.val[k])", "vals.append(A.val[k].T)"),
    "row_pointer_late": ("row_ptr.append(len(cols))", "row_ptr.append(max(len(cols) - 1, 0))"),
}


@pytest.mark.parametrize("mut", sorted(PRINCIPAL_MUTATIONS))
def test_principal_submatrix_pins_catch_planted_mistakes(mut):
    s = SYSTEMS["sc_overlap"]()
    f = _mutant(subspace, subspace.principal_submatrix, *PRINCIPAL_MUTATIONS[mut])
    try:
        ok = _principal_ok(f, s, _atom_sets(s, 1))
    except Exception:
        ok = False
    assert not ok, mut


# ----------------------------------------------------------- descriptor 17-25
def _chain():
    """Three atoms 0 - 1 - 2 in a line, two orbitals each, with the blocks below.

    H onsite: atom 0 [[1, .5], [.5, 2]], atom 1 [[-1, 0], [0, 3]], atom 2
    [[.5, 0], [0, -2]]; hopping H(1,0) = X = [[1, 2], [0, 1]], H(1,2) = Y =
    [[0, 1], [1, 1]], and H(0,1) = X^T, H(2,1) = Y^T.  S = I + NN blocks
    S(1,0) = [[.1, 0], [0, .2]], S(1,2) = [[.05, .1], [0, 0]] (and transposes).
    """
    X = np.array([[1.0, 2.0], [0.0, 1.0]])
    Y = np.array([[0.0, 1.0], [1.0, 1.0]])
    P = np.array([[0.1, 0.0], [0.0, 0.2]])
    Q = np.array([[0.05, 0.1], [0.0, 0.0]])
    on = [np.array([[1.0, 0.5], [0.5, 2.0]]), np.array([[-1.0, 0.0], [0.0, 3.0]]),
          np.array([[0.5, 0.0], [0.0, -2.0]])]
    rp = np.array([0, 2, 5, 7], np.int64)
    ci = np.array([0, 1, 0, 1, 2, 1, 2], np.int32)
    H = systems.Bsr(3, 2, rp, ci, np.stack([on[0], X.T, X, on[1], Y, Y.T, on[2]]))
    I2 = np.eye(2)
    S = systems.Bsr(3, 2, rp.copy(), ci.copy(), np.stack([I2, P.T, P, I2, Q, Q.T, I2]))
    spec = SystemSpec("chain", bdim=2)
    coords = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], np.int64)
    nbr_ptr = np.array([0, 1, 3, 4], np.int64)
    nbr = np.array([1, 0, 2, 1], np.int64)
    return systems.System(spec, 0, coords, nbr_ptr, nbr, H, S, 0)


# (row j, radius) -> entries 17..25 worked out by hand from the blocks above
CHAIN_EXPECTED = {
    # j = atom 1, orbital 0; O = {0, 1, 2}; diag(H_OO) = 1, 2, -1, 3, .5, -2
    (2, 1): {17: 0.1 ** 2 + 0.05 ** 2 + 0.1 ** 2,             # S row j: .1 | (1), 0 | .05, .1
             18: 3.5 / 6, 19: np.sqrt(19.25 / 6 - (3.5 / 6) ** 2), 20: -2.0, 21: 3.0,
             22: 1.0 + 4.0 + 1.0,                             # H row j: 1, 2 | (-1), 0 | 0, 1
             23: (np.sqrt(6.0) + np.sqrt(3.0)) / 2,           # ||X||_F, ||Y||_F
             24: 6 / 1000, 25: 2 / 3},                        # atoms 0 and 2 at the largest distance
    # j = atom 0, orbital 1; O = {0, 1} (atom 2 is two hops away); diag = 1, 2, -1, 3
    (1, 1): {17: 0.2 ** 2,                                    # S row j: 0, (1) | 0, .2
             18: 1.25, 19: np.sqrt(15 / 4 - 1.25 ** 2), 20: -1.0, 21: 3.0,
             22: 0.5 ** 2 + 2.0 ** 2 + 1.0 ** 2,              # H row j: .5, (2) | X^T row 1 = 2, 1
             23: np.sqrt(6.0),
             24: 4 / 1000, 25: 1 / 2},
    # j = atom 2, orbital 1, radius 2: all three atoms, only atom 0 at distance 2
    (5, 2): {17: 0.1 ** 2,                                    # S(2,1) = Q^T row 1 = .1, 0
             18: 3.5 / 6, 19: np.sqrt(19.25 / 6 - (3.5 / 6) ** 2), 20: -2.0, 21: 3.0,
             22: 1.0 + 1.0,                                   # H row j: Y^T row 1 = 1, 1 | 0, (-2)
             23: np.sqrt(3.0),
             24: 6 / 1000, 25: 1 / 3},
}


def _descriptor_ok(fn) -> bool:
    s = _chain()
    for (j, radius), exp in CHAIN_EXPECTED.items():
        d = fn(s, j, radius)
        for q, v in exp.items():
            if not abs(d[q] - v) <= 1e-14 * max(1.0, abs(v)):
                return False
        if np.any(d[26:] != 0.0):
            return False
    return True


def test_descriptor_entries_17_to_25_on_hand_built_chain():
    assert _descriptor_ok(descriptors.descriptor)


DESCRIPTOR_MUTATIONS = {
    "overlap_row_keeps_diagonal": ("        row[jl] = 0.0\n        d[17]", "        d[17]"),
    "std_as_variance": ("diag.std()", "diag.var()"),
    "hamiltonian_row_keeps_diagonal": ("    row[jl] = 0.0\n    d[22]", "    d[22]"),
    "surface_shell_off_by_one": ("if v == dmax)", "if v == dmax - 1)"),
    "neighbour_norm_of_row_block": ("Hs[la * b:(la + 1) * b, lc * b:(lc + 1) * b]",
                                    "Hs[la * b:(la + 1) * b, la * b:(la + 1) * b]"),
    "rows_as_atoms": ("d[24] = Hs.shape[0] / 1000.0", "d[24] = len(atoms) / 1000.0"),
}


@pytest.mark.parametrize("mut", sorted(DESCRIPTOR_MUTATIONS))
def test_descriptor_pins_catch_planted_mistakes(mut):
    f = _mutant(descriptors, descriptors.descriptor, *DESCRIPTOR_MUTATIONS[mut])
    assert not _descriptor_ok(f), mut
