"""Seeded synthetic workloads for the shifted Green's-function solve.

This module holds only input *definitions*: the tight-binding system
specifications, the complex shift grids, the choice of right-hand-side
orbitals and of local-subspace radii.  It contains none of the method's
arithmetic (no lattice construction, no matrix values, no solver), so both
the CPU oracle and the GPU library can take their inputs from here without
sharing any code of the method itself.

The five workloads follow the generalized shifted equation (zS - H) x = e_j
of Eq. 2 (Sec. 3) on synthetic tight-binding models whose matrices have the
structural properties stated in Sec. 8: real symmetric H and S, S positive
definite with unit diagonal and off-diagonal magnitudes below one.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Tuple

import numpy as np

# Lattice kinds
SC_PERIODIC = "sc_periodic"     # L^3 simple cubic, periodic, 6 nearest neighbours
FCC_CLUSTER = "fcc_cluster"     # n sites of FCC closest to the origin, open, <=12 NN

# Onsite-block kinds
ONSITE_UNIFORM = "uniform"          # u * I_b,  u ~ U[lo, hi]  (one draw per atom)
ONSITE_DIAG_NORMAL = "diag_normal"  # diag(d) + (N + N^T)/2,  N_kl ~ N(0, sigma)

# Hopping-block kinds
HOP_CONST = "const"    # t * I_b on every nearest-neighbour pair
HOP_NORMAL = "normal"  # X_kl ~ N(0, sigma), X_ji = X_ij^T

# Overlap kinds
S_IDENTITY = "identity"  # S = I
S_NORMAL = "normal"      # S = I + symmetric NN blocks N(0, s)
S_CONST = "const"        # S = I + s * I_b on every NN pair

DEFAULT_SEED = 1234


@dataclass(frozen=True)
class SystemSpec:
    """A synthetic tight-binding system: lattice, block size and value model."""

    lattice: str
    L: int = 0                 # SC edge length (atoms per edge)
    n_sites: int = 0           # FCC: number of lattice sites kept before removals
    bdim: int = 1              # orbitals per atom (block edge)
    onsite_mode: str = ONSITE_UNIFORM
    onsite_lo: float = 0.0
    onsite_hi: float = 0.0
    onsite_diag: Tuple[float, ...] = ()
    onsite_sigma: float = 0.0
    hop_mode: str = HOP_CONST
    hop_t: float = 0.0
    hop_sigma: float = 0.0
    s_mode: str = S_IDENTITY
    s_param: float = 0.0
    vacancy_frac: float = 0.0
    slab: bool = False
    subst_frac: float = 0.0
    subst_shift: float = 0.0

    @property
    def has_overlap(self) -> bool:
        return self.s_mode != S_IDENTITY


@dataclass(frozen=True)
class Workload:
    """One benchmark configuration: system, shifts and right-hand sides."""

    name: str
    system: SystemSpec
    n_shifts: int
    e_lo: float
    e_hi: float
    eta: float
    n_rhs: int
    rhs_rule: str              # "sample" | "subblock_orbital0" | "sample_local"
    tol: float
    seed: int = DEFAULT_SEED
    subblock: int = 0          # edge of the SC sub-block whose atoms give RHS
    radii: Tuple[int, ...] = ()  # local-subspace hop radii to draw from
    extra: dict = field(default_factory=dict)


def midpoint_shifts(n_z: int, e_lo: float, e_hi: float, eta: float) -> np.ndarray:
    """Complex energies z_m = E_m + i*eta on the midpoint grid of [e_lo, e_hi]."""
    m = np.arange(n_z, dtype=np.float64)
    e = e_lo + (m + 0.5) * (e_hi - e_lo) / n_z
    return e + 1j * eta


def random_shifts(n_z: int, e_lo: float, e_hi: float, eta: float, seed: int) -> np.ndarray:
    """Seeded random energies on [e_lo, e_hi] (robustness tests)."""
    rng = np.random.default_rng(seed)
    e = np.sort(rng.uniform(e_lo, e_hi, size=n_z))
    return e + 1j * eta


def n_atoms_nominal(spec: SystemSpec) -> int:
    if spec.lattice == SC_PERIODIC:
        return spec.L ** 3
    return spec.n_sites


def sample_rhs(n_rows: int, n_rhs: int, seed: int) -> np.ndarray:
    """n_rhs distinct orbital indices in [0, n_rows), sorted ascending."""
    rng = np.random.default_rng(seed + 7)
    cols = rng.choice(n_rows, size=min(n_rhs, n_rows), replace=False)
    return np.sort(cols).astype(np.int64)


def subblock_orbital0_rhs(L: int, sub: int, bdim: int) -> np.ndarray:
    """Orbital 0 of every atom of the SC sub-block [0, sub)^3 (atom a = x + L(y + L z))."""
    x, y, z = np.meshgrid(np.arange(sub), np.arange(sub), np.arange(sub), indexing="ij")
    a = (x + L * (y + L * z)).ravel()
    return np.sort(a * bdim).astype(np.int64)


def sample_local_rhs(n_atoms: int, bdim: int, n_rhs: int, radii: Tuple[int, ...], seed: int):
    """Seeded localized right-hand sides: (row index, subspace hop radius) per column.

    Atoms are drawn without replacement, the orbital uniformly in [0, bdim),
    and the radius uniformly from `radii`.
    """
    rng = np.random.default_rng(seed + 11)
    atoms = rng.choice(n_atoms, size=min(n_rhs, n_atoms), replace=False)
    orb = rng.integers(0, bdim, size=atoms.size)
    rad = rng.choice(np.asarray(radii, dtype=np.int64), size=atoms.size)
    rows = atoms.astype(np.int64) * bdim + orb
    order = np.argsort(rows, kind="stable")
    return rows[order], rad[order].astype(np.int32)


# ---------------------------------------------------------------------------
# The five configurations (sizes, distributions and tolerances as specified
# for the benchmark suite of this project).
# ---------------------------------------------------------------------------

C1_SYSTEM = SystemSpec(SC_PERIODIC, L=16, bdim=1, onsite_mode=ONSITE_UNIFORM,
                       onsite_lo=-1.0, onsite_hi=1.0, hop_mode=HOP_CONST, hop_t=-1.0)

C2_SYSTEM = SystemSpec(SC_PERIODIC, L=32, bdim=4, onsite_mode=ONSITE_DIAG_NORMAL,
                       onsite_diag=(-5.0, 1.0, 1.0, 1.0), onsite_sigma=0.1,
                       hop_mode=HOP_NORMAL, hop_sigma=0.5, s_mode=S_NORMAL, s_param=0.02)

C3_SYSTEM = SystemSpec(FCC_CLUSTER, n_sites=100_000, bdim=9, onsite_mode=ONSITE_UNIFORM,
                       onsite_lo=-0.5, onsite_hi=0.5, hop_mode=HOP_NORMAL, hop_sigma=0.3)

C4_SYSTEM = SystemSpec(FCC_CLUSTER, n_sites=1_000_000, bdim=4, onsite_mode=ONSITE_UNIFORM,
                       onsite_lo=-0.5, onsite_hi=0.5, hop_mode=HOP_NORMAL, hop_sigma=0.3,
                       s_mode=S_CONST, s_param=0.02, vacancy_frac=0.3, slab=True)

C5_SYSTEM = SystemSpec(SC_PERIODIC, L=216, bdim=4, onsite_mode=ONSITE_DIAG_NORMAL,
                       onsite_diag=(-5.0, 1.0, 1.0, 1.0), onsite_sigma=0.0,
                       hop_mode=HOP_NORMAL, hop_sigma=0.5, s_mode=S_CONST, s_param=0.02,
                       subst_frac=0.1, subst_shift=1.5)

C1 = Workload("anderson_sc16_b1", C1_SYSTEM, n_shifts=32, e_lo=-7.0, e_hi=7.0, eta=0.01,
              n_rhs=256, rhs_rule="sample", tol=1e-10)
C2 = Workload("sp3_sc32_b4_overlap", C2_SYSTEM, n_shifts=64, e_lo=-10.0, e_hi=6.0, eta=0.005,
              n_rhs=4096, rhs_rule="subblock_orbital0", tol=1e-5, subblock=16)
C3 = Workload("fcc100k_b9_local", C3_SYSTEM, n_shifts=128, e_lo=-8.0, e_hi=8.0, eta=0.002,
              n_rhs=20_000, rhs_rule="sample_local", tol=1e-5, radii=(2, 3, 4, 5))
C4 = Workload("fcc1m_b4_vacancy_slab", C4_SYSTEM, n_shifts=64, e_lo=-8.0, e_hi=8.0, eta=0.002,
              n_rhs=100_000, rhs_rule="sample_local", tol=1e-5, radii=(2, 3, 4, 5))
C5 = Workload("sc216_b4_subst", C5_SYSTEM, n_shifts=64, e_lo=-10.0, e_hi=6.0, eta=0.01,
              n_rhs=1_000_000, rhs_rule="sample_local", tol=1e-5, radii=(2, 3, 4, 5))

ALL = {w.name: w for w in (C1, C2, C3, C4, C5)}


def shifts_of(w: Workload) -> np.ndarray:
    return midpoint_shifts(w.n_shifts, w.e_lo, w.e_hi, w.eta)


def rhs_of(w: Workload, n_atoms: int | None = None):
    """Right-hand-side rows (and radii for local rules) of a workload."""
    spec = w.system
    if w.rhs_rule == "sample":
        n_rows = (n_atoms or n_atoms_nominal(spec)) * spec.bdim
        return sample_rhs(n_rows, w.n_rhs, w.seed)
    if w.rhs_rule == "subblock_orbital0":
        return subblock_orbital0_rhs(spec.L, w.subblock, spec.bdim)
    if w.rhs_rule == "sample_local":
        return sample_local_rhs(n_atoms or n_atoms_nominal(spec), spec.bdim, w.n_rhs,
                                w.radii, w.seed)
    raise ValueError(w.rhs_rule)


def scaled(spec: SystemSpec, **kw) -> SystemSpec:
    """A copy of `spec` with some fields changed (used for small test systems)."""
    return replace(spec, **kw)
