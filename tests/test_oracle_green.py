"""Pins of the oracle's Green's functions and of its shifted COCG (CPU only).

G_ij(z) = e_i^T (z S - H)^{-1} e_j is the solution of Eq. 2 (Sec. 3) with
b = e_j.  It is pinned by:
  * closed-form lattice Green's functions (finite Fourier sums; infinite chain);
  * two library routes that must agree (dense LU, generalized eigenpairs);
  * identities of the exact resolvent: complex symmetry G = G^T, G(conj z) =
    conj G(z), the resolvent identity G(z) - G(z') = (z' - z) G(z) S G(z');
  * for the shifted COCG: agreement with the exact G, the true residual at
    exit, the collinearity of the shifted residuals at an arbitrary
    iteration, and the reduction to plain CG for one real shift outside the
    spectrum.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import cocg, dense, gf, systems
from tests.helpers import out_layout, rel_err_per_shift
from workloads import (C1_SYSTEM, C2_SYSTEM, C3_SYSTEM, C4_SYSTEM, ONSITE_UNIFORM, midpoint_shifts,
                       scaled)


def _dense(s):
    return s.H.to_dense(), (None if s.S is None else s.S.to_dense())


def _csr(s):
    return s.H.to_csr(), (None if s.S is None else s.S.to_csr())


def test_chain_closed_form_and_infinite_limit():
    L, eps0, t = 40, 0.3, -1.0
    H = np.zeros((L, L))
    for i in range(L):
        H[i, i] = eps0
        H[i, (i + 1) % L] = H[(i + 1) % L, i] = t
    z = np.array([0.7 + 0.2j, -1.9 + 0.05j, 2.5 + 0.5j])
    G = dense.green_lu(H, None, z, [0, 3])
    for m, zm in enumerate(z):
        for c, j in enumerate([0, 3]):
            for i in (0, 1, 5, 17):
                assert abs(G[i, c, m] - dense.chain_green(L, eps0, t, zm, i, j)) < 1e-12
    # the finite periodic chain approaches the infinite chain as L grows
    zm = 0.4 + 0.3j
    g_inf = dense.infinite_chain_g00(eps0, t, zm)
    assert abs(dense.chain_green(4000, eps0, t, zm, 0, 0) - g_inf) < 1e-10
    assert g_inf.imag < 0


def test_sc_clean_closed_form_vs_lu_and_cocg(oracle_lib):
    L = 4
    spec = scaled(C1_SYSTEM, L=L, onsite_lo=0.25, onsite_hi=0.25)   # clean: eps0 = 0.25
    s = systems.build_system(spec, 1)
    H, _ = _dense(s)
    z = midpoint_shifts(6, -6.5, 6.5, 0.1)
    cols = np.array([0, 21])
    Glu = dense.green_lu(H, None, z, cols)
    sites = systems.sc_sites(L)
    for c, j in enumerate(cols):
        for i in (0, 1, 5, 21, 63):
            for m, zm in enumerate(z):
                ref = dense.sc_green(L, 0.25, -1.0, zm, sites[i], sites[j])
                assert abs(Glu[i, c, m] - ref) < 1e-12
    ptr, rows = out_layout([np.arange(L ** 3)] * 2)
    res = cocg.shifted_cocg(s.H.to_csr(), None, z, cols, ptr, rows, tol=1e-13)
    assert np.all(res.status == cocg.ST_CONVERGED)
    G = res.G.reshape(2, L ** 3, len(z)).transpose(1, 0, 2)
    assert np.abs(G - Glu).max() < 1e-10


@pytest.mark.parametrize("spec", [scaled(C1_SYSTEM, L=5), scaled(C2_SYSTEM, L=3),
                                  scaled(C3_SYSTEM, n_sites=120, bdim=4),
                                  scaled(C4_SYSTEM, n_sites=300)],
                         ids=["c1", "c2_overlap", "fcc_b4", "fcc_const_overlap"])
def test_lu_vs_eigen_routes(spec):
    s = systems.build_system(spec, 1234)
    H, S = _dense(s)
    z = midpoint_shifts(5, -9.0, 7.0, 0.05)
    cols = np.array([0, 7, H.shape[0] - 1])
    a = dense.green_lu(H, S, z, cols)
    b = dense.green_eig(H, S, z, cols)
    assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()


@pytest.mark.parametrize("spec,eta,tol,bound", [
    (scaled(C1_SYSTEM, L=6), 0.05, 1e-12, 1e-10),
    (scaled(C2_SYSTEM, L=4), 0.05, 1e-12, 1e-10),
    (scaled(C3_SYSTEM, n_sites=150, bdim=9), 0.05, 1e-12, 1e-10),
    (scaled(C4_SYSTEM, n_sites=400), 0.02, 1e-12, 1e-10),
    (scaled(C2_SYSTEM, L=4), 0.02, 1e-5, 2e-4),
], ids=["c1_sI", "c2_overlap", "fcc_b9", "fcc_overlap", "c2_loose"])
def test_cocg_matches_exact(oracle_lib, spec, eta, tol, bound):
    s = systems.build_system(spec, 1234)
    H, S = _dense(s)
    hc, sc = _csr(s)
    z = midpoint_shifts(12, -9.0, 7.0, eta)
    M = H.shape[0]
    cols = np.array([0, M // 2 + 1, M - 1])
    Gex = dense.green_lu(H, S, z, cols)
    # keep the block-pattern rows of each column (what the LDOS/DM need)
    rl = [systems.block_pattern_rows(s.H, j) for j in cols]
    ptr, rows = out_layout(rl)
    res = cocg.shifted_cocg(hc, sc, z, cols, ptr, rows, tol=tol)
    assert np.all(res.status == cocg.ST_CONVERGED)
    for c, j in enumerate(cols):
        Gc = res.G[ptr[c]:ptr[c + 1]]
        assert rel_err_per_shift(Gc, Gex[rl[c], c, :]).max() < bound
        assert np.all(res.resid[c] <= tol)


def test_true_residual_at_exit_and_symmetry(oracle_lib):
    s = systems.build_system(scaled(C2_SYSTEM, L=3), 99)
    H, S = _dense(s)
    hc, sc = _csr(s)
    M = H.shape[0]
    z = midpoint_shifts(8, -9.0, 7.0, 0.03)
    cols = np.array([2, 9, 40])
    ptr, rows = out_layout([np.arange(M)] * 3)
    tol = 1e-9
    res = cocg.shifted_cocg(hc, sc, z, cols, ptr, rows, tol=tol)
    X = res.G.reshape(3, M, len(z))
    for c, j in enumerate(cols):
        b = np.zeros(M)
        b[j] = 1
        for m, zm in enumerate(z):
            r = np.linalg.norm(b - (zm * S - H) @ X[c, :, m])
            assert r <= 10 * tol
            # the reported per-shift residual is the true residual of the returned x
            assert abs(res.resid[c, m] - r) <= 1e-3 * r + 1e-13
    # complex symmetry: G_ij = G_ji across the three columns
    for a in range(3):
        for b_ in range(3):
            assert np.abs(X[a, cols[b_], :] - X[b_, cols[a], :]).max() < 1e-8


def test_conjugate_shift_and_resolvent_identity(oracle_lib):
    s = systems.build_system(scaled(C2_SYSTEM, L=3), 5)
    H, S = _dense(s)
    hc, sc = _csr(s)
    M = H.shape[0]
    z1, z2 = -1.3 + 0.2j, 0.8 + 0.35j
    z = np.array([z1, np.conj(z1), z2])
    cols = np.arange(M)
    ptr, rows = out_layout([np.arange(M)] * M)
    res = cocg.shifted_cocg(hc, sc, z, cols, ptr, rows, tol=1e-13)
    Gall = res.G.reshape(M, M, 3).transpose(1, 0, 2)     # [i, j, m]
    assert np.abs(Gall[:, :, 1] - np.conj(Gall[:, :, 0])).max() < 1e-10
    lhs = Gall[:, :, 0] - Gall[:, :, 2]
    rhs = (z2 - z1) * Gall[:, :, 0] @ S @ Gall[:, :, 2]
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(lhs).max()


@pytest.mark.parametrize("overlap", [False, True])
def test_collinear_shifted_residuals(oracle_lib, overlap):
    spec = scaled(C2_SYSTEM, L=3) if overlap else scaled(C1_SYSTEM, L=5)
    s = systems.build_system(spec, 3)
    H, S = _dense(s)
    hc, sc = _csr(s)
    M = H.shape[0]
    Smat = np.eye(M) if S is None else S
    z = midpoint_shifts(10, -8.0, 6.0, 0.1)
    j = 4
    for stop in (3, 17, 40):
        ptr, rows = out_layout([np.arange(M)])
        res = cocg.shifted_cocg(hc, sc, z, [j], ptr, rows, tol=1e-14, max_iter=stop, keep_rt=True)
        assert res.iters[0] == stop
        X = res.G.reshape(M, len(z))
        b = np.zeros(M)
        b[j] = 1
        for m, zm in enumerate(z):
            if res.conv_it[0, m] >= 0:
                continue
            true_r = b - (zm * Smat - H) @ X[:, m]
            pred = res.rt[0] / res.pi[0, m]
            assert np.linalg.norm(true_r - pred) <= 1e-10 * max(1.0, np.linalg.norm(pred))


def test_single_real_shift_reduces_to_cg(oracle_lib):
    s = systems.build_system(scaled(C2_SYSTEM, L=4), 8)
    H, S = _dense(s)
    hc, sc = _csr(s)
    lam = dense.eigenpairs(H, S)[0]
    z = np.array([lam[0] - 1.0 + 0j])          # below the spectrum: z S - H negative definite
    cols = np.array([3, 50])
    M = H.shape[0]
    ptr, rows = out_layout([np.arange(M)] * 2)
    res = cocg.shifted_cocg(hc, sc, z, cols, ptr, rows, tol=1e-13)
    A = sp.csr_matrix(z[0].real * S - H)
    for c, j in enumerate(cols):
        b = np.zeros(M)
        b[j] = 1
        ref = spla.spsolve(A, b)
        x = res.G[ptr[c]:ptr[c + 1], 0]
        assert np.abs(x.imag).max() < 1e-12
        assert np.abs(x.real - ref).max() < 1e-10 * np.abs(ref).max()


def test_seed_choice_does_not_change_result(oracle_lib):
    s = systems.build_system(scaled(C1_SYSTEM, L=5), 21)
    hc, _ = _csr(s)
    z = midpoint_shifts(9, -7.0, 7.0, 0.08)
    ptr, rows = out_layout([systems.block_pattern_rows(s.H, 10)])
    a = cocg.shifted_cocg(hc, None, z, [10], ptr, rows, tol=1e-13, seed=0)
    b = cocg.shifted_cocg(hc, None, z, [10], ptr, rows, tol=1e-13, seed=8)
    assert np.abs(a.G - b.G).max() < 1e-10 * np.abs(a.G).max()


def test_ldos_total_dos_and_dm_identities():
    """Mulliken LDOS summed over all orbitals is the Lorentzian eigenvalue histogram
    (the DOS of Sec. 8); the DM equals its eigen-sum; each LDOS integrates to one."""
    s = systems.build_system(scaled(C2_SYSTEM, L=3), 4)
    H, S = _dense(s)
    M = H.shape[0]
    lam, Y = dense.eigenpairs(H, S)
    eta = 0.05
    E = np.linspace(-9.0, 7.0, 7)
    z = E + 1j * eta
    cols = np.arange(M)
    G = dense.green_lu(H, S, z, cols)                  # [i, j, m]
    total = np.zeros(len(z))
    for j in range(M):
        total += gf.ldos(G[:, j, :], S[:, j], None)
    lorentz = (eta / np.pi) / ((E[:, None] - lam[None, :]) ** 2 + eta ** 2)
    assert np.abs(total - lorentz.sum(axis=1)).max() < 1e-9 * total.max()
    # S = I: the LDOS is -Im G_jj / pi
    s0 = systems.build_system(scaled(C1_SYSTEM, L=3), 4)
    H0 = s0.H.to_dense()
    G0 = dense.green_lu(H0, None, z, [5])
    d = gf.ldos(G0[:, 0, :], None, 5)
    lam0, Y0 = dense.eigenpairs(H0, None)
    ref = (Y0[5, :] ** 2 * (eta / np.pi) / ((E[:, None] - lam0[None, :]) ** 2 + eta ** 2)).sum(axis=1)
    assert np.abs(d - ref).max() < 1e-10
    # DM at kT = 0: rho_ij = sum_k Y_ik Y_jk sum_m w_m f(E_m) L_eta(E_m - lambda_k)
    w = np.full(len(E), E[1] - E[0])
    mu = -1.0
    rho = gf.density_matrix(G[:, 3, :], E, w, mu, 0.0)
    weights = (w * gf.fermi(E, mu, 0.0))[:, None] * lorentz          # [m, k]
    ref = Y @ (Y[3, :] * weights.sum(axis=0))
    assert np.abs(rho - ref).max() < 1e-10
    # one LDOS integrates to one over the real line (fine grid, wide window)
    Ef = np.linspace(-400.0, 400.0, 400001)
    lf = (eta / np.pi) / ((Ef[:, None] - lam[None, :]) ** 2 + eta ** 2)
    j = 7
    weight_k = Y[j, :] * (S @ Y)[j, :]
    integral = np.trapezoid(lf @ weight_k, Ef)
    assert abs(integral - 1.0) < 2e-4
    assert abs(weight_k.sum() - 1.0) < 1e-12


def test_fermi_function():
    assert np.array_equal(gf.fermi(np.array([-1.0, 0.0, 1.0]), 0.0, 0.0), [1.0, 0.5, 0.0])
    x = np.array([-50.0, -1.0, 0.0, 2.0, 800.0])
    f = gf.fermi(x, 0.0, 0.5)
    assert np.allclose(f, 1.0 / (1.0 + np.exp(np.clip(x / 0.5, -700, 700))))
    assert np.allclose(f + gf.fermi(-x, 0.0, 0.5), 1.0)
