"""The oracle's pins catch plausible mistakes in its shifted COCG (CPU only).

Each case plants one mistake (a dropped term, a wrong sign, a wrong operand,
a conjugated form) in a copy of oracle/cocg.c, builds it in a temporary
directory and runs the comparison with the exact Green's function that
test_oracle_green.py uses.  The planted copy must disagree; the unmodified
source must agree.  Nothing here touches the GPU or the library.
"""
import importlib.util
import os
import subprocess

import numpy as np
import pytest

from oracle import dense, systems
from tests.helpers import out_layout, rel_err_per_shift
from workloads import C1_SYSTEM, C2_SYSTEM, midpoint_shifts, scaled

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

MUTATIONS = {
    "pi_sign": ("(1.0 + alpha * sig)", "(1.0 - alpha * sig)"),
    "beta_shift_square": ("ratio * ratio * beta_prev", "ratio * beta_prev"),
    "pi_three_term_alpha_prev": ("(alpha * beta_prev / alpha_prev)", "(alpha * beta_prev)"),
    "shift_residual_scale": ("r[rows[k]] / pi[m]", "r[rows[k]] * pi[m]"),
    "overlap_direction": ("Sp[i] = rt[i] + beta_prev * Sp[i]", "Sp[i] = r[i] + beta_prev * Sp[i]"),
    "operator_without_S": ("u[i] = zs * Sp[i] - q[i]", "u[i] = zs * p[i] - q[i]"),
    "residual_not_shifted": ("const double res = rnorm / cabs(pi[m]);", "const double res = rnorm;"),
    "beta_inverted": ("beta_prev = rho_next / rho;", "beta_prev = rho / rho_next;"),
    "conjugated_form": ("for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];",
                        "for (int64_t i = 0; i < n; ++i) s += conj(u[i]) * v[i];"),
}


def _load_variant(tmp_path, src_text, name):
    c_path = tmp_path / f"{name}.c"
    c_path.write_text(src_text)
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", str(c_path),
                           "-o", str(so), "-lm"])
    spec = importlib.util.spec_from_file_location(f"cocg_{name}", os.path.join(ORACLE_DIR, "cocg.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build = lambda force=False, _p=str(so): _p
    return mod


def _max_error(mod):
    """Worst relative error against dense LU over an S = I and an S != I case, and
    worst relative mismatch between the reported per-shift residual and the true
    residual of the returned solution at a loose tolerance."""
    worst = 0.0
    for spec in (scaled(C1_SYSTEM, L=4), scaled(C2_SYSTEM, L=3)):
        s = systems.build_system(spec, 11)
        H = s.H.to_dense()
        S = None if s.S is None else s.S.to_dense()
        z = midpoint_shifts(8, -8.0, 6.0, 0.1)
        cols = np.array([1, H.shape[0] - 2])
        rl = [np.arange(H.shape[0])] * 2
        ptr, rows = out_layout(rl)
        res = mod.shifted_cocg(s.H.to_csr(), None if s.S is None else s.S.to_csr(), z, cols, ptr,
                               rows, tol=1e-12, max_iter=3000)
        ex = dense.green_lu(H, S, z, cols)
        for c in range(2):
            err = rel_err_per_shift(res.G[ptr[c]:ptr[c + 1]], ex[:, c, :]).max()
            worst = max(worst, err if np.isfinite(err) else np.inf)
        loose = mod.shifted_cocg(s.H.to_csr(), None if s.S is None else s.S.to_csr(), z, cols, ptr,
                                 rows, tol=1e-6, max_iter=3000)
        Smat = np.eye(H.shape[0]) if S is None else S
        for c, j in enumerate(cols):
            b = np.zeros(H.shape[0])
            b[j] = 1.0
            for m, zm in enumerate(z):
                true_r = np.linalg.norm(b - (zm * Smat - H) @ loose.G[ptr[c]:ptr[c + 1], m])
                mis = abs(loose.resid[c, m] - true_r) / max(true_r, 1e-14)
                worst = max(worst, mis * 1e-3 if np.isfinite(mis) else np.inf)
    return worst


def test_unmodified_source_agrees(tmp_path):
    src = open(os.path.join(ORACLE_DIR, "cocg.c")).read()
    assert _max_error(_load_variant(tmp_path, src, "orig")) < 1e-9


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(os.path.join(ORACLE_DIR, "cocg.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mod = _load_variant(tmp_path, src.replace(old, new), name)
    assert not (_max_error(mod) < 1e-6)
