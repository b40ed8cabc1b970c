"""Python entry to the oracle's plain FP64 shifted COCG (oracle/cocg.c).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests/, the smoke
check and the benchmark's CPU-baseline leg may import anything under oracle/.

The C file is compiled on first use with gcc (-O3 -fopenmp, no host-specific
flags) into oracle/_build/.  The recurrences and their derivation are in the
header of cocg.c (generalized shifted COCG for Eq. 2, Sec. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_cocg.so")
_LOCK = threading.Lock()
_LIB = None

ST_CONVERGED, ST_MAX_ITER, ST_BREAKDOWN, ST_NONFINITE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile cocg.c (plain C, gcc) into oracle/_build/liboracle_cocg.so."""
    src = os.path.join(_HERE, "cocg.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", src,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_shifted_cocg.restype = ctypes.c_int
            lib.oracle_shifted_cocg.argtypes = [
                ctypes.c_int64, P, P, P, P, P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int64, P,
                P, P, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, P, P, P, P, P,
                P, P, P, ctypes.c_int]
            _LIB = lib
        return _LIB


@dataclass
class CocgResult:
    G: np.ndarray          # complex128 [out_total, nz]
    iters: np.ndarray      # int32 [ncols]
    resid: np.ndarray      # float64 [ncols, nz]  recurrence residual ||rt||/|pi|
    status: np.ndarray     # int32 [ncols]
    conv_it: np.ndarray    # int32 [ncols, nz]  iteration a shift converged at (-1: never)
    rt: np.ndarray | None  # complex128 [ncols, n]  final seed residual of the original equation
    pi: np.ndarray | None  # complex128 [ncols, nz] final pi^sigma
    inner_its: np.ndarray  # int32 [ncols] inner CG iterations (S != I)


def _ptr(a):
    return None if a is None else a.ctypes.data


def median_seed(z: np.ndarray) -> int:
    """Seed shift: the shift with the median real part (upper median, ties to the lower index)."""
    order = np.argsort(np.real(z), kind="stable")
    return int(order[len(z) // 2])


def shifted_cocg(csr_h, csr_s, z, cols, out_ptr, out_rows, tol, max_iter=100000, seed=None,
                 inner_tol=1e-14, inner_max=1000, keep_rt=False, nthreads=None) -> CocgResult:
    """Solve (z_m S - H) x = e_j for every column j and shift z_m; return x on the requested rows.

    csr_h, csr_s: (row_ptr int64, col int32, val float64) scalar CSR; csr_s None means S = I.
    """
    rp, ci, hv = (np.ascontiguousarray(csr_h[0], np.int64), np.ascontiguousarray(csr_h[1], np.int32),
                  np.ascontiguousarray(csr_h[2], np.float64))
    n = rp.size - 1
    if csr_s is not None:
        srp, sci, sv = (np.ascontiguousarray(csr_s[0], np.int64), np.ascontiguousarray(csr_s[1], np.int32),
                        np.ascontiguousarray(csr_s[2], np.float64))
    else:
        srp = sci = sv = None
    z = np.ascontiguousarray(z, np.complex128)
    nz = z.size
    cols = np.ascontiguousarray(cols, np.int64)
    out_ptr = np.ascontiguousarray(out_ptr, np.int64)
    out_rows = np.ascontiguousarray(out_rows, np.int64)
    ncols = cols.size
    if seed is None:
        seed = median_seed(z)
    G = np.zeros((int(out_ptr[-1]), nz), np.complex128)
    iters = np.zeros(ncols, np.int32)
    resid = np.zeros((ncols, nz), np.float64)
    status = np.zeros(ncols, np.int32)
    conv_it = np.zeros((ncols, nz), np.int32)
    rt = np.zeros((ncols, n), np.complex128) if keep_rt else None
    pi = np.zeros((ncols, nz), np.complex128) if keep_rt else None
    inner = np.zeros(ncols, np.int32)
    nthreads = nthreads or os.cpu_count() or 1
    rc = _lib().oracle_shifted_cocg(n, _ptr(rp), _ptr(ci), _ptr(hv), _ptr(srp), _ptr(sci), _ptr(sv),
                                    nz, _ptr(z), seed, ncols, _ptr(cols), _ptr(out_ptr),
                                    _ptr(out_rows), tol, max_iter, inner_tol, inner_max, _ptr(G),
                                    _ptr(iters), _ptr(resid), _ptr(status), _ptr(conv_it), _ptr(rt),
                                    _ptr(pi), _ptr(inner), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_shifted_cocg rejected its arguments ({rc})")
    return CocgResult(G, iters, resid, status, conv_it, rt, pi, inner)
