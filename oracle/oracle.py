"""ctypes front end of the C oracle in ``lc_oracle.c`` (test infrastructure).

The oracle computes the plain definitions of the paper's maps with a direct
O(n^2) sum in double-double arithmetic (Sec. 1, eq:directmv and eq:aij for
Legendre->Chebyshev; eq:Lxymod for Chebyshev->Legendre); see the header of
``lc_oracle.c``.  Nothing on the product path imports this module.

parity pins: see tests/test_oracle_pins.py (brute force at Chebyshev-Gauss
nodes in 50-digit arithmetic, mpmath inverse of A, textbook Legendre
expansions, structure of A, round trip, adjoint dot test).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig
from pathlib import Path

import numpy as np

L2C = 0
C2L = 1

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "lc_oracle.c"
_LIB_PATH = _HERE / "_build" / "liblc_oracle.so"
_lib = None


def build_oracle(force: bool = False) -> Path:
    """Compile lc_oracle.c with gcc (OpenMP when available) into _build/."""
    _LIB_PATH.parent.mkdir(parents=True, exist_ok=True)
    if (not force and _LIB_PATH.exists()
            and _LIB_PATH.stat().st_mtime >= _SRC.stat().st_mtime):
        return _LIB_PATH
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-fPIC", "-shared", "-std=c11", str(_SRC), "-lm"]
    tmp = _LIB_PATH.with_suffix(".so.tmp%d" % os.getpid())
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", str(tmp)],
                       check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", str(tmp)], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build_oracle()))
        i64, dp, ip = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
        lib.lco_lambda.argtypes = [i64, dp, dp]
        lib.lco_entry.argtypes = [ctypes.c_int, i64, i64, i64, dp]
        lib.lco_apply.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, i64, ip, dp]
        lib.lco_threads.argtypes = []
        lib.lco_dct.argtypes = [ctypes.c_int, i64, dp, dp]
        lib.lco_dct_rows.argtypes = [ctypes.c_int, i64, dp, i64, ip, dp]
        lib.lco_dct_rows.restype = ctypes.c_int
        lib.lco_apply_geg.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, i64, dp, i64, ip, dp]
        lib.lco_entry_geg.argtypes = [ctypes.c_int, ctypes.c_double, i64, i64, i64, dp]
        lib.lco_geg_tables.argtypes = [ctypes.c_int, ctypes.c_double, i64, dp, dp]
        for f in (lib.lco_lambda, lib.lco_entry, lib.lco_apply, lib.lco_threads, lib.lco_dct,
                  lib.lco_apply_geg, lib.lco_entry_geg, lib.lco_geg_tables):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads() -> int:
    """OpenMP threads the oracle uses for its row loop."""
    return int(_load().lco_threads())


def lambda_table(n: int):
    """Lambda(k) = Gamma(k+1/2)/Gamma(k+1) for k < n (eq:Lambda, eq:Lambdaint).

    Returns (hi, lo): hi is the double nearest the double-double value, lo its tail.
    """
    hi = np.empty(n, np.float64)
    lo = np.empty(n, np.float64)
    rc = _load().lco_lambda(n, _dptr(hi), _dptr(lo))
    if rc:
        raise RuntimeError("lco_lambda failed (%d)" % rc)
    return hi, lo


def entry(direction: int, n: int, i: int, j: int) -> float:
    """Entry (i, j) of C^{-1}A (L2C) or A^{-1}C (C2L) for size n."""
    out = ctypes.c_double()
    rc = _load().lco_entry(direction, n, i, j, ctypes.byref(out))
    if rc:
        raise ValueError("lco_entry failed (%d)" % rc)
    return out.value


def apply(direction: int, x, rows=None, adjoint: bool = False, alpha=None):
    """Apply the L2C (direction 0) or C2L (direction 1) map, or its transpose.

    x: 1-D float64 array of length n.  rows: optional int64 output indices;
    when given only those outputs are computed (in that order).
    alpha: None for the Legendre maps; otherwise the Gegenbauer parameter a
    (-1/2 < a, a != 0) of the maps between C_j^(a) and Chebyshev (Conclusions;
    the definitions are in the header of lc_oracle.c).
    """
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim != 1 or x.size == 0:
        raise ValueError("x must be a non-empty 1-D array")
    n = x.size
    lib = _load()
    if alpha is None:
        call = lambda nr, rp, op: lib.lco_apply(direction, int(adjoint), n, _dptr(x), nr, rp, op)
    else:
        a = float(alpha)
        call = lambda nr, rp, op: lib.lco_apply_geg(direction, int(adjoint), a, n, _dptr(x), nr, rp, op)
    if rows is None:
        out = np.empty(n, np.float64)
        rc = call(0, None, _dptr(out))
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(rows.size, np.float64)
        rc = call(rows.size, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(out))
    if rc:
        raise RuntimeError("oracle apply failed (%d)" % rc)
    return out


def geg_tables(direction: int, alpha: float, n: int):
    """The sequences behind the Gegenbauer entries, indices < n: direction 0
    returns g_k = (a)_k/k!; direction 1 returns (u, w) with u_l = (-a)_l/l!,
    w_m = (m-1)!/(a+2)_{m-1}, w_0 = 0 (header of lc_oracle.c)."""
    t0 = np.empty(n, np.float64)
    t1 = np.empty(n, np.float64)
    rc = _load().lco_geg_tables(direction, float(alpha), n, _dptr(t0), _dptr(t1))
    if rc:
        raise ValueError("lco_geg_tables failed (%d)" % rc)
    return t0 if direction == 0 else (t0, t1)


def entry_geg(direction: int, alpha: float, n: int, i: int, j: int) -> float:
    """Entry (i, j) of the Gegenbauer map for parameter alpha and size n."""
    out = ctypes.c_double()
    rc = _load().lco_entry_geg(direction, float(alpha), n, i, j, ctypes.byref(out))
    if rc:
        raise ValueError("lco_entry_geg failed (%d)" % rc)
    return out.value


def dense_matrix(direction: int, n: int, alpha=None):
    """The full n x n matrix of the map, column by column (small n only)."""
    m = np.zeros((n, n), np.float64)
    e = np.zeros(n, np.float64)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        m[:, j] = apply(direction, e, alpha=alpha)
    return m


def dct(kind: int, x, rows=None):
    """kind 0: v_m = sum_k x_k cos(pi k (2m+1)/(2n)) -- the Chebyshev series with
    coefficients x at the Chebyshev-Gauss points x_m = cos((m+1/2) pi/n);
    kind 1: its inverse, (2/n)/(1+[k=0]) sum_m x_m cos(pi k (2m+1)/(2n)).
    rows: optional output indices (then only those outputs, in that order)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if rows is None:
        out = np.empty_like(x)
        rc = _load().lco_dct(int(kind), x.size, _dptr(x), _dptr(out))
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(rows.size, np.float64)
        rc = _load().lco_dct_rows(int(kind), x.size, _dptr(x), rows.size,
                                  rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(out))
    if rc:
        raise RuntimeError("lco_dct failed (%d)" % rc)
    return out


def synthesis(f, alpha=None):
    """Values p(x_m) of p = sum_j f_j P_j at the n Chebyshev-Gauss points
    x_m = cos((m+1/2) pi/n): the L2C map, then the Chebyshev series at the
    points (Sec. 1: Legendre coefficients to values through the Chebyshev basis).
    With alpha, p = sum_j f_j C_j^(alpha)."""
    return dct(0, apply(L2C, f, alpha=alpha))


def analysis(v, alpha=None):
    """Legendre (or, with alpha, Gegenbauer) coefficients of the degree < n
    polynomial through the values v at the n Chebyshev-Gauss points: discrete
    Chebyshev transform, then C2L."""
    return apply(C2L, dct(1, v), alpha=alpha)
