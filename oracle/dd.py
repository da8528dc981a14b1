"""ORACLE (test infrastructure only): ctypes binding of ``dd.c``, the
double-double evaluator.  ``build()`` compiles it with gcc (OpenMP,
-ffp-contract=off) into ``oracle/_build/libeigref_dd.so``."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd.c")
_LIB = os.path.join(_HERE, "_build", "libeigref_dd.so")
_lib = None


def build(force=False):
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c99", _SRC, "-o", _LIB, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


_d = ctypes.c_double
_p = ctypes.c_void_p
_i64 = ctypes.c_int64


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _fcols(X):
    X = np.asarray(X, dtype=np.float64)
    if not X.flags.f_contiguous:
        X = np.asfortranarray(X)
    return X, X.shape[0]


def two_prod(a, b):
    hi, lo = _d(), _d()
    lib().dd_two_prod(_d(a), _d(b), ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def two_sum(a, b):
    hi, lo = _d(), _d()
    lib().dd_two_sum(_d(a), _d(b), ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def dot(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    hi, lo = _d(), _d()
    lib().dd_dot(_ptr(x), _ptr(y), _i64(len(x)), ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def residual_dense(A, X, shift=0.0):
    """(rq, res): Rayleigh quotients of A - shift I and ||B x - rq x|| / ||x||
    per column, in double-double."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    X, ldx = _fcols(X)
    n, k = X.shape
    rq, res = np.empty(k), np.empty(k)
    work = np.empty(2 * n * k)
    lib().dd_residual_dense(_ptr(A), _i64(n), _i64(A.shape[1]), _ptr(X), _i64(ldx), ctypes.c_int(k),
                            _d(shift), _ptr(rq), _ptr(res), _ptr(work), ctypes.c_int(0))
    return rq, res


def residual_csr(row_ptr, col_idx, val, X, shift=0.0):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    X, ldx = _fcols(X)
    n, k = X.shape
    rq, res = np.empty(k), np.empty(k)
    work = np.empty(2 * n * k)
    lib().dd_residual_csr(_ptr(rp), _ptr(ci), _ptr(v), _i64(n), _ptr(X), _i64(ldx), ctypes.c_int(k),
                          _d(shift), _ptr(rq), _ptr(res), _ptr(work))
    return rq, res


def orth_error(X):
    """X^T X - I evaluated in double-double (k x k)."""
    X, ldx = _fcols(X)
    n, k = X.shape
    out = np.empty((k, k), order="F")
    lib().dd_orth(_ptr(X), _i64(n), _i64(ldx), ctypes.c_int(k), _ptr(out))
    return out


def sin_angles(X, Q):
    """sin of the angle between column j of X and column j of Q, in dd."""
    X, ldx = _fcols(X)
    Q, ldq = _fcols(Q)
    n, k = X.shape
    out = np.empty(k)
    lib().dd_sin_angles(_ptr(X), _i64(ldx), _ptr(Q), _i64(ldq), _i64(n), ctypes.c_int(k), _ptr(out))
    return out


def product_entries(A, X, rows, cols, shift=0.0):
    """((A - shift I) X)[rows[t], cols[t]] in dd, as (hi, lo)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    X, ldx = _fcols(X)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    hi, lo = np.empty(len(rows)), np.empty(len(rows))
    lib().dd_product_entries(_ptr(A), _i64(A.shape[0]), _i64(A.shape[1]), _ptr(X), _i64(ldx), _d(shift),
                             _ptr(rows), _ptr(cols), _i64(len(rows)), _ptr(hi), _ptr(lo))
    return hi, lo
