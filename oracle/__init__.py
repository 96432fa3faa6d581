"""CPU oracle for the reproducible Jacobi-PCG hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``rpcg_oracle.c`` (plain C,
built with ``-O2 -ffp-contract=off``) through ctypes; it shares no code with
the CUDA library.  See the header of ``rpcg_oracle.c`` for what each routine
computes and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpcg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, NOT_CONVERGED, ERR_INVALID, ERR_NOT_SPD, ERR_NONFINITE = 0, 1, -1, -2, -3
PLAIN, EXACT = 0, 1

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, plain C11)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        P = ctypes.c_void_p
        L.oracle_dot_exact.restype = d
        L.oracle_dot_exact.argtypes = [i64, P, P, ctypes.c_int]
        L.oracle_sum_exact.restype = d
        L.oracle_sum_exact.argtypes = [i64, P]
        L.oracle_twosum.restype = None
        L.oracle_twosum.argtypes = [d, d, P, P]
        L.oracle_twoprod.restype = None
        L.oracle_twoprod.argtypes = [d, d, P, P]
        L.oracle_fpe_accumulate.restype = d
        L.oracle_fpe_accumulate.argtypes = [P, ctypes.c_int, d]
        L.oracle_fpesum.restype = ctypes.c_int
        L.oracle_fpesum.argtypes = [P, P, ctypes.c_int]
        L.oracle_dot_fpe.restype = d
        L.oracle_dot_fpe.argtypes = [i64, P, P, ctypes.c_int, ctypes.c_int, P]
        L.oracle_spmv.restype = None
        L.oracle_spmv.argtypes = [i32, P, P, P, P, P, ctypes.c_int]
        L.oracle_pcg_loop_seconds.restype = d
        L.oracle_pcg_loop_seconds.argtypes = []
        L.oracle_pcg_trace.restype = ctypes.c_int
        L.oracle_pcg_trace.argtypes = [i32, P, P, P, P, P, ctypes.c_int, d, i32, P, P, P, P]
        L.oracle_pcg.restype = ctypes.c_int
        L.oracle_pcg.argtypes = [i32, P, P, P, P, P, ctypes.c_int, d, i32, P, P, P, P, ctypes.c_int]
        _lib = L
    return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def dot_exact(a, b, nthreads: int = 1) -> float:
    """Correctly rounded value of sum(a_i * b_i), computed exactly (Sec. 2, long accumulator)."""
    a, b = _f64(a), _f64(b)
    assert a.shape == b.shape
    return _load().oracle_dot_exact(a.size, _ptr(a), _ptr(b), nthreads)


def sum_exact(x) -> float:
    """Correctly rounded value of sum(x_i)."""
    x = _f64(x)
    return _load().oracle_sum_exact(x.size, _ptr(x))


def twosum(a: float, b: float):
    """Alg. 1."""
    r, s = ctypes.c_double(), ctypes.c_double()
    _load().oracle_twosum(a, b, ctypes.byref(r), ctypes.byref(s))
    return r.value, s.value


def twoprod(a: float, b: float):
    """Alg. 2."""
    r, s = ctypes.c_double(), ctypes.c_double()
    _load().oracle_twoprod(a, b, ctypes.byref(r), ctypes.byref(s))
    return r.value, s.value


def fpe_accumulate(a: np.ndarray, x: float) -> float:
    """Alg. 4 with early exit; ``a`` (float64, length p) is updated in place.
    Returns the value carried out of the last term."""
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return _load().oracle_fpe_accumulate(_ptr(a), a.size, x)


def fpesum(a: np.ndarray, b: np.ndarray) -> bool:
    """Alg. 3; ``a`` is updated in place.  Returns True if a term was lost."""
    assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == b.size
    b = _f64(b)
    return bool(_load().oracle_fpesum(_ptr(a), _ptr(b), a.size))


def dot_fpe(a, b, p: int = 8, T: int = 1):
    """FPE dot (Listings 1-2, Algs. 1-4); returns (value, exact_flag)."""
    a, b = _f64(a), _f64(b)
    flag = ctypes.c_int()
    v = _load().oracle_dot_fpe(a.size, _ptr(a), _ptr(b), p, T, ctypes.byref(flag))
    return v, bool(flag.value)


def spmv(A, x, nthreads: int = 1) -> np.ndarray:
    """w = A x with each row summed left to right by fma from +0 (Sec. 4.3)."""
    x = _f64(x)
    y = np.empty(A.n, dtype=np.float64)
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    cl = np.ascontiguousarray(A.col, dtype=np.int32)
    vl = _f64(A.val)
    _load().oracle_spmv(A.n, _ptr(rp), _ptr(cl), _ptr(vl), _ptr(x), _ptr(y), nthreads)
    return y


def pcg(A, b, x0=None, variant: int = EXACT, tol: float = 1e-8, max_iter: int = 1000, nthreads: int = 1):
    """Jacobi-PCG (Fig. 1 with S8 next to S6 as in Fig. 2).

    Returns dict(x, status, iterations, relres, tau, history)."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    hist = np.full(max_iter + 1, np.nan)
    it, rr, tt = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    cl = np.ascontiguousarray(A.col, dtype=np.int32)
    vl = _f64(A.val)
    st = _load().oracle_pcg(A.n, _ptr(rp), _ptr(cl), _ptr(vl), _ptr(b), _ptr(x), variant, tol, max_iter,
                            _ptr(hist), ctypes.byref(it), ctypes.byref(rr), ctypes.byref(tt), nthreads)
    return dict(x=x, status=st, iterations=it.value, relres=rr.value, tau=tt.value,
                history=hist[: it.value + 1].copy(), loop_seconds=_load().oracle_pcg_loop_seconds())


def pcg_trace(A, b, variant: int = EXACT, tol: float = 0.0, max_iter: int = 2):
    """oracle_pcg with every loop test recorded (tiny systems): a list of
    dicts with dw, rho, beta, tau, gamma, relres and the vectors x, r, z, d
    after the set-up (entry 0) and after each loop body."""
    b = _f64(b)
    n = A.n
    x = np.zeros(n)
    rec = 6 + 4 * n
    tr = np.full((max_iter + 1) * rec, np.nan)
    it, rr, tt = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    cl = np.ascontiguousarray(A.col, dtype=np.int32)
    vl = _f64(A.val)
    st = _load().oracle_pcg_trace(n, _ptr(rp), _ptr(cl), _ptr(vl), _ptr(b), _ptr(x), variant, tol, max_iter,
                                  _ptr(tr), ctypes.byref(it), ctypes.byref(rr), ctypes.byref(tt))
    out = []
    for l in range(it.value + 1):
        t = tr[l * rec:(l + 1) * rec]
        out.append(dict(dw=t[0], rho=t[1], beta=t[2], tau=t[3], gamma=t[4], relres=t[5], x=t[6:6 + n].copy(),
                        r=t[6 + n:6 + 2 * n].copy(), z=t[6 + 2 * n:6 + 3 * n].copy(), d=t[6 + 3 * n:6 + 4 * n].copy()))
    return dict(status=st, iterations=it.value, trace=out)
