"""Reproducible Jacobi-PCG on one GB300 -- thin Python binding.

This module only marshals arguments into the C ABI declared in
``include/rpcg.h`` (``librpcg.so``, built from ``csrc/``): every step of
the solver and of the dot products runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  Importing works without a
GPU; any call that needs the library raises if ``librpcg.so`` is missing
(there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librpcg.so")

OK, NOT_CONVERGED, FPE_INEXACT = 0, 1, 2
ERR_INVALID, ERR_NOT_SPD, ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6
PLAIN, EXBLAS, FPE = 0, 1, 2
VARIANTS = {"plain": PLAIN, "exblas": EXBLAS, "fpe": FPE}

# every symbol the header declares (checked by the CPU tests)
EXPORTS = [
    "rpcg_opts_default", "rpcg_status_string", "rpcg_last_error", "rpcg_create", "rpcg_destroy",
    "rpcg_matrix_info", "rpcg_spmv", "rpcg_dot_exact", "rpcg_dot_fpe", "rpcg_dot_plain", "rpcg_solve",
    "rpcg_solve_host", "rpcg_solve_profiled", "rpcg_solve_path", "rpcg_solve_async", "rpcg_dot_exact_noalloc", "rpcg_batch_create",
    "rpcg_batch_destroy", "rpcg_batch_solve", "rpcg_batch_solve_profiled", "rpcg_batch_solve_async", "rpcg_batch_tuned", "rpcg_solve_batched", "rpcg_server_create",
    "rpcg_server_submit", "rpcg_server_wait", "rpcg_server_stats", "rpcg_server_destroy", "rpcg_server_register",
    "rpcg_server_submit_registered", "rpcg_server_unregister", "rpcg_eft_twosum",
    "rpcg_eft_twoprod",
]


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("fpe_size", ctypes.c_int32),
                ("fpe_strict", ctypes.c_int32), ("block", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("history", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32), ("relres", ctypes.c_double),
                ("tau", ctypes.c_double), ("fpe_inexact_count", ctypes.c_int32), ("fpe_size_used", ctypes.c_int32)]

    def as_dict(self):
        return dict(iterations=self.iterations, status=self.status, relres=self.relres, tau=self.tau,
                    fpe_inexact_count=self.fpe_inexact_count, fpe_size_used=self.fpe_size_used)


RESULT_BYTES = ctypes.sizeof(Result)


def result_from(buf) -> dict:
    """The rpcg_result in a tensor written by rpcg_solve_async (device or pinned host)."""
    raw = buf.cpu().numpy().tobytes()[:RESULT_BYTES]
    return Result.from_buffer_copy(raw).as_dict()


def results_from(buf, count) -> list:
    """The count rpcg_result records in a tensor written by rpcg_batch_solve_async."""
    raw = buf.cpu().numpy().tobytes()
    return [Result.from_buffer_copy(raw[k * RESULT_BYTES:(k + 1) * RESULT_BYTES]).as_dict() for k in range(count)]


class ServerTiming(ctypes.Structure):
    _fields_ = [("queue_us", ctypes.c_double), ("service_us", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("chunks", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64), ("matrices_cached", ctypes.c_uint64)]


class RpcgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


_lib = None


def lib():
    """Load librpcg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2005_07282_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.rpcg_opts_default.argtypes = [ctypes.POINTER(Opts)]
        L.rpcg_opts_default.restype = None
        L.rpcg_status_string.argtypes = [i32]
        L.rpcg_status_string.restype = ctypes.c_char_p
        L.rpcg_last_error.argtypes = []
        L.rpcg_last_error.restype = ctypes.c_char_p
        L.rpcg_create.argtypes = [ctypes.POINTER(P), i32, i32, P, P, P, i32, P]
        L.rpcg_destroy.argtypes = [P]
        L.rpcg_matrix_info.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.rpcg_spmv.argtypes = [P, P, P, P]
        L.rpcg_dot_exact.argtypes = [i64, P, P, P, P]
        L.rpcg_dot_fpe.argtypes = [i64, P, P, i32, P, P, P]
        L.rpcg_dot_exact_noalloc.argtypes = [i64, P, P, P, P]
        L.rpcg_eft_twosum.argtypes = [i64, P, P, P, P, P]
        L.rpcg_eft_twoprod.argtypes = [i64, P, P, P, P, P]
        L.rpcg_batch_create.argtypes = [ctypes.POINTER(P), i32, P]
        L.rpcg_batch_destroy.argtypes = [P]
        L.rpcg_batch_solve.argtypes = [P, P, P, i32, ctypes.POINTER(Opts), P, P]
        L.rpcg_batch_tuned.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.rpcg_solve_batched.argtypes = [i32, P, P, P, i32, ctypes.POINTER(Opts), P, P]
        L.rpcg_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_size_t, i32]
        L.rpcg_server_submit.argtypes = [P, i32, i32, P, P, P, P, P, i32, ctypes.POINTER(Opts),
                                         ctypes.POINTER(ctypes.c_uint64)]
        L.rpcg_server_register.argtypes = [P, i32, i32, P, P, P, ctypes.POINTER(ctypes.c_uint64)]
        L.rpcg_server_submit_registered.argtypes = [P, ctypes.c_uint64, P, P, i32, ctypes.POINTER(Opts),
                                                    ctypes.POINTER(ctypes.c_uint64)]
        L.rpcg_server_unregister.argtypes = [P, ctypes.c_uint64]
        L.rpcg_server_wait.argtypes = [P, ctypes.c_uint64, P, ctypes.POINTER(Result), ctypes.POINTER(ServerTiming),
                                       ctypes.c_int64]
        L.rpcg_server_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
        L.rpcg_server_destroy.argtypes = [P]
        L.rpcg_dot_plain.argtypes = [i64, P, P, P, P]
        L.rpcg_solve.argtypes = [P, P, P, i32, ctypes.POINTER(Opts), ctypes.POINTER(Result), P]
        L.rpcg_solve_host.argtypes = [P, P, P, i32, ctypes.POINTER(Opts), ctypes.POINTER(Result), P]
        L.rpcg_solve_profiled.argtypes = [P, P, P, i32, ctypes.POINTER(Opts), ctypes.POINTER(Result),
                                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32), P]
        for name in EXPORTS:
            fn = getattr(L, name)
            if fn.restype is ctypes.c_int or fn.restype is None and name not in ("rpcg_opts_default",):
                fn.restype = ctypes.c_int
        L.rpcg_opts_default.restype = None
        _lib = L
    return _lib


def _check(st: int, where: str, allow=(OK,)):
    if st not in allow:
        raise RpcgError(st, where, lib().rpcg_last_error().decode() or lib().rpcg_status_string(st).decode())
    return st


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def make_opts(tol=1e-8, max_iter=1000, fpe_size=8, fpe_strict=0, block=0, grid=0, tile=0, history=None) -> Opts:
    o = Opts()
    lib().rpcg_opts_default(ctypes.byref(o))
    o.tol, o.max_iter, o.fpe_size, o.fpe_strict, o.block, o.grid = tol, max_iter, fpe_size, fpe_strict, block, grid
    o.tile = tile
    o.history = None if history is None else _dptr(history).value
    return o


def dot_exact(a, b, out=None, stream=None):
    """rpcg_dot_exact on device tensors; returns a 0-d device tensor."""
    import torch
    out = torch.empty((), dtype=torch.float64, device=a.device) if out is None else out
    _check(lib().rpcg_dot_exact(a.numel(), _dptr(a), _dptr(b), ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "rpcg_dot_exact")
    return out


def dot_exact_noalloc(a, b, out=None, stream=None):
    """rpcg_dot_exact_noalloc: the exact dot using the library's fixed
    scratch array instead of allocating (see include/rpcg.h)."""
    import torch
    out = torch.empty((), dtype=torch.float64, device=a.device) if out is None else out
    _check(lib().rpcg_dot_exact_noalloc(a.numel(), _dptr(a), _dptr(b), ctypes.c_void_p(out.data_ptr()),
                                        _stream(stream)), "rpcg_dot_exact_noalloc")
    return out


def dot_fpe(a, b, p=8, stream=None):
    """rpcg_dot_fpe; returns (0-d value tensor, 0-d int32 exactness flag tensor)."""
    import torch
    out = torch.empty((), dtype=torch.float64, device=a.device)
    ex = torch.empty((), dtype=torch.int32, device=a.device)
    _check(lib().rpcg_dot_fpe(a.numel(), _dptr(a), _dptr(b), p, ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(ex.data_ptr()), _stream(stream)), "rpcg_dot_fpe")
    return out, ex


def eft(kind, a, b, stream=None):
    """Elementwise Alg. 1 (kind="twosum") or Alg. 2 (kind="twoprod"): returns (r, s)."""
    import torch
    r, s = torch.empty_like(a), torch.empty_like(a)
    fn = lib().rpcg_eft_twosum if kind == "twosum" else lib().rpcg_eft_twoprod
    _check(fn(a.numel(), _dptr(a), _dptr(b), _dptr(r), _dptr(s), _stream(stream)), "rpcg_eft_" + kind)
    return r, s


def dot_plain(a, b, stream=None):
    import torch
    out = torch.empty((), dtype=torch.float64, device=a.device)
    _check(lib().rpcg_dot_plain(a.numel(), _dptr(a), _dptr(b), ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "rpcg_dot_plain")
    return out


class Matrix:
    """A CSR matrix handle (rpcg_create / rpcg_destroy)."""

    def __init__(self, rowptr, col, val, n=None, stream=None):
        import torch
        self._h = ctypes.c_void_p()
        if isinstance(val, torch.Tensor) and val.is_cuda:
            n = rowptr.numel() - 1 if n is None else n
            nnz = val.numel()
            ptrs = [ctypes.c_void_p(t.data_ptr()) for t in (rowptr, col, val)]
            kind = 1
            self._keep = (rowptr, col, val)
        else:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val, dtype=np.float64)
            n = rowptr.size - 1 if n is None else n
            nnz = val.size
            ptrs = [ctypes.c_void_p(a.ctypes.data) for a in (rowptr, col, val)]
            kind = 0
        _check(lib().rpcg_create(ctypes.byref(self._h), n, nnz, *ptrs, kind, _stream(stream)), "rpcg_create")
        self.n, self.nnz = n, nnz

    @classmethod
    def from_csr(cls, A, stream=None):
        """From an object with rowptr/col/val numpy arrays (host)."""
        return cls(A.rowptr, A.col, A.val, n=A.n, stream=stream)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().rpcg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spmv(self, x, y=None, stream=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(lib().rpcg_spmv(self._h, _dptr(x), _dptr(y), _stream(stream)), "rpcg_spmv")
        return y

    def solve(self, b, x, variant="exblas", stream=None, **opts) -> dict:
        """rpcg_solve on device tensors; x is updated in place."""
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o = make_opts(**opts)
        r = Result()
        st = lib().rpcg_solve(self._h, _dptr(b), _dptr(x), v, ctypes.byref(o), ctypes.byref(r), _stream(stream))
        if st in (ERR_INVALID, ERR_OOM, ERR_CUDA):
            _check(st, "rpcg_solve")
        return r.as_dict()

    def solve_async(self, b, x, res, variant="exblas", stream=None, **opts):
        """rpcg_solve_async: enqueue the solve on the stream and return at once.
        res: a uint8 tensor of at least RESULT_BYTES bytes, on the device or
        in pinned host memory; read it with result_from() after the stream
        has reached that point."""
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o = make_opts(**opts)
        assert res.numel() * res.element_size() >= RESULT_BYTES and res.is_contiguous()
        _check(lib().rpcg_solve_async(self._h, _dptr(b), _dptr(x), v, ctypes.byref(o), ctypes.c_void_p(res.data_ptr()),
                                      _stream(stream)), "rpcg_solve_async")

    def solve_path(self, variant="exblas", **opts) -> str:
        """Which path rpcg_solve takes: "cluster" (one cluster-resident launch)
        or "graph" (grid-wide passes in a CUDA graph)."""
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o = make_opts(**opts)
        p = ctypes.c_int32()
        _check(lib().rpcg_solve_path(self._h, v, ctypes.byref(o), ctypes.byref(p)), "rpcg_solve_path")
        return "cluster" if p.value == 1 else "graph"

    def solve_profiled(self, b, x, variant="exblas", stream=None, **opts) -> dict:
        """rpcg_solve_profiled: the result plus per-pass event times (ms) and launch counts."""
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o = make_opts(**opts)
        r = Result()
        ms = (ctypes.c_float * 4)()
        cnt = (ctypes.c_int32 * 4)()
        st = lib().rpcg_solve_profiled(self._h, _dptr(b), _dptr(x), v, ctypes.byref(o), ctypes.byref(r), ms, cnt,
                                       _stream(stream))
        if st in (ERR_INVALID, ERR_OOM, ERR_CUDA):
            _check(st, "rpcg_solve_profiled")
        d = r.as_dict()
        d["pass_ms"] = dict(zip(("setup", "A", "B", "C"), list(ms)))
        d["launches"] = dict(zip(("setup", "A", "B", "C"), list(cnt)))
        return d

    def solve_host(self, b: np.ndarray, x: np.ndarray, variant="exblas", stream=None, **opts) -> dict:
        """rpcg_solve_host on host numpy arrays; x (float64, contiguous) is updated in place."""
        assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o = make_opts(**opts)
        r = Result()
        st = lib().rpcg_solve_host(self._h, ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(x.ctypes.data), v,
                                   ctypes.byref(o), ctypes.byref(r), _stream(stream))
        if st in (ERR_INVALID, ERR_OOM, ERR_CUDA):
            _check(st, "rpcg_solve_host")
        return r.as_dict()


class Batch:
    """A batch of matrix handles solved together (rpcg_batch_*)."""

    def __init__(self, mats):
        self.mats = list(mats)
        arr = (ctypes.c_void_p * len(self.mats))(*[m._h.value for m in self.mats])
        self._h = ctypes.c_void_p()
        _check(lib().rpcg_batch_create(ctypes.byref(self._h), len(self.mats), arr), "rpcg_batch_create")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().rpcg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, bs, xs, variant="exblas", stream=None, **opts):
        """Solve every system: bs, xs lists of device tensors (xs updated in place)."""
        n = len(self.mats)
        assert len(bs) == n and len(xs) == n
        barr = (ctypes.c_void_p * n)(*[_dptr(t).value for t in bs])
        xarr = (ctypes.c_void_p * n)(*[_dptr(t).value for t in xs])
        res = (Result * n)()
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o = make_opts(**opts)
        st = lib().rpcg_batch_solve(self._h, barr, xarr, v, ctypes.byref(o), res, _stream(stream))
        if st in (ERR_INVALID, ERR_OOM, ERR_CUDA):
            _check(st, "rpcg_batch_solve")
        return [r.as_dict() for r in res]

    def solve_async(self, bs, xs, res, variant="exblas", stream=None, **opts):
        """rpcg_batch_solve_async: enqueue and return; res: a uint8 tensor of at
        least len(mats) * RESULT_BYTES bytes (device or pinned host), read with
        results_from() once the stream has reached that point."""
        n = len(self.mats)
        assert len(bs) == n and len(xs) == n
        assert res.numel() * res.element_size() >= n * RESULT_BYTES and res.is_contiguous()
        barr = (ctypes.c_void_p * n)(*[_dptr(t).value for t in bs])
        xarr = (ctypes.c_void_p * n)(*[_dptr(t).value for t in xs])
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o = make_opts(**opts)
        _check(lib().rpcg_batch_solve_async(self._h, barr, xarr, v, ctypes.byref(o), ctypes.c_void_p(res.data_ptr()),
                                            _stream(stream)), "rpcg_batch_solve_async")

    def solve_profiled(self, bs, xs, variant="exblas", stream=None, **opts):
        """solve() launched pass by pass with events; returns (results,
        {pass: ms}, {pass: launches})."""
        n = len(self.mats)
        assert len(bs) == n and len(xs) == n
        barr = (ctypes.c_void_p * n)(*[_dptr(t).value for t in bs])
        xarr = (ctypes.c_void_p * n)(*[_dptr(t).value for t in xs])
        res = (Result * n)()
        ms = (ctypes.c_float * 5)()
        nl = (ctypes.c_int32 * 5)()
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        o = make_opts(**opts)
        st = lib().rpcg_batch_solve_profiled(self._h, barr, xarr, v, ctypes.byref(o), res, ms, nl, _stream(stream))
        if st in (ERR_INVALID, ERR_OOM, ERR_CUDA):
            _check(st, "rpcg_batch_solve_profiled")
        names = ("setup", "A", "B", "C", "list")
        return [r.as_dict() for r in res], dict(zip(names, list(ms))), dict(zip(names, list(nl)))

    def tuned(self):
        b, t = ctypes.c_int32(), ctypes.c_int32()
        lib().rpcg_batch_tuned(self._h, ctypes.byref(b), ctypes.byref(t))
        return b.value, t.value


class Server:
    """The serving loop (rpcg_server_*).  Host arrays passed to submit() are
    kept referenced until their ticket has been waited for."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 256):
        self._h = ctypes.c_void_p()
        _check(lib().rpcg_server_create(ctypes.byref(self._h), int(hbm_budget_bytes), int(max_slots)),
               "rpcg_server_create")
        self._keep = {}
        self._sizes = {}

    def register(self, A) -> int:
        """rpcg_server_register: the server copies A (host CSR); returns its id."""
        rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
        cl = np.ascontiguousarray(A.col, dtype=np.int32)
        vl = np.ascontiguousarray(A.val, dtype=np.float64)
        m = ctypes.c_uint64()
        _check(lib().rpcg_server_register(self._h, A.n, int(vl.size), rp.ctypes.data, cl.ctypes.data, vl.ctypes.data,
                                          ctypes.byref(m)), "rpcg_server_register")
        self._sizes[m.value] = A.n
        return m.value

    def unregister(self, matrix: int):
        _check(lib().rpcg_server_unregister(self._h, matrix), "rpcg_server_unregister")

    def submit_registered(self, matrix: int, b: np.ndarray, x0=None, tol=1e-8, max_iter=1000) -> int:
        """rpcg_server_submit_registered: a solve on a registered matrix."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        o = make_opts(tol=tol, max_iter=max_iter)
        t = ctypes.c_uint64()
        _check(lib().rpcg_server_submit_registered(self._h, matrix, b.ctypes.data,
                                                   None if x0 is None else x0.ctypes.data, EXBLAS, ctypes.byref(o),
                                                   ctypes.byref(t)), "rpcg_server_submit_registered")
        self._keep[t.value] = (b, x0, self._sizes[matrix])
        return t.value

    def submit(self, A, b: np.ndarray, x0=None, tol=1e-8, max_iter=1000) -> int:
        rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
        cl = np.ascontiguousarray(A.col, dtype=np.int32)
        vl = np.ascontiguousarray(A.val, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        o = make_opts(tol=tol, max_iter=max_iter)
        t = ctypes.c_uint64()
        _check(lib().rpcg_server_submit(self._h, A.n, int(vl.size), rp.ctypes.data, cl.ctypes.data, vl.ctypes.data,
                                        b.ctypes.data, None if x0 is None else x0.ctypes.data, EXBLAS,
                                        ctypes.byref(o), ctypes.byref(t)), "rpcg_server_submit")
        self._keep[t.value] = (rp, cl, vl, b, x0, A.n)
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1):
        """Returns (x, result dict with queue_us/service_us)."""
        n = self._keep[ticket][-1] if ticket in self._keep else 0
        x = np.empty(n, dtype=np.float64)
        r = Result()
        tm = ServerTiming()
        st = lib().rpcg_server_wait(self._h, ticket, x.ctypes.data if n else None, ctypes.byref(r),
                                    ctypes.byref(tm), timeout_us)
        if st == ERR_TIMEOUT:
            raise TimeoutError(f"ticket {ticket} not done within {timeout_us} us")
        if st in (ERR_INVALID, ERR_CUDA):
            _check(st, "rpcg_server_wait")
        self._keep.pop(ticket, None)
        d = r.as_dict()
        d["queue_us"], d["service_us"] = tm.queue_us, tm.service_us
        return x, d

    def stats(self) -> dict:
        s = ServerStats()
        lib().rpcg_server_stats(self._h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().rpcg_server_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._keep = {}
        self._sizes = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
