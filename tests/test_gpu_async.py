"""rpcg_solve_async: the solve is enqueued without synchronising the stream
and the result struct is written on the device; every result equals the
synchronous rpcg_solve bit for bit, on both solver paths."""
import numpy as np
import pytest

import synth
from conftest import bits

pytestmark = pytest.mark.gpu

SEED = synth.BASE_SEED + 21


def _dev(x, cuda):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(cuda)


def _res_buf(rpcg, cuda, pinned=False):
    import torch
    if pinned:
        return torch.zeros(rpcg.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    return torch.zeros(rpcg.RESULT_BYTES, dtype=torch.uint8, device=cuda)


def _sync(M, b, cuda, x0=None, **kw):
    import torch
    x = torch.zeros(M.n, dtype=torch.float64, device=cuda) if x0 is None else _dev(x0, cuda)
    r = M.solve(b, x, **kw)
    return r, x.cpu().numpy()


def _same(ra, xa, rs, xs):
    assert ra["status"] == rs["status"] and ra["iterations"] == rs["iterations"]
    assert bits([ra["relres"]])[0] == bits([rs["relres"]])[0]
    assert bits([ra["tau"]])[0] == bits([rs["tau"]])[0]
    assert ra["fpe_inexact_count"] == rs["fpe_inexact_count"] and ra["fpe_size_used"] == rs["fpe_size_used"]
    assert np.array_equal(bits(xa), bits(xs))


@pytest.mark.parametrize("kind,variant,kw,path", [
    ("p7_16", "exblas", {}, "cluster"),
    ("p27_30", "exblas", {}, "graph"),                 # 27000 rows: beyond the cluster path
    ("p7_16", "exblas", {"block": 256}, "graph"),
    ("p7_16", "plain", {}, "cluster"),
    ("p7_9", "fpe", {}, "cluster"),
    ("p7_9", "fpe", {"fpe_size": 2, "fpe_strict": 1}, "cluster"),
    ("p7_9", "fpe", {"fpe_size": 1}, "cluster"),
    ("p7_9", "fpe", {"block": 256}, "graph"),
    ("p7_9", "fpe", {"fpe_size": 2, "fpe_strict": 1, "block": 128}, "graph"),
])
def test_async_equals_sync(rpcg, cuda, oracle_lib, kind, variant, kw, path):
    import torch
    A = {"p7_16": lambda: synth.poisson7(16), "p27_30": lambda: synth.poisson27(30),
         "p7_9": lambda: synth.poisson7(9)}[kind]()
    M = rpcg.Matrix.from_csr(A)
    assert M.solve_path(variant, **kw) == path
    b = _dev(oracle_lib.spmv(A, synth.poisson_rhs_xtrue(A.n, SEED)), cuda)
    opts = dict(variant=variant, tol=1e-10, max_iter=2000, **kw)
    rs, xs = _sync(M, b, cuda, **opts)
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    res = _res_buf(rpcg, cuda)
    M.solve_async(b, x, res, **opts)
    torch.cuda.synchronize()
    _same(rpcg.result_from(res), x.cpu().numpy(), rs, xs)


@pytest.mark.parametrize("kind,kw", [("p7_12", {}), ("p27_14", {}), ("p7_12", {"block": 256}),
                                     ("p27_30", {})])
def test_async_back_to_back_on_one_handle(rpcg, cuda, oracle_lib, kind, kw):
    """Two solves enqueued on one handle before either runs, on the cluster
    path and on the graph path (whose x0 node is updated between the two
    launches): each sees its own arguments (passed by value at the call)."""
    import torch
    A = {"p7_12": lambda: synth.poisson7(12), "p27_14": lambda: synth.poisson27(14),
         "p27_30": lambda: synth.poisson27(30)}[kind]()
    M = rpcg.Matrix.from_csr(A)
    b1 = _dev(synth.rhs_uniform(A.n, SEED + 1), cuda)
    b2 = _dev(synth.rhs_uniform(A.n, SEED + 2), cuda)
    r1s, x1s = _sync(M, b1, cuda, tol=1e-9, max_iter=500, **kw)
    r2s, x2s = _sync(M, b2, cuda, x0=np.full(A.n, 0.5), tol=1e-6, max_iter=500, **kw)
    x1 = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    x2 = _dev(np.full(A.n, 0.5), cuda)
    res1, res2 = _res_buf(rpcg, cuda), _res_buf(rpcg, cuda, pinned=True)
    M.solve_async(b1, x1, res1, tol=1e-9, max_iter=500, **kw)
    M.solve_async(b2, x2, res2, tol=1e-6, max_iter=500, **kw)
    torch.cuda.synchronize()
    _same(rpcg.result_from(res1), x1.cpu().numpy(), r1s, x1s)
    _same(rpcg.result_from(res2), x2.cpu().numpy(), r2s, x2s)


def test_async_two_handles_two_streams(rpcg, cuda, oracle_lib):
    import torch
    As = [synth.diffusion7(20, SEED + 3)[0], synth.poisson27(40)]
    Ms = [rpcg.Matrix.from_csr(A) for A in As]
    bs = [_dev(synth.rhs_uniform(A.n, SEED + 4 + k), cuda) for k, A in enumerate(As)]
    ref = [_sync(M, b, cuda, tol=1e-10, max_iter=3000) for M, b in zip(Ms, bs)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    xs = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in As]
    res = [_res_buf(rpcg, cuda, pinned=True) for _ in As]
    torch.cuda.synchronize()
    for M, b, x, r, st in zip(Ms, bs, xs, res, streams):
        M.solve_async(b, x, r, tol=1e-10, max_iter=3000, stream=st)
    for st in streams:
        st.synchronize()
    for (rs, xsync), x, r in zip(ref, xs, res):
        _same(rpcg.result_from(r), x.cpu().numpy(), rs, xsync)


def test_async_statuses_decided_on_device(rpcg, cuda, oracle_lib):
    import scipy.sparse
    import torch
    A = synth.poisson7(10)
    M = rpcg.Matrix.from_csr(A)
    b = _dev(synth.rhs_uniform(A.n, SEED + 9), cuda)
    cases = [
        (b, dict(tol=1e-14, max_iter=4)),                 # NOT_CONVERGED
        (torch.zeros_like(b), dict(tol=1e-8, max_iter=50)),  # b = 0: x = 0, 0 iterations
        (b, dict(tol=1e-8, max_iter=0)),
    ]
    for bb, kw in cases:
        rs, xs = _sync(M, bb, cuda, x0=np.ones(A.n), **kw)
        x = _dev(np.ones(A.n), cuda)
        res = _res_buf(rpcg, cuda)
        M.solve_async(bb, x, res, **kw)
        torch.cuda.synchronize()
        _same(rpcg.result_from(res), x.cpu().numpy(), rs, xs)
    assert rpcg.result_from(res)["status"] == rpcg.NOT_CONVERGED
    # not SPD: status decided by the set-up on the device
    S = scipy.sparse.csr_matrix(np.array([[1.0, 2.0], [2.0, -1.0]]))
    An = synth.CSR(2, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))
    Mn = rpcg.Matrix.from_csr(An)
    bn = _dev(np.array([1.0, 1.0]), cuda)
    x = torch.zeros(2, dtype=torch.float64, device=cuda)
    res = _res_buf(rpcg, cuda)
    Mn.solve_async(bn, x, res, tol=1e-8, max_iter=10)
    torch.cuda.synchronize()
    assert rpcg.result_from(res)["status"] == rpcg.ERR_NOT_SPD
    # an empty system
    E = synth.CSR(0, np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    Me = rpcg.Matrix.from_csr(E)
    e = torch.zeros(0, dtype=torch.float64, device=cuda)
    res = _res_buf(rpcg, cuda)
    Me.solve_async(e, e, res)
    torch.cuda.synchronize()
    r = rpcg.result_from(res)
    assert r["status"] == 0 and r["iterations"] == 0 and r["relres"] == 0.0


def test_async_argument_errors_are_immediate(rpcg, cuda):
    import ctypes
    A = synth.poisson7(4)
    M = rpcg.Matrix.from_csr(A)
    st = rpcg.lib().rpcg_solve_async(M._h, None, None, 1, None, None, None)
    assert st == rpcg.ERR_INVALID
    assert b"NULL" in rpcg.lib().rpcg_last_error()
