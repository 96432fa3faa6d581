"""The serving loop: results are bit-identical alone and in the mix, work
that arrives while other solves run joins them (continuous batching), and
admission respects the HBM budget."""
import threading
import time

import numpy as np
import pytest

import synth
from conftest import bits

pytestmark = pytest.mark.gpu


def _alone(rpcg, cuda, A, b, x0=None, tol=1e-8):
    import torch
    M = rpcg.Matrix.from_csr(A)
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda) if x0 is None else torch.from_numpy(x0.copy()).to(cuda)
    r = M.solve(torch.from_numpy(b).to(cuda), x, variant="exblas", tol=tol, max_iter=2000)
    M.close()
    return r, x.cpu().numpy()


def test_server_results_identical_alone_and_in_mix(rpcg, cuda):
    sides = [6, 11, 16, 9, 6, 20, 11, 3]
    mats = {s: synth.poisson7(s) for s in set(sides)}  # repeated sides share one matrix
    reqs = []
    for k, s in enumerate(sides):
        A = mats[s]
        b = synth.rhs_uniform(A.n, 300 + k)
        x0 = synth.uniform_pm1(400 + k, A.n) if k % 3 == 0 else None
        reqs.append((A, b, x0))
    srv = rpcg.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    tickets = [srv.submit(A, b, x0=x0, tol=1e-8, max_iter=2000) for A, b, x0 in reqs]
    outs = [srv.wait(t, timeout_us=120_000_000) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["matrices_cached"] <= len(mats)
    for (A, b, x0), (x, res) in zip(reqs, outs):
        ra, xa = _alone(rpcg, cuda, A, b, x0)
        assert res["status"] == ra["status"] == 0
        assert res["iterations"] == ra["iterations"]
        assert bits([res["relres"]])[0] == bits([ra["relres"]])[0]
        assert np.array_equal(bits(x), bits(xa))
        assert res["queue_us"] >= 0 and res["service_us"] > 0


def test_server_admits_work_while_others_run(rpcg, cuda):
    """A long solve is running; short requests submitted afterwards finish
    before it does, so they were admitted alongside it."""
    big = synth.poisson27(48)
    b_big = synth.rhs_uniform(big.n, 9)
    small = synth.poisson7(8)
    srv = rpcg.Server(hbm_budget_bytes=4 << 30, max_slots=8)
    # tol 0: the big solve never meets the test (its residual shrinks by ~0.8
    # per iteration, 1e-30 at iteration 286), so it runs until max_iter or
    # until its residual underflows, thousands of iterations either way; the
    # short requests are submitted once it has run two chunks of iterations
    t_big = srv.submit(big, b_big, tol=0.0, max_iter=3000)
    t0 = time.time()
    while srv.stats()["chunks"] < 2 and time.time() - t0 < 60:
        time.sleep(0.0005)
    t_small = [srv.submit(small, synth.rhs_uniform(small.n, 50 + k), tol=1e-8) for k in range(5)]
    done_order, results = [], {}
    lock = threading.Lock()

    def waiter(t):
        x, r = srv.wait(t, timeout_us=120_000_000)
        with lock:
            done_order.append(t)
            results[t] = r

    ths = [threading.Thread(target=waiter, args=(t,)) for t in [t_big] + t_small]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    srv.close()
    assert results[t_big]["iterations"] > 1000, results[t_big]
    assert all(results[t]["status"] == 0 for t in t_small)
    assert done_order[-1] == t_big, done_order


def test_server_budget_and_errors(rpcg, cuda):
    # a 40^3 system needs ~9 MB for its matrix and ~3 MB for its vectors, a
    # 32^3 one ~5 + ~1.6 MB: a 20 MB budget holds only part of the requests at
    # once, so the rest wait for slots and memory, reuse or evict matrices
    A = synth.poisson7(40)
    other = synth.poisson7(32)
    srv = rpcg.Server(hbm_budget_bytes=20 << 20, max_slots=4)
    ts = [srv.submit(A if k % 2 == 0 else other, synth.rhs_uniform((A if k % 2 == 0 else other).n, k)) for k in range(6)]
    for t in ts:
        x, r = srv.wait(t, timeout_us=120_000_000)
        assert r["status"] == 0
    st = srv.stats()
    assert st["bytes_in_use"] <= 20 << 20
    # a request larger than the whole budget fails at once with OOM
    huge = synth.poisson7(80)
    th = srv.submit(huge, synth.rhs_uniform(huge.n, 1))
    x, r = srv.wait(th, timeout_us=60_000_000)
    assert r["status"] == rpcg.ERR_OOM
    # an unknown ticket is rejected; a short wait on a long solve times out
    with pytest.raises(rpcg.RpcgError):
        srv.wait(987654, timeout_us=1000)
    big = synth.poisson7(32)
    tb = srv.submit(big, synth.rhs_uniform(big.n, 3), tol=1e-14, max_iter=2000)
    with pytest.raises(TimeoutError):
        srv.wait(tb, timeout_us=1)
    x, r = srv.wait(tb, timeout_us=120_000_000)
    assert r["status"] in (0, rpcg.NOT_CONVERGED)
    srv.close()


def _wait_cached(srv, want, limit_s=10.0):
    """Poll the server's cache size until it reaches `want` (the scheduler
    frees the device copy of a matrix no ticket can name any more)."""
    t0 = time.time()
    while srv.stats()["matrices_cached"] != want and time.time() - t0 < limit_s:
        time.sleep(0.002)
    return srv.stats()["matrices_cached"]


def test_server_arrays_overwritten_after_collection_are_not_served_stale(rpcg, cuda):
    """The caller may change its arrays once a ticket is collected.  A new
    matrix written into the same host buffers (same shape, same addresses)
    must be solved as that new matrix: bit-identical to solving it alone,
    never the old device copy."""
    A = synth.poisson7(12)
    diag = np.array([k for i in range(A.n) for k in range(A.rowptr[i], A.rowptr[i + 1]) if A.col[k] == i])
    val_ptr = A.val.ctypes.data
    b = synth.rhs_uniform(A.n, 77)
    srv = rpcg.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    x1, r1 = srv.wait(srv.submit(A, b, tol=1e-10, max_iter=2000), timeout_us=60_000_000)
    assert r1["status"] == 0
    # nothing can name the first matrix any more: its device copy is freed
    assert _wait_cached(srv, 0) == 0
    # overwrite the values in place: diagonal 6 -> 8.5, off-diagonals -1 -> -1.25
    # (still diagonally dominant, so SPD)
    A.val[:] = -1.25
    A.val[diag] = 8.5
    assert A.val.ctypes.data == val_ptr
    x2, r2 = srv.wait(srv.submit(A, b, tol=1e-10, max_iter=2000), timeout_us=60_000_000)
    srv.close()
    ra, xa = _alone(rpcg, cuda, A, b, tol=1e-10)
    assert r2["status"] == ra["status"] == 0
    assert r2["iterations"] == ra["iterations"]
    assert np.array_equal(bits(x2), bits(xa))
    assert not np.array_equal(bits(x2), bits(x1))


def test_server_registered_matrix(rpcg, cuda):
    """A registered matrix is copied by the server: the caller's arrays can
    change at once, requests on it share one device copy, and each result is
    bit-identical to solving the registered matrix alone."""
    A = synth.poisson7(10)
    keep = synth.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy(), A.name)
    srv = rpcg.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    m = srv.register(A)
    A.val[:] = np.nan  # the server holds its own copy
    bs = [synth.rhs_uniform(keep.n, 600 + k) for k in range(4)]
    ts = [srv.submit_registered(m, b, tol=1e-9, max_iter=2000) for b in bs]
    outs = [srv.wait(t, timeout_us=60_000_000) for t in ts]
    assert srv.stats()["matrices_cached"] == 1
    # later requests reuse the cached copy after the earlier ones were collected
    x5, r5 = srv.wait(srv.submit_registered(m, bs[0], tol=1e-9, max_iter=2000), timeout_us=60_000_000)
    srv.unregister(m)
    with pytest.raises(rpcg.RpcgError):
        srv.submit_registered(m, bs[0])
    with pytest.raises(rpcg.RpcgError):
        srv.unregister(m)
    assert _wait_cached(srv, 0) == 0
    srv.close()
    for b, (x, r) in zip(bs, outs):
        ra, xa = _alone(rpcg, cuda, keep, b, tol=1e-9)
        assert r["status"] == ra["status"] == 0 and r["iterations"] == ra["iterations"]
        assert np.array_equal(bits(x), bits(xa))
    assert np.array_equal(bits(x5), bits(outs[0][0])) and r5["iterations"] == outs[0][1]["iterations"]
