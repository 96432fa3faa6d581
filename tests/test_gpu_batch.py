"""Batched solves: each system's result equals solving it alone, bit for
bit (exblas), for any tile size and with the autotuner; per-system
statuses are independent."""
import numpy as np
import pytest
import scipy.sparse

import synth
from conftest import bits

pytestmark = pytest.mark.gpu

SEED = synth.BASE_SEED + 4


def _dev(x, cuda):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(cuda)


def _csr_dense(M):
    S = scipy.sparse.csr_matrix(M)
    S.sort_indices()
    return synth.CSR(M.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def _systems():
    mats, rhs = [], []
    for k, s in enumerate([9, 3, 14, 1, 6, 11, 2, 8]):
        A, _ = synth.diffusion7(s, SEED + k)
        mats.append(A)
        rhs.append(synth.rhs_uniform(A.n, SEED + 100 + k))
    return mats, rhs


def _solo(rpcg, M, b, cuda, **kw):
    import torch
    x = torch.zeros(M.n, dtype=torch.float64, device=cuda)
    r = M.solve(b, x, **kw)
    return r, x.cpu().numpy()


@pytest.mark.parametrize("tile", [32, 100, 4096, 0])
def test_batch_bit_identical_to_solo(rpcg, cuda, tile):
    import torch
    mats, rhs = _systems()
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    bs = [_dev(b, cuda) for b in rhs]
    xs = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    B = rpcg.Batch(Ms)
    res = B.solve(bs, xs, variant="exblas", tol=1e-10, max_iter=3000, tile=tile, block=128 if tile == 100 else 0)
    for i, (M, b) in enumerate(zip(Ms, bs)):
        r, x = _solo(rpcg, M, b, cuda, variant="exblas", tol=1e-10, max_iter=3000)
        assert res[i]["iterations"] == r["iterations"], i
        assert res[i]["status"] == r["status"] == 0, i
        assert bits([res[i]["relres"]])[0] == bits([r["relres"]])[0]
        assert np.array_equal(bits(xs[i].cpu().numpy()), bits(x)), i
    if tile == 0:
        blk, tl = B.tuned()
        assert blk in (128, 256) and tl in (1024, 4096, 16384)
    B.close()


def test_batch_matches_oracle_and_history(rpcg, cuda, oracle_lib):
    import torch
    mats, rhs = _systems()
    mats, rhs = mats[:3], rhs[:3]
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    xs = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    hist = torch.full((3, 3001), float("nan"), dtype=torch.float64, device=cuda)
    B = rpcg.Batch(Ms)
    res = B.solve([_dev(b, cuda) for b in rhs], xs, tol=1e-10, max_iter=3000, tile=64, history=hist)
    for i, (A, b) in enumerate(zip(mats, rhs)):
        ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-10, max_iter=3000)
        assert res[i]["iterations"] == ref["iterations"]
        assert np.array_equal(bits(xs[i].cpu().numpy()), bits(ref["x"]))
        h = hist[i, : ref["iterations"] + 1].cpu().numpy()
        assert np.array_equal(bits(h), bits(ref["history"]))


def test_batch_mixed_statuses(rpcg, cuda, oracle_lib):
    import torch
    A0, _ = synth.diffusion7(5, SEED)
    mats = [A0, _csr_dense(np.array([[1.0, 2.0], [2.0, 1.0]])), _csr_dense(np.array([[4.0]])), A0]
    # the last system repeats A0's pattern but is a distinct handle with b = 0
    rhs = [synth.rhs_uniform(A0.n, 1), np.array([1.0, -1.0]), np.array([3.0]), np.zeros(A0.n)]
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    xs = [torch.ones(A.n, dtype=torch.float64, device=cuda) for A in mats]
    res = rpcg.Batch(Ms).solve([_dev(b, cuda) for b in rhs], xs, tol=1e-10, max_iter=50, tile=16)
    for i in range(4):
        x0 = np.ones(mats[i].n)
        ref = oracle_lib.pcg(mats[i], rhs[i], x0=x0, variant=oracle_lib.EXACT, tol=1e-10, max_iter=50)
        assert res[i]["status"] == ref["status"], (i, res[i], ref["status"])
        assert res[i]["iterations"] == ref["iterations"], i
        if ref["status"] >= 0:
            assert np.array_equal(bits(xs[i].cpu().numpy()), bits(ref["x"])), i
    assert res[1]["status"] == rpcg.ERR_NOT_SPD
    assert res[3]["iterations"] == 0 and not xs[3].any().item()


def test_batch_plain_converges(rpcg, cuda):
    import torch
    mats, rhs = _systems()
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    xs = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    res = rpcg.Batch(Ms).solve([_dev(b, cuda) for b in rhs], xs, variant="plain", tol=1e-10, max_iter=3000)
    assert all(r["status"] == 0 and r["relres"] < 1e-10 for r in res)


def test_batch_rejects_duplicates_and_bad_options(rpcg, cuda):
    import torch
    A, _ = synth.diffusion7(4, 1)
    M = rpcg.Matrix.from_csr(A)
    with pytest.raises(rpcg.RpcgError):
        rpcg.Batch([M, M])
    B = rpcg.Batch([M])
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    with pytest.raises(rpcg.RpcgError):
        B.solve([_dev(synth.rhs_uniform(A.n, 2), cuda)], [x], variant=7)
    with pytest.raises(rpcg.RpcgError):
        B.solve([_dev(synth.rhs_uniform(A.n, 2), cuda)], [x], variant="fpe", fpe_size=9)


@pytest.mark.parametrize("fpe_size,tile", [(8, 32), (2, 100), (1, 64), (0, 0), (8, 0)])
def test_batch_fpe_bit_identical_to_solo(rpcg, cuda, fpe_size, tile):
    """The fpe variant in a batch: every system's trajectory is the exact one
    (inexact dots are recomputed exactly, the other systems skip that pass),
    bit-identical to its solo solve; counts and sizes follow the solo rules."""
    import torch
    mats, rhs = _systems()
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    bs = [_dev(b, cuda) for b in rhs]
    xs = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    B = rpcg.Batch(Ms)
    res = B.solve(bs, xs, variant="fpe", tol=1e-10, max_iter=3000, tile=tile, fpe_size=fpe_size,
                  block=128 if tile == 100 else 0)
    for i, (M, b) in enumerate(zip(Ms, bs)):
        r, x = _solo(rpcg, M, b, cuda, variant="exblas", tol=1e-10, max_iter=3000)
        assert res[i]["status"] == r["status"] == 0, i
        assert res[i]["iterations"] == r["iterations"], i
        assert bits([res[i]["relres"]])[0] == bits([r["relres"]])[0], i
        assert np.array_equal(bits(xs[i].cpu().numpy()), bits(x)), i
        n = res[i]["fpe_inexact_count"]
        if fpe_size:
            assert res[i]["fpe_size_used"] == fpe_size, i
        else:
            assert res[i]["fpe_size_used"] == 3 if n == 0 else 3 < res[i]["fpe_size_used"] <= min(8, 3 + n)
    if fpe_size == 1:  # one term cannot hold the products' rounding errors
        assert sum(r["fpe_inexact_count"] for r in res) > 0
    B.close()


def test_batch_fpe_strict(rpcg, cuda):
    """fpe_strict = 1: nothing recomputed; with 8 terms nothing is lost on
    these systems and the batch equals the exact trajectory; with one term
    the systems that saw an inexact dot end with RPCG_FPE_INEXACT."""
    import torch
    mats, rhs = _systems()
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    bs = [_dev(b, cuda) for b in rhs]
    B = rpcg.Batch(Ms)
    x8 = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    r8 = B.solve(bs, x8, variant="fpe", tol=1e-10, max_iter=3000, tile=64, fpe_size=8, fpe_strict=1)
    for i, (M, b) in enumerate(zip(Ms, bs)):
        r, x = _solo(rpcg, M, b, cuda, variant="exblas", tol=1e-10, max_iter=3000)
        assert r8[i]["fpe_inexact_count"] == 0 and r8[i]["status"] == 0, i
        assert r8[i]["iterations"] == r["iterations"] and np.array_equal(bits(x8[i].cpu().numpy()), bits(x)), i
    x1 = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    r1 = B.solve(bs, x1, variant="fpe", tol=1e-10, max_iter=3000, tile=64, fpe_size=1, fpe_strict=1)
    assert any(r["fpe_inexact_count"] > 0 for r in r1)
    for r in r1:
        assert r["status"] == (rpcg.FPE_INEXACT if r["fpe_inexact_count"] > 0 else 0)
        assert r["relres"] < 1e-10


def test_batch_fpe_mixed_statuses(rpcg, cuda, oracle_lib):
    """Breakdowns, b = 0 and a one-row system in an fpe batch: the statuses,
    iteration counts and iterates of the exact-dot oracle."""
    import torch
    A0, _ = synth.diffusion7(5, SEED)
    mats = [A0, _csr_dense(np.array([[1.0, 2.0], [2.0, 1.0]])), _csr_dense(np.array([[4.0]])), A0]
    rhs = [synth.rhs_uniform(A0.n, 1), np.array([1.0, -1.0]), np.array([3.0]), np.zeros(A0.n)]
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    xs = [torch.ones(A.n, dtype=torch.float64, device=cuda) for A in mats]
    res = rpcg.Batch(Ms).solve([_dev(b, cuda) for b in rhs], xs, variant="fpe", tol=1e-10, max_iter=50, tile=16,
                               fpe_size=2)
    for i in range(4):
        ref = oracle_lib.pcg(mats[i], rhs[i], x0=np.ones(mats[i].n), variant=oracle_lib.EXACT, tol=1e-10, max_iter=50)
        assert res[i]["status"] == ref["status"], (i, res[i], ref["status"])
        assert res[i]["iterations"] == ref["iterations"], i
        if ref["status"] >= 0:
            assert np.array_equal(bits(xs[i].cpu().numpy()), bits(ref["x"])), i


@pytest.mark.parametrize("variant", ["exblas", "plain", "fpe"])
def test_batch_profiled_matches_graph(rpcg, cuda, variant):
    """The pass-by-pass form launches the same kernels in the same order:
    the same bits as the graph, one launch of A, B and C per iteration of the
    longest-running system, one list launch more."""
    import torch
    mats, rhs = _systems()
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    bs = [_dev(b, cuda) for b in rhs]
    B = rpcg.Batch(Ms)
    xg = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    rg = B.solve(bs, xg, variant=variant, tol=1e-10, max_iter=3000, tile=64, block=128)
    xp = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    rp, ms, nl = B.solve_profiled(bs, xp, variant=variant, tol=1e-10, max_iter=3000, tile=64, block=128)
    for i in range(len(mats)):
        assert rg[i]["iterations"] == rp[i]["iterations"]
        assert bits([rg[i]["relres"]])[0] == bits([rp[i]["relres"]])[0]
        assert np.array_equal(bits(xg[i].cpu().numpy()), bits(xp[i].cpu().numpy())), i
    for i in range(len(mats)):
        assert rg[i]["fpe_inexact_count"] == rp[i]["fpe_inexact_count"], i
    most = max(r["iterations"] for r in rg)
    assert nl == {"setup": 3, "A": most, "B": most, "C": most, "list": most + 1}
    assert all(v >= 0.0 for v in ms.values()) and ms["A"] > 0.0


def test_batch_more_systems_than_shared_prefix(rpcg, cuda, oracle_lib):
    """1100 systems: the unit prefix no longer fits the kernels' shared-memory
    copy and is searched in global memory; every system still matches the
    oracle bit for bit."""
    import torch
    mats, rhs = [], []
    for k in range(1100):
        A, _ = synth.diffusion7(1 + k % 3, SEED + 7 * k)
        mats.append(A)
        rhs.append(synth.rhs_uniform(A.n, SEED + 7 * k + 1))
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    xs = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    res = rpcg.Batch(Ms).solve([_dev(b, cuda) for b in rhs], xs, tol=1e-12, max_iter=100, tile=8, block=128)
    for i in range(0, 1100, 7):
        ref = oracle_lib.pcg(mats[i], rhs[i], variant=oracle_lib.EXACT, tol=1e-12, max_iter=100)
        assert res[i]["iterations"] == ref["iterations"] and res[i]["status"] == ref["status"], i
        assert np.array_equal(bits(xs[i].cpu().numpy()), bits(ref["x"])), i


def test_batch_async_equals_sync(rpcg, cuda, oracle_lib):
    """rpcg_batch_solve_async: enqueued without synchronising; the per-system
    results (device or pinned host memory) and iterates equal the synchronous
    batch solve, including a b = 0 system and an empty one."""
    import torch
    mats, rhs = _systems()
    E = synth.CSR(0, np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), np.zeros(0))
    mats = mats + [E, mats[0].__class__(mats[0].n, mats[0].rowptr.copy(), mats[0].col.copy(), mats[0].val.copy())]
    rhs = rhs + [np.zeros(0), np.zeros(mats[0].n)]
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    bs = [_dev(b, cuda) for b in rhs]
    B = rpcg.Batch(Ms)
    xs_sync = [torch.ones(A.n, dtype=torch.float64, device=cuda) for A in mats]
    rs = B.solve(bs, xs_sync, variant="exblas", tol=1e-10, max_iter=3000, tile=64, block=128)
    rf = B.solve(bs, [torch.ones(A.n, dtype=torch.float64, device=cuda) for A in mats], variant="fpe", tol=1e-10,
                 max_iter=3000, tile=64, block=128, fpe_size=1)
    xf = [torch.ones(A.n, dtype=torch.float64, device=cuda) for A in mats]
    resf = torch.zeros(len(mats) * rpcg.RESULT_BYTES, dtype=torch.uint8, device=cuda)
    B.solve_async(bs, xf, resf, variant="fpe", tol=1e-10, max_iter=3000, tile=64, block=128, fpe_size=1)
    torch.cuda.synchronize()
    for i, r in enumerate(rpcg.results_from(resf, len(mats))):
        assert r == rf[i], i
        assert torch.equal(xf[i].view(torch.int64), xs_sync[i].view(torch.int64)), i
    for pinned in (False, True):
        xs = [torch.ones(A.n, dtype=torch.float64, device=cuda) for A in mats]
        nbytes = len(mats) * rpcg.RESULT_BYTES
        res = torch.zeros(nbytes, dtype=torch.uint8).pin_memory() if pinned else \
            torch.zeros(nbytes, dtype=torch.uint8, device=cuda)
        B.solve_async(bs, xs, res, variant="exblas", tol=1e-10, max_iter=3000, tile=64, block=128)
        torch.cuda.synchronize()
        ra = rpcg.results_from(res, len(mats))
        for i in range(len(mats)):
            assert ra[i]["status"] == rs[i]["status"] and ra[i]["iterations"] == rs[i]["iterations"], i
            assert bits([ra[i]["relres"]])[0] == bits([rs[i]["relres"]])[0], i
            assert torch.equal(xs[i].view(torch.int64), xs_sync[i].view(torch.int64)), i
    assert ra[-1]["iterations"] == 0 and not xs[-1].any().item()   # b = 0: x = 0
    assert ra[-2] == {**ra[-2], "status": 0, "iterations": 0}     # the empty system
