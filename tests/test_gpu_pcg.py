"""GPU parity of SpMV and the full PCG trajectory against the CPU oracle.

exblas and fpe (fpe_strict = 0) must reproduce the oracle's exact-dot PCG
bit for bit: iteration count, every residual of the history, the solution.
The plain variant is checked by tolerance only (its dots are not exact)."""
import math

import numpy as np
import pytest

import synth
from conftest import bits

pytestmark = pytest.mark.gpu

SEED = synth.BASE_SEED


def _dev(x, cuda):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(cuda)


def _mats():
    yield synth.poisson7(16)                    # the 16^3 7-point system (4096 rows)
    yield synth.poisson27(12)
    yield synth.diffusion7(9, SEED + 3)[0]
    yield synth.poisson7(7)                     # rows not a multiple of a tile


@pytest.mark.parametrize("k", range(4))
def test_spmv_bit_exact(rpcg, cuda, oracle_lib, k):
    A = list(_mats())[k]
    x = synth.uniform_pm1(SEED + k, A.n)
    M = rpcg.Matrix.from_csr(A)
    y = M.spmv(_dev(x, cuda)).cpu().numpy()
    assert np.array_equal(bits(y), bits(oracle_lib.spmv(A, x)))


def test_spmv_long_rows_unstaged(rpcg, cuda, oracle_lib):
    """Rows longer than the staged slab take the direct path."""
    import scipy.sparse
    n = 600
    rng = np.random.default_rng(4)
    S = scipy.sparse.random(n, n, density=0.5, random_state=5, format="csr")
    S.sort_indices()
    A = synth.CSR(n, S.indptr.astype(np.int32), S.indices.astype(np.int32), rng.standard_normal(S.nnz))
    x = rng.standard_normal(n)
    y = rpcg.Matrix.from_csr(A).spmv(_dev(x, cuda)).cpu().numpy()
    assert np.array_equal(bits(y), bits(oracle_lib.spmv(A, x)))


def _system(kind):
    if kind == "p7_16":
        A = synth.poisson7(16)
    elif kind == "p27_10":
        A = synth.poisson27(10)
    elif kind == "diff_8":
        A = synth.diffusion7(8, SEED + 4)[0]
    return A


def _rhs(oracle_lib, A, seed):
    return oracle_lib.spmv(A, synth.poisson_rhs_xtrue(A.n, seed))


@pytest.mark.parametrize("variant", ["exblas", "fpe"])
@pytest.mark.parametrize("kind", ["p7_16", "p27_10", "diff_8"])
def test_pcg_bit_exact_vs_oracle(rpcg, cuda, oracle_lib, variant, kind):
    import torch
    A = _system(kind)
    tol = 1e-10 if kind == "diff_8" else 1e-8
    b = _rhs(oracle_lib, A, SEED)
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=tol, max_iter=2000, nthreads=4)
    M = rpcg.Matrix.from_csr(A)
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    hist = torch.full((2001,), float("nan"), dtype=torch.float64, device=cuda)
    r = M.solve(_dev(b, cuda), x, variant=variant, tol=tol, max_iter=2000, history=hist)
    assert r["status"] == ref["status"] == 0
    assert r["iterations"] == ref["iterations"]
    assert bits([r["relres"]])[0] == bits([ref["relres"]])[0]
    assert np.array_equal(bits(hist[: r["iterations"] + 1].cpu().numpy()), bits(ref["history"]))
    assert np.array_equal(bits(x.cpu().numpy()), bits(ref["x"]))


@pytest.mark.parametrize("variant", ["exblas", "fpe"])
def test_pcg_launch_shape_independent(rpcg, cuda, oracle_lib, variant):
    import torch
    A = synth.poisson7(16)
    b = _dev(_rhs(oracle_lib, A, SEED + 9), cuda)
    M = rpcg.Matrix.from_csr(A)
    outs = []
    for block, grid in [(256, 0), (128, 7), (512, 3), (256, 1), (128, 1000)]:
        x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            r = M.solve(b, x, variant=variant, block=block, grid=grid, stream=s)
        s.synchronize()
        outs.append((r["iterations"], bits(x.cpu().numpy()).tobytes(), bits([r["relres"]])[0]))
    assert len(set(outs)) == 1


def test_pcg_exblas_equals_fpe_small_p(rpcg, cuda, oracle_lib):
    """fpe with recompute-on-inexact follows the exact trajectory for any p."""
    import torch
    A = synth.diffusion7(8, SEED + 4)[0]
    b = _dev(_rhs(oracle_lib, A, SEED), cuda)
    M = rpcg.Matrix.from_csr(A)
    res = []
    for variant, p in [("exblas", 8), ("fpe", 1), ("fpe", 2), ("fpe", 8)]:
        x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
        r = M.solve(b, x, variant=variant, tol=1e-10, max_iter=2000, fpe_size=p)
        res.append((r["iterations"], bits(x.cpu().numpy()).tobytes()))
        if variant == "fpe" and p == 1:
            assert r["fpe_inexact_count"] > 0
    assert len(set(res)) == 1


@pytest.mark.parametrize("fpe_size", [1, 2, 0, 8])
@pytest.mark.parametrize("kw", [{}, {"block": 128, "grid": 37}])
def test_pcg_fpe_multipass_exact_trajectory(rpcg, cuda, oracle_lib, fpe_size, kw):
    """The multi-pass fpe solve (pass B as B1 + B2, part of the warps on the
    integer emulation) on systems too large for the cluster path: for every
    expansion size (1 and 2 lose bits in most dots and take the exact
    recomputation) the iterates, history and iteration count are the
    oracle's exact-dot ones, bit for bit."""
    import torch
    for A in (synth.poisson27(30), synth.diffusion7(27, SEED + 12)[0]):  # 27000 and 19683 rows
        M = rpcg.Matrix.from_csr(A)
        assert M.solve_path("fpe", **kw) == "graph"
        b = _rhs(oracle_lib, A, SEED + 13)
        ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-9, max_iter=3000, nthreads=4)
        x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
        hist = torch.full((3001,), float("nan"), dtype=torch.float64, device=cuda)
        r = M.solve(_dev(b, cuda), x, variant="fpe", tol=1e-9, max_iter=3000, fpe_size=fpe_size, history=hist, **kw)
        assert r["status"] == ref["status"] == 0
        assert r["iterations"] == ref["iterations"]
        assert np.array_equal(bits(x.cpu().numpy()), bits(ref["x"]))
        assert np.array_equal(bits(hist[: r["iterations"] + 1].cpu().numpy()), bits(ref["history"]))
        if fpe_size == 1:
            assert r["fpe_inexact_count"] > 0


def test_pcg_plain_converges(rpcg, cuda, oracle_lib):
    import torch
    A = synth.poisson7(16)
    b = _rhs(oracle_lib, A, SEED)
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-8)
    M = rpcg.Matrix.from_csr(A)
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    r = M.solve(_dev(b, cuda), x, variant="plain", tol=1e-8)
    assert r["status"] == 0 and r["relres"] < 1e-8
    assert abs(r["iterations"] - ref["iterations"]) <= max(1, 0.05 * ref["iterations"])
    assert np.allclose(x.cpu().numpy(), ref["x"], atol=1e-6)


def test_pcg_nonzero_x0_and_host_api(rpcg, cuda, oracle_lib):
    import torch
    A = synth.poisson27(8)
    b = _rhs(oracle_lib, A, SEED + 1)
    x0 = synth.uniform_pm1(SEED + 2, A.n)
    ref = oracle_lib.pcg(A, b, x0=x0, variant=oracle_lib.EXACT, tol=1e-9)
    M = rpcg.Matrix.from_csr(A)
    x = _dev(x0, cuda)
    r = M.solve(_dev(b, cuda), x, tol=1e-9)
    assert r["iterations"] == ref["iterations"]
    assert np.array_equal(bits(x.cpu().numpy()), bits(ref["x"]))
    xh = x0.copy()
    rh = M.solve_host(b, xh, tol=1e-9)
    assert rh == r and np.array_equal(bits(xh), bits(ref["x"]))


def test_pcg_edge_cases(rpcg, cuda, oracle_lib):
    import torch
    A = synth.poisson7(6)
    M = rpcg.Matrix.from_csr(A)
    # b = 0: x = 0 after 0 iterations
    x = torch.ones(A.n, dtype=torch.float64, device=cuda)
    r = M.solve(torch.zeros(A.n, dtype=torch.float64, device=cuda), x)
    assert r["status"] == 0 and r["iterations"] == 0 and not x.any().item()
    # max_iter = 0 -> not converged, x untouched
    b = _rhs(oracle_lib, A, SEED)
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    r = M.solve(_dev(b, cuda), x, max_iter=0)
    assert r["status"] == rpcg.NOT_CONVERGED and r["iterations"] == 0
    # a few iterations only: matches the oracle's truncated run
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-8, max_iter=3)
    r = M.solve(_dev(b, cuda), x, max_iter=3)
    assert r["status"] == ref["status"] == rpcg.NOT_CONVERGED and r["iterations"] == 3
    assert np.array_equal(bits(x.cpu().numpy()), bits(ref["x"]))
    # NaN in b
    bn = b.copy()
    bn[5] = math.nan
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    assert M.solve(_dev(bn, cuda), x)["status"] == rpcg.ERR_NONFINITE


def test_pcg_not_spd(rpcg, cuda, oracle_lib):
    import torch
    import scipy.sparse
    for Mx in (np.array([[1.0, 0.0], [0.0, -2.0]]), np.array([[1.0, 2.0], [2.0, 1.0]]),
               np.array([[1.0, 0.5], [0.5, 0.0]])):
        S = scipy.sparse.csr_matrix(Mx)
        S.sort_indices()
        A = synth.CSR(2, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))
        b = np.array([1.0, -1.0])
        ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-10, max_iter=10)
        M = rpcg.Matrix.from_csr(A)
        x = torch.zeros(2, dtype=torch.float64, device=cuda)
        r = M.solve(_dev(b, cuda), x, tol=1e-10, max_iter=10)
        assert r["status"] == ref["status"] == rpcg.ERR_NOT_SPD
        assert r["iterations"] == ref["iterations"]


def test_pcg_one_by_one_and_diagonal(rpcg, cuda, oracle_lib):
    import torch
    import scipy.sparse
    rng = np.random.default_rng(5)
    dvals = np.exp(rng.uniform(-5, 5, 300))
    S = scipy.sparse.csr_matrix(np.diag(dvals))
    A = synth.CSR(300, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))
    b = rng.uniform(-1, 1, 300)
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-12, max_iter=10)
    x = torch.zeros(300, dtype=torch.float64, device=cuda)
    r = rpcg.Matrix.from_csr(A).solve(_dev(b, cuda), x, tol=1e-12, max_iter=10)
    assert r["iterations"] == ref["iterations"] == 1
    assert np.array_equal(bits(x.cpu().numpy()), bits(ref["x"]))


def test_invalid_csr_rejected(rpcg, cuda):
    with pytest.raises(rpcg.RpcgError):
        rpcg.Matrix(np.array([0, 2, 3], np.int32), np.array([0, 5, 1], np.int32), np.ones(3))


@pytest.mark.parametrize("variant", ["exblas", "fpe", "plain"])
def test_profiled_solve_matches_graph_solve(rpcg, cuda, oracle_lib, variant):
    import torch
    A = synth.poisson27(10)
    b = _dev(_rhs(oracle_lib, A, SEED + 5), cuda)
    M = rpcg.Matrix.from_csr(A)
    x1 = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    x2 = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    # block 256 keeps the graph of grid-wide passes (the profiled form launches
    # the same kernels one by one; plain dots are only reproducible within a path)
    r1 = M.solve(b, x1, variant=variant, block=256)
    r2 = M.solve_profiled(b, x2, variant=variant)
    assert r1["iterations"] == r2["iterations"] == r2["launches"]["A"]
    assert np.array_equal(bits(x1.cpu().numpy()), bits(x2.cpu().numpy()))
    assert r2["pass_ms"]["A"] > 0


def test_band_matrix_spmv_and_pcg(rpcg, cuda, oracle_lib):
    """The band workload (rows of 2 bw + 1 entries) against the oracle."""
    import torch
    A = synth.band(3000, 40)
    x = synth.uniform_pm1(SEED + 11, A.n)
    M = rpcg.Matrix.from_csr(A)
    y = M.spmv(_dev(x, cuda)).cpu().numpy()
    assert np.array_equal(bits(y), bits(oracle_lib.spmv(A, x)))
    b = oracle_lib.spmv(A, np.ones(A.n))  # the paper's right-hand side: A times a vector of ones
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-8, max_iter=500)
    xd = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    r = M.solve(_dev(b, cuda), xd, tol=1e-8, max_iter=500)
    assert r["iterations"] == ref["iterations"] and r["status"] == 0
    assert np.array_equal(bits(xd.cpu().numpy()), bits(ref["x"]))


def test_pcg_fpe_adaptive_size(rpcg, cuda, oracle_lib):
    """fpe_size = 0 starts at 3 terms and grows after dots that lose bits;
    the trajectory stays the exact one."""
    import torch
    A = synth.diffusion7(9, SEED + 7)[0]
    b = _dev(_rhs(oracle_lib, A, SEED + 8), cuda)
    M = rpcg.Matrix.from_csr(A)
    xe = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    re = M.solve(b, xe, variant="exblas", tol=1e-10, max_iter=2000)
    xa = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    ra = M.solve(b, xa, variant="fpe", tol=1e-10, max_iter=2000, fpe_size=0)
    assert ra["iterations"] == re["iterations"]
    assert torch.equal(xa.view(torch.int64), xe.view(torch.int64))
    if ra["fpe_inexact_count"] == 0:
        assert ra["fpe_size_used"] == 3
    else:  # each finalisation that saw a lost dot adds one term
        assert 3 < ra["fpe_size_used"] <= min(8, 3 + ra["fpe_inexact_count"])
    x1 = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    r1 = M.solve(b, x1, variant="fpe", tol=1e-10, max_iter=2000, fpe_size=1)
    assert r1["fpe_size_used"] == 1 and r1["fpe_inexact_count"] > 0


def test_spmv_single_step_all_magnitudes(rpcg, cuda, oracle_lib):
    """A diagonal matrix makes every row a single step fma(a_ii, x_i, +0):
    normal, zero, subnormal, overflowing, infinite and NaN operands and
    results (and rounding ties) all equal the oracle's fma bit for bit (NaNs
    as NaNs)."""
    n = 1 << 20
    rng = np.random.default_rng(11)
    def draw(k):
        m = rng.uniform(1.0, 2.0, k) * rng.choice([-1.0, 1.0], k)
        e = rng.integers(-1074, 1024, k)
        v = np.ldexp(m, e)
        special = rng.random(k)
        v[special < 0.01] = 0.0
        v[(special >= 0.01) & (special < 0.015)] = -0.0
        v[(special >= 0.015) & (special < 0.02)] = np.inf
        v[(special >= 0.02) & (special < 0.022)] = np.nan
        v[(special >= 0.022) & (special < 0.05)] = np.ldexp(rng.uniform(0, 1, k), -1022)[(special >= 0.022) & (special < 0.05)]
        return v
    d, x = draw(n), draw(n)
    # products near the edges of the normal range and exact ties
    d[:1000] = np.ldexp(1.0 + np.arange(1000) * 2.0 ** -52, -511)
    x[:1000] = np.ldexp(1.0 + 2.0 ** -52, -511)
    d[1000:2000] = np.ldexp(1.5, 511)
    x[1000:2000] = np.ldexp(1.0 + np.arange(1000) * 2.0 ** -40, 512)
    A = synth.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    want = oracle_lib.spmv(A, x)
    got = rpcg.Matrix.from_csr(A).spmv(_dev(x, cuda)).cpu().numpy()
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(bits(got[~nan]), bits(want[~nan]))


@pytest.mark.parametrize("kw", [{}, {"block": 256}])
def test_pcg_storage_order_duplicates_and_stored_zeros(rpcg, cuda, oracle_lib, kw):
    """CSR as stored, not as a canonical matrix: columns unsorted within rows,
    explicitly stored zeros, and a diagonal entry stored twice (the last one
    in storage order is a_ii; the SpMV adds both).  Every row's fma chain
    follows storage order, so both solver paths match the oracle bit for bit."""
    import torch
    A0 = synth.poisson7(10)
    rng = np.random.default_rng(5)
    rowptr, cols, vals = [0], [], []
    for i in range(A0.n):
        c = list(A0.col[A0.rowptr[i]:A0.rowptr[i + 1]])
        v = list(A0.val[A0.rowptr[i]:A0.rowptr[i + 1]])
        perm = rng.permutation(len(c))
        c = [c[k] for k in perm]
        v = [v[k] for k in perm]
        if i % 3 == 0:                 # a stored zero
            c.append(c[0]); v.append(0.0)
        if i % 5 == 0:                 # the diagonal twice: 0.5 + 5.5 (the second one is a_ii)
            k = c.index(i)
            v[k] = 0.5
            c.append(i); v.append(5.5)
        rowptr.append(rowptr[-1] + len(c))
        cols += c
        vals += v
    A = synth.CSR(A0.n, np.array(rowptr, dtype=np.int32), np.array(cols, dtype=np.int32), np.array(vals))
    b = synth.rhs_uniform(A.n, SEED + 77)
    M = rpcg.Matrix.from_csr(A)
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    hist = torch.full((1001,), float("nan"), dtype=torch.float64, device=cuda)
    r = M.solve(_dev(b, cuda), x, variant="exblas", tol=1e-10, max_iter=1000, history=hist, **kw)
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-10, max_iter=1000)
    assert r["status"] == ref["status"] and r["iterations"] == ref["iterations"]
    assert np.array_equal(bits(x.cpu().numpy()), bits(ref["x"]))
    assert np.array_equal(bits(hist[: r["iterations"] + 1].cpu().numpy()), bits(ref["history"][: r["iterations"] + 1]))
    y = M.spmv(_dev(b, cuda)).cpu().numpy()
    assert np.array_equal(bits(y), bits(oracle_lib.spmv(A, b)))
