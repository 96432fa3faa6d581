"""The cluster-resident path for small systems (one launch of a thread-block
cluster runs the whole solve): bit-identical to the graph of grid-wide
passes and to the oracle, for the same statuses and edge cases."""
import numpy as np
import pytest
import scipy.sparse

import synth
from conftest import bits, pcg_2x2_golden

pytestmark = pytest.mark.gpu

SEED = synth.BASE_SEED + 11


def _dev(x, cuda):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(cuda)


def _csr_dense(M):
    S = scipy.sparse.csr_matrix(M)
    S.sort_indices()
    return synth.CSR(M.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def _system(kind):
    if kind == "p7_16":          # the 16^3 7-point system (4096 rows)
        return synth.poisson7(16)
    if kind == "p27_10":
        return synth.poisson27(10)
    if kind == "diff_9":
        return synth.diffusion7(9, SEED)[0]
    if kind == "p7_25":          # 15625 rows: 16 CTAs of 1024 rows, the last one partial
        return synth.poisson7(25)
    if kind == "p7_3":           # 27 rows: one CTA
        return synth.poisson7(3)
    if kind == "one":
        return _csr_dense(np.array([[4.0]]))
    if kind == "band":
        return synth.band(3000, 6)
    raise KeyError(kind)


def _solve(M, b, cuda, variant, x0=None, **kw):
    import torch
    n = M.n
    x = torch.zeros(n, dtype=torch.float64, device=cuda) if x0 is None else _dev(x0, cuda)
    maxit = kw.get("max_iter", 3000)
    hist = torch.full((maxit + 1,), float("nan"), dtype=torch.float64, device=cuda)
    r = M.solve(_dev(b, cuda), x, variant=variant, history=hist, **kw)
    h = hist[: max(r["iterations"], 0) + 1].cpu().numpy()
    return r, x.cpu().numpy(), h


@pytest.mark.parametrize("kind", ["p7_16", "p27_10", "diff_9", "p7_25", "p7_3", "one", "band"])
def test_cluster_equals_graph_and_oracle(rpcg, cuda, oracle_lib, kind):
    A = _system(kind)
    b = oracle_lib.spmv(A, synth.poisson_rhs_xtrue(A.n, SEED + 1))
    M = rpcg.Matrix.from_csr(A)
    assert M.solve_path("exblas") == "cluster"
    assert M.solve_path("exblas", block=256) == "graph"
    assert M.solve_path("fpe") == "cluster"
    assert M.solve_path("fpe", grid=4) == "graph"
    kw = dict(tol=1e-10, max_iter=3000)
    rc, xc, hc = _solve(M, b, cuda, "exblas", **kw)
    rg, xg, hg = _solve(M, b, cuda, "exblas", block=256, **kw)
    assert M.solve_path("exblas") == "cluster"  # the cluster was resident
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-10, max_iter=3000, nthreads=4)
    assert rc["status"] == rg["status"] == ref["status"] == 0
    assert rc["iterations"] == rg["iterations"] == ref["iterations"]
    assert np.array_equal(bits(xc), bits(xg)) and np.array_equal(bits(xc), bits(ref["x"]))
    assert np.array_equal(bits(hc), bits(hg)) and np.array_equal(bits(hc), bits(ref["history"]))
    assert bits([rc["relres"]])[0] == bits([ref["relres"]])[0]
    assert bits([rc["tau"]])[0] == bits([rg["tau"]])[0]


def test_cluster_too_large_takes_graph(rpcg, cuda):
    M = rpcg.Matrix.from_csr(synth.poisson7(26))  # 17576 rows
    assert M.solve_path("exblas") == "graph"
    # 27-point rows at 16384 rows do not fit the shared-memory slabs either
    M2 = rpcg.Matrix.from_csr(synth.poisson27(25))
    assert M2.solve_path("exblas") == "graph"


def test_cluster_nonzero_x0_host_api_and_fpe(rpcg, cuda, oracle_lib):
    A = synth.diffusion7(10, SEED + 2)[0]
    b = synth.rhs_uniform(A.n, SEED + 3)
    x0 = synth.uniform_pm1(SEED + 4, A.n)
    M = rpcg.Matrix.from_csr(A)
    ref = oracle_lib.pcg(A, b, x0=x0, variant=oracle_lib.EXACT, tol=1e-9, max_iter=3000, nthreads=4)
    rc, xc, _ = _solve(M, b, cuda, "exblas", x0=x0, tol=1e-9, max_iter=3000)
    assert rc["iterations"] == ref["iterations"] and np.array_equal(bits(xc), bits(ref["x"]))
    xh = x0.copy()
    rh = M.solve_host(b, xh, variant="exblas", tol=1e-9, max_iter=3000)
    assert rh["iterations"] == ref["iterations"] and np.array_equal(bits(xh), bits(ref["x"]))
    # fpe (exact recompute on inexact dots) lands on the same bits, on both paths
    rf, xf, _ = _solve(M, b, cuda, "fpe", x0=x0, tol=1e-9, max_iter=3000)
    assert rf["iterations"] == ref["iterations"] and np.array_equal(bits(xf), bits(ref["x"]))
    rg, xg, _ = _solve(M, b, cuda, "fpe", x0=x0, block=256, tol=1e-9, max_iter=3000)
    assert rg["iterations"] == ref["iterations"] and np.array_equal(bits(xg), bits(ref["x"]))


@pytest.mark.parametrize("kind", ["p7_16", "p27_10", "diff_9", "p7_25", "band"])
@pytest.mark.parametrize("fpe_size", [1, 2, 8, 0])
def test_cluster_fpe_follows_the_exact_trajectory(rpcg, cuda, oracle_lib, kind, fpe_size):
    """The fpe variant on the cluster path: per-thread expansions of Algs. 2-4
    whose terms meet exactly in the long accumulator; a dot whose expansions
    lost bits is recomputed exactly, so every size (and the adaptive one,
    fpe_size = 0) follows the oracle's exact-dot trajectory bit for bit."""
    A = _system(kind)
    b = oracle_lib.spmv(A, synth.poisson_rhs_xtrue(A.n, SEED + 21))
    M = rpcg.Matrix.from_csr(A)
    assert M.solve_path("fpe") == "cluster"
    kw = dict(tol=1e-10, max_iter=3000)
    r, x, h = _solve(M, b, cuda, "fpe", fpe_size=fpe_size, **kw)
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, nthreads=4, **kw)
    assert r["status"] == ref["status"] == 0
    assert r["iterations"] == ref["iterations"]
    assert np.array_equal(bits(x), bits(ref["x"])) and np.array_equal(bits(h), bits(ref["history"]))
    assert bits([r["relres"]])[0] == bits([ref["relres"]])[0]
    if fpe_size == 1:  # one term cannot hold a product's rounding error
        assert r["fpe_inexact_count"] > 0 and r["fpe_size_used"] == 1
    elif fpe_size == 0:
        n = r["fpe_inexact_count"]  # each phase that saw an inexact dot adds one term
        assert r["fpe_size_used"] == 3 if n == 0 else 3 < r["fpe_size_used"] <= min(8, 3 + n)
    else:
        assert r["fpe_size_used"] == fpe_size


def test_cluster_fpe_strict(rpcg, cuda, oracle_lib):
    """fpe_strict = 1: inexact dots are reported, not recomputed.  With 8
    terms nothing is lost on the 16^3 system and the result is the exact
    trajectory; with one term the solve still converges and reports
    RPCG_FPE_INEXACT with the count, as the multi-pass path does."""
    A = _system("p7_16")
    b = oracle_lib.spmv(A, synth.poisson_rhs_xtrue(A.n, SEED + 22))
    M = rpcg.Matrix.from_csr(A)
    kw = dict(tol=1e-10, max_iter=3000)
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, nthreads=4, **kw)
    r8, x8, _ = _solve(M, b, cuda, "fpe", fpe_size=8, fpe_strict=1, **kw)
    assert r8["status"] == 0 and r8["fpe_inexact_count"] == 0
    assert r8["iterations"] == ref["iterations"] and np.array_equal(bits(x8), bits(ref["x"]))
    r1, x1, _ = _solve(M, b, cuda, "fpe", fpe_size=1, fpe_strict=1, **kw)
    assert r1["status"] == rpcg.FPE_INEXACT and r1["fpe_inexact_count"] > 0
    assert r1["relres"] < 1e-10 and abs(r1["iterations"] - ref["iterations"]) <= 3
    g1, _, _ = _solve(M, b, cuda, "fpe", fpe_size=1, fpe_strict=1, block=256, **kw)
    assert g1["status"] == rpcg.FPE_INEXACT and g1["fpe_inexact_count"] > 0


def _edge_cases():
    A7 = synth.poisson7(6)
    n = A7.n
    neg = _csr_dense(np.diag([2.0, -1.0, 3.0]))                     # a_22 < 0
    nodiag = _csr_dense(np.array([[2.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 2.0]]))
    indef = _csr_dense(np.array([[1.0, 2.0], [2.0, 1.0]]))          # <d,w> <= 0 at some step
    b_nan = synth.rhs_uniform(n, 5)
    b_nan[7] = np.nan
    return [
        ("b zero", A7, np.zeros(n), None, dict(tol=1e-8, max_iter=100)),
        ("max_iter 0", A7, synth.rhs_uniform(n, 6), None, dict(tol=1e-8, max_iter=0)),
        ("max_iter 3", A7, synth.rhs_uniform(n, 7), None, dict(tol=1e-14, max_iter=3)),
        ("tol 0", A7, synth.rhs_uniform(n, 8), None, dict(tol=0.0, max_iter=40)),
        ("nan in b", A7, b_nan, None, dict(tol=1e-8, max_iter=100)),
        ("negative diagonal", neg, np.array([1.0, 1.0, 1.0]), None, dict(tol=1e-8, max_iter=100)),
        ("missing diagonal", nodiag, np.array([1.0, 2.0, 3.0]), None, dict(tol=1e-8, max_iter=100)),
        ("indefinite", indef, np.array([1.0, -1.0]), np.ones(2), dict(tol=1e-10, max_iter=50)),
        ("converged at x0", A7, np.zeros(n) + 1.0, None, dict(tol=1e30, max_iter=100)),
    ]


@pytest.mark.parametrize("variant", ["exblas", "fpe"])
@pytest.mark.parametrize("case", range(9))
def test_cluster_edge_cases_match_graph_and_oracle(rpcg, cuda, oracle_lib, case, variant):
    name, A, b, x0, kw = _edge_cases()[case]
    M = rpcg.Matrix.from_csr(A)
    assert M.solve_path(variant) == "cluster"
    rc, xc, hc = _solve(M, b, cuda, variant, x0=x0, **kw)
    rg, xg, hg = _solve(M, b, cuda, variant, x0=x0, block=128, **kw)
    assert rc["status"] == rg["status"], name
    assert rc["iterations"] == rg["iterations"], name
    assert np.array_equal(bits(xc), bits(xg)), name
    if rc["status"] >= 0:
        assert np.array_equal(bits(hc), bits(hg)), name
    ref = oracle_lib.pcg(A, b, x0=x0, variant=oracle_lib.EXACT, **kw)
    assert rc["status"] == ref["status"], (name, rc, ref["status"])
    assert rc["iterations"] == ref["iterations"], name
    if ref["status"] >= 0:
        assert np.array_equal(bits(xc), bits(ref["x"])), name


def test_cluster_plain_converges_and_is_deterministic(rpcg, cuda, oracle_lib):
    A = synth.poisson7(16)
    b = oracle_lib.spmv(A, synth.poisson_rhs_xtrue(A.n, SEED + 9))
    M = rpcg.Matrix.from_csr(A)
    assert M.solve_path("plain") == "cluster"
    r1, x1, h1 = _solve(M, b, cuda, "plain", tol=1e-8, max_iter=1000)
    r2, x2, h2 = _solve(M, b, cuda, "plain", tol=1e-8, max_iter=1000)
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-8, max_iter=1000)
    assert r1["status"] == 0 and r1["relres"] < 1e-8
    assert abs(r1["iterations"] - ref["iterations"]) <= max(2, ref["iterations"] // 20)
    assert r1["iterations"] == r2["iterations"] and np.array_equal(bits(x1), bits(x2))
    assert np.array_equal(bits(h1), bits(h2))


@pytest.mark.parametrize("n", [16384, 16385, 16383, 1025])
def test_cluster_size_boundary(rpcg, cuda, oracle_lib, n):
    """Band systems (7 entries per row) at the cluster path's limit: 16384 rows
    fill 16 CTAs of 1024 rows exactly; 16385 rows take the graph path; 16383 and
    1025 leave a ragged last CTA.  Both paths agree with the oracle."""
    A = synth.band(n, 3)
    b = synth.rhs_uniform(n, SEED + n)
    M = rpcg.Matrix.from_csr(A)
    assert M.solve_path("exblas") == ("graph" if n > 16384 else "cluster")
    rc, xc, hc = _solve(M, b, cuda, "exblas", tol=1e-12, max_iter=200)
    rg, xg, hg = _solve(M, b, cuda, "exblas", block=256, tol=1e-12, max_iter=200)
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-12, max_iter=200, nthreads=4)
    assert rc["iterations"] == rg["iterations"] == ref["iterations"]
    assert np.array_equal(bits(xc), bits(ref["x"])) and np.array_equal(bits(xg), bits(ref["x"]))
    assert np.array_equal(bits(hc), bits(ref["history"]))


@pytest.mark.parametrize("variant", ["exblas", "fpe"])
@pytest.mark.parametrize("path", ["cluster", "graph"])
def test_2x2_hand_worked_trace(rpcg, cuda, variant, path):
    """The CUDA solve of the 2x2 system of tests/golden/pcg_2x2_trace.txt
    after one and after two loop bodies: x, tau and every relres equal the
    trace worked out by hand (exact rational arithmetic, one rounding per
    operation with the fma forms of Sec. 4.3), on both paths."""
    A, b, want = pcg_2x2_golden()
    M = rpcg.Matrix.from_csr(A)
    kw = {} if path == "cluster" else dict(block=128, grid=1)
    assert M.solve_path(variant, **kw) == path
    for its in (1, 2):
        r, x, h = _solve(M, b, cuda, variant, tol=0.0, max_iter=its, **kw)
        assert r["status"] == rpcg.NOT_CONVERGED and r["iterations"] == its
        assert np.array_equal(bits(x), bits(want[its]["x"]))
        assert bits([r["tau"]])[0] == bits(want[its]["tau"])[0]
        assert np.array_equal(bits(h), bits([want[l]["relres"][0] for l in range(its + 1)]))
    M.close()
