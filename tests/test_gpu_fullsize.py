"""Parity at the full benchmark sizes, in the launch configuration bench.py
times: exact dots of 2^28 elements against the oracle, and the 27-point
Poisson 256^3 solve -- its first iterations bit for bit against the oracle,
and properties of the complete solve that hold at any size."""
import numpy as np
import pytest

import synth
from conftest import bits

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def big_system(oracle_lib):
    A = synth.poisson27(256)
    xt = synth.poisson_rhs_xtrue(A.n, synth.BASE_SEED + 2)
    b = oracle_lib.spmv(A, xt, nthreads=oracle_lib.default_threads())
    return A, b


@pytest.mark.parametrize("fam", ["a", "b"])
def test_exact_dot_2p28(rpcg, cuda, oracle_lib, fam):
    import torch
    n = 1 << 28
    a, b = getattr(synth, f"dot_family_{fam}")(n, synth.BASE_SEED + 1)
    want = oracle_lib.dot_exact(a, b, nthreads=oracle_lib.default_threads())
    ta, tb = torch.from_numpy(a).to(cuda), torch.from_numpy(b).to(cuda)
    got = rpcg.dot_exact(ta, tb).item()
    assert bits([got])[0] == bits([want])[0]


def test_exact_dot_2p28_unaligned_view(rpcg, cuda, oracle_lib):
    """The instance for operands not on 16-byte boundaries (one element at a
    time) at the full size, where every thread spills its shared digits to
    the global ones more than once."""
    import torch
    n = 1 << 28
    a, b = synth.dot_family_a(n + 1, synth.BASE_SEED + 4)
    want = oracle_lib.dot_exact(a[1:], b[1:], nthreads=oracle_lib.default_threads())
    ta, tb = torch.from_numpy(a).to(cuda), torch.from_numpy(b).to(cuda)
    got = rpcg.dot_exact(ta[1:], tb[1:]).item()
    assert bits([got])[0] == bits([want])[0]


def test_exact_dot_family_c_2p26(rpcg, cuda, oracle_lib):
    import torch
    a, b = synth.dot_family_c(1 << 26, 1e32, synth.BASE_SEED + 1)
    want = oracle_lib.dot_exact(a, b, nthreads=oracle_lib.default_threads())
    got = rpcg.dot_exact(torch.from_numpy(a).to(cuda), torch.from_numpy(b).to(cuda)).item()
    assert bits([got])[0] == bits([want])[0]


def test_poisson27_256_first_iterations_bit_exact(rpcg, cuda, oracle_lib, big_system):
    import torch
    A, b = big_system
    k = 2
    ref = oracle_lib.pcg(A, b, variant=oracle_lib.EXACT, tol=1e-8, max_iter=k,
                         nthreads=oracle_lib.default_threads())
    M = rpcg.Matrix.from_csr(A)
    x = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    hist = torch.full((k + 1,), float("nan"), dtype=torch.float64, device=cuda)
    r = M.solve(torch.from_numpy(b).to(cuda), x, variant="exblas", tol=1e-8, max_iter=k, history=hist)
    assert r["iterations"] == ref["iterations"] == k
    assert np.array_equal(bits(hist.cpu().numpy()), bits(ref["history"]))
    assert np.array_equal(bits(x.cpu().numpy()), bits(ref["x"]))


def test_poisson27_256_full_solve_properties(rpcg, cuda, big_system):
    """Converges; the true residual recomputed independently meets the
    tolerance; exblas and fpe agree bit for bit; another launch shape gives
    the same bits."""
    import scipy.sparse
    import torch
    A, b = big_system
    M = rpcg.Matrix.from_csr(A)
    db = torch.from_numpy(b).to(cuda)
    x1 = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    r1 = M.solve(db, x1, variant="exblas", tol=1e-8, max_iter=5000)
    assert r1["status"] == 0 and r1["relres"] < 1e-8
    x = x1.cpu().numpy()
    S = scipy.sparse.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    true_rel = np.linalg.norm(b - S @ x) / np.linalg.norm(b)
    assert true_rel < 1e-8 * 1.01
    x2 = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    r2 = M.solve(db, x2, variant="exblas", tol=1e-8, max_iter=5000, block=128, grid=300)
    assert r2["iterations"] == r1["iterations"]
    assert torch.equal(x1.view(torch.int64), x2.view(torch.int64))
    x3 = torch.zeros(A.n, dtype=torch.float64, device=cuda)
    r3 = M.solve(db, x3, variant="fpe", tol=1e-8, max_iter=5000)
    assert r3["iterations"] == r1["iterations"]
    assert torch.equal(x1.view(torch.int64), x3.view(torch.int64))


def test_batch_256_full_config(rpcg, cuda, oracle_lib):
    """The batched configuration at its full size (256 diffusion systems,
    s ~ U{8..64}, tol 1e-10), autotuned as bench.py runs it: every system
    bit-identical to solving it alone, and sampled systems (the three
    smallest and one of median size) bit-identical to the oracle."""
    import torch
    mats, rhs = synth.diffusion_batch(256, synth.BASE_SEED + 3)
    Ms = [rpcg.Matrix.from_csr(A) for A in mats]
    bs = [torch.from_numpy(b).to(cuda) for b in rhs]
    xs = [torch.zeros(A.n, dtype=torch.float64, device=cuda) for A in mats]
    res = rpcg.Batch(Ms).solve(bs, xs, variant="exblas", tol=1e-10, max_iter=5000)
    assert all(r["status"] == 0 for r in res)
    for i, (M, b) in enumerate(zip(Ms, bs)):
        x = torch.zeros(M.n, dtype=torch.float64, device=cuda)
        r = M.solve(b, x, variant="exblas", tol=1e-10, max_iter=5000)
        assert r["iterations"] == res[i]["iterations"], i
        assert bits([r["relres"]])[0] == bits([res[i]["relres"]])[0], i
        assert torch.equal(x.view(torch.int64), xs[i].view(torch.int64)), i
    order = sorted(range(len(mats)), key=lambda k: mats[k].n)
    for i in order[:3] + [order[len(order) // 2]]:
        ref = oracle_lib.pcg(mats[i], rhs[i], variant=oracle_lib.EXACT, tol=1e-10, max_iter=5000,
                             nthreads=oracle_lib.default_threads())
        assert ref["iterations"] == res[i]["iterations"], i
        assert np.array_equal(bits(xs[i].cpu().numpy()), bits(ref["x"])), i
