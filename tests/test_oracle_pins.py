"""Pins for the CPU oracle: each check ties it to something other than
itself -- rational brute force, math.fsum, values worked by hand from the
paper's algorithms, closed-form eigenpairs, and library solvers."""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.linalg

import synth
from conftest import pcg_2x2_golden

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OVER = Fraction(2) ** 1024 * (1 - Fraction(1, 2 ** 54))


def rn(q: Fraction) -> float:
    """Round a rational to the nearest binary64, ties to even (Python's int
    true division is correctly rounded; overflow maps to +-inf)."""
    if q == 0:
        return 0.0
    if abs(q) >= OVER:
        return math.inf if q > 0 else -math.inf
    return q.numerator / q.denominator


def exact_dot_bruteforce(a, b) -> float:
    if not all(map(math.isfinite, list(a) + list(b))):
        return math.nan
    return rn(sum((Fraction(x) * Fraction(y) for x, y in zip(a, b)), Fraction(0)))


def rand_double(rng, lo=-1074, hi=1023):
    """A random double with an exponent spread from subnormal to huge."""
    e = rng.randint(lo, hi)
    m = rng.getrandbits(52)
    if e < -1022:
        v = math.ldexp(m, -1074)
    else:
        v = math.ldexp((1 << 52) | m, e - 52)
    return -v if rng.random() < 0.5 else v


def same(x: float, y: float) -> bool:
    if math.isnan(x) or math.isnan(y):
        return math.isnan(x) and math.isnan(y)
    return x == y and math.copysign(1, x) == math.copysign(1, y)


# ------------------------------------------------------------------ exact dot

def test_exact_dot_golden(oracle_lib):
    n = 0
    for line in open(os.path.join(GOLDEN, "exact_dot_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b, e = (part.split() for part in line.split(";"))
        a = [float.fromhex(t) for t in a]
        b = [float.fromhex(t) for t in b]
        want = float.fromhex(e[0]) if e[0] != "inf" else math.inf
        assert same(oracle_lib.dot_exact(a, b), want), line
        assert same(exact_dot_bruteforce(a, b), want), line
        n += 1
    assert n >= 10


@pytest.mark.parametrize("seed", range(12))
def test_exact_dot_vs_fraction_wide(oracle_lib, seed):
    rng = random.Random(seed)
    n = rng.choice([1, 2, 3, 7, 16, 33, 64])
    # exponents spread so that some products are subnormal and none overflow
    a = [rand_double(rng, -1074, 500) for _ in range(n)]
    b = [rand_double(rng, -1074, 500) for _ in range(n)]
    assert same(oracle_lib.dot_exact(a, b), exact_dot_bruteforce(a, b))


@pytest.mark.parametrize("seed", range(8))
def test_exact_dot_vs_fraction_clustered(oracle_lib, seed):
    """Narrow exponent range with heavy cancellation (many ties likely)."""
    rng = random.Random(100 + seed)
    n = 64
    a = [rng.choice([-1, 1]) * rng.randint(1, 2 ** 27) * 2.0 ** rng.randint(-30, -20) for _ in range(n)]
    b = [rng.choice([-1, 1]) * rng.randint(1, 2 ** 27) * 2.0 ** rng.randint(-30, -20) for _ in range(n)]
    a += [-x for x in a[: n // 2]]
    b += b[: n // 2]
    assert same(oracle_lib.dot_exact(a, b), exact_dot_bruteforce(a, b))


def test_exact_dot_extreme_exponents(oracle_lib):
    rng = random.Random(7)
    for _ in range(40):
        n = rng.randint(1, 12)
        a = [rand_double(rng, -1074, 1023) for _ in range(n)]
        b = [rand_double(rng, -1074, 0) for _ in range(n)]
        assert same(oracle_lib.dot_exact(a, b), exact_dot_bruteforce(a, b))


def test_exact_dot_single_pair_is_hardware_product(oracle_lib):
    rng = random.Random(11)
    for _ in range(500):
        a, b = rand_double(rng, -600, 500), rand_double(rng, -600, 500)
        p = a * b
        want = 0.0 if (a == 0 or b == 0) else p
        assert same(oracle_lib.dot_exact([a], [b]), want)


def test_exact_dot_is_fsum_with_unit_weights(oracle_lib):
    rng = np.random.default_rng(3)
    for n in (1, 10, 1000, 20000):
        x = rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, n))
        assert oracle_lib.dot_exact(x, np.ones(n)) == math.fsum(x)
        assert oracle_lib.sum_exact(x) == math.fsum(x)


def test_exact_dot_counts_and_cancellation(oracle_lib):
    for n in (0, 1, 5, 4096, 100000):
        assert oracle_lib.dot_exact(np.ones(n), np.ones(n)) == float(n)
    x = synth.uniform_pm1(5, 5000)
    v = oracle_lib.dot_exact(np.concatenate([x, -x]), np.concatenate([x, x]))
    assert same(v, 0.0)


def test_exact_dot_nonfinite(oracle_lib):
    assert math.isnan(oracle_lib.dot_exact([1.0, math.inf], [1.0, 1.0]))
    assert math.isnan(oracle_lib.dot_exact([1.0, math.nan], [1.0, 0.0]))


def test_exact_dot_thread_count_independent(oracle_lib):
    for fam in ("a", "b"):
        x, y = getattr(synth, f"dot_family_{fam}")(100003, 17)
        vals = {oracle_lib.dot_exact(x, y, nthreads=t) for t in (1, 2, 3, 8, 13)}
        assert len(vals) == 1


@pytest.mark.parametrize("fam", ["a", "b"])
def test_exact_dot_families_vs_fraction(oracle_lib, fam):
    x, y = getattr(synth, f"dot_family_{fam}")(3000, 5)
    assert same(oracle_lib.dot_exact(x, y), exact_dot_bruteforce(x.tolist(), y.tolist()))


def test_exact_dot_family_c_vs_fraction(oracle_lib):
    for cond in (1e8, 1e24, 1e40):
        x, y = synth.dot_family_c(2000, cond, 9)
        assert same(oracle_lib.dot_exact(x, y), exact_dot_bruteforce(x.tolist(), y.tolist()))


# ---------------------------------------------------------------- EFTs, FPEs

def test_twosum_error_free(oracle_lib):
    rng = random.Random(21)
    for _ in range(3000):
        a, b = rand_double(rng, -300, 300), rand_double(rng, -300, 300)
        r, s = oracle_lib.twosum(a, b)
        assert r == a + b
        assert Fraction(r) + Fraction(s) == Fraction(a) + Fraction(b)


def test_twoprod_error_free(oracle_lib):
    rng = random.Random(22)
    for _ in range(3000):
        a, b = rand_double(rng, -400, 400), rand_double(rng, -400, 400)
        r, s = oracle_lib.twoprod(a, b)
        assert r == a * b
        if abs(r) >= 2.0 ** -969:
            assert Fraction(r) + Fraction(s) == Fraction(a) * Fraction(b)


def _parse_fpe_golden():
    for line in open(os.path.join(GOLDEN, "fpe_accumulate.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        p, before, x, after, out = (t.strip() for t in line.split("|"))
        yield (int(p), [float.fromhex(t) for t in before.split()], float.fromhex(x),
               [float.fromhex(t) for t in after.split()], float.fromhex(out))


def test_fpe_accumulate_golden(oracle_lib):
    cases = list(_parse_fpe_golden())
    assert len(cases) >= 6
    for p, before, x, after, out in cases:
        a = np.array(before, dtype=np.float64)
        carried = oracle_lib.fpe_accumulate(a, x)
        assert [same(u, v) for u, v in zip(a.tolist(), after)] == [True] * p
        assert same(carried, out)


def test_fpe_accumulate_invariant(oracle_lib):
    """sum(after) + carried == sum(before) + x exactly (Alg. 4 is error free)."""
    rng = random.Random(23)
    for p in (1, 2, 3, 8):
        a = np.zeros(p)
        for _ in range(400):
            x = rand_double(rng, -200, 200)
            before = sum(map(Fraction, a.tolist()), Fraction(0))
            c = oracle_lib.fpe_accumulate(a, x)
            after = sum(map(Fraction, a.tolist()), Fraction(0))
            assert after + Fraction(c) == before + Fraction(x)


def _parse_fpesum_golden():
    for line in open(os.path.join(GOLDEN, "fpesum.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        p, a, b, after, lost = (t.strip() for t in line.split("|"))
        yield (int(p), [float.fromhex(t) for t in a.split()], [float.fromhex(t) for t in b.split()],
               [float.fromhex(t) for t in after.split()], bool(int(lost)))


def test_fpesum_golden(oracle_lib):
    """Alg. 3 on multi-term expansions, worked by hand: term order of b,
    cancellation leaving overlapping terms, and losses at p = 1, 2, 3."""
    cases = list(_parse_fpesum_golden())
    assert len(cases) >= 8
    for p, a, b, after, lost in cases:
        assert len(a) == len(b) == len(after) == p
        x = np.array(a, dtype=np.float64)
        got_lost = oracle_lib.fpesum(x, np.array(b, dtype=np.float64))
        assert [same(u, v) for u, v in zip(x.tolist(), after)] == [True] * p, (a, b, x.tolist(), after)
        assert got_lost == lost, (a, b)


def test_pcg_2x2_hand_worked_trace(oracle_lib):
    """Every scalar and vector of two loop bodies (Fig. 1/Fig. 2 with the
    fma forms of Sec. 4.3) against a trace worked out by hand with exact
    rational arithmetic.  The system is chosen so that each single-rounding
    form differs from its two-rounding neighbour somewhere (r, x, d) and the
    Jacobi multiply by RN(1/a_ii) differs from a division by a_ii."""
    A, b, want = pcg_2x2_golden()
    got = oracle_lib.pcg_trace(A, b, tol=0.0, max_iter=2)
    assert got["status"] == oracle_lib.NOT_CONVERGED and got["iterations"] == 2
    assert sorted(want) == [0, 1, 2]
    for l, names in want.items():
        rec = got["trace"][l]
        for name, vals in names.items():
            have = np.atleast_1d(rec[name]).tolist()
            assert [same(u, v) for u, v in zip(have, vals)] == [True] * len(vals), (l, name, have, vals)


def test_fpesum_invariant(oracle_lib):
    rng = random.Random(24)
    for p in (2, 3, 8):
        for _ in range(100):
            a = np.zeros(p)
            b = np.zeros(p)
            for _ in range(5):
                oracle_lib.fpe_accumulate(a, rand_double(rng, -100, 100))
                oracle_lib.fpe_accumulate(b, rand_double(rng, -100, 100))
            total = sum(map(Fraction, a.tolist() + b.tolist()), Fraction(0))
            lost = oracle_lib.fpesum(a, b)
            if not lost:
                assert sum(map(Fraction, a.tolist()), Fraction(0)) == total


def test_fpe_one_product_identities(oracle_lib):
    """The identities a thread holding one product relies on (Algs. 2-4):
    Alg. 4 into an empty expansion stores the value whole and carries
    nothing out; Alg. 3 of the twoprod pair's one-term expansions (r) and
    (s) is one twosum whose error becomes the second term, lost only when
    p = 1.  Checked against the oracle's own Algs. 3 and 4 and against
    rational arithmetic."""
    rng = random.Random(31)
    for _ in range(3000):
        a, b = rand_double(rng, -300, 300), rand_double(rng, -300, 300)
        r, s = oracle_lib.twoprod(a, b)
        assert Fraction(r) + Fraction(s) == Fraction(a) * Fraction(b)  # exponents keep the error representable
        for p in (1, 2, 3, 8):
            res, err = np.zeros(p), np.zeros(p)
            assert oracle_lib.fpe_accumulate(res, r) == 0.0 and res[0] == r and not res[1:].any()
            if s != 0.0:
                assert oracle_lib.fpe_accumulate(err, s) == 0.0 and err[0] == s
            lost = oracle_lib.fpesum(res, err)
            r1, s1 = oracle_lib.twosum(r, s)
            assert same(res[0], r1)
            if p >= 2:
                assert not lost and (same(res[1], s1) or (s1 == 0.0 and res[1] == 0.0))
                assert Fraction(res[0]) + Fraction(res[1]) == Fraction(a) * Fraction(b)
            else:
                assert lost == (s1 != 0.0)


@pytest.mark.parametrize("fam", ["a", "c8", "c16"])
@pytest.mark.parametrize("T", [1, 4, 7])
def test_fpe_dot_equals_exact_when_flagged(oracle_lib, fam, T):
    if fam == "a":
        x, y = synth.dot_family_a(5000, 31)
    else:
        x, y = synth.dot_family_c(5000, 1e8 if fam == "c8" else 1e16, 31)
    v, flag = oracle_lib.dot_fpe(x, y, p=8, T=T)
    assert flag
    assert same(v, oracle_lib.dot_exact(x, y))
    assert same(v, exact_dot_bruteforce(x.tolist(), y.tolist()))


def test_fpe_dot_flag_forced_off(oracle_lib):
    x, y = synth.dot_family_c(4000, 1e40, 32)
    v, flag = oracle_lib.dot_fpe(x, y, p=2, T=1)
    assert not flag
    # the tiny-product case: twoprod cannot keep its error term
    v, flag = oracle_lib.dot_fpe([2.0 ** -500, 1.0], [2.0 ** -500, 1.0], p=8, T=1)
    assert not flag
    v, flag = oracle_lib.dot_fpe([1.0, math.inf], [1.0, 1.0], p=8, T=1)
    assert not flag and math.isnan(v)


def test_fpe_size3_is_enough_on_poisson_vectors(oracle_lib):
    """Sec. 4.3: FPE3 keeps every bit for Poisson-type dots (checked here on
    the dots of the first PCG step of a 7-point Poisson system)."""
    A = synth.poisson7(12)
    xt = synth.poisson_rhs_xtrue(A.n, 1)
    b = oracle_lib.spmv(A, xt)
    v, flag = oracle_lib.dot_fpe(b, b, p=3, T=4)
    assert flag and v == oracle_lib.dot_exact(b, b)


# ---------------------------------------------------------------- SpMV

def _fma_chain_fraction(vals, xs):
    acc = 0.0
    for v, x in zip(vals, xs):
        acc = rn(Fraction(v) * Fraction(x) + Fraction(acc))
        if acc == 0.0:
            acc = 0.0  # fma(v, x, +0) with an exact-zero result is +0 unless both are -0
    return acc


def test_spmv_fma_chain_bruteforce(oracle_lib):
    A, _ = synth.diffusion7(5, 3)
    x = synth.uniform_pm1(44, A.n)
    y = oracle_lib.spmv(A, x)
    for i in range(A.n):
        lo, hi = A.rowptr[i], A.rowptr[i + 1]
        want = _fma_chain_fraction(A.val[lo:hi].tolist(), x[A.col[lo:hi]].tolist())
        assert y[i] == want


@pytest.mark.parametrize("kind", ["7", "27"])
def test_spmv_poisson_eigenpairs(oracle_lib, kind):
    s = 12
    A = synth.poisson7(s) if kind == "7" else synth.poisson27(s)
    g = np.arange(1, s + 1) / (s + 1)
    for (j, k, l) in [(1, 1, 1), (2, 3, 5), (s, 1, 7), (4, 4, 4)]:
        vx, vy, vz = np.sin(j * np.pi * g), np.sin(k * np.pi * g), np.sin(l * np.pi * g)
        v = (vz[:, None, None] * vy[None, :, None] * vx[None, None, :]).reshape(-1)
        th = np.pi * np.array([j, k, l]) / (s + 1)
        if kind == "7":
            lam = 6 - 2 * np.cos(th).sum()
        else:
            lam = 27 - np.prod(1 + 2 * np.cos(th))
        Av = oracle_lib.spmv(A, v)
        assert np.linalg.norm(Av - lam * v) / np.linalg.norm(lam * v) <= 1e-12


def test_spmv_threads_and_scipy(oracle_lib):
    A = synth.poisson27(10)
    x = synth.uniform_pm1(3, A.n)
    y1 = oracle_lib.spmv(A, x, nthreads=1)
    y4 = oracle_lib.spmv(A, x, nthreads=5)
    assert np.array_equal(y1, y4)
    S = scipy.sparse.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    assert np.allclose(S @ x, y1, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- PCG

def _csr_from_dense(M):
    S = scipy.sparse.csr_matrix(M)
    S.sort_indices()
    return synth.CSR(M.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def test_pcg_diagonal_converges_in_one_iteration(oracle_lib):
    rng = np.random.default_rng(5)
    dvals = np.exp(rng.uniform(-5, 5, 50))
    A = _csr_from_dense(np.diag(dvals))
    b = rng.uniform(-1, 1, 50)
    r = oracle_lib.pcg(A, b, tol=1e-12, max_iter=10)
    assert r["status"] == 0 and r["iterations"] == 1
    assert np.allclose(r["x"], b / dvals, rtol=1e-15)


def test_pcg_one_by_one(oracle_lib):
    for a, b in [(3.0, 7.0), (1e-3, 2.5), (7.25, -1e5)]:
        r = oracle_lib.pcg(_csr_from_dense(np.array([[a]])), np.array([b]), tol=1e-14, max_iter=5)
        assert r["status"] == 0 and r["iterations"] == 1
        assert abs(r["x"][0] - b / a) <= 2 * np.spacing(abs(b / a))


def test_pcg_zero_rhs(oracle_lib):
    A = synth.poisson7(4)
    r = oracle_lib.pcg(A, np.zeros(A.n), x0=np.ones(A.n), tol=1e-8)
    assert r["status"] == 0 and r["iterations"] == 0 and not r["x"].any()


def test_pcg_finite_termination_small_spd(oracle_lib):
    """CG on an n x n SPD system reaches a tiny residual in about n steps."""
    rng = np.random.default_rng(9)
    for n in (3, 5, 8):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        M = Q @ np.diag(np.linspace(1, 4, n)) @ Q.T
        M = (M + M.T) / 2
        A = _csr_from_dense(M)
        b = rng.uniform(-1, 1, n)
        r = oracle_lib.pcg(A, b, tol=1e-13, max_iter=4 * n)
        assert r["status"] == 0 and r["iterations"] <= n + 3
        assert np.allclose(M @ r["x"], b, atol=1e-11)


@pytest.mark.parametrize("variant", [0, 1])
def test_pcg_poisson_vs_scipy_cg(oracle_lib, variant):
    A = synth.poisson7(16)
    xt = synth.poisson_rhs_xtrue(A.n, 2005072820)
    b = oracle_lib.spmv(A, xt)
    r = oracle_lib.pcg(A, b, variant=variant, tol=1e-8, max_iter=1000)
    assert r["status"] == 0
    S = scipy.sparse.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    res = np.linalg.norm(b - S @ r["x"]) / np.linalg.norm(b)
    assert res < 1e-8 * 1.01
    assert r["relres"] < 1e-8 and r["history"][-1] == r["relres"]
    iters = []
    Minv = scipy.sparse.diags(1.0 / S.diagonal())
    x_sp, info = scipy.sparse.linalg.cg(S, b, rtol=1e-8, maxiter=1000, M=Minv,
                                        callback=lambda xk: iters.append(1))
    assert info == 0
    assert abs(len(iters) - r["iterations"]) <= max(2, 0.05 * r["iterations"])
    assert np.allclose(r["x"], x_sp, atol=1e-6)


def test_pcg_threads_bit_identical(oracle_lib):
    A, _ = synth.diffusion7(10, 4)
    b = synth.rhs_uniform(A.n, 4)
    r1 = oracle_lib.pcg(A, b, tol=1e-10, max_iter=2000, nthreads=1)
    r5 = oracle_lib.pcg(A, b, tol=1e-10, max_iter=2000, nthreads=5)
    assert r1["iterations"] == r5["iterations"]
    assert np.array_equal(r1["x"], r5["x"]) and np.array_equal(r1["history"], r5["history"])


def test_pcg_not_spd_detected(oracle_lib):
    A = _csr_from_dense(np.array([[1.0, 0.0], [0.0, -2.0]]))
    r = oracle_lib.pcg(A, np.array([1.0, 1.0]), tol=1e-10)
    assert r["status"] == -2
    A = _csr_from_dense(np.array([[1.0, 2.0], [2.0, 1.0]]))  # indefinite, positive diagonal
    r = oracle_lib.pcg(A, np.array([1.0, -1.0]), tol=1e-10, max_iter=10)
    assert r["status"] == -2


def test_pcg_exact_and_plain_agree_closely(oracle_lib):
    A = synth.poisson27(12)
    xt = synth.poisson_rhs_xtrue(A.n, 77)
    b = oracle_lib.spmv(A, xt)
    re = oracle_lib.pcg(A, b, variant=1, tol=1e-8)
    rp = oracle_lib.pcg(A, b, variant=0, tol=1e-8)
    assert re["status"] == rp["status"] == 0
    assert abs(re["iterations"] - rp["iterations"]) <= max(1, 0.05 * re["iterations"])
