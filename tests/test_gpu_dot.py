"""GPU parity of the three dot products against the CPU oracle (exact
results compared bit for bit; element-by-element inputs shared through the
seeded generators)."""
import math
import os
import random

import numpy as np
import pytest

import synth
from conftest import bits

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIZES = [0, 1, 2, 3, 31, 257, 4097, 65537, 1000003]  # several tiles and ragged tails


def _dev(x, cuda):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(cuda)


def _exact_gpu(rpcg, a, b, cuda):
    return rpcg.dot_exact(_dev(a, cuda), _dev(b, cuda)).item()


def same(x, y):
    return bits([x])[0] == bits([y])[0] or (math.isnan(x) and math.isnan(y))


@pytest.mark.parametrize("fam", ["a", "b", "c8", "c24", "c40"])
@pytest.mark.parametrize("n", SIZES)
def test_dot_exact_families(rpcg, cuda, oracle_lib, fam, n):
    if fam.startswith("c"):
        if n < 4:
            pytest.skip("family c needs n >= 4")
        a, b = synth.dot_family_c(n, float("1e" + fam[1:]), synth.BASE_SEED + 1)
    else:
        a, b = getattr(synth, f"dot_family_{fam}")(n, synth.BASE_SEED + 1)
    want = oracle_lib.dot_exact(a, b, nthreads=oracle_lib.default_threads())
    assert same(_exact_gpu(rpcg, a, b, cuda), want)


def test_dot_exact_golden(rpcg, cuda, oracle_lib):
    for line in open(os.path.join(GOLDEN, "exact_dot_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b, _ = (part.split() for part in line.split(";"))
        a = [float.fromhex(t) for t in a]
        b = [float.fromhex(t) for t in b]
        assert same(_exact_gpu(rpcg, a, b, cuda), oracle_lib.dot_exact(a, b)), line


def _rand_double(rng, lo, hi):
    e = rng.randint(lo, hi)
    m = rng.getrandbits(52)
    v = math.ldexp(m, -1074) if e < -1022 else math.ldexp((1 << 52) | m, e - 52)
    return -v if rng.random() < 0.5 else v


@pytest.mark.parametrize("seed", range(6))
def test_dot_exact_extreme_exponents(rpcg, cuda, oracle_lib, seed):
    """Subnormal operands, products far below 2^-1074 and near 2^2046."""
    rng = random.Random(seed)
    n = 5000
    a = [_rand_double(rng, -1074, 1023) for _ in range(n)]
    b = [_rand_double(rng, -1074, 1023 if seed % 2 else 0) for _ in range(n)]
    assert same(_exact_gpu(rpcg, a, b, cuda), oracle_lib.dot_exact(a, b))


def _wide_values(rng, n, hi=1023):
    """n doubles with exponents uniform over [-1074, hi] (subnormals below
    -1022), random significands and signs."""
    e = rng.integers(-1074, hi + 1, n)
    m = rng.integers(0, 1 << 52, n, dtype=np.int64)
    normal = np.ldexp((m | (1 << 52)).astype(np.float64), np.maximum(e, -1022) - 52)
    sub = np.ldexp(m.astype(np.float64), np.full(n, -1074))
    v = np.where(e < -1022, sub, normal)
    return np.where(rng.random(n) < 0.5, -v, v)


@pytest.mark.parametrize("n", [65536, 70001, 1000003])
@pytest.mark.parametrize("layout", ["wide", "mixed"])
def test_dot_exact_wide_exponents_large(rpcg, cuda, oracle_lib, n, layout):
    """Products spread over the whole exponent range, at sizes with many
    CTAs: every pair ("wide"), or every seventh pair among U[-1, 1] pairs
    ("mixed": each thread's register windows keep moving); through both
    entry points."""
    rng = np.random.default_rng(n)
    a, b = synth.dot_family_a(n, 17)
    wa, wb = _wide_values(rng, n, hi=1000), _wide_values(rng, n, hi=0)
    if layout == "wide":
        a, b = wa, wb
    else:
        a[::7], b[::7] = wa[::7], wb[::7]
    want = oracle_lib.dot_exact(a, b, nthreads=oracle_lib.default_threads())
    assert math.isfinite(want)
    assert same(_exact_gpu(rpcg, a, b, cuda), want)
    assert same(rpcg.dot_exact_noalloc(_dev(a, cuda), _dev(b, cuda)).item(), want)


def test_dot_exact_special_values(rpcg, cuda, oracle_lib):
    n = 3000
    a, b = synth.dot_family_a(n, 5)
    for bad in (math.inf, -math.inf, math.nan):
        a2 = a.copy()
        a2[1234] = bad
        assert math.isnan(_exact_gpu(rpcg, a2, b, cuda))
    # exact cancellation is +0, n ones is n
    x = synth.uniform_pm1(3, 4097)
    assert same(_exact_gpu(rpcg, np.concatenate([x, -x]), np.concatenate([x, x]), cuda), 0.0)
    assert _exact_gpu(rpcg, np.ones(100001), np.ones(100001), cuda) == 100001.0
    # tiny negative values that round to zero keep their sign
    assert same(_exact_gpu(rpcg, [-2.0 ** -600], [2.0 ** -500], cuda), oracle_lib.dot_exact([-2.0 ** -600], [2.0 ** -500]))


def test_dot_exact_misaligned_and_strided_views(rpcg, cuda, oracle_lib):
    import torch
    a, b = synth.dot_family_b(20001, 8)
    ta, tb = _dev(a, cuda), _dev(b, cuda)
    for off in (1, 3):
        va, vb = ta[off:], tb[:-off]
        want = oracle_lib.dot_exact(a[off:], b[:-off])
        assert same(rpcg.dot_exact(va, vb).item(), want)


def test_dot_exact_order_independent(rpcg, cuda, oracle_lib):
    a, b = synth.dot_family_c(200000, 1e30, 44)
    v0 = _exact_gpu(rpcg, a, b, cuda)
    perm = np.random.default_rng(1).permutation(a.size)
    assert same(_exact_gpu(rpcg, a[perm], b[perm], cuda), v0)
    assert same(v0, oracle_lib.dot_exact(a, b, nthreads=4))


@pytest.mark.parametrize("fam", ["a", "c8", "c16", "c40"])
@pytest.mark.parametrize("p", [2, 3, 8])
def test_dot_fpe_equals_exact_when_flagged(rpcg, cuda, oracle_lib, fam, p):
    n = 300001
    if fam == "a":
        a, b = synth.dot_family_a(n, 9)
    else:
        a, b = synth.dot_family_c(n, float("1e" + fam[1:]), 9)
    v, ex = rpcg.dot_fpe(_dev(a, cuda), _dev(b, cuda), p=p)
    want = oracle_lib.dot_exact(a, b, nthreads=4)
    if ex.item():
        assert same(v.item(), want)
    if fam == "a" and p >= 3:
        assert ex.item() == 1
    if fam == "c40" and p == 2:
        assert ex.item() == 0


def test_dot_fpe_flag_cases(rpcg, cuda):
    v, ex = rpcg.dot_fpe(_dev([2.0 ** -500, 1.0], cuda), _dev([2.0 ** -500, 1.0], cuda), p=8)
    assert ex.item() == 0
    v, ex = rpcg.dot_fpe(_dev([1.0, math.inf], cuda), _dev([1.0, 1.0], cuda), p=8)
    assert ex.item() == 0 and math.isnan(v.item())
    v, ex = rpcg.dot_fpe(_dev([], cuda), _dev([], cuda), p=8)
    assert ex.item() == 1 and same(v.item(), 0.0)


def _one_thread(vals_a, vals_b, t, n=2048, nthr=256):
    """Arrays of n pairs whose non-zero products all land in thread t of the
    FPE dot's single CTA (thread t takes elements t, t + 256, ...; up to
    n = 4096 the dot runs as one CTA of 256 threads)."""
    a, b = np.zeros(n), np.zeros(n)
    for k, (x, y) in enumerate(zip(vals_a, vals_b)):
        a[t + k * nthr], b[t + k * nthr] = x, y
    return a, b


@pytest.mark.parametrize("p", [1, 2, 8])
def test_dot_fpe_integer_and_fp64_warps_agree(rpcg, cuda, oracle_lib, p):
    """A thread's expansions depend only on its own products, so the same
    products placed in any thread (of any warp, whichever pipe runs its
    Accumulate cascades) give the same value and flag, bit for bit, and the
    paper's one-thread FPE dot gives them too: lossy ill-conditioned sums,
    products below twoprod's exact range, subnormal products, sums that
    overflow, cancellation to zero."""
    rng = np.random.default_rng(5)
    c40a, c40b = synth.dot_family_c(8, 1e40, 3)
    cases = [
        (c40a, c40b),
        (rng.uniform(-1, 1, 8), rng.uniform(-1, 1, 8)),
        ([2.0 ** -600, 1.0, -3.0, 2.0 ** -500, 5.0, 7.0, 1e-300, 9.0], [2.0 ** -500, 1.0, 3.0, 2.0 ** -560, 1.5, 1.0, 1e-20, 2.0]),
        ([1.5 * 2.0 ** 1000] * 8, [1.9 * 2.0 ** 23] * 8),                  # the running sum overflows
        ([1.0, -1.0, 2.0 ** 60, -(2.0 ** 60), 3.0, -3.0, 0.5, -0.5], [1.0] * 8),  # cancels to +0
        ([2.0 ** -1074, 3.0, 2.0 ** -1000, 1.0, 1.0, 1.0, 1.0, 1.0], [1.0, 2.0 ** -1074, 2.0 ** -30, 1e-16, 1.0, -1e-16, 3.0, 2.0 ** 52]),
    ]
    # threads in the first and last warps of the CTA and in between
    for va, vb in cases:
        got = []
        for t in (0, 40, 95, 96, 160, 255):
            a, b = _one_thread(va, vb, t)
            v, ex = rpcg.dot_fpe(_dev(a, cuda), _dev(b, cuda), p=p)
            got.append((bits([v.item()])[0] if not math.isnan(v.item()) else "nan", ex.item()))
        assert len(set(got)) == 1, (va, got)
        # one thread holds every product, so no cross-thread merge happens and
        # the paper's one-thread FPE dot gives the value and flag, lossy or not
        a, b = _one_thread(va, vb, 0)
        want_v, want_ex = oracle_lib.dot_fpe(a, b, p=p, T=1)
        assert same(v.item(), want_v) and ex.item() == int(want_ex), (va, v.item(), ex.item(), want_v, want_ex)
        if got[0][1] == 1:
            assert same(v.item(), oracle_lib.dot_exact(a, b))


@pytest.mark.parametrize("p", [2, 3, 8])
def test_dot_fpe_one_thread_random_exponents(rpcg, cuda, oracle_lib, p):
    """The twosums of both expansions on products spread over the whole
    exponent range (subnormal and near-overflow ones included), with equal
    and opposite products, products that are exact powers of two and
    operands of equal magnitude among them: 16 products in one thread
    against the oracle's one-thread FPE dot, value and flag bit for bit."""
    for seed in range(40):
        rng = np.random.default_rng(1000 + seed)
        k = 16
        hi = 1000 if seed % 4 else 1023  # every fourth set may overflow
        va = _wide_values(rng, k, hi=hi // 2)
        vb = _wide_values(rng, k, hi=hi // 2)
        if seed % 3 == 0:  # pairs that cancel exactly
            va[1::2] = -va[0::2]
            vb[1::2] = vb[0::2]
        if seed % 5 == 0:  # powers of two of one magnitude
            va[:8] = np.ldexp(1.0, rng.integers(-60, 60, 8)) * np.where(rng.random(8) < 0.5, -1, 1)
            vb[:8] = np.ldexp(1.0, rng.integers(-60, 60, 8))
        a, b = _one_thread(va, vb, 37, n=4096)
        v, ex = rpcg.dot_fpe(_dev(a, cuda), _dev(b, cuda), p=p)
        want_v, want_ex = oracle_lib.dot_fpe(a, b, p=p, T=1)
        assert same(v.item(), want_v) and ex.item() == int(want_ex), (seed, v.item(), ex.item(), want_v, want_ex)


@pytest.mark.parametrize("cond", [1e8, 1e24, 1e40])
@pytest.mark.parametrize("p", [1, 2, 3, 8])
def test_dot_fpe_one_thread_equals_oracle_fpe(rpcg, cuda, oracle_lib, cond, p):
    """Sec. 4.2's FPE dot (Algs. 2 and 4 with the early exit, Alg. 3, then the
    correctly rounded sum of the terms) against the oracle's, value and flag
    bit for bit, including every case where the expansion loses bits.  All
    16 products of an ill-conditioned family-(c) input are placed in one
    thread (of an integer-pipe warp or of an FP64 warp) of the FPE dot's
    single CTA; every other element is zero.  With one thread the GPU's
    exact cross-thread merge and the paper's fpesum merge coincide, so the
    oracle's one-thread dot is the expected result."""
    va, vb = synth.dot_family_c(16, cond, 3)
    want_exact = oracle_lib.dot_exact(va, vb)
    flags = set()
    for t in (0, 40, 95, 96, 160, 255):
        a, b = _one_thread(va, vb, t, n=4096)
        v, ex = rpcg.dot_fpe(_dev(a, cuda), _dev(b, cuda), p=p)
        want_v, want_ex = oracle_lib.dot_fpe(a, b, p=p, T=1)
        assert same(v.item(), want_v), (t, v.item(), want_v)
        assert ex.item() == int(want_ex), (t, ex.item(), want_ex)
        flags.add(int(want_ex))
    # the cases cover both outcomes: p = 1 always loses bits on these inputs,
    # p = 8 never does (then the value is the exact dot)
    if p == 1:
        assert flags == {0}
        assert not same(v.item(), want_exact)
    if p == 8:
        assert flags == {1} and same(v.item(), want_exact)


def test_dot_plain_close(rpcg, cuda, oracle_lib):
    a, b = synth.dot_family_a(1000003, 12)
    want = oracle_lib.dot_exact(a, b, nthreads=4)
    got = rpcg.dot_plain(_dev(a, cuda), _dev(b, cuda)).item()
    # fp64 error bound of a summation tree: n * u * sum|a_i b_i|
    assert abs(got - want) <= 1e-16 * a.size * float(np.abs(a * b).sum())


def test_dot_exact_repeat_is_deterministic(rpcg, cuda):
    a, b = synth.dot_family_b(777777, 3)
    ta, tb = _dev(a, cuda), _dev(b, cuda)
    vals = {bits([rpcg.dot_exact(ta, tb).item()])[0] for _ in range(5)}
    assert len(vals) == 1


def test_dot_exact_window_anchor_edges(rpcg, cuda, oracle_lib):
    """The register window's first anchor: a product at the lowest digit
    (two subnormal operands), leading zero products, and a tiny product
    followed by ordinary ones, in every lane position of a warp."""
    tiny = 2.0 ** -1074
    rng = np.random.default_rng(3)
    for n in (1, 2, 33, 4096, 100001):
        base_a, base_b = synth.dot_family_a(n, 123)
        for pattern in ("tiny_first", "zeros_first", "tiny_everywhere"):
            a, b = base_a.copy(), base_b.copy()
            if pattern == "tiny_first":
                a[: min(n, 64)] = tiny
                b[: min(n, 64)] = tiny * 3
            elif pattern == "zeros_first":
                a[: min(n, 5000)] = 0.0
            else:
                idx = rng.choice(n, size=max(1, n // 7), replace=False)
                a[idx] = tiny
                b[idx] = -tiny
            assert same(_exact_gpu(rpcg, a, b, cuda), oracle_lib.dot_exact(a, b)), (n, pattern)
