"""The FPE dot's error-free transformations -- twosum (Alg. 1) as exact
integer arithmetic on the bit patterns, twoprod (Alg. 2) in FP64 -- against
the oracle's FP64 Alg. 1 and Alg. 2, element by element, on random and
adversarial inputs."""
import math
import random

import numpy as np
import pytest

import synth
from conftest import bits

pytestmark = pytest.mark.gpu


def _rand(rng, n, lo, hi):
    out = []
    for _ in range(n):
        e = rng.randint(lo, hi)
        m = rng.getrandbits(52)
        v = math.ldexp(m, -1074) if e < -1022 else math.ldexp((1 << 52) | m, e - 52)
        out.append(-v if rng.random() < 0.5 else v)
    return np.array(out)


def _cases(seed):
    rng = random.Random(seed)
    n = 40000
    yield _rand(rng, n, -60, 60), _rand(rng, n, -60, 60)            # overlapping ranges
    yield _rand(rng, n, -1074, 1023), _rand(rng, n, -1074, 1023)    # everything
    a = _rand(rng, n, -10, 10)
    yield a, -a * (1 + np.ldexp(np.array([rng.getrandbits(20) for _ in range(n)], float), -52))  # cancellation
    yield _rand(rng, n, -1074, -1000), _rand(rng, n, -1074, -1000)  # subnormal neighbourhood
    x = synth.uniform_pm1(seed, n)
    yield x, np.ldexp(x[::-1].copy(), 53)                           # exponent gaps near 53..55
    ties = np.ldexp(np.ones(n), 0)
    yield ties, np.ldexp(np.array([rng.choice([1, 3, 5, 7]) for _ in range(n)], float), -53)  # exact ties
    yield np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** 1023, -2.0 ** 1023, 2.0 ** -1074, math.inf, math.nan]), \
        np.array([-0.0, -0.0, -1.0, 1.0, 2.0 ** 1023, 2.0 ** 1023, -2.0 ** -1074, 1.0, 1.0])


def _same(got, want):
    g, w = bits(got), bits(want)
    both_nan = np.isnan(got) & np.isnan(want)
    return np.all((g == w) | both_nan)


@pytest.mark.parametrize("seed", [1, 2])
def test_twosum_matches_oracle(rpcg, cuda, oracle_lib, seed):
    import torch
    for a, b in _cases(seed):
        r, s = rpcg.eft("twosum", torch.from_numpy(a).to(cuda), torch.from_numpy(b).to(cuda))
        want = [oracle_lib.twosum(float(x), float(y)) for x, y in zip(a, b)]
        assert _same(r.cpu().numpy(), np.array([w[0] for w in want]))
        assert _same(s.cpu().numpy(), np.array([w[1] for w in want]))


@pytest.mark.parametrize("seed", [3, 4])
def test_twoprod_matches_oracle(rpcg, cuda, oracle_lib, seed):
    import torch
    for a, b in _cases(seed):
        r, s = rpcg.eft("twoprod", torch.from_numpy(a).to(cuda), torch.from_numpy(b).to(cuda))
        want = [oracle_lib.twoprod(float(x), float(y)) for x, y in zip(a, b)]
        assert _same(r.cpu().numpy(), np.array([w[0] for w in want]))
        assert _same(s.cpu().numpy(), np.array([w[1] for w in want]))


def test_fpe_dot_integer_pipe_matches_fp64_semantics(rpcg, cuda, oracle_lib):
    """The FPE dot (its Accumulate cascades on the integer pipe) equals the
    exact dot whenever its flag holds, on small ill-conditioned cases and
    every expansion size."""
    import torch
    for fam_c in (1e8, 1e24, 1e40):
        a, b = synth.dot_family_c(64, fam_c, 5)
        for p in (1, 2, 3, 8):
            v, ex = rpcg.dot_fpe(torch.from_numpy(a).to(cuda), torch.from_numpy(b).to(cuda), p=p)
            if ex.item():
                assert bits([v.item()])[0] == bits([oracle_lib.dot_exact(a, b)])[0]
