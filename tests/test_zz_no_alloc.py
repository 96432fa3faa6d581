"""The exact dot that allocates nothing (rpcg_dot_exact_noalloc).

It serves callers that cannot let the library allocate device memory, such
as a framework whose allocator already holds the whole GPU.  Its scratch is
a fixed array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test; it
passes both alone in a fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _call(rpcg, fn, a, b, out):
    L = rpcg.lib()
    import torch
    st = getattr(L, fn)(a.numel(), ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == rpcg.OK, L.rpcg_last_error()


def test_noalloc_matches_allocating_exact_dot_twice(rpcg, cuda):
    import torch
    cases = [synth.dot_family_a(1000003, 71), synth.dot_family_c(300000, 1e32, 72)]
    for a_np, b_np in cases:
        a = torch.from_numpy(a_np).to(cuda)
        b = torch.from_numpy(b_np).to(cuda)
        ref = torch.empty((), dtype=torch.float64, device=cuda)
        _call(rpcg, "rpcg_dot_exact", a, b, ref)
        # two calls in a row: the shared scratch must start clean each time
        for _ in range(2):
            got = torch.full((), float("nan"), dtype=torch.float64, device=cuda)
            _call(rpcg, "rpcg_dot_exact_noalloc", a, b, got)
            torch.cuda.synchronize()
            # exact dots are bit-exact: the tolerance used by these tests is zero ulps
            assert np.float64(got.item()).view(np.int64) == np.float64(ref.item()).view(np.int64)


def test_noalloc_empty_and_unaligned_after_a_large_call(rpcg, cuda):
    """A large call leaves the shared array holding its digits, counter and
    flags; the calls right after it on the same stream must start clean.
    n = 0 gives +0, and views offset by one element (not 16-byte aligned,
    the other instance of the kernel) give rpcg_dot_exact's bits."""
    import torch
    a_np, b_np = synth.dot_family_b(2000001, 73)
    a = torch.from_numpy(a_np).to(cuda)
    b = torch.from_numpy(b_np).to(cuda)
    big = torch.empty((), dtype=torch.float64, device=cuda)
    empty = torch.full((), float("nan"), dtype=torch.float64, device=cuda)
    got = torch.full((), float("nan"), dtype=torch.float64, device=cuda)
    ref = torch.empty((), dtype=torch.float64, device=cuda)
    _call(rpcg, "rpcg_dot_exact_noalloc", a, b, big)
    _call(rpcg, "rpcg_dot_exact_noalloc", a[:0], b[:0], empty)
    _call(rpcg, "rpcg_dot_exact_noalloc", a[1:], b[1:], got)
    _call(rpcg, "rpcg_dot_exact", a[1:], b[1:], ref)
    torch.cuda.synchronize()
    assert np.float64(empty.item()).view(np.int64) == 0  # +0, not -0 or NaN
    assert np.float64(got.item()).view(np.int64) == np.float64(ref.item()).view(np.int64)
    _call(rpcg, "rpcg_dot_exact", a, b, ref)
    torch.cuda.synchronize()
    assert np.float64(big.item()).view(np.int64) == np.float64(ref.item()).view(np.int64)


def test_noalloc_rejects_sizes_beyond_its_maximum(rpcg, cuda):
    L = rpcg.lib()
    st = L.rpcg_dot_exact_noalloc((1 << 30) + 1, ctypes.c_void_p(8), ctypes.c_void_p(8), ctypes.c_void_p(8), None)
    assert st == rpcg.ERR_INVALID
    assert b"2^30" in L.rpcg_last_error()
