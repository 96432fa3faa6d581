"""The seeded input generators (shared by the oracle and the CUDA path, no
method arithmetic): structure and determinism of every workload's matrices,
checked on CPU with SciPy."""
import numpy as np
import pytest
import scipy.sparse

import synth


def _sp(A):
    return scipy.sparse.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))


def _check_csr(A):
    rp, col = A.rowptr.astype(np.int64), A.col.astype(np.int64)
    assert A.rowptr.dtype == np.int32 and A.col.dtype == np.int32 and A.val.dtype == np.float64
    assert rp[0] == 0 and rp[-1] == A.nnz == col.size and np.all(np.diff(rp) >= 0)
    assert col.size == 0 or (col.min() >= 0 and col.max() < A.n)
    for i in range(A.n):  # columns ascending in every row: the storage order of the fma chains
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0), i


@pytest.mark.parametrize("make", [lambda: synth.poisson7(5), lambda: synth.poisson27(4),
                                  lambda: synth.band(200, 7), lambda: synth.diffusion7(5, 11)[0]])
def test_matrices_symmetric_sorted_and_dominant(make):
    A = make()
    _check_csr(A)
    S = _sp(A)
    assert (S != S.T).nnz == 0  # exactly symmetric
    d = S.diagonal()
    off = np.asarray(abs(S).sum(axis=1)).ravel() - np.abs(d)
    assert np.all(d > 0)
    assert np.all(d - off >= -1e-12 * d)  # (weakly) diagonally dominant, irreducible: SPD


def test_poisson_and_band_values():
    P7, P27, B = _sp(synth.poisson7(4)), _sp(synth.poisson27(4)), _sp(synth.band(50, 3))
    assert set(P7.diagonal()) == {6.0} and set(P27.diagonal()) == {26.0} and set(B.diagonal()) == {7.0}
    for S in (P7, P27, B):
        offd = S - scipy.sparse.diags(S.diagonal())
        offd.eliminate_zeros()
        assert set(offd.data) == {-1.0}


def test_diffusion_rows_exceed_offdiagonal_sum_by_sigma_and_boundary():
    A, sigma = synth.diffusion7(6, 5)
    S = _sp(A)
    d = S.diagonal()
    off = np.asarray(abs(S).sum(axis=1)).ravel() - d
    assert 0.0 <= sigma <= 1.0
    assert np.all(d - off >= sigma - 1e-12 * d)  # interior rows: sigma (up to the rounding of the sums)
    coef = -(S - scipy.sparse.diags(d)).data
    assert coef.min() >= 1e-2 * (1 - 1e-12) and coef.max() <= 1e2 * (1 + 1e-12)  # c_f = 10^U[-2, 2]


def test_generators_deterministic_and_seeded():
    a1, b1 = synth.dot_family_b(1000, 3)
    a2, b2 = synth.dot_family_b(1000, 3)
    a3, _ = synth.dot_family_b(1000, 4)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and not np.array_equal(a1, a3)
    D1, D2 = synth.diffusion7(4, 9)[0], synth.diffusion7(4, 9)[0]
    assert np.array_equal(D1.val, D2.val) and not np.array_equal(D1.val, synth.diffusion7(4, 10)[0].val)
    x = synth.uniform_pm1(7, 100000)
    assert x.min() >= -1.0 and x.max() < 1.0 and abs(x.mean()) < 0.02
    # a counter-based stream: a window equals the same range of the full draw
    assert np.array_equal(synth.uniform_pm1(7, 100, start=500), x[500:600])


def test_diffusion_batch_sizes():
    mats, rhs = synth.diffusion_batch(12, 77)
    assert len(mats) == len(rhs) == 12
    for A, b in zip(mats, rhs):
        s = round(A.n ** (1 / 3))
        assert s ** 3 == A.n and 8 <= s <= 64 and b.shape == (A.n,)


def test_family_c_realised_condition_number(oracle_lib):
    """The ill-conditioned family's realised condition number
    2 sum|a_i b_i| / |a . b| (denominator from the oracle's exact dot) stays
    within a small factor of the requested one, at small and large n."""
    import numpy as np
    for cond in (1e8, 1e16, 1e24, 1e32, 1e40):
        for n in (4096, 1 << 18):
            a, b = synth.dot_family_c(n, cond, synth.BASE_SEED + 1)
            realised = 2.0 * float(np.sum(np.abs(a) * np.abs(b))) / abs(oracle_lib.dot_exact(a, b))
            assert cond / 10 <= realised <= cond * 30, (cond, n, realised)
