"""Seeded synthetic inputs for the reproducible Jacobi-PCG hot path.

This module is shared by the CPU oracle, the tests and the benchmark, and it
holds none of the method's arithmetic: no products are summed, no SpMV, no
dot product and no PCG step happens here.  It only draws random numbers and
lays out CSR matrices whose entries are given directly (stencil constants,
face coefficients and their plain sums on the diagonal).

Random numbers come from one counter-based generator: the SplitMix64
finaliser of Steele, Lea and Flood ("Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``seed + (i + 1) * golden_gamma``.
Element ``i`` of a stream depends only on ``(seed, i)``, so any slice of any
stream can be regenerated independently and both sides of a comparison see
the same numbers.

Workloads (the paper's experiments use a 3D Poisson operator, Sec. 5.1;
its SuiteSparse and band matrices are not available, so these synthetic
operators stand in for them):

* ``poisson7(s)``: 7-point 3D Poisson on an s^3 grid, diagonal 6,
  off-diagonals -1, Dirichlet boundary.
* ``poisson27(s)``: 27-point 3D Poisson on an s^3 grid, diagonal 26,
  off-diagonals -1 (the paper's stencil, Sec. 5.1).
* ``diffusion7(s, seed)``: variable-coefficient 7-point diffusion operator,
  face coefficients log-uniform in [1e-2, 1e2] plus a shift sigma*I.
* ``dot_family_a/b/c``: the three families of dot-product inputs.

Columns in every row are stored in ascending order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
BASE_SEED = 2005072820

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_seed(seed: int, tag: int) -> int:
    """Derive the seed of an independent stream ``tag`` of a base ``seed``."""
    z = np.array([(seed * 0x9E3779B97F4A7C15 + tag * 0xD1B54A32D192ED03 + 1) & (2**64 - 1)], dtype=np.uint64)
    return int(_mix64(z)[0])


def u64(seed: int, start: int, count: int) -> np.ndarray:
    """Elements ``start .. start+count-1`` of the uint64 stream of ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        state = np.uint64(seed & (2**64 - 1)) + idx * GOLDEN_GAMMA
    return _mix64(state)


def uniform_pm1(seed: int, n: int, start: int = 0) -> np.ndarray:
    """U[-1, 1] doubles: 2 * (u >> 11) * 2^-53 - 1 (every value exact)."""
    u = u64(seed, start, n) >> np.uint64(11)
    return u.astype(np.float64) * (2.0 ** -52) - 1.0


def uniform_01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """U[0, 1) doubles: (u >> 11) * 2^-53."""
    u = u64(seed, start, n) >> np.uint64(11)
    return u.astype(np.float64) * (2.0 ** -53)


def uniform_int(seed: int, n: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), by multiply-shift of the top 32 bits."""
    span = hi - lo + 1
    top = (u64(seed, start, n) >> np.uint64(32)).astype(np.uint64)
    return (lo + ((top * np.uint64(span)) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


# ---------------------------------------------------------------- matrices

@dataclass
class CSR:
    """CSR matrix with int32 row pointers and column indices, float64 values."""
    n: int
    rowptr: np.ndarray  # int32[n+1]
    col: np.ndarray     # int32[nnz]
    val: np.ndarray     # float64[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _stencil_csr(s: int, offsets, values, name: str) -> CSR:
    """Lay out a constant-coefficient stencil on an s^3 grid (x fastest).

    ``offsets`` are (dk, dj, di) triples; they are sorted so that column
    indices come out ascending within each row.
    """
    n = s * s * s
    if n >= 2**31:
        raise ValueError("grid too large for int32 indices")
    order = sorted(range(len(offsets)), key=lambda t: offsets[t])
    offsets = [offsets[t] for t in order]
    values = [values[t] for t in order]
    idx = np.arange(n, dtype=np.int64)
    ii = idx % s
    jj = (idx // s) % s
    kk = idx // (s * s)
    del idx
    counts = np.zeros(n, dtype=np.int32)
    masks = []
    for dk, dj, di in offsets:
        m = np.ones(n, dtype=bool)
        if di:
            m &= (ii + di >= 0) & (ii + di < s)
        if dj:
            m &= (jj + dj >= 0) & (jj + dj < s)
        if dk:
            m &= (kk + dk >= 0) & (kk + dk < s)
        masks.append(m)
        counts += m
    del ii, jj, kk
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    if nnz >= 2**31:
        raise ValueError("too many nonzeros for int32 row pointers")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    pos = rowptr[:-1].copy()
    rows_all = np.arange(n, dtype=np.int64)
    for (dk, dj, di), v, m in zip(offsets, values, masks):
        rows = rows_all[m] if not m.all() else rows_all
        p = pos[rows]
        col[p] = (rows + di + dj * s + dk * s * s).astype(np.int32)
        val[p] = v
        pos[rows] += 1
    return CSR(n, rowptr.astype(np.int32), col, val, name)


def poisson7(s: int) -> CSR:
    """7-point 3D Poisson, diagonal 6, off-diagonals -1, on an s^3 grid."""
    offs = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
    vals = [6.0] + [-1.0] * 6
    return _stencil_csr(s, offs, vals, f"poisson7_{s}")


def poisson27(s: int) -> CSR:
    """27-point 3D Poisson, diagonal 26, off-diagonals -1, on an s^3 grid (Sec. 5.1)."""
    offs = [(dk, dj, di) for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
    vals = [26.0 if o == (0, 0, 0) else -1.0 for o in offs]
    return _stencil_csr(s, offs, vals, f"poisson27_{s}")


def diffusion7(s: int, seed: int) -> tuple[CSR, float]:
    """Variable-coefficient 7-point diffusion operator on an s^3 grid.

    Each face carries a coefficient c_f = 10^U[-2, 2] shared by the two cells
    it separates; Dirichlet boundary faces have their own coefficient and
    only add to the diagonal.  a_ii = (c_-x + c_+x) + ... + sigma with the
    six faces summed in the order -x, +x, -y, +y, -z, +z and then sigma,
    sigma ~ U[0, 1]; a_ij = -c_f.  The operator is SPD (strictly diagonally
    dominant or irreducibly dominant with positive boundary faces).
    Returns the CSR matrix and sigma.
    """
    n = s * s * s
    sig = float(uniform_01(stream_seed(seed, 99), 1)[0])
    cx = 10.0 ** (2.0 * uniform_pm1(stream_seed(seed, 1), (s + 1) * s * s)).reshape(s, s, s + 1)
    cy = 10.0 ** (2.0 * uniform_pm1(stream_seed(seed, 2), s * (s + 1) * s)).reshape(s, s + 1, s)
    cz = 10.0 ** (2.0 * uniform_pm1(stream_seed(seed, 3), (s + 1) * s * s)).reshape(s + 1, s, s)
    diag = (cx[:, :, :-1] + cx[:, :, 1:])
    diag = diag + cy[:, :-1, :]
    diag = diag + cy[:, 1:, :]
    diag = diag + cz[:-1, :, :]
    diag = diag + cz[1:, :, :]
    diag = (diag + sig).reshape(n)
    # off-diagonal coefficients per row for each neighbour direction
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    coef = {
        (0, 0, -1): -cx[:, :, :-1].reshape(n), (0, 0, 1): -cx[:, :, 1:].reshape(n),
        (0, -1, 0): -cy[:, :-1, :].reshape(n), (0, 1, 0): -cy[:, 1:, :].reshape(n),
        (-1, 0, 0): -cz[:-1, :, :].reshape(n), (1, 0, 0): -cz[1:, :, :].reshape(n),
        (0, 0, 0): diag,
    }
    A = _stencil_csr(s, offs, [0.0] * 7, f"diffusion7_{s}")
    # fill values row by row in the (ascending) column order
    idx = np.arange(n, dtype=np.int64)
    ii, jj, kk = idx % s, (idx // s) % s, idx // (s * s)
    pos = A.rowptr[:-1].astype(np.int64).copy()
    for dk, dj, di in sorted(offs):
        m = np.ones(n, dtype=bool)
        if di:
            m &= (ii + di >= 0) & (ii + di < s)
        if dj:
            m &= (jj + dj >= 0) & (jj + dj < s)
        if dk:
            m &= (kk + dk >= 0) & (kk + dk < s)
        rows = idx[m]
        A.val[pos[rows]] = coef[(dk, dj, di)][rows]
        pos[rows] += 1
    return A, sig


def band(n: int, bw: int) -> CSR:
    """Band matrix with half-bandwidth bw: row i holds columns
    max(0, i-bw) .. min(n-1, i+bw), diagonal 2 bw + 1 and off-diagonals -1
    (strictly diagonally dominant, so SPD).  The paper's performance runs use
    a band version of its Poisson matrix (Sec. 5.1) without giving the entry
    values; these values are this module's choice."""
    rows = np.arange(n, dtype=np.int64)
    lo = np.maximum(rows - bw, 0)
    hi = np.minimum(rows + bw, n - 1)
    counts = (hi - lo + 1).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    if nnz >= 2**31:
        raise ValueError("too many nonzeros for int32 row pointers")
    col = np.empty(nnz, dtype=np.int32)
    val = np.full(nnz, -1.0, dtype=np.float64)
    # entry k of row i is column lo_i + k
    for start in range(0, n, 1 << 20):
        stop = min(n, start + (1 << 20))
        c = counts[start:stop]
        base = np.repeat(lo[start:stop] - rowptr[start:stop], c)  # column minus position
        pos = np.arange(rowptr[start], rowptr[stop], dtype=np.int64)
        col[rowptr[start]:rowptr[stop]] = (pos + base).astype(np.int32)
    diag_pos = rowptr[:-1] + (rows - lo)
    val[diag_pos] = float(2 * bw + 1)
    return CSR(n, rowptr.astype(np.int32), col, val, f"band_{n}_{bw}")


# ---------------------------------------------------------------- dot inputs

def dot_family_a(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Family (a): both vectors U[-1, 1]."""
    return uniform_pm1(stream_seed(seed, 11), n), uniform_pm1(stream_seed(seed, 12), n)


def _family_b_vec(n: int, seed: int) -> np.ndarray:
    u = u64(seed, 0, n)
    mant = 1.0 + (u >> np.uint64(12)).astype(np.float64) * (2.0 ** -52)
    e = uniform_int(stream_seed(seed, 1), n, -300, 300)
    sign = np.where((u & np.uint64(1)) == 1, -1.0, 1.0)
    return sign * np.ldexp(mant, e.astype(np.int32))


def dot_family_b(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Family (b): m * 2^e with m ~ U[1, 2) (52 random bits), e uniform in [-300, 300], random sign."""
    return _family_b_vec(n, stream_seed(seed, 21)), _family_b_vec(n, stream_seed(seed, 22))


def dot_family_c(n: int, cond: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Family (c): ill-conditioned pairs built by cancellation.

    Half of the terms are random with large exponents; the other half cancel
    them.  Layout before a random permutation: m "large" pairs
    (x_i, y_i) = (u 2^e, v 2^f) with e, f uniform integers in [0, E];
    m partner pairs (-x_i, y_i) whose products cancel the large ones
    exactly; and k = max(2, n // 8) small pairs with x, y ~ U[-1, 1] that
    carry the O(1) value of the dot.  E is chosen from the target condition
    number 2 sum|x_i y_i| / |x . y| ~ cond; the realised condition number is
    measured by the caller.  (Sequential generators that cancel a running
    sum need the sum itself, which this module does not compute.)
    """
    if n < 4:
        raise ValueError("family c needs n >= 4")
    k = max(2, n // 8)
    m = (n - k) // 2
    k = n - 2 * m
    # expected sum|p| ~ 2 m 2^(2E) / (4 E^2 ln2^2) * 1/4 ; |dot| ~ sqrt(k)/3
    lc = math.log2(max(cond, 2.0))
    E = 1
    for e_try in range(1, 600):
        est = 2 * (2 * m * (2.0 ** (2 * e_try)) / max(1.0, (e_try * math.log(2)) ** 2) / 4.0) / (math.sqrt(k) / 3.0)
        if math.log2(est) >= lc:
            E = e_try
            break
        E = e_try
    s1, s2, s3, s4, s5, s6, s7 = (stream_seed(seed, 30 + t) for t in range(7))
    ex = uniform_int(s1, m, 0, E)
    ey = uniform_int(s2, m, 0, E)
    xl = np.ldexp(uniform_pm1(s3, m), ex.astype(np.int32))
    yl = np.ldexp(uniform_pm1(s4, m), ey.astype(np.int32))
    xs = uniform_pm1(s5, k)
    ys = uniform_pm1(s6, k)
    x = np.concatenate([xl, -xl, xs])
    y = np.concatenate([yl, yl, ys])
    perm = np.argsort(u64(s7, 0, n), kind="stable")
    return x[perm], y[perm]


def poisson_rhs_xtrue(n: int, seed: int) -> np.ndarray:
    """x_true ~ U[-1, 1] for a system of size n (b = A x_true is formed by the caller)."""
    return uniform_pm1(stream_seed(seed, 7), n)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """A right-hand side b ~ U[-1, 1] drawn directly."""
    return uniform_pm1(stream_seed(seed, 8), n)


def diffusion_batch(count: int, seed: int) -> tuple[list, list]:
    """The batched workload: `count` variable-coefficient 7-point diffusion
    systems on s^3 grids with s uniform in [8, 64], b ~ U[-1, 1] per system.
    Returns (list of CSR, list of right-hand sides)."""
    sides = uniform_int(stream_seed(seed, 50), count, 8, 64)
    mats, rhs = [], []
    for i, s in enumerate(sides.tolist()):
        A, _ = diffusion7(int(s), stream_seed(seed, 1000 + i))
        mats.append(A)
        rhs.append(rhs_uniform(A.n, stream_seed(seed, 5000 + i)))
    return mats, rhs

