/*
 * CPU oracle for the reproducible Jacobi-PCG hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the GPU path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA
 * library: every routine here is written out independently from the paper
 * (Iakymchuk, Barreda, Graillat, Aliaga, Quintana-Orti, "Reproducibility of
 * Parallel Preconditioned Conjugate Gradient in Hybrid Programming
 * Environments") and from the IEEE 754 definitions it relies on.
 *
 * Build: plain C11, -O2 -ffp-contract=off, no -ffast-math, so that every
 * a*b and a+b below is one IEEE binary64 operation rounded to nearest even
 * and every fma() is the correctly rounded fused multiply-add (C99 7.12.13).
 *
 * Contents
 *   exact dot      Sec. 2 (long accumulator idea, Kulisch): sum of a_i*b_i
 *                  computed exactly as a big two's-complement integer and
 *                  rounded once to nearest-even.  Defined for all finite
 *                  inputs; any NaN/Inf input gives NaN.
 *   FPE dot        Alg. 1 (twosum), Alg. 2 (twoprod), Alg. 4 (Accumulate,
 *                  with the early exit of Sec. 4.2), Alg. 3 (fpesum),
 *                  Listing 2's per-thread FPEs merged in thread order; the
 *                  final rounding is the correctly rounded value of the
 *                  FPE's exact sum (what NearSum returns, Sec. 4.3).
 *   SpMV           Sec. 4.3: rows summed left to right with explicit fma.
 *   PCG            Fig. 1 / Fig. 2 (S8 merged next to S6), Jacobi
 *                  preconditioner as an elementwise multiply by the inverse
 *                  diagonal (Sec. 3.1, Sec. 4.3), AXPYs with fma (Sec. 4.3).
 *
 * Readings where the paper is silent (the same list appears in the design
 * notes): z0 = inv.*r0, d0 = z0, beta0 = <z0,r0>, tau0 = <r0,r0>;
 * inv_i = RN(1/a_ii); stop when RN(RN_sqrt(tau)/bnorm) < tol with
 * bnorm = RN_sqrt(<b,b>), tested at the loop top; rho = RN(beta/<d,w>);
 * x = fma(rho,d,x); r = fma(-rho,w,r); gamma = RN(beta_new/beta_old);
 * d = fma(gamma,d,z); SpMV accumulator starts at +0.0.
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ------------------------------------------------------------------ */
/* Status codes (the oracle's own copy of the values the solver reports) */
enum {
    OR_OK = 0,
    OR_NOT_CONVERGED = 1,
    OR_ERR_INVALID = -1,
    OR_ERR_NOT_SPD = -2,
    OR_ERR_NONFINITE = -3
};

/* ------------------------------------------------------------------ */
/* Big integer: the long accumulator.
 *
 * A finite double is +-m * 2^e with integer 0 <= m < 2^53 and e >= -1074.
 * A product of two doubles is +-M * 2^E with M < 2^106 and E >= -2148.
 * We keep two non-negative big integers P (positive products) and N
 * (negative products), both in units of 2^-2148, and the value is P - N.
 * The largest product is below 2^2048, so a sum of up to 2^63 products is
 * below 2^(2048 + 2148 + 63) = 2^4259; BIG_W 32-bit words hold 4480 bits.
 */
#define BIG_W 140
#define BIG_SCALE 2148 /* value = integer * 2^-2148 */

typedef struct {
    uint32_t w[BIG_W]; /* little-endian words, unsigned magnitude */
} big_t;

static void big_zero(big_t *a) { memset(a->w, 0, sizeof(a->w)); }

/* a += v * 2^shift, with v a 128-bit unsigned integer given as hi:lo. */
static void big_add_shifted(big_t *a, uint64_t hi, uint64_t lo, int shift) {
    /* split v into four 32-bit words */
    uint32_t v[4] = {(uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32)};
    int q = shift / 32, r = shift % 32;
    /* v << r occupies five words */
    uint32_t s[5];
    for (int k = 0; k < 5; k++) {
        uint64_t cur = (k < 4) ? v[k] : 0;
        uint64_t prev = (k > 0) ? v[k - 1] : 0;
        uint64_t word = (cur << r) | (r ? (prev >> (32 - r)) : 0);
        s[k] = (uint32_t)word;
    }
    uint64_t carry = 0;
    int k = 0;
    for (int j = q; j < BIG_W; j++, k++) {
        uint64_t add = (k < 5) ? s[k] : 0;
        if (k >= 5 && carry == 0) break;
        uint64_t t = (uint64_t)a->w[j] + add + carry;
        a->w[j] = (uint32_t)t;
        carry = t >> 32;
    }
}

/* a += b */
static void big_add(big_t *a, const big_t *b) {
    uint64_t carry = 0;
    for (int j = 0; j < BIG_W; j++) {
        uint64_t t = (uint64_t)a->w[j] + b->w[j] + carry;
        a->w[j] = (uint32_t)t;
        carry = t >> 32;
    }
}

/* returns -1, 0, +1 for a < b, a == b, a > b */
static int big_cmp(const big_t *a, const big_t *b) {
    for (int j = BIG_W - 1; j >= 0; j--) {
        if (a->w[j] != b->w[j]) return a->w[j] < b->w[j] ? -1 : 1;
    }
    return 0;
}

/* d = a - b, requires a >= b */
static void big_sub(big_t *d, const big_t *a, const big_t *b) {
    int64_t borrow = 0;
    for (int j = 0; j < BIG_W; j++) {
        int64_t t = (int64_t)a->w[j] - (int64_t)b->w[j] - borrow;
        borrow = t < 0;
        d->w[j] = (uint32_t)(t + (borrow ? ((int64_t)1 << 32) : 0));
    }
}

static int big_bit(const big_t *a, int i) { return (a->w[i / 32] >> (i % 32)) & 1u; }

static int big_msb(const big_t *a) {
    for (int j = BIG_W - 1; j >= 0; j--) {
        if (a->w[j]) {
            int b = 31;
            while (!((a->w[j] >> b) & 1u)) b--;
            return j * 32 + b;
        }
    }
    return -1;
}

/* Round the magnitude D * 2^-2148 to the nearest binary64, ties to even,
 * with gradual underflow; values at or above the overflow threshold give inf. */
static double big_round(const big_t *D, int negative) {
    int t = big_msb(D);
    if (t < 0) return 0.0; /* exact zero is +0 */
    /* bit index of the last kept bit: 53 significant bits, but never below
       2^-1074 (bit index 1074 in units of 2^-2148) */
    int lsb = t - 52;
    if (lsb < 1074) lsb = 1074;
    uint64_t mant = 0;
    for (int i = t; i >= lsb; i--) mant = (mant << 1) | (uint64_t)big_bit(D, i);
    int round_bit = (lsb - 1 >= 0) ? big_bit(D, lsb - 1) : 0;
    int sticky = 0;
    for (int i = lsb - 2; i >= 0 && !sticky; i--) sticky = big_bit(D, i);
    if (round_bit && (sticky || (mant & 1u))) mant += 1;
    /* mant <= 2^53 is exact in binary64; the scaling by a power of two is
       exact unless it overflows, in which case ldexp returns inf, which is
       the correct round-to-nearest result there. */
    double v = ldexp((double)mant, lsb - BIG_SCALE);
    return negative ? -v : v;
}

/* ------------------------------------------------------------------ */
/* Splitting a double into sign, integer significand and exponent. */
typedef struct {
    int neg;
    uint64_t m; /* 0 <= m < 2^53 */
    int e;      /* value = (-1)^neg * m * 2^e */
    int finite;
} parts_t;

static parts_t split_double(double x) {
    uint64_t bits;
    memcpy(&bits, &x, 8);
    parts_t p;
    p.neg = (int)(bits >> 63);
    int E = (int)((bits >> 52) & 0x7ff);
    uint64_t frac = bits & ((UINT64_C(1) << 52) - 1);
    p.finite = (E != 0x7ff);
    if (E == 0) {
        p.m = frac;
        p.e = -1074;
    } else {
        p.m = frac | (UINT64_C(1) << 52);
        p.e = E - 1075;
    }
    return p;
}

/* Accumulate the exact product a*b into (P, N).  Returns 0 if a or b is not finite. */
static int acc_product(big_t *P, big_t *N, double a, double b) {
    parts_t pa = split_double(a), pb = split_double(b);
    if (!pa.finite || !pb.finite) return 0;
    if (pa.m == 0 || pb.m == 0) return 1;
    unsigned __int128 M = (unsigned __int128)pa.m * (unsigned __int128)pb.m;
    int shift = pa.e + pb.e + BIG_SCALE; /* >= 0 */
    big_add_shifted((pa.neg ^ pb.neg) ? N : P, (uint64_t)(M >> 64), (uint64_t)M, shift);
    return 1;
}

static double round_pn(const big_t *P, const big_t *N) {
    big_t D;
    int c = big_cmp(P, N);
    if (c == 0) return 0.0;
    if (c > 0) {
        big_sub(&D, P, N);
        return big_round(&D, 0);
    }
    big_sub(&D, N, P);
    return big_round(&D, 1);
}

/* ---- threaded exact dot: each thread owns (P, N) for a contiguous range;
        the thread results are added (integer addition is associative, so the
        result does not depend on the thread count). */
typedef struct {
    const double *a, *b;
    int64_t lo, hi;
    big_t P, N;
    int ok;
} dot_job_t;

static void *dot_worker(void *arg) {
    dot_job_t *j = (dot_job_t *)arg;
    big_zero(&j->P);
    big_zero(&j->N);
    j->ok = 1;
    for (int64_t i = j->lo; i < j->hi; i++) {
        if (!acc_product(&j->P, &j->N, j->a[i], j->b[i])) j->ok = 0;
    }
    return NULL;
}

double oracle_dot_exact(int64_t n, const double *a, const double *b, int nthreads) {
    if (n <= 0) return 0.0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > n) nthreads = (int)n;
    dot_job_t *jobs = (dot_job_t *)calloc((size_t)nthreads, sizeof(dot_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; t++) {
        jobs[t].a = a;
        jobs[t].b = b;
        jobs[t].lo = n * t / nthreads;
        jobs[t].hi = n * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, dot_worker, &jobs[t]);
    dot_worker(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    int ok = 1;
    for (int t = 1; t < nthreads; t++) {
        big_add(&jobs[0].P, &jobs[t].P);
        big_add(&jobs[0].N, &jobs[t].N);
    }
    for (int t = 0; t < nthreads; t++) ok &= jobs[t].ok;
    double r = ok ? round_pn(&jobs[0].P, &jobs[0].N) : NAN;
    free(jobs);
    free(th);
    return r;
}

/* Exactly rounded sum of an array (a dot with all-ones weights). */
double oracle_sum_exact(int64_t n, const double *x) {
    big_t P, N;
    big_zero(&P);
    big_zero(&N);
    for (int64_t i = 0; i < n; i++) {
        if (!acc_product(&P, &N, x[i], 1.0)) return NAN;
    }
    return round_pn(&P, &N);
}

/* ------------------------------------------------------------------ */
/* Error-free transformations and floating-point expansions.           */

/* Alg. 1: r + s = a + b exactly (unless r overflows). */
void oracle_twosum(double a, double b, double *r, double *s) {
    double rr = a + b;
    double z = rr - a;
    double ss = (a - (rr - z)) + (b - z);
    *r = rr;
    *s = ss;
}

/* Alg. 2: r + s = a * b exactly (unless the product under- or overflows). */
void oracle_twoprod(double a, double b, double *r, double *s) {
    double rr = a * b;
    *r = rr;
    *s = fma(a, b, -rr);
}

/* Alg. 4 with the early exit of Sec. 4.2: add x into the p-term expansion a.
 * Returns the value carried out of the last term (0 when nothing is lost). */
double oracle_fpe_accumulate(double *a, int p, double x) {
    for (int i = 0; i < p; i++) {
        double r, s;
        oracle_twosum(a[i], x, &r, &s);
        a[i] = r;
        x = s;
        if (x == 0.0) break; /* early exit: stop propagating a zero error */
    }
    return x;
}

/* Alg. 3: a := a + b for two p-term expansions.  Returns nonzero if any
 * Accumulate carried a nonzero value out of the last term. */
int oracle_fpesum(double *a, const double *b, int p) {
    int lost = 0;
    for (int i = 0; i < p; i++) {
        if (oracle_fpe_accumulate(a, p, b[i]) != 0.0) lost = 1;
    }
    return lost;
}

/* The smallest |r| for which twoprod's error term is always representable:
 * |a*b| >= 2^-969 implies e_a + e_b >= -970 (binary64: e_min = -1022, p = 53). */
#define TWOPROD_SAFE 0x1p-969

/* FPE dot (Listing 2 with the per-element body of Listing 1): T logical
 * threads, thread t handles elements [n*t/T, n*(t+1)/T) in order with a
 * result expansion and an error expansion of p terms each (Sec. 4.2: two
 * FPEs, merged before rounding).  Threads are merged in index order with
 * fpesum.  The returned value is the correctly rounded exact sum of the
 * merged expansion.  *exact is 1 iff no term was lost (no carry out of the
 * last term), no twoprod could have lost its error term (|r| < 2^-969 with
 * nonzero operands) and every term stayed finite. */
double oracle_dot_fpe(int64_t n, const double *a, const double *b, int p, int T, int *exact) {
    if (p < 1 || p > 64 || T < 1) {
        *exact = 0;
        return NAN;
    }
    double *res = (double *)calloc((size_t)T * p, sizeof(double));
    double *err = (double *)calloc((size_t)p, sizeof(double));
    int ok = 1;
    for (int t = 0; t < T; t++) {
        double *R = res + (size_t)t * p;
        memset(err, 0, sizeof(double) * (size_t)p);
        int64_t lo = n * t / T, hi = n * (t + 1) / T;
        for (int64_t i = lo; i < hi; i++) {
            double r, s;
            if (!isfinite(a[i]) || !isfinite(b[i])) ok = 0;
            oracle_twoprod(a[i], b[i], &r, &s);
            if (a[i] != 0.0 && b[i] != 0.0 && fabs(r) < TWOPROD_SAFE) ok = 0;
            if (oracle_fpe_accumulate(R, p, r) != 0.0) ok = 0;
            if (oracle_fpe_accumulate(err, p, s) != 0.0) ok = 0;
        }
        if (oracle_fpesum(R, err, p)) ok = 0;
    }
    for (int t = 1; t < T; t++) {
        if (oracle_fpesum(res, res + (size_t)t * p, p)) ok = 0;
    }
    /* the rounded sum of the terms is returned even when a term was lost;
       non-finite terms give NaN */
    int fin = 1;
    for (int i = 0; i < p; i++) fin &= isfinite(res[i]) ? 1 : 0;
    if (!fin) ok = 0;
    double v = fin ? oracle_sum_exact(p, res) : NAN;
    *exact = ok;
    free(res);
    free(err);
    return v;
}

/* ------------------------------------------------------------------ */
/* SpMV, Sec. 4.3: y_i = fma(val_k, x_col_k, acc) left to right from +0. */
typedef struct {
    int32_t lo, hi;
    const int32_t *rowptr, *col;
    const double *val, *x;
    double *y;
} spmv_job_t;

static void *spmv_worker(void *arg) {
    spmv_job_t *j = (spmv_job_t *)arg;
    for (int32_t i = j->lo; i < j->hi; i++) {
        double acc = 0.0;
        for (int32_t k = j->rowptr[i]; k < j->rowptr[i + 1]; k++) acc = fma(j->val[k], j->x[j->col[k]], acc);
        j->y[i] = acc;
    }
    return NULL;
}

void oracle_spmv(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const double *x, double *y,
                 int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > n) nthreads = n > 0 ? n : 1;
    spmv_job_t *jobs = (spmv_job_t *)calloc((size_t)nthreads, sizeof(spmv_job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = (spmv_job_t){(int32_t)((int64_t)n * t / nthreads), (int32_t)((int64_t)n * (t + 1) / nthreads),
                               rowptr, col, val, x, y};
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, spmv_worker, &jobs[t]);
    spmv_worker(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
}

/* ------------------------------------------------------------------ */
/* PCG (Fig. 1, with S8 next to S6 as in Fig. 2).                      */

/* plain dot: one rounding per multiply and per add, in index order */
static double dot_plain(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double p = a[i] * b[i];
        s = s + p;
    }
    return s;
}

static double dot_v(int variant, int64_t n, const double *a, const double *b, int nthreads) {
    return variant == 0 ? dot_plain(n, a, b) : oracle_dot_exact(n, a, b, nthreads);
}

/*
 * variant: 0 = plain dots, 1 = exact dots (the exblas trajectory; the fpe
 * variant with recompute-on-inexact follows the same trajectory).
 * x: in = x0, out = final iterate.
 * history (optional, max_iter + 1 entries): relative residual at the top of
 * every loop test, history[l] for l = 0 .. iterations.
 * Returns a status code.
 */
static double now_seconds(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* Instrumentation only: wall-clock seconds spent in the iteration loop of
 * the last oracle_pcg call (excludes the set-up).  Used to time the oracle
 * as a CPU baseline; it does not influence any result. */
static double g_loop_seconds = 0.0;
double oracle_pcg_loop_seconds(void) { return g_loop_seconds; }

/* Optional per-loop-test record (for checking every scalar and vector of a
 * tiny solve against a hand-worked trace): record l holds
 * [<d,w>, rho, beta, tau, gamma, relres, x[0..n), r[0..n), z[0..n), d[0..n)]
 * after the set-up (l = 0; <d,w>, rho, gamma are NaN there) and after each
 * loop body l = 1, 2, ...  It only copies values; no arithmetic. */
static void trace_record(double *trace, int32_t l, int32_t n, double dw, double rho, double beta, double tau,
                         double gamma, double rel, const double *x, const double *r, const double *z, const double *d) {
    if (!trace) return;
    double *t = trace + (size_t)l * (6 + 4 * (size_t)n);
    t[0] = dw;
    t[1] = rho;
    t[2] = beta;
    t[3] = tau;
    t[4] = gamma;
    t[5] = rel;
    memcpy(t + 6, x, sizeof(double) * (size_t)n);
    memcpy(t + 6 + n, r, sizeof(double) * (size_t)n);
    memcpy(t + 6 + 2 * (size_t)n, z, sizeof(double) * (size_t)n);
    memcpy(t + 6 + 3 * (size_t)n, d, sizeof(double) * (size_t)n);
}

static int pcg_core(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const double *b, double *x,
                    int variant, double tol, int32_t max_iter, double *history, int32_t *iterations, double *relres_out,
                    double *tau_out, int nthreads, double *trace) {
    g_loop_seconds = 0.0;
    *iterations = 0;
    *relres_out = NAN;
    *tau_out = NAN;
    if (n < 0 || max_iter < 0) return OR_ERR_INVALID;
    if (n == 0) {
        *relres_out = 0.0;
        *tau_out = 0.0;
        if (history) history[0] = 0.0;
        return OR_OK;
    }
    size_t sz = (size_t)n * sizeof(double);
    double *inv = (double *)malloc(sz), *r = (double *)malloc(sz), *z = (double *)malloc(sz);
    double *d = (double *)malloc(sz), *w = (double *)malloc(sz);
    int status = OR_OK;

    /* Compute preconditioner: inverse of the diagonal (Sec. 4.3). */
    for (int32_t i = 0; i < n && status == OR_OK; i++) {
        double aii = 0.0;
        int found = 0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
            if (col[k] == i) {
                aii = val[k];
                found = 1;
            }
        }
        if (!found || !(aii > 0.0)) status = isfinite(aii) ? OR_ERR_NOT_SPD : OR_ERR_NONFINITE;
        else inv[i] = 1.0 / aii;
    }
    if (status != OR_OK) goto done;

    /* r0 = b - A x0 */
    oracle_spmv(n, rowptr, col, val, x, w, nthreads);
    for (int32_t i = 0; i < n; i++) r[i] = b[i] - w[i];
    for (int32_t i = 0; i < n; i++) z[i] = inv[i] * r[i];
    for (int32_t i = 0; i < n; i++) d[i] = z[i];
    double beta = dot_v(variant, n, z, r, nthreads);
    double tau = dot_v(variant, n, r, r, nthreads);
    double bb = dot_v(variant, n, b, b, nthreads);
    if (!isfinite(beta) || !isfinite(tau) || !isfinite(bb)) {
        status = OR_ERR_NONFINITE;
        goto done;
    }
    double bnorm = sqrt(bb);
    if (bnorm == 0.0) {
        /* b = 0: the solution is x = 0 */
        for (int32_t i = 0; i < n; i++) x[i] = 0.0;
        *relres_out = 0.0;
        *tau_out = 0.0;
        if (history) history[0] = 0.0;
        goto done;
    }
    int32_t l = 0;
    double rel = sqrt(tau) / bnorm;
    if (history) history[0] = rel;
    trace_record(trace, 0, n, NAN, NAN, beta, tau, NAN, rel, x, r, z, d);
    double t_loop = now_seconds();
    while (rel >= tol && l < max_iter) {
        double beta_old = beta;
        /* S1 */
        oracle_spmv(n, rowptr, col, val, d, w, nthreads);
        /* S2 */
        double dw = dot_v(variant, n, d, w, nthreads);
        if (!isfinite(dw)) {
            status = OR_ERR_NONFINITE;
            break;
        }
        if (!(dw > 0.0)) {
            status = OR_ERR_NOT_SPD;
            break;
        }
        double rho = beta / dw;
        /* S3, S4, S5 */
        for (int32_t i = 0; i < n; i++) x[i] = fma(rho, d[i], x[i]);
        for (int32_t i = 0; i < n; i++) r[i] = fma(-rho, w[i], r[i]);
        for (int32_t i = 0; i < n; i++) z[i] = inv[i] * r[i];
        /* S6 and S8 */
        beta = dot_v(variant, n, z, r, nthreads);
        tau = dot_v(variant, n, r, r, nthreads);
        if (!isfinite(beta) || !isfinite(tau)) {
            status = OR_ERR_NONFINITE;
            l++;
            break;
        }
        /* S7 */
        double gamma = beta / beta_old;
        for (int32_t i = 0; i < n; i++) d[i] = fma(gamma, d[i], z[i]);
        l++;
        rel = sqrt(tau) / bnorm;
        if (history) history[l] = rel;
        trace_record(trace, l, n, dw, rho, beta, tau, gamma, rel, x, r, z, d);
        if (tau > 0.0 && !(beta > 0.0)) {
            status = OR_ERR_NOT_SPD;
            break;
        }
    }
    g_loop_seconds = now_seconds() - t_loop;
    *iterations = l;
    *relres_out = rel;
    *tau_out = tau;
    if (status == OR_OK && rel >= tol) status = OR_NOT_CONVERGED;
done:
    free(inv);
    free(r);
    free(z);
    free(d);
    free(w);
    return status;
}

int oracle_pcg(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const double *b, double *x,
               int variant, double tol, int32_t max_iter, double *history, int32_t *iterations, double *relres_out,
               double *tau_out, int nthreads) {
    return pcg_core(n, rowptr, col, val, b, x, variant, tol, max_iter, history, iterations, relres_out, tau_out,
                    nthreads, NULL);
}

/* oracle_pcg with the per-loop-test record of trace_record: `trace` holds
 * (max_iter + 1) * (6 + 4 n) doubles. */
int oracle_pcg_trace(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const double *b,
                     double *x, int variant, double tol, int32_t max_iter, double *trace, int32_t *iterations,
                     double *relres_out, double *tau_out) {
    return pcg_core(n, rowptr, col, val, b, x, variant, tol, max_iter, NULL, iterations, relres_out, tau_out, 1,
                    trace);
}
