/*
 * Oracle (TEST INFRASTRUCTURE ONLY): plain C Berends-Giele recursion.
 *
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline / reference leg of
 * bench.py may load or run this file's library.  It shares no code, header or
 * constant with the CUDA library: it is a second, literal statement of the
 * recursion of arXiv:2502.07060, Sec. 2.2, used for bulk parity checks and as
 * the timed CPU baseline.  One OpenMP iteration per phase-space point.
 *
 * Recursion (Sec. 2.2, currents and the three- and four-gluon vertices), with
 * the vertices contracted and the factors of i cancelled against the
 * propagator -i/P^2:
 *
 *   R(i,j) = sum_s   (JA.JB)(PA - PB) + 2 (PB.JA) JB - 2 (PA.JB) JA
 *          + sum_s<t 2 (JA.JC) JB - (JB.JC) JA - (JA.JB) JC
 *   J(i,j) = R(i,j) / P_{i,j}^2   for internal ranges,   A = eps_n . R(1,n-1)
 *
 * F_p: p an odd prime below 2^31 (Sec. 3), operands canonical in [0,p), every
 * product formed in 64 bits and reduced with %, inverses by the extended
 * Euclidean algorithm (Sec. 3, the finite-field division).
 * C64: C99 double complex, the library's complex division for 1/P^2.
 * C64DD: the same recursion in double-double complex arithmetic (about 106
 * significant bits: Knuth's TwoSum and an FMA-based exact product, the
 * classic error-free transformations), used as the high-precision reference
 * that FP64 results are measured against.  Outputs (re_hi, re_lo, im_hi,
 * im_lo) per point.
 *
 * Metric: 0 = mostly minus (Sec. 2.3), 1 = alternating (Sec. 3.1).
 * Momenta are d-dimensional and zero padded to D_s (Sec. 2.3), so a dot with a
 * range momentum runs over its first d components.
 * A singular propagator (P^2 == 0 for an internal range) gives status 1 and
 * amplitude 0.
 *
 * Layouts: k[E][n][d], eps[E][n][Ds], out[E]; complex values are interleaved
 * (re, im) doubles.  Return value 0 on success, -1 on bad arguments.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BGO_NMAX 16
#define BGO_DMAX 16

typedef double complex cplx;

static int sign_of(int metric, int mu) {
    if (metric == 0) return mu == 0 ? 1 : -1;
    return (mu % 2 == 0) ? 1 : -1;
}

/* ---------------------------------------------------------------- F_p ---- */

static uint32_t fp_add(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)(((uint64_t)a + b) % p); }
static uint32_t fp_sub(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)(((uint64_t)a + p - b) % p); }
static uint32_t fp_mul(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)(((uint64_t)a * b) % p); }

/* Inverse by the extended Euclidean algorithm; a != 0 (mod p). */
static uint32_t fp_inv(uint32_t a, uint32_t p) {
    int64_t r0 = p, r1 = a, s0 = 0, s1 = 1;
    while (r1 != 0) {
        int64_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    /* r0 == 1 since p is prime and a != 0 */
    s0 %= (int64_t)p;
    if (s0 < 0) s0 += p;
    return (uint32_t)s0;
}

static uint32_t fp_dot(const uint32_t* a, const uint32_t* b, int dims, int metric, uint32_t p) {
    uint32_t acc = 0;
    for (int mu = 0; mu < dims; ++mu) {
        uint32_t t = fp_mul(a[mu], b[mu], p);
        acc = sign_of(metric, mu) > 0 ? fp_add(acc, t, p) : fp_sub(acc, t, p);
    }
    return acc;
}

/* acc[0..dims) += c * v[0..dims) */
static void fp_axpy(uint32_t* acc, uint32_t c, const uint32_t* v, int dims, uint32_t p) {
    for (int mu = 0; mu < dims; ++mu) acc[mu] = fp_add(acc[mu], fp_mul(c, v[mu], p), p);
}

static int fp_point(int n, int d, int Ds, uint32_t p, int metric,
                    const uint32_t* k, const uint32_t* eps, uint32_t* out) {
    const int N = n - 1;
    static __thread uint32_t J[BGO_NMAX][BGO_NMAX][BGO_DMAX];
    static __thread uint32_t P[BGO_NMAX][BGO_NMAX][BGO_DMAX];
    uint32_t R[BGO_DMAX], diff[BGO_DMAX];

    for (int i = 0; i < N; ++i) {
        uint32_t acc[BGO_DMAX] = {0};
        for (int j = i; j < N; ++j) {
            for (int mu = 0; mu < d; ++mu) acc[mu] = fp_add(acc[mu], k[j * d + mu], p);
            memcpy(P[i][j], acc, sizeof(uint32_t) * d);
        }
        memcpy(J[i][i], eps + i * Ds, sizeof(uint32_t) * Ds);
    }
    for (int m = 2; m <= N; ++m) {
        for (int i = 0; i + m - 1 < N; ++i) {
            const int j = i + m - 1;
            memset(R, 0, sizeof R);
            for (int s = i; s < j; ++s) {                      /* three-gluon vertex */
                const uint32_t *JA = J[i][s], *JB = J[s + 1][j];
                const uint32_t *PA = P[i][s], *PB = P[s + 1][j];
                uint32_t jj = fp_dot(JA, JB, Ds, metric, p);
                uint32_t pb_ja = fp_dot(PB, JA, d, metric, p);
                uint32_t pa_jb = fp_dot(PA, JB, d, metric, p);
                for (int mu = 0; mu < d; ++mu) diff[mu] = fp_sub(PA[mu], PB[mu], p);
                fp_axpy(R, jj, diff, d, p);
                fp_axpy(R, fp_add(pb_ja, pb_ja, p), JB, Ds, p);
                fp_axpy(R, fp_sub(0, fp_add(pa_jb, pa_jb, p), p), JA, Ds, p);
            }
            for (int s = i; s < j - 1; ++s) {                  /* four-gluon vertex */
                for (int t = s + 1; t < j; ++t) {
                    const uint32_t *JA = J[i][s], *JB = J[s + 1][t], *JC = J[t + 1][j];
                    uint32_t ac = fp_dot(JA, JC, Ds, metric, p);
                    uint32_t bc = fp_dot(JB, JC, Ds, metric, p);
                    uint32_t ab = fp_dot(JA, JB, Ds, metric, p);
                    fp_axpy(R, fp_add(ac, ac, p), JB, Ds, p);
                    fp_axpy(R, fp_sub(0, bc, p), JA, Ds, p);
                    fp_axpy(R, fp_sub(0, ab, p), JC, Ds, p);
                }
            }
            if (m < N) {
                uint32_t p2 = fp_dot(P[i][j], P[i][j], d, metric, p);
                if (p2 == 0) { *out = 0; return 1; }
                uint32_t inv = fp_inv(p2, p);
                for (int mu = 0; mu < Ds; ++mu) J[i][j][mu] = fp_mul(inv, R[mu], p);
            }
        }
    }
    *out = fp_dot(eps + (n - 1) * Ds, R, Ds, metric, p);
    return 0;
}

static int check_args(int n, int d, int Ds, int metric) {
    if (n < 4 || n > BGO_NMAX || d < 1 || Ds < d || Ds > BGO_DMAX) return -1;
    if (metric != 0 && metric != 1) return -1;
    return 0;
}

int bgo_amp_fp(int n, int d, int Ds, uint32_t p, int metric, int64_t E,
               const uint32_t* k, const uint32_t* eps, uint32_t* out, uint8_t* status,
               int nthreads) {
    if (check_args(n, d, Ds, metric) || p < 3 || p >= (1u << 31) || E < 0) return -1;
    if (E > 0 && (!k || !eps || !out)) return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
    for (int64_t e = 0; e < E; ++e) {
        int st = fp_point(n, d, Ds, p, metric, k + e * n * d, eps + e * n * Ds, out + e);
        if (status) status[e] = (uint8_t)st;
    }
    return 0;
}

/* ---------------------------------------------------------------- C64 ---- */

static cplx c_dot(const cplx* a, const cplx* b, int dims, int metric) {
    cplx acc = 0;
    for (int mu = 0; mu < dims; ++mu) {
        cplx t = a[mu] * b[mu];
        acc = sign_of(metric, mu) > 0 ? acc + t : acc - t;
    }
    return acc;
}

static void c_axpy(cplx* acc, cplx c, const cplx* v, int dims) {
    for (int mu = 0; mu < dims; ++mu) acc[mu] += c * v[mu];
}

static int c_point(int n, int d, int Ds, int metric, const cplx* k, const cplx* eps, cplx* out) {
    const int N = n - 1;
    static __thread cplx J[BGO_NMAX][BGO_NMAX][BGO_DMAX];
    static __thread cplx P[BGO_NMAX][BGO_NMAX][BGO_DMAX];
    cplx R[BGO_DMAX], diff[BGO_DMAX];

    for (int i = 0; i < N; ++i) {
        cplx acc[BGO_DMAX];
        for (int mu = 0; mu < BGO_DMAX; ++mu) acc[mu] = 0;
        for (int j = i; j < N; ++j) {
            for (int mu = 0; mu < d; ++mu) acc[mu] += k[j * d + mu];
            memcpy(P[i][j], acc, sizeof(cplx) * d);
        }
        memcpy(J[i][i], eps + i * Ds, sizeof(cplx) * Ds);
    }
    for (int m = 2; m <= N; ++m) {
        for (int i = 0; i + m - 1 < N; ++i) {
            const int j = i + m - 1;
            for (int mu = 0; mu < BGO_DMAX; ++mu) R[mu] = 0;
            for (int s = i; s < j; ++s) {
                const cplx *JA = J[i][s], *JB = J[s + 1][j];
                const cplx *PA = P[i][s], *PB = P[s + 1][j];
                cplx jj = c_dot(JA, JB, Ds, metric);
                cplx pb_ja = c_dot(PB, JA, d, metric);
                cplx pa_jb = c_dot(PA, JB, d, metric);
                for (int mu = 0; mu < d; ++mu) diff[mu] = PA[mu] - PB[mu];
                c_axpy(R, jj, diff, d);
                c_axpy(R, pb_ja + pb_ja, JB, Ds);
                c_axpy(R, -(pa_jb + pa_jb), JA, Ds);
            }
            for (int s = i; s < j - 1; ++s) {
                for (int t = s + 1; t < j; ++t) {
                    const cplx *JA = J[i][s], *JB = J[s + 1][t], *JC = J[t + 1][j];
                    cplx ac = c_dot(JA, JC, Ds, metric);
                    cplx bc = c_dot(JB, JC, Ds, metric);
                    cplx ab = c_dot(JA, JB, Ds, metric);
                    c_axpy(R, ac + ac, JB, Ds);
                    c_axpy(R, -bc, JA, Ds);
                    c_axpy(R, -ab, JC, Ds);
                }
            }
            if (m < N) {
                cplx p2 = c_dot(P[i][j], P[i][j], d, metric);
                if (p2 == 0) { *out = 0; return 1; }
                cplx inv = 1.0 / p2;
                for (int mu = 0; mu < Ds; ++mu) J[i][j][mu] = inv * R[mu];
            }
        }
    }
    *out = c_dot(eps + (n - 1) * Ds, R, Ds, metric);
    return 0;
}

int bgo_amp_c64(int n, int d, int Ds, int metric, int64_t E,
                const double* k, const double* eps, double* out, uint8_t* status,
                int nthreads) {
    if (check_args(n, d, Ds, metric) || E < 0) return -1;
    if (E > 0 && (!k || !eps || !out)) return -1;
    const cplx* kc = (const cplx*)k;
    const cplx* ec = (const cplx*)eps;
    cplx* oc = (cplx*)out;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
    for (int64_t e = 0; e < E; ++e) {
        int st = c_point(n, d, Ds, metric, kc + e * n * d, ec + e * n * Ds, oc + e);
        if (status) status[e] = (uint8_t)st;
    }
    return 0;
}

/* ------------------------------------------------------ double-double ---- */

typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; } cdd;

static dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = {s, e};
    return r;
}
static dd fast_two_sum(double a, double b) {   /* |a| >= |b| */
    double s = a + b;
    dd r = {s, b - (s - a)};
    return r;
}
static dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);          /* exact error of the product */
    e += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p, e);
}
static dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul((dd){q1, 0.0}, b));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul((dd){q2, 0.0}, b));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add(q, (dd){q3, 0.0});
}
static cdd c_add(cdd a, cdd b) { cdd r = {dd_add(a.re, b.re), dd_add(a.im, b.im)}; return r; }
static cdd c_sub(cdd a, cdd b) { cdd r = {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; return r; }
static cdd c_mul(cdd a, cdd b) {
    cdd r = {dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)),
             dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
    return r;
}
static cdd c_inv(cdd z) {
    dd w = dd_add(dd_mul(z.re, z.re), dd_mul(z.im, z.im));
    cdd r = {dd_div(z.re, w), dd_neg(dd_div(z.im, w))};
    return r;
}
static int c_iszero(cdd z) { return z.re.hi == 0.0 && z.im.hi == 0.0; }
static const cdd CDD_ZERO = {{0.0, 0.0}, {0.0, 0.0}};

static cdd cdd_dot(const cdd* a, const cdd* b, int dims, int metric) {
    cdd acc = CDD_ZERO;
    for (int mu = 0; mu < dims; ++mu) {
        cdd t = c_mul(a[mu], b[mu]);
        acc = sign_of(metric, mu) > 0 ? c_add(acc, t) : c_sub(acc, t);
    }
    return acc;
}

static void cdd_axpy(cdd* acc, cdd c, const cdd* v, int dims) {
    for (int mu = 0; mu < dims; ++mu) acc[mu] = c_add(acc[mu], c_mul(c, v[mu]));
}

static int dd_point(int n, int d, int Ds, int metric, const double* k, const double* eps, double* out) {
    const int N = n - 1;
    static __thread cdd J[BGO_NMAX][BGO_NMAX][BGO_DMAX];
    static __thread cdd P[BGO_NMAX][BGO_NMAX][BGO_DMAX];
    cdd R[BGO_DMAX], diff[BGO_DMAX];

    for (int i = 0; i < N; ++i) {
        cdd acc[BGO_DMAX];
        for (int mu = 0; mu < BGO_DMAX; ++mu) acc[mu] = CDD_ZERO;
        for (int j = i; j < N; ++j) {
            for (int mu = 0; mu < d; ++mu) {
                cdd x = {{k[2 * (j * d + mu)], 0.0}, {k[2 * (j * d + mu) + 1], 0.0}};
                acc[mu] = c_add(acc[mu], x);
            }
            memcpy(P[i][j], acc, sizeof(cdd) * d);
        }
        for (int mu = 0; mu < Ds; ++mu) {
            cdd x = {{eps[2 * (i * Ds + mu)], 0.0}, {eps[2 * (i * Ds + mu) + 1], 0.0}};
            J[i][i][mu] = x;
        }
    }
    for (int m = 2; m <= N; ++m) {
        for (int i = 0; i + m - 1 < N; ++i) {
            const int j = i + m - 1;
            for (int mu = 0; mu < BGO_DMAX; ++mu) R[mu] = CDD_ZERO;
            for (int s = i; s < j; ++s) {
                const cdd *JA = J[i][s], *JB = J[s + 1][j];
                const cdd *PA = P[i][s], *PB = P[s + 1][j];
                cdd jj = cdd_dot(JA, JB, Ds, metric);
                cdd pb_ja = cdd_dot(PB, JA, d, metric);
                cdd pa_jb = cdd_dot(PA, JB, d, metric);
                for (int mu = 0; mu < d; ++mu) diff[mu] = c_sub(PA[mu], PB[mu]);
                cdd_axpy(R, jj, diff, d);
                cdd_axpy(R, c_add(pb_ja, pb_ja), JB, Ds);
                cdd_axpy(R, c_sub(CDD_ZERO, c_add(pa_jb, pa_jb)), JA, Ds);
            }
            for (int s = i; s < j - 1; ++s) {
                for (int t = s + 1; t < j; ++t) {
                    const cdd *JA = J[i][s], *JB = J[s + 1][t], *JC = J[t + 1][j];
                    cdd ac = cdd_dot(JA, JC, Ds, metric);
                    cdd bc = cdd_dot(JB, JC, Ds, metric);
                    cdd ab = cdd_dot(JA, JB, Ds, metric);
                    cdd_axpy(R, c_add(ac, ac), JB, Ds);
                    cdd_axpy(R, c_sub(CDD_ZERO, bc), JA, Ds);
                    cdd_axpy(R, c_sub(CDD_ZERO, ab), JC, Ds);
                }
            }
            if (m < N) {
                cdd p2 = cdd_dot(P[i][j], P[i][j], d, metric);
                if (c_iszero(p2)) { out[0] = out[1] = out[2] = out[3] = 0.0; return 1; }
                cdd inv = c_inv(p2);
                for (int mu = 0; mu < Ds; ++mu) J[i][j][mu] = c_mul(inv, R[mu]);
            }
        }
    }
    cdd last[BGO_DMAX];
    for (int mu = 0; mu < Ds; ++mu) {
        cdd x = {{eps[2 * ((n - 1) * Ds + mu)], 0.0}, {eps[2 * ((n - 1) * Ds + mu) + 1], 0.0}};
        last[mu] = x;
    }
    cdd a = cdd_dot(last, R, Ds, metric);
    out[0] = a.re.hi; out[1] = a.re.lo; out[2] = a.im.hi; out[3] = a.im.lo;
    return 0;
}

int bgo_amp_c64dd(int n, int d, int Ds, int metric, int64_t E,
                  const double* k, const double* eps, double* out4, uint8_t* status,
                  int nthreads) {
    if (check_args(n, d, Ds, metric) || E < 0) return -1;
    if (E > 0 && (!k || !eps || !out4)) return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int64_t e = 0; e < E; ++e) {
        int st = dd_point(n, d, Ds, metric, k + 2 * e * n * d, eps + 2 * e * n * Ds, out4 + 4 * e);
        if (status) status[e] = (uint8_t)st;
    }
    return 0;
}

int bgo_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
