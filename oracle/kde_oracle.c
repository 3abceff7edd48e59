/*
 * kde_oracle.c -- CPU reference of the PLUGIN bandwidth selector, written from
 * Algorithm 1 (Steps I-VII) and Eqs. (6)-(7) of Gramacki, Sawerwain & Gramacki.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline leg of the benchmark.  The product path never links it.
 *
 * Readings of the paper taken here:
 *  - Step I prints the one-pass form sum(X^2)/(n-1) - (sum X)^2/(n(n-1)).  The
 *    same estimator is computed two-pass, sum((X - mean)^2)/(n-1), which is
 *    algebraically identical and does not cancel when the data carry a large
 *    offset.
 *  - No z-score standardisation (Eqs. 3-4): it is optional in the paper's
 *    flowchart and h * sigma on standardised data equals h on raw data.
 *  - K^6(0), K^4(0) in Steps III and V are the kernel's 6th / 4th derivatives
 *    at zero, as the printed values -15/sqrt(2 pi) and 3/sqrt(2 pi) show.
 *  - The double sums of Steps IV and VI run over all i and j, i = j included;
 *    Eqs. (6)-(7) give the same value as 2 * sum_{i<j} plus n K^(r)(0).
 *  - psi6 >= 0 or psi4 <= 0 leaves g2 or h undefined (a root of a negative
 *    number); that is reported as ORACLE_ERR_DOMAIN.
 *
 * Sums are Neumaier-compensated: each row i is summed over j, then the row sums
 * are summed in row order.  Threads only decide who computes which row, never
 * the order of any addition, so the result does not depend on the thread count.
 */
#include "kde_oracle.h"

#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>

/* ---- constants of Algorithm 1 (Gaussian kernel K = phi, Eq. 2) ---------- */
static const double PI = 3.14159265358979323846264338327950288;

static double inv_sqrt_2pi(void) { return 1.0 / sqrt(2.0 * PI); }

/* ---- Neumaier compensated summation ---------------------------------------- */
typedef struct { double s, c; } csum;

static void csum_add(csum* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double csum_value(const csum* a) { return a->s + a->c; }

/* ---- Step I ----------------------------------------------------------------- */
int oracle_moments(const double* x, int64_t n, double* mean, double* var) {
    if (!x || n < 2 || !mean || !var) return ORACLE_ERR_INVALID;
    csum s = {0, 0};
    for (int64_t i = 0; i < n; ++i) csum_add(&s, x[i]);
    double mu = csum_value(&s) / (double)n;
    csum q = {0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double c = x[i] - mu;
        csum_add(&q, c * c);
    }
    *mean = mu;
    *var = csum_value(&q) / (double)(n - 1);
    if (!isfinite(*mean) || !isfinite(*var)) return ORACLE_ERR_INVALID;
    return ORACLE_OK;
}

/* ---- kernel derivatives, Steps IV and VI ------------------------------------ */
/* K^(6)(x) = (x^6 - 15 x^4 + 45 x^2 - 15) exp(-x^2/2) / sqrt(2 pi)
 * K^(4)(x) = (x^4 - 6 x^2 + 3) exp(-x^2/2) / sqrt(2 pi)
 * and, for the stages above Algorithm 1's two, the same Hermite form:
 * K^(8)(x)  = (x^8 - 28 x^6 + 210 x^4 - 420 x^2 + 105) exp(-x^2/2) / sqrt(2 pi)
 * K^(10)(x) = (x^10 - 45 x^8 + 630 x^6 - 3150 x^4 + 4725 x^2 - 945) exp(-x^2/2) / sqrt(2 pi) */
double oracle_kernel_deriv(int r, double x) {
    double x2 = x * x;
    double e = exp(-0.5 * x2);
    double x4 = x2 * x2, x6 = x4 * x2, x8 = x4 * x4;
    if (r == 6) return inv_sqrt_2pi() * (x6 - 15.0 * x4 + 45.0 * x2 - 15.0) * e;
    if (r == 4) return inv_sqrt_2pi() * (x4 - 6.0 * x2 + 3.0) * e;
    if (r == 8) return inv_sqrt_2pi() * (x8 - 28.0 * x6 + 210.0 * x4 - 420.0 * x2 + 105.0) * e;
    if (r == 10)
        return inv_sqrt_2pi() * (x8 * x2 - 45.0 * x8 + 630.0 * x6 - 3150.0 * x4 + 4725.0 * x2 - 945.0) * e;
    return NAN;
}

static int valid_order(int r) { return r == 4 || r == 6 || r == 8 || r == 10; }

/* ---- the O(n^2) functional ---------------------------------------------------- */
typedef struct {
    const double* x;
    int64_t n;
    int r;
    double g;
    int form;
    double* row;          /* row[i]: compensated sum of row i */
    int64_t next;         /* next row block to take (shared, atomic) */
} psi_job;

#define ROW_BLOCK 16

static void psi_row(const psi_job* jb, int64_t i) {
    csum acc = {0, 0};
    int64_t j0 = (jb->form == ORACLE_FORM_FULL) ? 0 : i + 1;
    for (int64_t j = j0; j < jb->n; ++j) {
        double u = (jb->x[i] - jb->x[j]) / jb->g;
        csum_add(&acc, oracle_kernel_deriv(jb->r, u));
    }
    jb->row[i] = csum_value(&acc);
}

static void* psi_worker(void* arg) {
    psi_job* jb = (psi_job*)arg;
    for (;;) {
        int64_t b = __atomic_fetch_add(&jb->next, 1, __ATOMIC_RELAXED);
        int64_t i0 = b * ROW_BLOCK;
        if (i0 >= jb->n) break;
        int64_t i1 = i0 + ROW_BLOCK < jb->n ? i0 + ROW_BLOCK : jb->n;
        for (int64_t i = i0; i < i1; ++i) psi_row(jb, i);
    }
    return NULL;
}

int oracle_psi(const double* x, int64_t n, int r, double g, int form, int nthreads,
               double* psi) {
    if (!x || !psi || n < 1 || !valid_order(r) || !(g > 0) || !isfinite(g))
        return ORACLE_ERR_INVALID;
    if (form != ORACLE_FORM_FULL && form != ORACLE_FORM_SYMMETRIC) return ORACLE_ERR_INVALID;
    psi_job jb = {x, n, r, g, form, (double*)malloc(sizeof(double) * (size_t)n), 0};
    if (!jb.row) return ORACLE_ERR_INVALID;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    if (nthreads == 1) {
        psi_worker(&jb);
    } else {
        pthread_t th[1024];
        int started = 0;
        for (int t = 0; t < nthreads; ++t)
            if (pthread_create(&th[t], NULL, psi_worker, &jb) == 0) ++started;
        if (started == 0) psi_worker(&jb);
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    csum tot = {0, 0};
    for (int64_t i = 0; i < n; ++i) csum_add(&tot, jb.row[i]);
    free(jb.row);
    double s = csum_value(&tot);
    if (form == ORACLE_FORM_SYMMETRIC) /* Eqs. (6)-(7) */
        s = 2.0 * s + (double)n * oracle_kernel_deriv(r, 0.0);
    double nn = (double)n;
    *psi = s / (nn * nn * pow(g, (double)(r + 1)));
    return ORACLE_OK;
}

int oracle_psi_block(const double* x, int64_t n, int64_t i0, int64_t i1, int64_t j0,
                     int64_t j1, int r, double g, double* sum, double* abs_sum) {
    if (!x || !sum || !abs_sum || !valid_order(r) || !(g > 0)) return ORACLE_ERR_INVALID;
    if (i0 < 0 || j0 < 0 || i1 > n || j1 > n) return ORACLE_ERR_INVALID;
    csum s = {0, 0}, a = {0, 0};
    for (int64_t i = i0; i < i1; ++i) {
        for (int64_t j = (j0 > i + 1 ? j0 : i + 1); j < j1; ++j) {
            double k = oracle_kernel_deriv(r, (x[i] - x[j]) / g);
            csum_add(&s, k);
            csum_add(&a, fabs(k));
        }
    }
    *sum = csum_value(&s);
    *abs_sum = csum_value(&a);
    return ORACLE_OK;
}

/* ---- Algorithm 1 ----------------------------------------------------------------- */
static void fill_nan(oracle_result* o) {
    o->mean = o->sigma = o->psi8 = o->g1 = o->psi6 = o->g2 = o->psi4 = o->h = NAN;
}

int oracle_plugin(const double* x, int64_t n, int form, int nthreads, oracle_result* out) {
    if (!out) return ORACLE_ERR_INVALID;
    fill_nan(out);
    out->status = ORACLE_ERR_INVALID;
    if (!x || n < 2) return out->status;
    const double mu2 = 1.0;                              /* mu_2(K) = 1 */
    const double k6_0 = -15.0 * inv_sqrt_2pi();          /* K^(6)(0), Step III */
    const double k4_0 = 3.0 * inv_sqrt_2pi();            /* K^(4)(0), Step V */
    const double RK = 1.0 / (2.0 * sqrt(PI));            /* R(K), Step VII */
    double nn = (double)n, mean, var;

    /* Step I */
    int st = oracle_moments(x, n, &mean, &var);
    if (st != ORACLE_OK) { out->status = st; return st; }
    out->mean = mean;
    out->sigma = sqrt(var);
    if (!(out->sigma > 0)) { out->status = ORACLE_ERR_DEGENERATE; return out->status; }
    /* Step II */
    out->psi8 = 105.0 / (32.0 * sqrt(PI) * pow(out->sigma, 9.0));
    /* Step III */
    out->g1 = pow(-2.0 * k6_0 / (mu2 * out->psi8 * nn), 1.0 / 9.0);
    /* Step IV */
    st = oracle_psi(x, n, 6, out->g1, form, nthreads, &out->psi6);
    if (st != ORACLE_OK) { out->status = st; return st; }
    if (!(out->psi6 < 0)) { out->status = ORACLE_ERR_DOMAIN; return out->status; }
    /* Step V */
    out->g2 = pow(-2.0 * k4_0 / (mu2 * out->psi6 * nn), 1.0 / 7.0);
    /* Step VI */
    st = oracle_psi(x, n, 4, out->g2, form, nthreads, &out->psi4);
    if (st != ORACLE_OK) { out->status = st; return st; }
    if (!(out->psi4 > 0)) { out->status = ORACLE_ERR_DOMAIN; return out->status; }
    /* Step VII */
    out->h = pow(RK / (mu2 * mu2 * out->psi4 * nn), 1.0 / 5.0);
    out->status = ORACLE_OK;
    return ORACLE_OK;
}

/* ---- the l-stage direct plug-in: Algorithm 1 with l estimated functionals --------- */
/* Stage count l: psi_{2l+4} by the normal scale (Step II's formula, general r:
 * (-1)^(r/2) r! / ((2 sigma)^(r+1) (r/2)! sqrt(pi))), then for r = 2l+2, ..., 4
 * the pilot g_r = (-2 K^(r)(0) / (mu2 psi_{r+2} n))^(1/(r+3)) (Steps III and V)
 * and psi_r(g_r) (Steps IV and VI), then h (Step VII).  l = 2 is Algorithm 1. */
static double kernel_deriv_at_zero(int r) {          /* K^(r)(0) = He_r(0) / sqrt(2 pi) */
    double he = 1.0;                                  /* He_r(0) = (-1)^(r/2) (r-1)!! */
    for (int k = r - 1; k > 1; k -= 2) he *= (double)k;
    return ((r / 2) % 2 ? -he : he) * inv_sqrt_2pi();
}

static double normal_scale_psi(int r, double sigma) {
    double num = 1.0, den = 1.0;                      /* r! and (r/2)! */
    for (int k = 2; k <= r; ++k) num *= (double)k;
    for (int k = 2; k <= r / 2; ++k) den *= (double)k;
    double v = num / (pow(2.0 * sigma, (double)(r + 1)) * den * sqrt(PI));
    return (r / 2) % 2 ? -v : v;
}

int oracle_plugin_stages(const double* x, int64_t n, int stages, int form, int nthreads,
                         oracle_stage_result* out) {
    if (!out) return ORACLE_ERR_INVALID;
    out->mean = out->sigma = out->h = NAN;
    for (int k = 0; k < 6; ++k) out->psi[k] = out->g[k] = NAN;
    out->stages = stages;
    out->status = ORACLE_ERR_INVALID;
    if (!x || n < 2 || stages < 1 || stages > 4) return out->status;
    double nn = (double)n, mean, var;
    int st = oracle_moments(x, n, &mean, &var);                 /* Step I */
    if (st != ORACLE_OK) { out->status = st; return st; }
    out->mean = mean;
    out->sigma = sqrt(var);
    if (!(out->sigma > 0)) { out->status = ORACLE_ERR_DEGENERATE; return out->status; }
    int top = 2 * stages + 4;
    double psi_up = normal_scale_psi(top, out->sigma);          /* Step II */
    out->psi[top / 2 - 2] = psi_up;
    for (int r = top - 2; r >= 4; r -= 2) {
        double ratio = -2.0 * kernel_deriv_at_zero(r) / (psi_up * nn);   /* mu2 = 1 */
        if (!(ratio > 0)) { out->status = ORACLE_ERR_DOMAIN; return out->status; }
        double g = pow(ratio, 1.0 / (double)(r + 3));             /* Steps III, V */
        out->g[r / 2 - 2] = g;
        st = oracle_psi(x, n, r, g, form, nthreads, &psi_up);      /* Steps IV, VI */
        if (st != ORACLE_OK) { out->status = st; return st; }
        out->psi[r / 2 - 2] = psi_up;
    }
    if (!(psi_up > 0)) { out->status = ORACLE_ERR_DOMAIN; return out->status; }
    out->h = pow(1.0 / (2.0 * sqrt(PI)) / (psi_up * nn), 1.0 / 5.0);   /* Step VII */
    out->status = ORACLE_OK;
    return ORACLE_OK;
}

/* ---- long double brute force -------------------------------------------------------- */
int oracle_long_double_mantissa_bits(void) { return LDBL_MANT_DIG; }

static long double kernel_deriv_ld(int r, long double x) {
    const long double PIL = 3.141592653589793238462643383279502884L;
    long double x2 = x * x, e = expl(-0.5L * x2), c = 1.0L / sqrtl(2.0L * PIL);
    if (r == 6) return c * (x2 * x2 * x2 - 15.0L * x2 * x2 + 45.0L * x2 - 15.0L) * e;
    return c * (x2 * x2 - 6.0L * x2 + 3.0L) * e;
}

int oracle_psi_ld(const double* x, int64_t n, int r, long double g, long double* psi) {
    if (!x || !psi || n < 1 || (r != 4 && r != 6) || !(g > 0)) return ORACLE_ERR_INVALID;
    long double s = 0.0L;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            s += kernel_deriv_ld(r, ((long double)x[i] - (long double)x[j]) / g);
    long double nn = (long double)n;
    *psi = s / (nn * nn * powl(g, (long double)(r + 1)));
    return ORACLE_OK;
}

int oracle_plugin_ld(const double* x, int64_t n, oracle_result_ld* out) {
    if (!out) return ORACLE_ERR_INVALID;
    out->mean = out->sigma = out->psi8 = out->g1 = out->psi6 = out->g2 = out->psi4 = out->h = NAN;
    out->status = ORACLE_ERR_INVALID;
    if (!x || n < 2) return out->status;
    const long double PIL = 3.141592653589793238462643383279502884L;
    const long double c = 1.0L / sqrtl(2.0L * PIL);
    long double nn = (long double)n, s = 0.0L, q = 0.0L;
    for (int64_t i = 0; i < n; ++i) s += (long double)x[i];
    out->mean = s / nn;
    for (int64_t i = 0; i < n; ++i) {
        long double d = (long double)x[i] - out->mean;
        q += d * d;
    }
    out->sigma = sqrtl(q / (nn - 1.0L));
    if (!(out->sigma > 0)) { out->status = ORACLE_ERR_DEGENERATE; return out->status; }
    out->psi8 = 105.0L / (32.0L * sqrtl(PIL) * powl(out->sigma, 9.0L));
    out->g1 = powl(-2.0L * (-15.0L * c) / (out->psi8 * nn), 1.0L / 9.0L);
    oracle_psi_ld(x, n, 6, out->g1, &out->psi6);
    if (!(out->psi6 < 0)) { out->status = ORACLE_ERR_DOMAIN; return out->status; }
    out->g2 = powl(-2.0L * (3.0L * c) / (out->psi6 * nn), 1.0L / 7.0L);
    oracle_psi_ld(x, n, 4, out->g2, &out->psi4);
    if (!(out->psi4 > 0)) { out->status = ORACLE_ERR_DOMAIN; return out->status; }
    out->h = powl((1.0L / (2.0L * sqrtl(PIL))) / (out->psi4 * nn), 1.0L / 5.0L);
    out->status = ORACLE_OK;
    return ORACLE_OK;
}

/* ---- Eq. (1) with the Gaussian kernel of Eq. (2): the density estimate -------- */
/* fhat(t_j) = (1 / (n h)) sum_i K((t_j - X_i) / h), one compensated sum per point. */
typedef struct {
    const double* x;
    int64_t n;
    double h;
    const double* t;
    int64_t m;
    double* out;
    int64_t next;
} eval_job;

static void* eval_worker(void* arg) {
    eval_job* jb = (eval_job*)arg;
    for (;;) {
        int64_t j = __atomic_fetch_add(&jb->next, 1, __ATOMIC_RELAXED);
        if (j >= jb->m) break;
        csum acc = {0, 0};
        for (int64_t i = 0; i < jb->n; ++i) {
            double u = (jb->t[j] - jb->x[i]) / jb->h;
            csum_add(&acc, inv_sqrt_2pi() * exp(-0.5 * u * u));
        }
        jb->out[j] = csum_value(&acc) / ((double)jb->n * jb->h);
    }
    return NULL;
}

int oracle_kde_eval(const double* x, int64_t n, double h, const double* t, int64_t m,
                    int nthreads, double* out) {
    if (!x || !t || !out || n < 1 || m < 0 || !(h > 0) || !isfinite(h)) return ORACLE_ERR_INVALID;
    eval_job jb = {x, n, h, t, m, out, 0};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    if (nthreads == 1 || m < 2) {
        eval_worker(&jb);
    } else {
        pthread_t th[1024];
        int started = 0;
        for (int k = 0; k < nthreads; ++k)
            if (pthread_create(&th[k], NULL, eval_worker, &jb) == 0) ++started;
        if (started == 0) eval_worker(&jb);
        for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
    }
    return ORACLE_OK;
}

/* ---- Q32.32 fixed point: the paper's arithmetic (Section 4.1) for the pair terms ----- */
/* Values are int64 raw with value = raw * 2^-32: 31 integer bits, 32 fractional bits,
 * a sign bit.  Products keep the high part of the exact 128-bit product, i.e. they
 * truncate toward minus infinity.  The data are z-scored first (Eq. 3), so the
 * pair differences are in units of the sample standard deviation; u = d * sigma / g. */
typedef int64_t q32;
#define Q_ONE ((q32)1 << 32)

q32 oracle_q32_mul(q32 a, q32 b) { return (q32)(((__int128)a * (__int128)b) >> 32); }

/* floor(2^32 exp(-w / 2)) for w = w_raw * 2^-32 >= 0, in long double. */
q32 oracle_q32_exp_half(q32 w) {
    long double wr = (long double)w / 4294967296.0L;
    long double e = expl(-0.5L * wr) * 4294967296.0L;
    return (q32)floorl(e);
}

/* One pair term He_r(u) exp(-u^2/2) in Q32.32 (without 1/sqrt(2 pi)); |He_r| into *pabs.
 * Pairs with |u| >= 64 or u^2 >= 45 give 0: there floor(2^32 exp(-u^2/2)) is already 0. */
static q32 q32_term(int r, q32 d, q32 ginv, double* pabs) {
    *pabs = 0.0;
    if (fabs((double)d * (double)ginv) >= 64.0 * 18446744073709551616.0) return 0;
    q32 u = oracle_q32_mul(d, ginv);
    q32 w = oracle_q32_mul(u, u);
    if (w >= 45 * Q_ONE) return 0;
    q32 p;
    if (r == 6) {          /* ((w - 15) w + 45) w - 15 */
        p = oracle_q32_mul(w - 15 * Q_ONE, w) + 45 * Q_ONE;
        p = oracle_q32_mul(p, w) - 15 * Q_ONE;
    } else {               /* (w - 6) w + 3 */
        p = oracle_q32_mul(w - 6 * Q_ONE, w) + 3 * Q_ONE;
    }
    *pabs = fabs((double)p) / 4294967296.0;
    return oracle_q32_mul(p, oracle_q32_exp_half(w));
}

typedef struct {
    const q32* z;
    int64_t n;
    int r;
    q32 ginv;
    __int128* row;
    double* rowabs;
    int64_t next;
} q32_job;

static void* q32_worker(void* arg) {
    q32_job* jb = (q32_job*)arg;
    for (;;) {
        int64_t b = __atomic_fetch_add(&jb->next, 1, __ATOMIC_RELAXED);
        int64_t i0 = b * ROW_BLOCK;
        if (i0 >= jb->n) break;
        int64_t i1 = i0 + ROW_BLOCK < jb->n ? i0 + ROW_BLOCK : jb->n;
        for (int64_t i = i0; i < i1; ++i) {
            __int128 s = 0;
            double a = 0.0, pa;
            for (int64_t j = i + 1; j < jb->n; ++j) {
                /* K^(r) is even (Eq. 5), but a truncating product is not odd in its
                   operand: the term is taken on the magnitude of the difference. */
                q32 dz = jb->z[i] - jb->z[j];
                s += q32_term(jb->r, dz < 0 ? -dz : dz, jb->ginv, &pa);
                a += pa;
            }
            jb->row[i] = s;
            jb->rowabs[i] = a;
        }
    }
    return NULL;
}

/* psi_r(g) with the pair sum of Eqs. (6)-(7) in Q32.32 on z = (x - mean) / sigma
 * (z truncated to Q32.32), everything else in binary64.  *sum_abs_he receives
 * sum_{i<j} |He_r(u_ij)| (in the same units as the terms) for error bounds. */
int oracle_psi_q32(const double* x, int64_t n, int r, double g, double mean, double sigma,
                   int nthreads, double* psi, double* sum_abs_he) {
    if (!x || !psi || n < 1 || (r != 4 && r != 6) || !(g > 0) || !(sigma > 0)) return ORACLE_ERR_INVALID;
    q32* z = (q32*)malloc(sizeof(q32) * (size_t)n);
    __int128* row = (__int128*)malloc(sizeof(__int128) * (size_t)n);
    double* rowabs = (double*)malloc(sizeof(double) * (size_t)n);
    if (!z || !row || !rowabs) { free(z); free(row); free(rowabs); return ORACLE_ERR_INVALID; }
    for (int64_t i = 0; i < n; ++i) {
        double zi = (x[i] - mean) / sigma;                        /* Eq. (3) */
        if (!(fabs(zi) < 536870912.0)) { free(z); free(row); free(rowabs); return ORACLE_ERR_INVALID; }
        z[i] = (q32)floor(zi * 4294967296.0);
    }
    q32_job jb = {z, n, r, (q32)floor(sigma / g * 4294967296.0), row, rowabs, 0};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    if (nthreads == 1) {
        q32_worker(&jb);
    } else {
        pthread_t th[1024];
        int started = 0;
        for (int t = 0; t < nthreads; ++t)
            if (pthread_create(&th[t], NULL, q32_worker, &jb) == 0) ++started;
        if (started == 0) q32_worker(&jb);
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    __int128 tot = 0;
    double abs_tot = 0.0;
    for (int64_t i = 0; i < n; ++i) { tot += row[i]; abs_tot += rowabs[i]; }
    free(z); free(row); free(rowabs);
    double he0 = (r == 6) ? -15.0 : 3.0;
    double nn = (double)n;
    double s = (double)tot / 4294967296.0;                        /* sum_{i<j} He_r exp(-u^2/2) */
    *psi = (2.0 * s + nn * he0) * inv_sqrt_2pi() / (nn * nn * pow(g, (double)(r + 1)));
    if (sum_abs_he) *sum_abs_he = abs_tot;
    return ORACLE_OK;
}

/* Algorithm 1 with the pair sums of Steps IV and VI in Q32.32 on z-scored data
 * (Eq. 3), the scalar steps in binary64; h comes out in the units of x (Eq. 4). */
int oracle_plugin_q32(const double* x, int64_t n, int nthreads, oracle_result* out) {
    if (!out) return ORACLE_ERR_INVALID;
    fill_nan(out);
    out->status = ORACLE_ERR_INVALID;
    if (!x || n < 2) return out->status;
    double nn = (double)n, mean, var;
    int st = oracle_moments(x, n, &mean, &var);
    if (st != ORACLE_OK) { out->status = st; return st; }
    out->mean = mean;
    out->sigma = sqrt(var);
    if (!(out->sigma > 0)) { out->status = ORACLE_ERR_DEGENERATE; return out->status; }
    out->psi8 = 105.0 / (32.0 * sqrt(PI) * pow(out->sigma, 9.0));
    out->g1 = pow(-2.0 * (-15.0 * inv_sqrt_2pi()) / (out->psi8 * nn), 1.0 / 9.0);
    st = oracle_psi_q32(x, n, 6, out->g1, mean, out->sigma, nthreads, &out->psi6, NULL);
    if (st != ORACLE_OK) { out->status = st; return st; }
    if (!(out->psi6 < 0)) { out->status = ORACLE_ERR_DOMAIN; return out->status; }
    out->g2 = pow(-2.0 * (3.0 * inv_sqrt_2pi()) / (out->psi6 * nn), 1.0 / 7.0);
    st = oracle_psi_q32(x, n, 4, out->g2, mean, out->sigma, nthreads, &out->psi4, NULL);
    if (st != ORACLE_OK) { out->status = st; return st; }
    if (!(out->psi4 > 0)) { out->status = ORACLE_ERR_DOMAIN; return out->status; }
    out->h = pow(1.0 / (2.0 * sqrt(PI)) / (out->psi4 * nn), 1.0 / 5.0);
    out->status = ORACLE_OK;
    return ORACLE_OK;
}
