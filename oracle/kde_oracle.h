/*
 * kde_oracle.h -- plain, slow, obviously correct CPU reference for the PLUGIN
 * bandwidth selector (Algorithm 1 of Gramacki, Sawerwain & Gramacki,
 * "FPGA-Based Bandwidth Selection for Kernel Density Estimation Using High
 * Level Synthesis Approach").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this library; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA library.
 *
 * Everything is IEEE binary64 except the *_ld brute-force entry points, which
 * use long double (binary128 on aarch64, x87 80-bit on x86-64).
 */
#ifndef KDE_ORACLE_H
#define KDE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORACLE_OK = 0,
    ORACLE_ERR_INVALID = 1,     /* null pointer, n < 2, r not in {4, 6}, g <= 0 or not finite */
    ORACLE_ERR_DEGENERATE = 2,  /* sigma == 0 */
    ORACLE_ERR_DOMAIN = 3       /* psi6 >= 0 (g2 undefined) or psi4 <= 0 (h undefined) */
};

/* How the O(n^2) double sum of Steps IV and VI is taken. */
enum {
    ORACLE_FORM_FULL = 0,       /* sum over all i and all j, as printed in Steps IV / VI */
    ORACLE_FORM_SYMMETRIC = 1   /* 2 * sum_{i<j} + n K^(r)(0), Eqs. (6) and (7) */
};

typedef struct {
    double mean, sigma, psi8, g1, psi6, g2, psi4, h;
    int status;
} oracle_result;

typedef struct {
    long double mean, sigma, psi8, g1, psi6, g2, psi4, h;
    int status;
} oracle_result_ld;

/* l-stage plug-in: psi[k] and g[k] belong to r = 2k + 4 (psi_4 .. psi_14);
 * the top one is the normal-scale functional (its g is NaN), unused ones NaN. */
typedef struct {
    double mean, sigma;
    double psi[6];
    double g[6];
    double h;
    int stages;
    int status;
} oracle_stage_result;

/* Step I: mean and unbiased variance (divisor n-1), two-pass. */
int oracle_moments(const double* x, int64_t n, double* mean, double* var);

/* K^(r)(u) for r in {4, 6} (the printed Hermite forms of Steps IV and VI) and
 * r in {8, 10} (the same form, for the stages above Algorithm 1's two). */
double oracle_kernel_deriv(int r, double u);

/* psi_r(g) = n^-2 g^-(r+1) sum_i sum_j K^(r)((X_i - X_j)/g), Steps IV / VI. */
int oracle_psi(const double* x, int64_t n, int r, double g, int form, int nthreads,
               double* psi);

/* Unnormalised block sum over i in [i0,i1), j in [j0,j1) with i < j of
 * K^(r)((X_i - X_j)/g); also the sum of absolute values of the same terms. */
int oracle_psi_block(const double* x, int64_t n, int64_t i0, int64_t i1, int64_t j0,
                     int64_t j1, int r, double g, double* sum, double* abs_sum);

/* The whole of Algorithm 1, Steps I-VII. */
int oracle_plugin(const double* x, int64_t n, int form, int nthreads, oracle_result* out);

/* The l-stage direct plug-in, l = stages in 1..4: psi_{2l+4} by the normal
 * scale, then psi_{2l+2}, ..., psi_4 each at the pilot bandwidth computed from
 * the one above it (the form of Steps III and V), then h (Step VII).  l = 2 is
 * Algorithm 1.  K^(r) for r in {4, 6, 8, 10}. */
int oracle_plugin_stages(const double* x, int64_t n, int stages, int form, int nthreads,
                         oracle_stage_result* out);

/* Brute force in long double: full double loop, plain summation. */
int oracle_plugin_ld(const double* x, int64_t n, oracle_result_ld* out);
int oracle_psi_ld(const double* x, int64_t n, int r, long double g, long double* psi);
int oracle_long_double_mantissa_bits(void);

/* Eq. (1) with the Gaussian kernel of Eq. (2): fhat(t_j) = (1/(n h)) sum_i
 * K((t_j - X_i)/h) for j < m, into out[j].  Threads over points; per-point
 * compensated sums, so the bits do not depend on the thread count. */
int oracle_kde_eval(const double* x, int64_t n, double h, const double* t, int64_t m,
                    int nthreads, double* out);

/* Q32.32 fixed point (Section 4.1): int64 raw, value = raw * 2^-32; products
 * keep the high part of the exact 128-bit product (truncation toward -inf). */
int64_t oracle_q32_mul(int64_t a, int64_t b);
/* floor(2^32 exp(-w/2)) for the Q32.32 value w >= 0 (long double). */
int64_t oracle_q32_exp_half(int64_t w);
/* psi_r(g), r in {4, 6}, with the pair sum in Q32.32 on z = (x - mean)/sigma
 * (Eq. 3, truncated to Q32.32), u = z-difference * (sigma/g) in Q32.32; the
 * exponential is the exactly truncated value.  *sum_abs_he (may be NULL) gets
 * sum_{i<j} |He_r(u_ij)| for error bounds. */
int oracle_psi_q32(const double* x, int64_t n, int r, double g, double mean, double sigma,
                   int nthreads, double* psi, double* sum_abs_he);
/* Algorithm 1 with the Steps IV / VI pair sums in Q32.32 (as oracle_psi_q32). */
int oracle_plugin_q32(const double* x, int64_t n, int nthreads, oracle_result* out);

#ifdef __cplusplus
}
#endif
#endif
