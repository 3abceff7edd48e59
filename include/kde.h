/*
 * kde.h -- C ABI of libkde, a GB300 (sm_103a) implementation of the two-stage
 * direct plug-in (PLUGIN) bandwidth selector for univariate Gaussian kernel
 * density estimation (Gramacki, Sawerwain & Gramacki, "FPGA-Based Bandwidth
 * Selection for Kernel Density Estimation Using High Level Synthesis Approach",
 * Algorithm 1 and Eqs. 1-8).
 *
 * Notation.  K = phi, the standard normal density (Eq. 2).  K^(r) is its r-th
 * derivative; for even r, K^(r)(u) = He_r(u) phi(u) with He_r the probabilists'
 * Hermite polynomial: He_4 = u^4 - 6u^2 + 3, He_6 = u^6 - 15u^4 + 45u^2 - 15
 * (Algorithm 1, Steps IV and VI).
 *
 * Conventions shared by every entry point.
 *  - All functions return a kde_status; none throws or aborts.  A non-OK return
 *    leaves a thread-local message readable with kde_last_error().
 *  - Pointers may be host or device memory unless stated otherwise; the library
 *    asks the CUDA runtime which, copies host data itself, and never keeps a
 *    caller pointer after the call returns (the server copies at submit).
 *  - The caller owns every buffer it passes.  The library owns its own device
 *    workspaces and frees them in kde_shutdown() or at process exit.  Each
 *    (device, stream) has one workspace; it keeps the plan of its last call
 *    (tiling and work-list) and a CUDA graph per plan, so a repeated call of the
 *    same shape does no host planning and replays one graph.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  When every
 *    output pointer is device memory the call only enqueues work on `stream`
 *    and returns; the status words in the device outputs are then the result.
 *    When an output is host memory the call waits for `stream` before it
 *    returns.
 *  - Precision: KDE_FP32 evaluates the O(n^2) pair terms in binary32 (exact
 *    differences on a per-sample fixed grid, exp on the FMA pipe, compensated
 *    per-thread sums) with sorting, moments, block and final sums and all
 *    scalar steps in binary64; KDE_FP64 does everything in binary64.
 *  - Every sample is sorted on the device first, so results do not depend on
 *    the order of the input values (bitwise).
 *  - psi values use the paper's normalisation n^-2 g^-(r+1) sum_i sum_j
 *    K^(r)((X_i - X_j)/g), diagonal i = j included (Steps IV and VI).
 *  - A pair evaluation is one unique unordered pair i < j (Eqs. 6-7 add the
 *    diagonal analytically); kde_psi on n values does n(n-1)/2 of them.
 */
#ifndef KDE_H
#define KDE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KDE_API __attribute__((visibility("default")))
#else
#define KDE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KDE_OK = 0,
    KDE_ERR_INVALID = 1,     /* null pointer, n < 2, r not in {4,6,8,10}, g <= 0 or not finite,
                                non-finite data, or data whose range overflows the format */
    KDE_ERR_DEGENERATE = 2,  /* sample standard deviation is zero (Step I) */
    KDE_ERR_DOMAIN = 3,      /* psi6 >= 0 (g2 undefined, Step V) or psi4 <= 0 (h undefined,
                                Step VII); fields after the failing step are NaN */
    KDE_ERR_OOM = 4,         /* device memory could not be reserved */
    KDE_ERR_CUDA = 5,        /* a CUDA runtime call failed; see kde_last_error() */
    KDE_ERR_TIMEOUT = 6,     /* a bounded wait ran out (server poll) */
    KDE_ERR_BUSY = 7         /* admission refused: request larger than the server's budget,
                                or the server is shutting down */
} kde_status;

/* KDE_FP32 holds each sample on a grid of step g 2^-F around its median, with
 * F = 21 - floor(log2(R / g)) for R the smaller of twice the 0.1%-99.9%
 * quantile radius and the largest deviation; pair differences on the grid are
 * exact.  When the grid is coarse (F < 16) the rounding residual of each value
 * is added to every difference as well.  Rounding only drops below the stated
 * accuracy for extreme R / g (e.g. clusters thousands of bandwidths apart),
 * where KDE_FP64 is the safer choice. */
/* KDE_Q32 is the paper's arithmetic (Section 4.1): the data are z-scored
 * (Eq. 3) and each pair term of Steps IV / VI is taken in Q32.32 fixed point
 * (int64, 32 fractional bits, products truncated toward -inf, exp by a Remez
 * polynomial), summed exactly; the scalar steps are binary64.  Its error on h
 * is of the scale of the paper's Table 4.  r in {4, 6} only; not served by
 * the continuous-batching server. */
typedef enum {
    KDE_FP32 = 0,            /* binary32 pair terms, binary64 elsewhere */
    KDE_FP64 = 1,            /* binary64 everywhere */
    KDE_Q32 = 2              /* Q32.32 fixed-point pair terms on z-scored data */
} kde_precision;

/* Every scalar of Algorithm 1 for one sample.  In a device-memory output the
 * struct is written by the GPU; status is KDE_OK when all fields are valid. */
typedef struct {
    double mean;   /* sample mean (used only to centre the data) */
    double sigma;  /* Step I: sqrt of the unbiased variance, divisor n-1 */
    double psi8;   /* Step II: normal-scale psi8 = 105 / (32 sqrt(pi) sigma^9) */
    double g1;     /* Step III: (-2 K^(6)(0) / (mu2 psi8 n))^(1/9) */
    double psi6;   /* Step IV: psi6(g1), Eq. 6 */
    double g2;     /* Step V: (-2 K^(4)(0) / (mu2 psi6 n))^(1/7) */
    double psi4;   /* Step VI: psi4(g2), Eq. 7 */
    double h;      /* Step VII: (R(K) / (mu2^2 psi4 n))^(1/5), in the units of x */
    int32_t status;/* kde_status of this sample */
    int32_t reserved;
} kde_result;

/* Results of the l-stage plug-in (kde_plugin_h_stages).  psi[k] and g[k]
 * belong to the order r = 2k + 4 (psi_4, psi_6, ..., psi_14): g[k] is the pilot
 * bandwidth psi_r was estimated at; the top order 2l + 4 holds the normal-scale
 * value (its g is NaN); unused entries are NaN. */
typedef struct {
    double mean, sigma;
    double psi[6];
    double g[6];
    double h;
    int32_t stages;
    int32_t status;
} kde_stage_result;

/*
 * kde_psi -- the functional psi_r(g) of Steps IV / VI (Eqs. 6-7) for a given g.
 *   x      n samples, binary64, host or device, contiguous.
 *   n      number of samples, n >= 2.
 *   r      derivative order, 4 or 6 (Steps IV, VI), or 8 or 10 (the same
 *          Hermite form, for plug-in stages above Algorithm 1's two).
 *   g      bandwidth > 0, in the units of x.
 *   prec   KDE_FP32 or KDE_FP64.
 *   out    one double, host or device: psi_r(g).  With a device `out` the call is
 *          asynchronous and a failed run writes NaN there.
 *   stream cudaStream_t or NULL.
 * Errors: KDE_ERR_INVALID (arguments, non-finite data), KDE_ERR_OOM, KDE_ERR_CUDA.
 */
KDE_API kde_status kde_psi(const double* x, int64_t n, int r, double g, kde_precision prec,
                   double* out, void* stream);

/*
 * kde_plugin_h -- Algorithm 1, Steps I-VII, for one sample: the bandwidth h and
 * every intermediate scalar.  x: n binary64 values (host or device); out: one
 * kde_result (host or device).  The steps run back to back on the device; no
 * scalar returns to the host between them.
 * Errors: as kde_psi, plus KDE_ERR_DEGENERATE and KDE_ERR_DOMAIN (also in
 * out->status).
 */
KDE_API kde_status kde_plugin_h(const double* x, int64_t n, kde_precision prec, kde_result* out,
                        void* stream);

/* As kde_plugin_h for binary32 samples (the pair path is the same; the moments
 * read the binary32 values and widen them to binary64). */
KDE_API kde_status kde_plugin_h_f32(const float* x, int64_t n, kde_precision prec, kde_result* out,
                            void* stream);

/*
 * kde_plugin_h_batch -- Algorithm 1 for m independent samples in one pass:
 * one moments launch, one persistent psi6 launch and one persistent psi4 launch
 * over a work-list of (sample, chunk of tile pairs) items, captured once in a
 * CUDA graph per batch shape and replayed.
 *   x_packed  all samples back to back, binary64, host or device.
 *   offsets   m+1 int64 offsets into x_packed (HOST memory), offsets[0] = 0,
 *             non-decreasing; sample k is x_packed[offsets[k] .. offsets[k+1]).
 *   m         number of samples, m >= 1.
 *   out       m kde_result, host or device.  A sample with n < 2 gets
 *             KDE_ERR_INVALID in its own status; the others still run.
 * Each sample's result is bitwise the same as kde_plugin_h on that sample alone
 * (the tiling and the summation order depend only on its n).
 */
KDE_API kde_status kde_plugin_h_batch(const double* x_packed, const int64_t* offsets, int64_t m,
                              kde_precision prec, kde_result* out, void* stream);

/*
 * kde_plugin_h_stages -- the l-stage direct plug-in, of which Algorithm 1 is
 * the case l = 2: psi_{2l+4} by the normal scale (Step II's formula for general
 * even order), then for r = 2l+2, ..., 4 the pilot bandwidth
 * g_r = (-2 K^(r)(0) / (mu2 psi_{r+2} n))^(1/(r+3)) (the form of Steps III and
 * V) and psi_r(g_r) (Steps IV and VI), then h (Step VII).
 *   stages  l in 1..4 (orders up to psi_10 are estimated from the data).
 *   out     one kde_stage_result, host or device (device: asynchronous).
 * Errors as kde_plugin_h; out->status holds the sample's status.
 */
KDE_API kde_status kde_plugin_h_stages(const double* x, int64_t n, int stages, kde_precision prec,
                                       kde_stage_result* out, void* stream);

/*
 * kde_psi_slots -- verification view of kde_psi: the per-chunk partial sums the
 * pair kernel writes before its final reduction.  The library first sorts the
 * sample in increasing order (psi_r does not depend on the order); indices
 * below refer to that sorted sample X_(1) <= ... <= X_(n).  Slot k holds the
 * sum of He_r(u) exp(-u^2/2), u = (X_(i) - X_(j))/g, over the unique pairs i < j
 * of chunk k of the upper triangle of tile pairs, tile side `tile` (tile pairs
 * (I, J), I <= J, numbered row by row; chunk k is tile pairs
 * [k*chunk, (k+1)*chunk)).
 *   slots     host array of capacity `cap` doubles (may be NULL to query sizes).
 *   info      host int64[4]: {tile, chunk, n_tile_pairs, n_slots}.
 * Errors: KDE_ERR_INVALID when cap < n_slots and slots != NULL.
 */
KDE_API kde_status kde_psi_slots(const double* x, int64_t n, int r, double g, kde_precision prec,
                         double* slots, int64_t cap, int64_t* info);

/* ---- density estimate -------------------------------------------------------- */

/*
 * kde_eval -- the kernel density estimate of Eq. 1 with the Gaussian kernel of
 * Eq. 2 at m points: out[j] = (1 / (n h)) sum_i K((t[j] - x[i]) / h), usually
 * with the h of kde_plugin_h.
 *   x      n >= 1 binary64 sample values, host or device (read only).
 *   t      m >= 1 binary64 evaluation points, host or device (read only).
 *   h      bandwidth, finite and > 0.
 *   prec   KDE_FP32: differences as double-float pairs, MUFU ex2, compensated
 *          binary32 group sums folded into binary64 (every term is positive,
 *          so nothing cancels); points farther than ~13.2 h from every sample
 *          underflow to 0.  KDE_FP64: binary64 throughout.
 *   out    m doubles, host or device.  Host: the call waits.  Device:
 *          asynchronous on `stream`; invalid inputs then show as NaN in out.
 * Errors: KDE_ERR_INVALID for null pointers, n < 1, m < 1, bad h or precision,
 * a non-finite x or t, or (KDE_FP32) a value more than 1e7 bandwidths from the
 * sample median.  Deterministic for given (n, m, device).
 */
KDE_API kde_status kde_eval(const double* x, int64_t n, double h, const double* t, int64_t m,
                            kde_precision prec, double* out, void* stream);

/* ---- tile-configuration autotuner -------------------------------------------- */

/*
 * kde_autotune -- time every tile configuration of the pair kernel for `prec`
 * on the current device and use the fastest per size class from now on.  The
 * paper has no counterpart (its design is a fixed FPGA pipeline).  Each
 * configuration runs psi_6 (Step IV) on synthetic normal samples of n = 2^10,
 * 2^12, 2^14, 2^16 and 2^18 (device-resident, best of 3 after a warm-up); the
 * fastest is recorded for the size class n in [2^(k-1), 2^(k+1)) around each,
 * and 2^18 also serves every larger n.  The built-in choice is kept unless
 * another configuration is at least 3% faster.  Every later plan on this device
 * (kde_psi, kde_plugin_h, batch, server, static) consults the table.
 *   chosen  host int32[cap], cap >= 5, or NULL: the configuration index chosen
 *           for each size class, smallest first.
 * Tuning allocates a few MB of device memory and takes about a second for
 * KDE_FP32 (several seconds for KDE_FP64).  Results computed with another
 * configuration may differ in the last bits (within the stated tolerance).
 * Environment KDE_FP32_TILE_CONFIG / KDE_FP64_TILE_CONFIG still take priority.
 */
KDE_API kde_status kde_autotune(kde_precision prec, int32_t* chosen, int cap);
/* Forget the tuned table of `prec` on the current device: the built-in rule
 * applies again. */
KDE_API kde_status kde_autotune_clear(kde_precision prec);
/* The tile configuration a plan for n values of `prec` uses now on the current
 * device: info[0] configuration index, info[1] threads per block, info[2] rows
 * per thread (tile side T = threads x rows).  host int32[3]. */
KDE_API kde_status kde_tile_config(kde_precision prec, int64_t n, int32_t* info);

/* ---- allocation-free variant ---------------------------------------------------- */

/* Largest n kde_psi_static accepts. */
#define KDE_STATIC_MAX_N 65536

/*
 * kde_psi_static -- psi_r(g) as kde_psi computes it, for n <= KDE_STATIC_MAX_N,
 * using only a fixed scratch area of
 * about 1.6 MB compiled into the library as a device variable.  The paper has
 * no counterpart: this exists for callers that must not allocate device memory
 * on the call path, e.g. a process whose framework allocator already holds
 * most of HBM, or a latency-bound loop where cudaMalloc / cudaFree would
 * synchronise the device.  The call itself performs no device allocation.
 *   x       n binary64 values, host or device pointer (read only).
 *   out     1 double, host or device.  Host: the call waits for the result.
 *           Device: asynchronous on `stream`.
 * Set-up: the first call on a device, with that device current, looks up the
 * scratch area's address once (cudaGetSymbolAddress) and caches it; make that
 * first call before any stream capture.
 * Concurrency: one scratch area per device.  Calls from several host threads on
 * the same stream are serialised by a lock held while the call enqueues its
 * work; calls that overlap on the device (different streams) race on the area
 * -- order them on one stream.
 * Device reset: call kde_shutdown before cudaDeviceReset; the next call then
 * looks the scratch address up again (and is again a set-up call).
 * Errors: KDE_ERR_INVALID for n > KDE_STATIC_MAX_N (message says so), n < 2,
 * r not in {4, 6, 8, 10}, g <= 0 or not finite, null pointers, a bad precision.
 */
KDE_API kde_status kde_psi_static(const double* x, int64_t n, int r, double g, kde_precision prec,
                                  double* out, void* stream);

/* ---- serving: continuous batching of bandwidth-selection requests ---------- */

typedef struct kde_server kde_server;

typedef struct {
    size_t hbm_budget_bytes;   /* device memory the server may hold for requests */
    int32_t max_inflight;      /* admitted requests at most (>= 1) */
    int32_t device;            /* CUDA device ordinal */
    double tick_target_ms;     /* device time per scheduling tick (<= 0: default) */
} kde_server_config;

/* Per-request timing, host clock, nanoseconds since server creation, and the
 * unique pairs the r = 6 and r = 4 pair kernels skipped as far tile pairs
 * (every term below 1e-31 of the diagonal in binary32, exactly 0 in binary64):
 * the request evaluated n(n-1) - skipped6 - skipped4 pair terms. */
typedef struct {
    int64_t n;
    int32_t precision;
    int32_t status;
    int64_t t_submit_ns, t_admit_ns, t_done_ns;
    uint64_t skipped6, skipped4;
} kde_request_times;

/* Create a server; it reserves its device arena and starts its host thread. */
KDE_API kde_status kde_server_create(const kde_server_config* cfg, kde_server** out);
/* Enqueue one request; x (host, n binary32 values) is copied before return. */
KDE_API kde_status kde_server_submit(kde_server* s, const float* x, int64_t n, kde_precision prec,
                             uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a ticket; KDE_ERR_TIMEOUT if not done.
 * A finished ticket's result is returned once and then forgotten. */
KDE_API kde_status kde_server_poll(kde_server* s, uint64_t ticket, int32_t timeout_ms,
                           kde_result* out, kde_request_times* times);
/* Stop accepting, finish admitted work, free everything. */
KDE_API void kde_server_destroy(kde_server* s);

/* ---- profiling ----------------------------------------------------------------- */

/* Turn kernel timing on or off (process-wide, off by default).  While on, every
 * run records CUDA events around its kernels on the caller's stream (inside the
 * captured graph too). */
KDE_API kde_status kde_profile_enable(int on);
/* Wait for the last profiled run on `stream` and write the device time in ms of
 * its kernels: ms[0] init, sort, moments (Steps I-III) and the first prescale;
 * ms[1] pairs r = 6 (Steps IV-V; for kde_psi the one pairs launch); ms[2] the
 * second prescale; ms[3] pairs r = 4 (Steps VI-VII).  ms[2] and ms[3] are 0 for
 * kde_psi.  If cap >= 5, ms[4] is the number of kernel launches of that run
 * (the kernel nodes its CUDA graph replays).  If cap >= 7, ms[5] and ms[6] are
 * the unique pairs the r = 6 and r = 4 pair kernels skipped as far tile pairs
 * (every term at most |He_r(13.16)| 2^-125 in binary32, exactly 0 in binary64), summed over the
 * run's samples; this waits for the run.  cap >= 4.  KDE_ERR_INVALID if no
 * profiled run happened there. */
KDE_API kde_status kde_profile_last(void* stream, double* ms, int cap);

/* Measure sustained per-SM throughputs with dedicated microbenchmark kernels on
 * the current device (every block resident, CUDA-event timing): out[0] FP32 FMA
 * lane-operations per second per SM, out[1] MUFU ex2 results per second per SM,
 * out[2] FP64 FMA lane-operations per second per SM, out[3] SM count, out[4]
 * ticks per second of the SM cycle counter during the FP32 run.  cap >= 5.
 * Divided by the SM clock these size the ALU roofline of the pair kernels. */
KDE_API kde_status kde_probe_pipe_rates(double* out, int cap);

/* ---- misc -------------------------------------------------------------------- */

/* Thread-local text of the last error on this thread ("" if none). */
KDE_API const char* kde_last_error(void);
/* Library version string. */
KDE_API const char* kde_version(void);
/* Free the library's cached device workspaces and graphs (optional). */
KDE_API void kde_shutdown(void);

#ifdef __cplusplus
}
#endif
#endif /* KDE_H */
