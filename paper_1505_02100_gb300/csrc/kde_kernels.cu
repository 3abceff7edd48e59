// kde_kernels.cu -- device code of libkde.
//
// Algorithm 1 of Gramacki, Sawerwain & Gramacki runs as these kernels per batch:
//   moments_kernel   Step I (mean, unbiased variance), Steps II-III (psi8^NS, g1)
//   pairs_kernel<6>  Step IV (psi6(g1), Eq. 6) and Step V (g2)
//   pairs_kernel<4>  Step VI (psi4(g2), Eq. 7) and Step VII (h)
// The last CTA to finish a sample's share of a kernel takes that sample's next
// scalar step, so no scalar goes back to the host between steps.
//
// Before them, every sample is sorted (kde_sort.cu) and, per psi, scaled once
// (prescale_kernel): binary32 samples onto an exact-difference grid, binary64
// samples to u-units (X - median) / g.  The pair kernels evaluate K^(r)(u) =
// He_r(u) phi(u) for every unique pair, u = (X_i - X_j) / g: the binary32 path
// spends an exact FADD for the difference, an FMUL for u^2, a clamp, 6
// instructions of range reduction and exponent insertion plus an 8-FFMA
// polynomial for exp(-u^2/2), r/2 Horner FFMAs on the integer Hermite
// coefficients, one FMUL for the term and four instructions of compensated
// accumulation.  The 1/sqrt(2 pi), the factor 2 and the diagonal n K^(r)(0)
// of Eqs. 6-7 are applied once, in binary64, at the end.
#include "kde_internal.cuh"

#include <math_constants.h>

#include <cfloat>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

namespace kde {
namespace {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ex2_approx_ftz(float t) {
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(t));
  return e;
}

__device__ __forceinline__ double load_x(const void* x, int f32, int64_t i) {
  return f32 ? static_cast<double>(__ldg(static_cast<const float*>(x) + i))
             : __ldg(static_cast<const double*>(x) + i);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order (warp trees, then warps in index order);
// every thread gets the result.  `red` holds THREADS/32 + 1 doubles.
template <int THREADS>
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < THREADS / 32; ++i) s += red[i];
    red[THREADS / 32] = s;
  }
  __syncthreads();
  const double r = red[THREADS / 32];
  __syncthreads();
  return r;
}

template <int THREADS, bool MAX>
__device__ double block_minmax(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_down_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, u) : fmin(v, u);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = red[0];
    for (int i = 1; i < THREADS / 32; ++i) s = MAX ? fmax(s, red[i]) : fmin(s, red[i]);
    red[THREADS / 32] = s;
  }
  __syncthreads();
  const double r = red[THREADS / 32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void set_nan_result(kde_result& r) {
  const double q = CUDART_NAN;
  r.mean = r.sigma = r.psi8 = r.g1 = r.psi6 = r.g2 = r.psi4 = r.h = q;
}

// Representation of the next psi evaluation at bandwidth g (see the notes in
// kde_internal.cuh): scale, binary32 grid exponent F and padding values.  Returns false (and sets KDE_ERR_INVALID) when g or the data
// range cannot be represented.  Padding sits kPadMargin bandwidths beyond the
// data on either side, so every term that involves it is exactly zero.
__device__ bool set_psi_scale(SampleState* st, double g, int prec) {
  if (!(g > 0.0) || !isfinite(g)) {
    st->res.status = KDE_ERR_INVALID;
    return false;
  }
  const double c = st->center;
  const double W = fmax(st->xmax - c, c - st->xmin) / g;   // max |u| of any sample from c
  st->g_cur = g;
  if (prec == KDE_FP32) {
    // bulk radius in u-units: the window [-2^(22-F), 2^(22-F)) holds it
    const double bulk = fmax(st->qhi - c, c - st->qlo) / g;
    const double zr = fmin(W, 2.0 * bulk);
    int F = kFMax;
    if (zr > 0.0) F = 21 - static_cast<int>(floor(log2(zr)));
    F = F < kFMin ? kFMin : (F > kFMax ? kFMax : F);
    const double two_f = ldexp(1.0, F);
    if (!(W * two_f < kFp32RangeLimit)) {
      st->res.status = KDE_ERR_INVALID;
      return false;
    }
    const double P = (W + kPadMargin) * two_f;
    st->F = F;
    st->scale = two_f / g;
    st->pad_lo = kYBias - P;
    st->pad_hi = kYBias + P;
  } else if (prec == KDE_Q32) {
    // z-scored values (Eq. 3); the kernel takes u = z-difference * (sigma / g)
    const double sigma = st->res.sigma;
    if (!(sigma > 0.0)) {
      st->res.status = KDE_ERR_DEGENERATE;
      return false;
    }
    const double zmax = fmax(st->xmax - st->res.mean, st->res.mean - st->xmin) / sigma;
    if (!(zmax < kQ32ZLimit)) {
      st->res.status = KDE_ERR_INVALID;
      return false;
    }
    st->F = 0;
    st->scale = sigma / g;
    st->pad_hi = kQ32ZLimit + 1.0;   // z units: padding is never within 64 bandwidths
    st->pad_lo = -st->pad_hi;
  } else {
    if (!(W < kFp64RangeLimit)) {
      st->res.status = KDE_ERR_INVALID;
      return false;
    }
    st->F = 0;
    st->scale = 1.0 / g;
    st->pad_hi = W + kPadMargin;
    st->pad_lo = -st->pad_hi;
  }
  return true;
}

// K^(r)(0) = He_r(0) / sqrt(2 pi)
__device__ __forceinline__ double kernel_deriv_at_zero(int r) {
  return (r == 4 ? 3.0 : r == 6 ? -15.0 : r == 8 ? 105.0 : r == 10 ? -945.0 : 10395.0) /
         sqrt(2.0 * kPi);
}

// psi_r by the normal scale (Step II's formula for general even r):
// (-1)^(r/2) r! / ((2 sigma)^(r+1) (r/2)! sqrt(pi)).
__device__ __forceinline__ double normal_scale_psi(int r, double sigma) {
  double num = 1.0, den = 1.0;
  for (int k = 2; k <= r; ++k) num *= k;
  for (int k = 2; k <= r / 2; ++k) den *= k;
  const double v = num / (pow(2.0 * sigma, r + 1.0) * den * sqrt(kPi));
  return (r / 2) % 2 ? -v : v;
}

// Record psi_r (and the pilot it was taken at) in the stage results and in the
// Algorithm-1 fields that correspond to it.
__device__ __forceinline__ void record_psi(SampleState* st, int r, double psi, double g) {
  st->sres.psi[r / 2 - 2] = psi;
  st->sres.g[r / 2 - 2] = g;
  if (r == 8) st->res.psi8 = psi;
  if (r == 6) { st->res.psi6 = psi; st->res.g1 = g; }
  if (r == 4) { st->res.psi4 = psi; st->res.g2 = g; }
}

// Pilot bandwidth for psi_r from psi_{r+2} (Steps III and V, mu2 = 1); sets the
// scale of the next pair launch for precision `prec`.  false (DOMAIN) if the
// ratio is not positive.
__device__ bool next_pilot(SampleState* st, int r, double psi_up, double n, int prec) {
  const double ratio = -2.0 * kernel_deriv_at_zero(r) / (psi_up * n);
  if (!(ratio > 0.0)) {
    st->res.status = KDE_ERR_DOMAIN;
    return false;
  }
  const double g = pow(ratio, 1.0 / (r + 3.0));
  st->sres.g[r / 2 - 2] = g;
  if (r == 6) st->res.g1 = g;
  if (r == 4) st->res.g2 = g;
  return set_psi_scale(st, g, prec);
}

// ---------------------------------------------------------------------------
// init: every result field NaN, status OK (or INVALID for n < 2), counters 0
// ---------------------------------------------------------------------------

__global__ void init_states_kernel(const SampleDesc* desc, SampleState* state, int64_t m,
                                   unsigned long long* counters, int n_counters) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n_counters) counters[k] = 0ull;
  if (k >= m) return;
  SampleState* st = state + k;
  set_nan_result(st->res);
  st->res.status = desc[k].n >= 2 ? KDE_OK : KDE_ERR_INVALID;
  st->res.reserved = 0;
  st->xmin = st->xmax = st->g_cur = st->scale = st->pad_lo = st->pad_hi = st->psi_out = CUDART_NAN;
  st->center = st->qlo = st->qhi = CUDART_NAN;
  st->F = 0;
  st->reserved = 0;
  st->done_mom = 0;
  st->done_pairs = 0;
  st->skipped[0] = st->skipped[1] = 0;
  st->sres.mean = st->sres.sigma = st->sres.h = CUDART_NAN;
  for (int q = 0; q < 6; ++q) st->sres.psi[q] = st->sres.g[q] = CUDART_NAN;
  st->sres.stages = desc[k].stages;
}

// The l-stage result of each sample from its state (after the last pair launch).
__global__ void stage_results_kernel(SampleState* state, int64_t m) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= m) return;
  SampleState* st = state + k;
  st->sres.mean = st->res.mean;
  st->sres.sigma = st->res.sigma;
  st->sres.h = st->res.h;
  st->sres.status = st->res.status;
}

// ---------------------------------------------------------------------------
// Step I (+ Steps II-III): per-block two-pass moments, merged in block order
// ---------------------------------------------------------------------------

struct Moments {
  double cnt, mean, m2, mn, mx;
};

// Chan, Golub & LeVeque pairwise update of (count, mean, M2).
__device__ __forceinline__ Moments merge(const Moments& a, const Moments& b) {
  if (b.cnt == 0.0) return a;
  if (a.cnt == 0.0) return b;
  Moments r;
  r.cnt = a.cnt + b.cnt;
  const double delta = b.mean - a.mean;
  r.mean = a.mean + delta * (b.cnt / r.cnt);
  r.m2 = a.m2 + b.m2 + delta * delta * (a.cnt * b.cnt / r.cnt);
  r.mn = fmin(a.mn, b.mn);
  r.mx = fmax(a.mx, b.mx);
  return r;
}

__global__ void __launch_bounds__(kMomThreads) moments_kernel(MomentsArgs a) {
  __shared__ double red[kMomThreads / 32 + 1];
  __shared__ Moments tup[kMomMaxBlocks];
  __shared__ int s_last;
  const int tid = threadIdx.x;

  // which sample does this block belong to (prefix sums of blocks per sample)
  const int64_t b = blockIdx.x;
  int64_t lo = 0, hi = a.m;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (a.mprefix[mid] <= b) lo = mid; else hi = mid;
  }
  const int64_t k = a.ids ? static_cast<int64_t>(a.ids[lo]) : lo;
  const SampleDesc d = a.desc[k];
  SampleState* st = a.state + k;
  const int64_t lb = b - a.mprefix[lo];
  const int64_t i0 = lb * d.mchunk;
  const int64_t i1 = (i0 + d.mchunk < d.n) ? i0 + d.mchunk : d.n;

  // pass 1: block-local mean
  double s = 0.0;
  for (int64_t i = i0 + tid; i < i1; i += kMomThreads) s += load_x(a.x, a.x_is_f32, d.x_off + i);
  const double cnt = static_cast<double>(i1 - i0);
  const double lmean = block_sum<kMomThreads>(s, red) / cnt;
  // pass 2: sum of squared deviations from the local mean, min, max
  double q = 0.0, mn = CUDART_INF, mx = -CUDART_INF;
  for (int64_t i = i0 + tid; i < i1; i += kMomThreads) {
    const double v = load_x(a.x, a.x_is_f32, d.x_off + i);
    const double c = v - lmean;
    q += c * c;
    mn = fmin(mn, v);
    mx = fmax(mx, v);
    if (!isfinite(v)) q = CUDART_NAN;   // propagate: non-finite data is invalid
  }
  q = block_sum<kMomThreads>(q, red);
  mn = block_minmax<kMomThreads, false>(mn, red);
  mx = block_minmax<kMomThreads, true>(mx, red);

  if (tid == 0) {
    double* t = a.mslots + d.mslot_off + lb * 5;
    t[0] = cnt; t[1] = lmean; t[2] = q; t[3] = mn; t[4] = mx;
    __threadfence();
    const unsigned prev = atomicAdd(&st->done_mom, 1u);
    s_last = (prev + 1 == static_cast<unsigned>(d.mblocks));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // last block of this sample: merge the block tuples in a fixed tree order
  const int nb = static_cast<int>(d.mblocks);
  if (tid < nb) {
    const double* t = a.mslots + d.mslot_off + tid * 5;
    tup[tid] = Moments{__ldcg(t), __ldcg(t + 1), __ldcg(t + 2), __ldcg(t + 3), __ldcg(t + 4)};
  }
  __syncthreads();
  for (int stride = 1; stride < nb; stride <<= 1) {
    if ((tid % (2 * stride)) == 0 && tid + stride < nb) tup[tid] = merge(tup[tid], tup[tid + stride]);
    __syncthreads();
  }
  if (tid != 0) return;

  st->done_mom = 0;
  const Moments M = tup[0];
  const double n = static_cast<double>(d.n);
  st->res.mean = M.mean;
  st->xmin = M.mn;
  st->xmax = M.mx;
  if (!isfinite(M.mean) || !isfinite(M.m2) || !isfinite(M.mn) || !isfinite(M.mx)) {
    st->res.status = KDE_ERR_INVALID;
    return;
  }
  const double sigma = sqrt(M.m2 / (n - 1.0));            // Step I
  st->res.sigma = sigma;
  {  // the sample is sorted: median and 0.1% / 99.9% quantiles by index
    const int64_t ilo = (d.n - 1) / 1000, ihi = d.n - 1 - ilo, imid = (d.n - 1) / 2;
    st->center = load_x(a.x, a.x_is_f32, d.x_off + imid);
    st->qlo = load_x(a.x, a.x_is_f32, d.x_off + ilo);
    st->qhi = load_x(a.x, a.x_is_f32, d.x_off + ihi);
  }
  double g;
  if (d.g_fixed > 0.0) {
    g = d.g_fixed;                                          // stand-alone psi_r(g)
  } else {
    if (!(sigma > 0.0)) {
      st->res.status = KDE_ERR_DEGENERATE;
      return;
    }
    // Step II: the top functional by the normal scale (psi_8 for Algorithm 1's
    // two stages, psi_{2l+4} for l stages); Step III: the first pilot
    const int top = 2 * d.stages + 4;
    const double psi_ns = normal_scale_psi(top, sigma);
    st->sres.psi[top / 2 - 2] = psi_ns;
    if (top == 8) st->res.psi8 = psi_ns;
    if (top == 6) st->res.psi6 = psi_ns;
    next_pilot(st, top - 2, psi_ns, n, d.prec);
    return;
  }
  set_psi_scale(st, g, d.prec);
}

// ---------------------------------------------------------------------------
// Scaled values for the pair kernel, once per sample and psi (O(n))
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kPrescaleThreads) prescale_kernel(PrescaleArgs a) {
  const int64_t b = blockIdx.x;
  int64_t lo = 0, hi = a.m;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (a.bprefix[mid] <= b) lo = mid; else hi = mid;
  }
  const int64_t k = a.ids ? static_cast<int64_t>(a.ids[lo]) : lo;
  const SampleDesc& d = a.desc[k];
  const int64_t i = (b - a.bprefix[lo]) * kPrescaleThreads + threadIdx.x;
  if (i >= d.n) return;
  const SampleState& st = a.state[k];
  if (st.res.status != KDE_OK) return;
  const double z = __dmul_rn(__dsub_rn(load_x(a.x, a.x_is_f32, d.x_off + i), st.center), st.scale);
  if (d.prec == KDE_Q32) {
    // Eq. 3 in binary64, then truncated to Q32.32
    const double zz = __ddiv_rn(__dsub_rn(load_x(a.x, a.x_is_f32, d.x_off + i), st.res.mean), st.res.sigma);
    static_cast<long long*>(a.y)[d.y_off + i] = static_cast<long long>(floor(__dmul_rn(zz, 4294967296.0)));
    return;
  }
  if (d.prec == KDE_FP32) {
    // grid value and what rounding to it left over: hi + lo = kYBias + z to ~2^-24
    // the grid scaled by 2^-F (exact): differences come out in u-units
    const float hi_grid = static_cast<float>(kYBias + rint(z));
    const float hi = ldexpf(hi_grid, -st.F);
    const float lo = static_cast<float>(ldexp((kYBias + z) - static_cast<double>(hi_grid), -st.F));
    static_cast<float2*>(a.y)[d.y_off + i] = make_float2(hi, lo);
  } else {
    static_cast<double*>(a.y)[d.y_off + i] = z;
  }
}

// ---------------------------------------------------------------------------
// Steps IV / VI: persistent triangular-tile pair kernel
// ---------------------------------------------------------------------------

// T: the arithmetic type of the pair terms; Y: the stored scaled value
// (binary32: grid value and rounding residual; binary64: u-units).
template <int PREC> struct Arith;
template <> struct Arith<KDE_FP32> { using T = float; using Y = float2; };
template <> struct Arith<KDE_FP64> { using T = double; using Y = double; };
__device__ __forceinline__ float hi_of(float2 v) { return v.x; }
__device__ __forceinline__ float lo_of(float2 v) { return v.y; }
__device__ __forceinline__ double hi_of(double v) { return v; }
__device__ __forceinline__ float lo_of(double) { return 0.0f; }

// The polynomial (non-factorised) binary32 path always adds the rounding
// residuals to each difference (two more FADDs per pair), so that every pair term
// sees the exact data.  Grid values alone would perturb each value by up to half
// a grid step: on a grid of step g 2^-F that moves psi_r by up to ~1e-5 at F = 13,
// and even on fine grids the per-tile-pair effect (~1e-6 of a tile pair's sum of
// |terms|) only cancels over the whole triangle when every pair sees the same
// rounded data -- it does not once the factorised path (which works on the exact
// values) takes some of the tile pairs.

// Hermite factor of K^(r) on v = u^2, u = (X_i - X_j)/g, with the integer
// coefficients printed in Steps IV and VI (exact in binary32):
//   He_6 = ((v - 15) v + 45) v - 15,   He_4 = (v - 6) v + 3.
// `h` = 1/2 halves every coefficient exactly (diagonal tile pairs).  Rounding
// these coefficients (e.g. after absorbing a base change into them) would
// distort He_r, and the pair sum cancels so strongly (sum |terms| / |sum| grows
// like (sigma/g)^6, ~1e4 at n = 2^20) that binary32 would lose several digits.
template <typename T, int RORD>
struct Coef {
  // Horner coefficients, highest power first.  r <= 6: polynomial in v with the
  // powers of p2 folded in (exact: integers times powers of two).  r >= 8:
  // polynomial in w = v p2 = u^2 (integer coefficients), because p2^(r/2)
  // would leave the binary32 range for fine grids.
  static constexpr int K = RORD / 2 + 1;
  static constexpr bool kOnW = RORD >= 8;
  T c[K];
  // h = 1 or 1/2; p2 = 2^(-2F) turns v in grid units into u^2 (exact)
  __device__ void set(double h, double p2) {
    // He_r(u) = sum_k a[k] u^(2 (K-1-k)), coefficients of the Hermite forms
    // printed in Steps IV and VI and their continuation for r = 8, 10
    const double a4[3] = {1.0, -6.0, 3.0};
    const double a6[4] = {1.0, -15.0, 45.0, -15.0};
    const double a8[5] = {1.0, -28.0, 210.0, -420.0, 105.0};
    const double a10[6] = {1.0, -45.0, 630.0, -3150.0, 4725.0, -945.0};
    const double* a = RORD == 4 ? a4 : RORD == 6 ? a6 : RORD == 8 ? a8 : a10;
    for (int k = 0; k < K; ++k) {
      double scale = h;
      if (!kOnW)
        for (int e = 0; e < K - 1 - k; ++e) scale *= p2;
      c[k] = static_cast<T>(a[k] * scale);
    }
  }
  template <typename U>
  __device__ __forceinline__ U horner(U x) const {   // x = v (r <= 6) or w (r >= 8)
    U p = c[0];
#pragma unroll
    for (int k = 1; k < K; ++k) p = fma(p, x, c[k]);
    return p;
  }
};

// He_r(0) for the diagonal: (-1)^(r/2) (r - 1)!!
template <int RORD>
__host__ __device__ constexpr double he_at_zero() {
  return RORD == 4 ? 3.0 : RORD == 6 ? -15.0 : RORD == 8 ? 105.0 : -945.0;
}

// exp(-u^2/2) in binary32 on the FMA pipe, as 2^t with t = -u^2 / (2 ln 2).
// With w = u^2 (the values are stored in u-units), t = -w c with c = 1 / (2 ln 2)
// = kCHi + c_lo split into two binary32 values.  k = round(w kCHi) by the
// 1.5 * 2^23 rounding trick, f = k - w kCHi in [-1/2, 1/2] from one FFMA (the
// exact value of a 48-bit product minus an integer, rounded once), 2^f by a
// degree-8 minimax polynomial (a Remez fit, p(0) = 1 exactly; with its
// coefficients in binary32 its relative error is 1.3e-9, from float32(ln 2)),
// and k goes straight into the exponent field.
// That is exp(-u^2/2) scaled by 2^(-w c_lo) = 1 - w c_lo ln 2 + O(1e-12).
//
// The c_lo factor is not applied to f or to the term: there it would be a
// smooth correction a few units in the last place, added to a value already
// on the binary32 grid, and rounding would drop the same fraction of it from
// every term -- a bias.  Instead the caller sums term * v per row in binary32
// (one FFMA per pair) and subtracts c_lo ln 2 times that sum, in binary64,
// from a correction total of its own.  (Folding it into the Kahan sum does
// not work: the compensation term keeps only the bits above half an ulp of
// the next, much larger, partial sum added to it.)
//
// The pair sum cancels so strongly (sum |terms| / |sum| ~ 2e4 for psi6 at
// n = 2^20, growing like (sigma/g)^6) that any bias of the exponential at the
// 1e-10 level shows.  Measured or projected exactly over every grid distance
// on normal data at n = 2^20: the MUFU ex2 unit (~3e-8 rms) costs 1.6e-4 on
// psi6; rounding c to one binary32 (a dilation of the Gaussian but not of
// He_r) ~2e-6 on psi4; folding c_lo into f ~1e-5 on psi6; a natural-base
// reduction whose last step rounds a value on a grid coarser than its result
// (t - k ln2_hi with t large) ~8e-6 on psi6.
// u^2 is clamped to 125 * 2 ln 2 (~173): beyond it every term is below 1e-31,
// the exponent stays normal and He_r stays finite.  Tile pairs whose largest
// distance is below the clamp skip it (CLAMP = false).  Since every scaling by
// 2^-F is exact, these terms are bit for bit those of the grid units.
constexpr float kRoundMagic = 12582912.0f;                 // 1.5 * 2^23
constexpr double kInvTwoLn2 = 0.72134752044448170367996234050095;
constexpr float kMinT = 125.0f;
// The binary32 pair terms work in u-units (w = u^2): c = 1 / (2 ln 2) = kCHi + c_lo
constexpr float kCHi = static_cast<float>(kInvTwoLn2);
constexpr double kCLoLn2 = (kInvTwoLn2 - static_cast<double>(kCHi)) * 0.69314718055994530942;
constexpr float kWMax = kMinT / kCHi;   // u^2 clamp (~173)

__device__ __forceinline__ float exp2_reduced(float f) {
  float q = 1.3344183e-06f;
  q = __fmaf_rn(q, f, 1.5314209e-05f);
  q = __fmaf_rn(q, f, 1.5403098e-04f);
  q = __fmaf_rn(q, f, 1.3333434e-03f);
  q = __fmaf_rn(q, f, 9.6181296e-03f);
  q = __fmaf_rn(q, f, 5.5504110e-02f);
  q = __fmaf_rn(q, f, 2.4022651e-01f);
  q = __fmaf_rn(q, f, 6.9314718e-01f);
  return __fmaf_rn(q, f, 1.0f);
}

// One pair term, binary32, without its 2^(-w c_lo) factor: d = u = y_i - y_j
// (exact on the grid, in u-units).  The constants are compile-time immediates:
// Hermite coefficients are the integers of Steps IV / VI (and their
// continuation for r = 8, 10); a diagonal tile pair halves its sum afterwards.
// `wout` receives w = u^2: the term is too large by the relative amount w c_lo ln 2.
template <int RORD, bool CLAMP>
__device__ __forceinline__ float term32(float d, float& wout) {
  const float w = CLAMP ? fminf(__fmul_rn(d, d), kWMax) : __fmul_rn(d, d);   // u^2
  const float yb = __fmaf_rn(w, -kCHi, kRoundMagic);      // low bits: k = round(t)
  const float kf = __fsub_rn(yb, kRoundMagic);
  const float f = __fmaf_rn(w, -kCHi, -kf);               // t - k (c_hi part)
  const float e = __int_as_float(__float_as_int(exp2_reduced(f)) + (__float_as_int(yb) << 23));
  float p;
  if (RORD == 4) p = __fmaf_rn(__fadd_rn(w, -6.0f), w, 3.0f);
  else if (RORD == 6) p = __fmaf_rn(__fmaf_rn(__fadd_rn(w, -15.0f), w, 45.0f), w, -15.0f);
  else if (RORD == 8)
    p = __fmaf_rn(__fmaf_rn(__fmaf_rn(__fadd_rn(w, -28.0f), w, 210.0f), w, -420.0f), w, 105.0f);
  else
    p = __fmaf_rn(__fmaf_rn(__fmaf_rn(__fmaf_rn(__fadd_rn(w, -45.0f), w, 630.0f), w, -3150.0f), w, 4725.0f),
                  w, -945.0f);
  wout = w;
  return __fmul_rn(p, e);
}

template <int RORD>
__device__ __forceinline__ double term64(double a, double b, const Coef<double, RORD>& cf,
                                         double acc) {
  const double d = __dsub_rn(a, b);
  const double v = __dmul_rn(d, d);
  const double p = cf.horner(v);   // u-units: v = u^2 = w
  return fma(p, exp(-0.5 * v), acc);
}

// Compensated (Kahan) accumulator, binary32.  The sum is s - c.
struct Kahan32 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const {
    return static_cast<double>(s) - static_cast<double>(c);
  }
};

// ---------------------------------------------------------------------------
// Binary32 pair terms with the Gaussian factorised over a tile pair
// ---------------------------------------------------------------------------
// The sample is sorted, so a row tile and a segment of a column tile each hold a
// narrow range of values.  With row values a_i = a0 + alpha_i, column values
// b_j = b0 + beta_j and Delta = a0 - b0 (u-units), u = a_i - b_j satisfies
//   -u^2/2 = -alpha_i (Delta + alpha_i/2) + [beta_j (Delta - beta_j/2) - Delta^2/2]
//            + alpha_i beta_j,
// so exp(-u^2/2) = R_i C_j exp(alpha_i beta_j) exactly.  R_i (per row) and C_j
// (per column, with exp(-Delta^2/2) folded in) are evaluated once per row and
// column of a segment by an accurate exponential; the coupling factor is the
// Taylor polynomial of exp(p), p = alpha_i beta_j, to order K:
//   K = 2: 1 + p + p^2/2, truncation p^3/6 <= 1.7e-10 while A B <= kFacP2,
//   K = 1: 1 + p,         truncation p^2/2 <= 8e-12   while A B <= kFacP1
// (A, B: half-widths of the row tile and the segment).  Every pair term
// He_r(u^2) exp(-u^2/2) is still evaluated on its own:
//   u = (a_i - b0) - beta_j,  w = u^2,  He_r(w) by Horner,
//   e = C_j + alpha_i (C_j beta_j) [+ (alpha_i^2/2) (C_j beta_j^2)],
//   row sum += He_r(w) e,
// and R_i multiplies the row's sum once per segment: r/2 + 4 (K = 1) or r/2 + 5
// (K = 2) FMA-pipe operations per pair.  The factors carry only rounding errors
// (no smooth bias), and no term depends on a rounded constant, so the c_lo
// correction of the polynomial path is not needed here.
//
// Segments are aligned power-of-two column ranges of 32 ... 512.  A tile pair
// takes one width and order from the column tile's overall half-width (the
// cheaper of K = 1 at the widest width it allows and K = 2 at the widest width
// it allows); every segment
// then checks its own half-width and falls back to K = 2, or to the polynomial
// path, where needed.  A segment of width w costs each thread about
// (kSegRowOps + kSegFixedOps / ROWS) / w slots per pair on top of the pairs.
constexpr int kSub = 128;                        // columns per binary64 sub-tile
constexpr int kSegMax = 512, kSegMin = 32;       // binary32 segment widths
constexpr float kFacP1 = 4.0e-6f;                // A B bound for the 2-term coupling
constexpr float kFacP2 = 1.0e-3f;                // A B bound for the 3-term coupling
constexpr float kFacXMax = 2.0f;                 // |exponent| bound of R_i and of C_j / exp(-Delta^2/2)
// Issue slots a segment costs each thread, beyond its pairs: ~24 per row (R_i, the
// fold into the accumulator) and ~50 shared (column factors, barriers, the checks).
constexpr float kSegRowOps = 24.0f, kSegFixedOps = 50.0f;
constexpr double kLog2e = 1.4426950408889634074;
constexpr float kLog2eHi = static_cast<float>(kLog2e);
constexpr float kLog2eLo = static_cast<float>(kLog2e - static_cast<double>(kLog2eHi));

// e^(xh + xl) in binary32 for a double-float exponent xh + xl <= 3 (|xl| <= 3, xl
// carrying what xh cannot), 0 below -86 (such factors only reach terms under e^-86
// of the diagonal).  k = round((xh + xl) log2 e).  xh (log2 e)_hi = ph + pl exactly
// (product and its FMA residual); ph - k is exact (an integer taken from a nearby
// binary32), so f = (ph - k) + xl (log2 e)_hi rounds once at |f| <= 1/2, and the
// small parts pl + xh (log2 e)_lo follow.  2^f by the degree-8 polynomial above,
// k into the exponent field (a normal result: -125 <= k <= 5).
__device__ __forceinline__ float exp_factor(float xh, float xl) {
  const float s = __fadd_rn(xh, xl);
  if (s < -86.0f) return 0.0f;
  const float kb = __fmaf_rn(s, kLog2eHi, kRoundMagic);
  const float kf = __fsub_rn(kb, kRoundMagic);
  const float ph = __fmul_rn(xh, kLog2eHi);
  const float pl = __fmaf_rn(xh, kLog2eHi, -ph);
  float f = __fmaf_rn(xl, kLog2eHi, __fsub_rn(ph, kf));
  f = __fadd_rn(f, __fmaf_rn(xh, kLog2eLo, pl));
  return __int_as_float(__float_as_int(exp2_reduced(f)) + (__float_as_int(kb) << 23));
}

// e^x for |x| <= 3 (the row factors): k = round(x log2 e), f = x (log2 e)_hi - k
// from the exact product minus an integer, rounded once (|f| <= 1/2), plus
// x (log2 e)_lo; 2^f by the degree-8 polynomial, k into the exponent field.
__device__ __forceinline__ float exp_small(float x) {
  const float kb = __fmaf_rn(x, kLog2eHi, kRoundMagic);
  const float kf = __fsub_rn(kb, kRoundMagic);
  float f = __fmaf_rn(x, kLog2eHi, -kf);
  f = __fmaf_rn(x, kLog2eLo, f);
  return __int_as_float(__float_as_int(exp2_reduced(f)) + (__float_as_int(kb) << 23));
}

// He_r on w = u^2 with the integer coefficients of Steps IV / VI (and their
// continuation for r = 8, 10), exact in binary32.
template <int RORD>
__device__ __forceinline__ float hermite_w(float w) {
  if (RORD == 4) return __fmaf_rn(__fadd_rn(w, -6.0f), w, 3.0f);
  if (RORD == 6) return __fmaf_rn(__fmaf_rn(__fadd_rn(w, -15.0f), w, 45.0f), w, -15.0f);
  if (RORD == 8)
    return __fmaf_rn(__fmaf_rn(__fmaf_rn(__fadd_rn(w, -28.0f), w, 210.0f), w, -420.0f), w, 105.0f);
  return __fmaf_rn(__fmaf_rn(__fmaf_rn(__fmaf_rn(__fadd_rn(w, -45.0f), w, 630.0f), w, -3150.0f), w, 4725.0f),
                   w, -945.0f);
}

// He_r straight from u for r = 4 and 6.  In t = u^2 - (r - 1) the second-highest
// power of He_r(u) vanishes (r - 1 is the mean of its roots in u^2):
//   He_4 = t^2 - 6,          t = u^2 - 3,
//   He_6 = (t^2 - 30) t - 40, t = u^2 - 5,
// so the square folds into the first FMA, one operation fewer than Horner in
// w = u^2.  t is rounded once; near u = 0 its error (half an ulp of r - 1), times
// He_r's slope there, is about 1e-6 of the term -- an unbiased rounding like the
// others, which the pair sums average out.  Higher orders keep the Horner form in
// w, where the same shift would be amplified 30-45 times more.
template <int RORD>
__device__ __forceinline__ float hermite_u(float u) {
  if (RORD == 4) {
    const float t = __fmaf_rn(u, u, -3.0f);
    return __fmaf_rn(t, t, -6.0f);
  }
  if (RORD == 6) {
    const float t = __fmaf_rn(u, u, -5.0f);
    return __fmaf_rn(__fmaf_rn(t, t, -30.0f), t, -40.0f);
  }
  return hermite_w<RORD>(__fmul_rn(u, u));
}

// The column factors of one segment of `width` columns: fac[j] = (beta_j, C_j,
// C_j beta_j, C_j beta_j^2) with C_j = exp(beta_j (Delta - beta_j/2) - Delta^2/2);
// the exponent is formed as a double-float (Delta^2 split exactly by an FMA).
// Columns past the sample (j >= vc) get zero factors, so their terms vanish.
template <int THREADS>
__device__ __forceinline__ void column_factors(const float* __restrict__ tile, const float* __restrict__ tile_lo,
                                               int width, int vc, float b0, float delta,
                                               float4* __restrict__ fac) {
  const float dh = __fmul_rn(delta, delta);
  const float dl = __fmaf_rn(delta, delta, -dh);
  for (int j = threadIdx.x; j < width; j += THREADS) {
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (j < vc) {
      const float beta = __fadd_rn(__fsub_rn(tile[j], b0), tile_lo[j]);
      const float q = __fmaf_rn(beta, -0.5f, delta);
      const float xl = __fmaf_rn(beta, q, -0.5f * dl);
      const float c = exp_factor(-0.5f * dh, xl);
      const float cb = __fmul_rn(c, beta);
      v = make_float4(beta, c, cb, __fmul_rn(cb, beta));
    }
    fac[j] = v;
  }
}

// One segment, factorised: this thread's ROWS rows against `width` columns (a
// multiple of 16).  ap = a_i - b0, al = alpha_i, ah = alpha_i^2 / 2.  Per row,
// groups of 16 terms are accumulated by FMA (one rounding per term, the product
// exact) and each group goes into the row's Kahan sum; rs gets the compensated
// row sums (before R_i).
template <int RORD, int ROWS, int K>
__device__ __forceinline__ void tile_pass_fac(const float4* __restrict__ fac, int width, const float (&ap)[ROWS],
                                              const float (&al)[ROWS], const float (&ah)[ROWS],
                                              float (&rs)[ROWS]) {
  float sum[ROWS], comp[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) sum[r] = comp[r] = 0.0f;
#pragma unroll 1
  for (int jj = 0; jj < width; jj += 16) {
    float grp[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) grp[r] = 0.0f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float4 f = fac[jj + q];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const float h = hermite_u<RORD>(__fsub_rn(ap[r], f.x));
        float e = __fmaf_rn(al[r], f.z, f.y);
        if (K == 2) e = __fmaf_rn(ah[r], f.w, e);
        grp[r] = __fmaf_rn(h, e, grp[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const float y = __fsub_rn(grp[r], comp[r]);
      const float t = __fadd_rn(sum[r], y);
      comp[r] = __fsub_rn(__fsub_rn(t, sum[r]), y);
      sum[r] = t;
    }
  }
#pragma unroll
  for (int r = 0; r < ROWS; ++r) rs[r] = __fsub_rn(sum[r], comp[r]);
}

// One tile pair, FP32: this thread's ROWS rows against the TILE columns in
// shared memory.  Per row, each group of CJ terms (CJ / 4 float4s of columns)
// is summed as a tree and added to the row's Kahan-compensated sum; the row sums
// are folded into the thread's running Kahan sum once per tile pair.  Sorted
// tiles make the terms one accumulator sees nearly equal; plain binary32
// summation of such runs drifts systematically, which the cancellation of the
// pair sum would amplify.  Per row, sum(term * v) feeds the c_lo correction
// (see term32), which goes to the thread's binary64 total `cacc`.
template <int RORD, int ROWS, int CJ, bool CLAMP, bool LO>
__device__ __forceinline__ void tile_pass(const float* __restrict__ tile, const float* __restrict__ tile_lo,
                                          int ncol, const float (&w)[ROWS], const float (&wl)[ROWS], float half,
                                          Kahan32& acc, double& cacc) {
  static_assert(CJ == 4 || CJ == 8, "one or two float4s of columns per group of terms");
  float sum[ROWS], comp[ROWS], tv[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) sum[r] = comp[r] = tv[r] = 0.0f;
#pragma unroll 1
  for (int jj = 0; jj < ncol; jj += CJ) {
    float b[CJ], bl[CJ];
#pragma unroll
    for (int q4 = 0; q4 < CJ; q4 += 4) {
      const float4 v4 = *reinterpret_cast<const float4*>(tile + jj + q4);
      b[q4] = v4.x; b[q4 + 1] = v4.y; b[q4 + 2] = v4.z; b[q4 + 3] = v4.w;
      if (LO) {
        const float4 l4 = *reinterpret_cast<const float4*>(tile_lo + jj + q4);
        bl[q4] = l4.x; bl[q4 + 1] = l4.y; bl[q4 + 2] = l4.z; bl[q4 + 3] = l4.w;
      }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      float t[CJ];
#pragma unroll
      for (int q = 0; q < CJ; ++q) {
        float v;
        // grid difference (exact), plus the residuals when the grid is coarse
        const float d = LO ? __fadd_rn(__fsub_rn(w[r], b[q]), __fsub_rn(wl[r], bl[q])) : __fsub_rn(w[r], b[q]);
        t[q] = term32<RORD, CLAMP>(d, v);
        tv[r] = __fmaf_rn(t[q], v, tv[r]);
      }
      float g = __fadd_rn(__fadd_rn(t[0], t[1]), __fadd_rn(t[2], t[3]));
      if (CJ == 8) g = __fadd_rn(g, __fadd_rn(__fadd_rn(t[CJ / 2], t[CJ / 2 + 1]), __fadd_rn(t[CJ / 2 + 2], t[CJ / 2 + 3])));
      const float y = __fsub_rn(g, comp[r]);
      const float tt = __fadd_rn(sum[r], y);
      comp[r] = __fsub_rn(__fsub_rn(tt, sum[r]), y);
      sum[r] = tt;
    }
  }
  float tvsum = 0.0f;
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    acc.add(__fmul_rn(half, __fsub_rn(sum[r], comp[r])));   // half = 1/2 on a diagonal tile: exact
    tvsum = __fadd_rn(tvsum, tv[r]);
  }
  cacc -= static_cast<double>(tvsum) * static_cast<double>(half) * kCLoLn2;
}

// One tile pair, FP64 (plain binary64 accumulation, accurate exp).
template <int RORD, int ROWS, int TILE>
__device__ __forceinline__ void tile_pass64(const double* __restrict__ tile,
                                            const double (&w)[ROWS],
                                            const Coef<double, RORD>& cf, double& acc) {
  double part[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) part[r] = 0.0;
#pragma unroll 2
  for (int jj = 0; jj < TILE; jj += 2) {
    const double2 b = *reinterpret_cast<const double2*>(tile + jj);
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      part[r] = term64<RORD>(w[r], b.x, cf, part[r]);
      part[r] = term64<RORD>(w[r], b.y, cf, part[r]);
    }
  }
  double seg = part[0];
#pragma unroll
  for (int r = 1; r < ROWS; ++r) seg += part[r];
  acc += seg;
}

// Binary64 pair terms with the Gaussian factorised over a tile pair: the same
// identity as the binary32 path (exp(-u^2/2) = R_i C_j exp(alpha_i beta_j)), with
// the coupling factor taken to p^4/24 (truncation p^5/120 < 3e-19 for
// |alpha| |beta| <= kFac64PMax) and every factor from the binary64 exp.  Per pair:
//   u = (a_i - b0) - beta_j,  w = u^2,  He_r(w) by Horner,
//   e = c0 + alpha (c1 + alpha (c2 + alpha (c3 + alpha c4))),  c_k = C_j beta_j^k / k!,
//   row sum += He_r(w) e,
// ten binary64 operations for r = 6 instead of the ~25 of a term with its own exp.
constexpr double kFac64PMax = 5.0e-4;
constexpr double kFac64XMax = 8.0;

// Column factors of one sub-tile, three double2 per column:
// (beta, c0), (c1, c2), (c3, c4); zero past the sample.
template <int THREADS>
__device__ __forceinline__ void column_factors64(const double* __restrict__ tile, int vc, double b0,
                                                 double delta, double2* __restrict__ fac) {
  const double dh = delta * delta;
  const double dl = fma(delta, delta, -dh);
#pragma unroll
  for (int j = threadIdx.x; j < kSub; j += THREADS) {
    double2 f0 = make_double2(0.0, 0.0), f1 = f0, f2 = f0;
    if (j < vc) {
      const double beta = tile[j] - b0;
      // beta (delta - beta/2) - delta^2/2, with delta^2 split exactly
      const double x = fma(beta, fma(beta, -0.5, delta), -0.5 * dh) - 0.5 * dl;
      const double c0 = exp(x);
      const double c1 = c0 * beta;
      const double c2 = c1 * beta * 0.5;
      const double c3 = c2 * beta * (1.0 / 3.0);
      const double c4 = c3 * beta * 0.25;
      f0 = make_double2(beta, c0);
      f1 = make_double2(c1, c2);
      f2 = make_double2(c3, c4);
    }
    fac[3 * j] = f0;
    fac[3 * j + 1] = f1;
    fac[3 * j + 2] = f2;
  }
}

// One sub-tile, binary64 factorised: rs gets the row sums (before R_i).
template <int RORD, int ROWS>
__device__ __forceinline__ void tile_pass_fac64(const double2* __restrict__ fac, const double (&ap)[ROWS],
                                                const double (&al)[ROWS], const Coef<double, RORD>& cf,
                                                double (&rs)[ROWS]) {
#pragma unroll
  for (int r = 0; r < ROWS; ++r) rs[r] = 0.0;
#pragma unroll 2
  for (int j = 0; j < kSub; ++j) {
    const double2 f0 = fac[3 * j], f1 = fac[3 * j + 1], f2 = fac[3 * j + 2];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const double u = __dsub_rn(ap[r], f0.x);
      const double h = cf.horner(__dmul_rn(u, u));
      const double e = fma(al[r], fma(al[r], fma(al[r], fma(al[r], f2.y, f2.x), f1.y), f1.x), f0.y);
      rs[r] = fma(h, e, rs[r]);
    }
  }
}

// Tile pair number p of the upper triangle (I <= J, row by row) -> (I, J).
// Row I starts at S(I) = I nt - I (I - 1) / 2.  The root of the quadratic gives a
// first guess (binary32: a few rows off at most for nt <= 2^16, which the integer
// steps below correct exactly).
__device__ __forceinline__ void tri_index(int64_t p, int64_t nt, int64_t& I, int64_t& J) {
  const float b = 2.0f * static_cast<float>(nt) + 1.0f;
  const float disc = fmaxf(b * b - 8.0f * static_cast<float>(p), 0.0f);
  int64_t i = static_cast<int64_t>(floorf((b - sqrtf(disc)) * 0.5f));
  if (i > nt - 1) i = nt - 1;
  if (i < 0) i = 0;
  auto S = [nt](int64_t q) { return q * nt - q * (q - 1) / 2; };
  while (i > 0 && S(i) > p) --i;
  while (i + 1 < nt && S(i + 1) <= p) ++i;
  I = i;
  J = i + (p - S(i));
}

template <int PREC, int RORD>
__device__ void finish_psi(const PairArgs& a, const SampleDesc& d, SampleState* st, double s);

template <int PREC, int THREADS, int ROWS, int RORD>
__device__ void finalize_pairs(const PairArgs& a, const SampleDesc& d, SampleState* st,
                               double* red) {
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < d.nchunks; i += THREADS) s += __ldcg(a.slots + d.slot_off + i);
  s = block_sum<THREADS>(s, red);
  if (threadIdx.x != 0) return;
  st->done_pairs = 0;
  if (st->res.status != KDE_OK) return;
  finish_psi<PREC, RORD>(a, d, st, s);
}

// psi_r from the pair sum s = sum_{i<j} He_r(u) exp(-u^2/2) (Eqs. 6-7), then the
// next step of the chain.  Thread 0 only.
template <int PREC, int RORD>
__device__ void finish_psi(const PairArgs& a, const SampleDesc& d, SampleState* st, double s) {
  const double n = static_cast<double>(d.n);
  const double g = st->g_cur;
  // Eqs. 6-7: [2 sum_{i<j} K^(r) + n K^(r)(0)] / (n^2 g^(r+1)), K^(r) = He_r phi
  const double psi = (2.0 * s + n * he_at_zero<RORD>()) / (sqrt(2.0 * kPi) * n * n * pow(g, RORD + 1.0));
  if (!a.chain) {
    st->psi_out = psi;
    if (RORD == 6) st->res.psi6 = psi;
    if (RORD == 4) st->res.psi4 = psi;
    return;
  }
  record_psi(st, RORD, psi, g);
  if (RORD > 4) {
    next_pilot(st, RORD - 2, psi, n, PREC);   // Steps V (and their continuation above)
    return;
  }
  if (!(psi > 0.0)) {
    st->res.status = KDE_ERR_DOMAIN;
    return;
  }
  const double RK = 1.0 / (2.0 * sqrt(kPi));                 // R(K)
  st->res.h = pow(RK / (psi * n), 1.0 / 5.0);                 // Step VII, mu2 = 1
}

// Register budget per thread: binary32 64 with 4 rows and r <= 6 (the fast
// path needs no more), 96 with 8 rows or r >= 8; binary64 is left to the
// compiler (its inlined exp takes ~170; the FP64 pipe, not occupancy, bounds it).
template <int PREC, int ROWS, int RORD>
constexpr int pair_reg_budget() {
  return PREC != KDE_FP32 ? 65536 : (ROWS >= 8 || RORD >= 8) ? 96 : 64;
}
template <int PREC, int THREADS, int ROWS, int RORD>
constexpr int pair_min_blocks() {
  return 65536 / (pair_reg_budget<PREC, ROWS, RORD>() * THREADS) > 0
             ? 65536 / (pair_reg_budget<PREC, ROWS, RORD>() * THREADS)
             : 1;
}

template <int PREC, int THREADS, int ROWS, int CJ, int RORD>
__global__ void __launch_bounds__(THREADS, (pair_min_blocks<PREC, THREADS, ROWS, RORD>())) pairs_kernel(PairArgs a) {
  using T = typename Arith<PREC>::T;
  constexpr int TILE = THREADS * ROWS;
  static_assert(TILE % 8 == 0, "tile");
  static_assert(TILE % kSub == 0, "whole sub-tiles");
  __shared__ __align__(16) T tile[TILE];
  __shared__ __align__(16) float tile_lo[PREC == KDE_FP32 ? TILE : 4];
  __shared__ __align__(16) float4 fac[PREC == KDE_FP32 ? (kSegMax < TILE ? kSegMax : TILE) : 1];
  __shared__ __align__(16) double2 fac64[PREC == KDE_FP64 ? 3 * kSub : 1];
  __shared__ double red[THREADS / 32 + 1];
  __shared__ long long s_item;
  __shared__ int s_last;
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) s_item = static_cast<long long>(atomicAdd(a.counters, 1ull));
    __syncthreads();
    const long long item = s_item;
    if (item >= a.n_items) break;
    const uint64_t wi = a.items[item];
    const int64_t k = static_cast<int64_t>(wi >> 32);
    const int64_t c = static_cast<int64_t>(wi & 0xffffffffull);
    const SampleDesc d = a.desc[k];
    SampleState* st = a.state + k;

    double part = 0.0;
    int64_t diag_units = 0;
    if (st->res.status == KDE_OK) {
      using Y = typename Arith<PREC>::Y;
      const Y* __restrict__ y = static_cast<const Y*>(a.y) + d.y_off;
      // binary32: grid values were stored in u-units (scaled by 2^-F); the pads too
      const double unit = PREC == KDE_FP32 ? ldexp(1.0, -st->F) : 1.0;
      const T pad_lo = static_cast<T>(st->pad_lo * unit), pad_hi = static_cast<T>(st->pad_hi * unit);
      Coef<T, RORD> full, half;   // binary64 terms (u-units)
      full.set(1.0, 1.0);
      half.set(0.5, 1.0);
      int64_t p = c * d.chunk;
      const int64_t pend = (p + d.chunk < d.ntp) ? p + d.chunk : d.ntp;
      // the first tile pair of the chunk
      int64_t I, J;
      tri_index(p, d.nt, I, J);
      T w[ROWS];
      float wl[ROWS];
      // binary32 factorised path: row-tile centre a0 (a grid value), half-width A,
      // alpha_i = a_i - a0 and alpha_i^2 / 2 per row; first and last valid rows
      float a0 = 0.0f, halfA = 0.0f, row_first = 0.0f, row_last = 0.0f;
      float al[ROWS], ah[ROWS];
      // binary64 factorised path: the same geometry in u-units
      double a064 = 0.0, halfA64 = 0.0, row_first64 = 0.0, row_last64 = 0.0;
      double al64[ROWS];
      unsigned row_ok = 0u;
      const float unit_f = static_cast<float>(unit);
      // row slot r of this thread holds sample I*TILE + tid*ROWS + r
      auto load_rows = [&](int64_t I_) {
        row_ok = 0u;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const int64_t i = I_ * TILE + static_cast<int64_t>(tid) * ROWS + r;
          if (i < d.n) {
            const Y v = y[i];
            w[r] = hi_of(v);
            wl[r] = lo_of(v);
            row_ok |= 1u << r;
          } else {
            w[r] = pad_lo;
            wl[r] = 0.0f;
          }
        }
        if constexpr (PREC == KDE_FP64) {
          const int64_t vr64 = d.n - I_ * TILE;
          const int vr = vr64 < TILE ? static_cast<int>(vr64) : TILE;
          row_first64 = hi_of(y[I_ * TILE]);
          row_last64 = hi_of(y[I_ * TILE + vr - 1]);
          a064 = hi_of(y[I_ * TILE + (vr - 1) / 2]);
          halfA64 = fmax(a064 - row_first64, row_last64 - a064);
#pragma unroll
          for (int r = 0; r < ROWS; ++r) al64[r] = ((row_ok >> r) & 1u) ? static_cast<double>(w[r]) - a064 : 0.0;
        }
        if constexpr (PREC == KDE_FP32) {
          const int64_t vr64 = d.n - I_ * TILE;
          const int vr = vr64 < TILE ? static_cast<int>(vr64) : TILE;
          row_first = static_cast<float>(hi_of(y[I_ * TILE]));
          row_last = static_cast<float>(hi_of(y[I_ * TILE + vr - 1]));
          a0 = static_cast<float>(hi_of(y[I_ * TILE + (vr - 1) / 2]));
          halfA = __fadd_rn(fmaxf(__fsub_rn(a0, row_first), __fsub_rn(row_last, a0)), unit_f);
#pragma unroll
          for (int r = 0; r < ROWS; ++r) {
            const bool ok = (row_ok >> r) & 1u;
            al[r] = ok ? __fadd_rn(__fsub_rn(static_cast<float>(w[r]), a0), wl[r]) : 0.0f;
            ah[r] = __fmul_rn(0.5f, __fmul_rn(al[r], al[r]));
          }
        }
      };
      load_rows(I);
      Kahan32 acc32;
      double cacc = 0.0;
      double acc64 = 0.0;
      // Far tile pairs are skipped: the sample is sorted, so the smallest distance
      // of an off-diagonal tile pair is its first column minus its last row.  Beyond
      // the binary32 clamp every term is below 1e-31; beyond 40 bandwidths every
      // binary64 term underflows to exactly 0.
      const double far2 = (PREC == KDE_FP32) ? static_cast<double>(kWMax) : 1600.0;
      int64_t skipped_pairs = 0;
      for (; p < pend; ++p) {
        bool far = false;
        if (J > I) {
          if constexpr (PREC == KDE_FP32) {   // binary32 on the grid (block-uniform test)
            const float gap = __fsub_rn(__fsub_rn(hi_of(y[J * TILE]), hi_of(y[I * TILE + TILE - 1])), unit_f);
            far = gap > 0.0f && __fmul_rn(gap, gap) > kWMax;
          } else {
            const double gap = static_cast<double>(hi_of(y[J * TILE])) - static_cast<double>(hi_of(y[I * TILE + TILE - 1]));
            far = gap > 0.0 && gap * gap > far2;
          }
        }
        if (far) {
          const int64_t cols = d.n - J * TILE;
          skipped_pairs += static_cast<int64_t>(TILE) * (cols < TILE ? cols : TILE);
        } else {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const int64_t j = J * TILE + tid + r * THREADS;
          if (j < d.n) {
            const Y v = y[j];
            tile[tid + r * THREADS] = hi_of(v);
            if (PREC == KDE_FP32) tile_lo[tid + r * THREADS] = lo_of(v);
          } else {
            tile[tid + r * THREADS] = pad_hi;
            if (PREC == KDE_FP32) tile_lo[tid + r * THREADS] = 0.0f;
          }
        }
        __syncthreads();
        // A diagonal tile pair (I == J) is evaluated in full with halved
        // coefficients: the i < j and j < i terms are bitwise equal, and the
        // i == j terms are He_r(0) / 2 (to rounding), removed below.
        const bool diag = (I == J);
        const Coef<T, RORD>& cf = diag ? half : full;
        if constexpr (PREC == KDE_FP32) {
          const float hf = diag ? 0.5f : 1.0f;
          // the polynomial path clamps on tiles with padding (rows or columns)
          const bool full_tiles = (J + 1) * TILE <= d.n;
          const int64_t vct64 = d.n - J * TILE;
          const int vct = vct64 < TILE ? static_cast<int>(vct64) : TILE;
          // width and coupling order of the tile pair's segments, estimated from the
          // column tile's half-width scaled to each width (each segment checks its own)
          int kord = 0, segw = kSub;
          {
            const float abt = __fmul_rn(halfA, __fadd_rn(__fmul_rn(0.5f, __fsub_rn(tile[vct - 1], tile[0])), unit_f));
            int w1 = 0, w2 = 0;
#pragma unroll
            for (int wd = (kSegMax < TILE ? kSegMax : TILE); wd >= kSegMin; wd >>= 1) {
              const float est = abt * (static_cast<float>(wd) / static_cast<float>(TILE));
              if (w2 == 0 && est <= kFacP2) w2 = wd;
              if (w1 == 0 && est <= kFacP1) w1 = wd;
            }
            constexpr float seg_cost = kSegRowOps + kSegFixedOps / ROWS;
            if (w1 > 0 && seg_cost / static_cast<float>(w1) <=
                              (w2 > 0 ? 1.0f + seg_cost / static_cast<float>(w2) : 1e30f)) {
              kord = 1;
              segw = w1;
            } else if (w2 > 0) {
              kord = 2;
              segw = w2;
            }
          }
#pragma unroll 1
          for (int c0i = 0; c0i < vct; c0i += segw) {
            const int vc = vct - c0i < segw ? vct - c0i : segw;
            const float* __restrict__ sub = tile + c0i;
            const float* __restrict__ sub_lo = tile_lo + c0i;
            if (J > I) {   // a far segment: its first column is beyond the clamp from the last row
              const float gap = __fsub_rn(__fsub_rn(sub[0], row_last), unit_f);
              if (gap > 0.0f && __fmul_rn(gap, gap) > kWMax) {
                skipped_pairs += static_cast<int64_t>(TILE) * vc;
                continue;
              }
            }
            const float b0 = sub[(vc - 1) / 2];
            const float halfB = __fadd_rn(fmaxf(__fsub_rn(b0, sub[0]), __fsub_rn(sub[vc - 1], b0)), unit_f);
            const float delta = __fsub_rn(a0, b0);
            const float ad = fabsf(delta);
            const float ab = __fmul_rn(halfA, halfB);
            const bool xok = __fmul_rn(halfA, __fadd_rn(ad, halfA)) <= kFacXMax &&
                             __fmul_rn(halfB, __fadd_rn(ad, halfB)) <= kFacXMax;
            const int K = !xok ? 0 : (kord == 1 && ab <= kFacP1) ? 1 : (ab <= kFacP2 ? 2 : 0);
            if (K > 0) {
              __syncthreads();   // the previous segment's factors are no longer read
              column_factors<THREADS>(sub, sub_lo, segw, vc, b0, delta, fac);
              __syncthreads();
              float ap[ROWS], rsum[ROWS];
#pragma unroll
              for (int r = 0; r < ROWS; ++r)   // rows past the sample: u = -beta_j stays small, R_i = 0
                ap[r] = ((row_ok >> r) & 1u) ? __fadd_rn(__fsub_rn(static_cast<float>(w[r]), b0), wl[r]) : 0.0f;
              if (K == 1) tile_pass_fac<RORD, ROWS, 1>(fac, segw, ap, al, ah, rsum);
              else tile_pass_fac<RORD, ROWS, 2>(fac, segw, ap, al, ah, rsum);
#pragma unroll
              for (int r = 0; r < ROWS; ++r) {
                const float x = -__fmul_rn(al[r], __fmaf_rn(al[r], 0.5f, delta));
                const float R = ((row_ok >> r) & 1u) ? exp_small(x) : 0.0f;
                acc32.add(__fmul_rn(hf, __fmul_rn(rsum[r], R)));
              }
            } else {
              // The largest |y_i - y_j| of the segment against the row tile: its last column
              // minus the first row, or (on a diagonal tile pair, where rows lie above the
              // segment too) the last row minus its first column.
              const float span = __fadd_rn(fmaxf(__fsub_rn(sub[vc - 1], row_first), __fsub_rn(row_last, sub[0])),
                                           unit_f);
              const bool near = full_tiles && __fmul_rn(span, span) <= kWMax;
              if (near) tile_pass<RORD, ROWS, CJ, false, true>(sub, sub_lo, segw, w, wl, hf, acc32, cacc);
              else tile_pass<RORD, ROWS, CJ, true, true>(sub, sub_lo, segw, w, wl, hf, acc32, cacc);
            }
          }
        } else {
          const double hd = diag ? 0.5 : 1.0;
#pragma unroll 1
          for (int c0i = 0; c0i < TILE; c0i += kSub) {
            const int64_t vc64 = d.n - (J * TILE + c0i);
            if (vc64 <= 0) break;   // the rest of the tile is padding
            const int vc = vc64 < kSub ? static_cast<int>(vc64) : kSub;
            const T* __restrict__ sub = tile + c0i;
            if (J > I) {   // far sub-tile: every term underflows to exactly 0
              const double gap = static_cast<double>(sub[0]) - row_last64;
              if (gap > 0.0 && gap * gap > far2) {
                skipped_pairs += static_cast<int64_t>(TILE) * vc;
                continue;
              }
            }
            const double b0 = sub[(vc - 1) / 2];
            const double halfB = fmax(b0 - sub[0], sub[vc - 1] - b0);
            const double delta = a064 - b0;
            const double ad = fabs(delta);
            const bool fac_ok = halfA64 * halfB <= kFac64PMax && halfA64 * (ad + halfA64) <= kFac64XMax &&
                                halfB * (ad + halfB) <= kFac64XMax;
            if (fac_ok) {
              __syncthreads();   // the previous sub-tile's factors are no longer read
              column_factors64<THREADS>(sub, vc, b0, delta, fac64);
              __syncthreads();
              double ap[ROWS], rsum[ROWS];
#pragma unroll
              for (int r = 0; r < ROWS; ++r) ap[r] = ((row_ok >> r) & 1u) ? static_cast<double>(w[r]) - b0 : 0.0;
              tile_pass_fac64<RORD, ROWS>(fac64, ap, al64, full, rsum);
              double seg = 0.0;
#pragma unroll
              for (int r = 0; r < ROWS; ++r) {
                const double R = ((row_ok >> r) & 1u) ? exp(-al64[r] * fma(al64[r], 0.5, delta)) : 0.0;
                seg = fma(rsum[r], R, seg);
              }
              acc64 += hd * seg;
            } else {
              tile_pass64<RORD, ROWS, kSub>(sub, w, cf, acc64);
            }
          }
        }
        if (diag) {
          const int64_t valid = d.n - I * TILE;
          diag_units += valid < TILE ? valid : TILE;
        }
        }
        if (++J == d.nt) {
          ++I;
          J = I;
          if (p + 1 < pend) load_rows(I);
        }
      }
      part = (PREC == KDE_FP32) ? acc32.value() + cacc : acc64;
      if (tid == 0 && skipped_pairs > 0)
        atomicAdd(&st->skipped[RORD == 6 ? 0 : 1], static_cast<unsigned long long>(skipped_pairs));
    }
    const double tot = block_sum<THREADS>(part, red);
    if (tid == 0) {
      a.slots[d.slot_off + c] = tot - 0.5 * he_at_zero<RORD>() * static_cast<double>(diag_units);
      __threadfence();
      const unsigned prev = atomicAdd(&st->done_pairs, 1u);
      s_last = (prev + 1 == static_cast<unsigned>(d.nchunks));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      finalize_pairs<PREC, THREADS, ROWS, RORD>(a, d, st, red);
    }
    __syncthreads();
  }
  if (tid == 0) {
    const unsigned long long e = atomicAdd(a.counters + 1, 1ull);
    if (e + 1 == gridDim.x) {
      a.counters[0] = 0ull;
      a.counters[1] = 0ull;
    }
  }
}


// ---------------------------------------------------------------------------
// Q32.32 fixed point (Section 4.1): the paper's arithmetic for the pair terms
// ---------------------------------------------------------------------------
// int64 raw values, value = raw * 2^-32.  Products keep the high part of the
// exact 128-bit product (truncation toward -inf).  z-scored data (Eq. 3),
// u = (z_i - z_j) * (sigma / g), w = u^2, He_r(w) by Horner, exp(-w/2) as
// 2^-t with t = w / (2 ln 2) = k + f, 2^-f by a degree-8 minimax polynomial
// on [0, 1) (absolute error 0.002 of the last place; coefficients fitted by
// our own Remez exchange), shifted right by k.  Sums are exact in int64 per
// work item and int128 per sample, so the result does not depend on order.

constexpr long long kQOne = 1LL << 32;
constexpr long long kQInvTwoLn2 = 3098164009LL;   // round(2^32 / (2 ln 2))

__device__ __forceinline__ long long qmul(long long a, long long b) {
  const long long hi = __mul64hi(a, b);
  const unsigned long long lo = static_cast<unsigned long long>(a) * static_cast<unsigned long long>(b);
  return static_cast<long long>((static_cast<unsigned long long>(hi) << 32) | (lo >> 32));
}

// 2^32 exp(-w/2) for the Q32.32 value w >= 0
__device__ __forceinline__ long long q_exp_half(long long w) {
  const long long t = qmul(w, kQInvTwoLn2);
  const long long k = t >> 32;
  if (k >= 63) return 0;
  const long long f = t & 0xffffffffLL;
  long long q = 4028LL;
  q = qmul(q, f) - 62610LL;
  q = qmul(q, f) + 658738LL;
  q = qmul(q, f) - 5725081LL;
  q = qmul(q, f) + 41308991LL;
  q = qmul(q, f) - 238388224LL;
  q = qmul(q, f) + 1031764981LL;
  q = qmul(q, f) - 2977044471LL;
  q = qmul(q, f) + 4294967296LL;
  return q >> k;
}

// He_r(u) exp(-u^2/2) in Q32.32 for the z-difference d; 0 where the truncated
// exponential is 0 anyway (|u| >= 64 or u^2 >= 45)
template <int RORD>
__device__ __forceinline__ long long q_term(long long d, long long ginv, double ginv_d) {
  if (fabs(static_cast<double>(d) * ginv_d) >= 64.0 * 18446744073709551616.0) return 0;
  const long long u = qmul(d, ginv);
  const long long w = qmul(u, u);
  if (w >= 45 * kQOne) return 0;
  long long p;
  if (RORD == 6) {
    p = qmul(w - 15 * kQOne, w) + 45 * kQOne;
    p = qmul(p, w) - 15 * kQOne;
  } else {
    p = qmul(w - 6 * kQOne, w) + 3 * kQOne;
  }
  return qmul(p, q_exp_half(w));
}

template <int THREADS>
__device__ long long block_sum_i64(long long v, long long* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < THREADS; ++i) t += red[i];
    red[0] = t;
  }
  __syncthreads();
  const long long r = red[0];
  __syncthreads();
  return r;
}

template <int THREADS, int RORD>
__device__ void finalize_q32(const PairArgs& a, const SampleDesc& d, SampleState* st, __int128* red) {
  __int128 s = 0;
  for (int64_t i = threadIdx.x; i < d.nchunks; i += THREADS)
    s += static_cast<__int128>(__double_as_longlong(__ldcg(a.slots + d.slot_off + i)));
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x != 0) return;
  __int128 t = 0;
  for (int i = 0; i < THREADS; ++i) t += red[i];
  st->done_pairs = 0;
  if (st->res.status != KDE_OK) return;
  const long long hi = static_cast<long long>(t >> 64);
  const unsigned long long lo = static_cast<unsigned long long>(t);
  const double sum = (static_cast<double>(hi) * 18446744073709551616.0 + static_cast<double>(lo)) / 4294967296.0;
  finish_psi<KDE_Q32, RORD>(a, d, st, sum);
}

template <int THREADS, int ROWS, int RORD>
__global__ void __launch_bounds__(THREADS) pairs_q32_kernel(PairArgs a) {
  constexpr int TILE = THREADS * ROWS;
  __shared__ long long tile[TILE];
  __shared__ __int128 red[THREADS];
  __shared__ long long s_item;
  __shared__ int s_last;
  long long* red64 = reinterpret_cast<long long*>(red);
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) s_item = static_cast<long long>(atomicAdd(a.counters, 1ull));
    __syncthreads();
    const long long item = s_item;
    if (item >= a.n_items) break;
    const uint64_t wi = a.items[item];
    const int64_t k = static_cast<int64_t>(wi >> 32);
    const int64_t c = static_cast<int64_t>(wi & 0xffffffffull);
    const SampleDesc d = a.desc[k];
    SampleState* st = a.state + k;
    long long acc_off = 0, acc_diag = 0;
    int64_t diag_units = 0, skipped_pairs = 0;
    if (st->res.status == KDE_OK) {
      const long long* __restrict__ y = static_cast<const long long*>(a.y) + d.y_off;
      const long long pad_lo = static_cast<long long>(floor(st->pad_lo * 4294967296.0));
      const long long pad_hi = static_cast<long long>(floor(st->pad_hi * 4294967296.0));
      const long long ginv = static_cast<long long>(floor(st->scale * 4294967296.0));
      const double ginv_d = static_cast<double>(ginv);
      int64_t p = c * d.chunk;
      const int64_t pend = (p + d.chunk < d.ntp) ? p + d.chunk : d.ntp;
      int64_t I, J;
      tri_index(p, d.nt, I, J);
      long long w[ROWS];
      auto load_rows = [&](int64_t I_) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const int64_t i = I_ * TILE + static_cast<int64_t>(tid) * ROWS + r;
          w[r] = i < d.n ? y[i] : pad_lo;
        }
      };
      load_rows(I);
      for (; p < pend; ++p) {
        bool far = false;
        if (J > I) {   // sorted: smallest distance = first column - last row; u >= 6.8 gives 0
          const double gap = static_cast<double>(y[J * TILE] - y[I * TILE + TILE - 1]) * ginv_d *
                             (1.0 / 18446744073709551616.0);
          far = gap >= 6.8;
        }
        if (far) {
          const int64_t cols = d.n - J * TILE;
          skipped_pairs += static_cast<int64_t>(TILE) * (cols < TILE ? cols : TILE);
        } else {
          __syncthreads();
#pragma unroll
          for (int r = 0; r < ROWS; ++r) {
            const int64_t j = J * TILE + tid + r * THREADS;
            tile[tid + r * THREADS] = j < d.n ? y[j] : pad_hi;
          }
          __syncthreads();
          long long acc = 0;
#pragma unroll 2
          for (int jj = 0; jj < TILE; ++jj) {
            const long long b = tile[jj];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
              const long long dz = w[r] - b;   // the term is even: take |dz| (truncation is not odd)
              acc += q_term<RORD>(dz < 0 ? -dz : dz, ginv, ginv_d);
            }
          }
          if (I == J) {   // full square: symmetric pairs twice, the diagonal once
            acc_diag += acc;
            const int64_t valid = d.n - I * TILE;
            diag_units += valid < TILE ? valid : TILE;
          } else {
            acc_off += acc;
          }
        }
        if (++J == d.nt) {
          ++I;
          J = I;
          if (p + 1 < pend) load_rows(I);
        }
      }
      if (tid == 0 && skipped_pairs > 0)
        atomicAdd(&st->skipped[RORD == 6 ? 0 : 1], static_cast<unsigned long long>(skipped_pairs));
    }
    const long long off = block_sum_i64<THREADS>(acc_off, red64);
    const long long dg = block_sum_i64<THREADS>(acc_diag, red64);
    if (tid == 0) {
      // the diagonal terms are exactly He_r(0) (u = 0, exp = 1); the rest of a
      // diagonal tile holds each unordered pair twice
      const long long he0 = static_cast<long long>(he_at_zero<RORD>()) * kQOne;
      const long long item_sum = off + (dg - diag_units * he0) / 2;
      a.slots[d.slot_off + c] = __longlong_as_double(item_sum);
      __threadfence();
      const unsigned prev = atomicAdd(&st->done_pairs, 1u);
      s_last = (prev + 1 == static_cast<unsigned>(d.nchunks));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      finalize_q32<THREADS, RORD>(a, d, st, red);
    }
    __syncthreads();
  }
  if (tid == 0) {
    const unsigned long long e = atomicAdd(a.counters + 1, 1ull);
    if (e + 1 == gridDim.x) {
      a.counters[0] = 0ull;
      a.counters[1] = 0ull;
    }
  }
}

// ---------------------------------------------------------------------------
// configuration table
// ---------------------------------------------------------------------------

using PairKernel = void (*)(PairArgs);

struct ConfigEntry {
  PairConfig cfg;
  PairKernel k4, k6, k8, k10;
};

#define KDE_CFG(P, TH, RW, CJ)                                                       \
  { {TH, RW}, pairs_kernel<P, TH, RW, CJ, 4>, pairs_kernel<P, TH, RW, CJ, 6>,         \
    pairs_kernel<P, TH, RW, CJ, 8>, pairs_kernel<P, TH, RW, CJ, 10> }

const ConfigEntry kFp32Configs[] = {
    KDE_CFG(KDE_FP32, 128, 4, 8),   // T = 512
    KDE_CFG(KDE_FP32, 64, 8, 8),    // T = 512
    KDE_CFG(KDE_FP32, 256, 4, 8),   // T = 1024
    KDE_CFG(KDE_FP32, 64, 4, 8),    // T = 256
    KDE_CFG(KDE_FP32, 128, 2, 8),   // T = 256
};
const ConfigEntry kFp64Configs[] = {
    KDE_CFG(KDE_FP64, 128, 2, 4),   // T = 256
    KDE_CFG(KDE_FP64, 128, 4, 4),   // T = 512
    KDE_CFG(KDE_FP64, 64, 4, 4),    // T = 256
};
#undef KDE_CFG
const ConfigEntry kQ32Configs[] = {
    {{128, 2}, pairs_q32_kernel<128, 2, 4>, pairs_q32_kernel<128, 2, 6>, nullptr, nullptr},   // T = 256
};

const ConfigEntry& entry(int prec, int cfg) {
  return prec == KDE_FP32 ? kFp32Configs[cfg] : prec == KDE_Q32 ? kQ32Configs[cfg] : kFp64Configs[cfg];
}

}  // namespace

int pair_config_count(int prec) {
  return prec == KDE_FP32  ? static_cast<int>(sizeof(kFp32Configs) / sizeof(kFp32Configs[0]))
         : prec == KDE_Q32 ? static_cast<int>(sizeof(kQ32Configs) / sizeof(kQ32Configs[0]))
                           : static_cast<int>(sizeof(kFp64Configs) / sizeof(kFp64Configs[0]));
}

PairConfig pair_config(int prec, int cfg) { return entry(prec, cfg).cfg; }

// Resident blocks per SM of a pair kernel, cached per (device, precision,
// configuration, order).  Devices of one process may differ, so the current
// device is part of the key; the cache is shared by every host thread.
namespace {
std::mutex g_occ_mu;
std::map<std::tuple<int, int, int, int>, int> g_occ;

int occupancy_cached(int prec, int cfg, int r, PairKernel k, int threads) {
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, prec, cfg, r);
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    const auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
  }
  int v = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k, threads, 0);
  if (v < 1) v = 1;
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ[key] = v;
  return v;
}
}  // namespace

int pair_blocks_per_sm(int prec, int cfg) {
  const ConfigEntry& e = entry(prec, cfg);
  const int b4 = occupancy_cached(prec, cfg, 4, e.k4, e.cfg.threads);
  const int b6 = occupancy_cached(prec, cfg, 6, e.k6, e.cfg.threads);
  return b4 < b6 ? b4 : b6;
}

cudaError_t launch_stage_results(SampleState* state, int64_t m, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  stage_results_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(state, m);
  return cudaGetLastError();
}

cudaError_t launch_init(const SampleDesc* desc, SampleState* state, int64_t m,
                        unsigned long long* counters, int n_counters, cudaStream_t s) {
  const int64_t work = m > n_counters ? m : n_counters;
  const int blocks = static_cast<int>((work + 255) / 256);
  init_states_kernel<<<blocks, 256, 0, s>>>(desc, state, m, counters, n_counters);
  return cudaGetLastError();
}

cudaError_t launch_moments(const MomentsArgs& a, int64_t total_blocks, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  moments_kernel<<<static_cast<unsigned>(total_blocks), kMomThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_prescale(const PrescaleArgs& a, int64_t total_blocks, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  prescale_kernel<<<static_cast<unsigned>(total_blocks), kPrescaleThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pairs(int prec, int cfg, const PairArgs& a, int grid, cudaStream_t s) {
  if (a.n_items <= 0 || grid <= 0) return cudaSuccess;
  const ConfigEntry& e = entry(prec, cfg);
  PairKernel k = a.r == 6 ? e.k6 : a.r == 8 ? e.k8 : a.r == 10 ? e.k10 : e.k4;
  if (a.r >= 8) {   // the higher orders may hold more registers: at most their resident count
    const int cap = occupancy_cached(prec, cfg, a.r, k, e.cfg.threads) * num_sms();
    if (grid > cap) grid = cap;
  }
  k<<<grid, e.cfg.threads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace kde
