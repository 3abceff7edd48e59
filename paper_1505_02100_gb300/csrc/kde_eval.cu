// kde_eval.cu -- the density estimate of Eq. 1 with the Gaussian kernel of
// Eq. 2, fhat(t) = (1 / (n h)) sum_i K((t - X_i) / h), at m points.
//
// Unlike psi_r, every term is positive, so the sum does not cancel. A per-term
// relative error that is small and nearly unbiased stays small in the sum, and
// the MUFU ex2 unit (about 3e-8 rms, bias about -5e-8) is accurate enough here.
// The precision risk is elsewhere:
// - Differences t - X_i taken in binary32 lose digits when the values are far
//   from the origin. Both sides are therefore held as double-float pairs
//   z = hi + lo of (value - median) / h * sqrt(1 / (2 ln 2)), so that
//   K(u) = 2^(-(z_t - z_i)^2) / sqrt(2 pi). One pair difference
//   (hi_t - hi_i) + (lo_t - lo_i) is then good to about 2^-48 |z|.
// - Long binary32 runs of similar positive terms drift. Each point therefore
//   sums its terms in groups of 4 (a tree) with one Kahan step per group, and
//   folds into binary64 once per shared-memory tile of samples.
//
// Flow, all on the stream:
//   copy x and t -> (binary32) radix-sort the copy of x for its median -> prescale
//   -> eval_pairs (2-D grid: point tiles x sample chunks, binary64 partial per
//      (chunk, point)) -> reduce over chunks in fixed order, scale by 1/(n h sqrt(2 pi)).
// Results are deterministic: the chunking depends only on (n, m, device).
#include "kde_internal.cuh"

#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>

namespace kde {
namespace {

constexpr int kEvalThreads = 128;
constexpr int kEvalPPT = 4;                            // points per thread
constexpr int kEvalPoints = kEvalThreads * kEvalPPT;   // points per block
constexpr int kEvalTile = 1024;                        // samples per shared-memory tile
constexpr double kEvalRangeLimit = 1.0e7;              // binary32 path: max |z| of any value
constexpr double kInvSqrt2Ln2 = 0.84932180028801904272;   // sqrt(1 / (2 ln 2))

__device__ __forceinline__ float ex2_neg(float v) {   // 2^(-v), MUFU
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-v));
  return e;
}

struct EvalArgs {
  const double* xs;   // sorted sample (for the median)
  int64_t n;
  const double* t;
  int64_t m;
  double scale;       // binary32: sqrt(1/(2 ln 2)) / h
  float* zx;          // binary32: hi[n], lo[n]   (n padded to whole tiles)
  float* zt;          // binary32: hi[m], lo[m]
  double* zx64;       // binary64: raw values x[n] (n padded to whole tiles)
  double* zt64;       // binary64: raw points t[m]
  int64_t n_pad;
  int prec;
  int* flag;          // set to 1 for a non-finite value, or (binary32) one beyond kEvalRangeLimit
};

__global__ void eval_setup_kernel(SampleDesc d, int64_t sblocks, SampleDesc* desc, int64_t* prefix,
                                  int* flag) {
  *desc = d;
  prefix[0] = 0;
  prefix[1] = sblocks;
  *flag = 0;
}

// binary32: z = (value - median) * scale, split into hi + lo; binary64: the raw
// values.  The sample is padded to whole tiles with values whose terms vanish.
__global__ void eval_prescale_kernel(EvalArgs a) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const double c = a.xs[(a.n - 1) / 2];
  const int64_t total = a.n_pad + a.m;
  if (i >= total) return;
  const bool is_x = i < a.n_pad;
  const int64_t k = is_x ? i : i - a.n_pad;
  const bool pad = is_x && k >= a.n;
  if (a.prec == KDE_FP64) {
    // binary64 keeps the raw values: t - X_i is then exact for nearby pairs,
    // wherever they lie (centring would cost digits far from the median)
    const double v = is_x ? (pad ? 1.0e300 : a.xs[k]) : a.t[k];
    if (!pad && !isfinite(v)) atomicExch(a.flag, 1);
    (is_x ? a.zx64 : a.zt64)[k] = v;
    return;
  }
  double z;
  if (is_x) z = pad ? 1.0e30 : (a.xs[k] - c) * a.scale;   // padding: terms underflow to 0
  else z = (a.t[k] - c) * a.scale;
  if (!pad && !(fabs(z) <= kEvalRangeLimit)) atomicExch(a.flag, 1);
  {
    const float hi = static_cast<float>(z);
    const float lo = static_cast<float>(z - static_cast<double>(hi));
    float* base = is_x ? a.zx : a.zt;
    const int64_t len = is_x ? a.n_pad : a.m;
    base[k] = hi;
    base[len + k] = lo;
  }
}

// Block (bx, by): points [bx * kEvalPoints, +kEvalPoints) against samples of
// chunk by.  part[by * m + j] = sum over the chunk of 2^(-(z_t - z_i)^2)
// (binary32) or exp(-(t - x_i)^2 / (2 h^2)) (binary64).
__global__ void __launch_bounds__(kEvalThreads) eval_pairs32_kernel(const float* __restrict__ zx,
                                                                    const float* __restrict__ zt,
                                                                    int64_t n_pad, int64_t m,
                                                                    int64_t chunk, double* part) {
  __shared__ __align__(16) float sh[kEvalTile];
  __shared__ __align__(16) float sl[kEvalTile];
  const int tid = threadIdx.x;
  const int64_t p0 = blockIdx.x * static_cast<int64_t>(kEvalPoints);
  float th[kEvalPPT], tl[kEvalPPT];
#pragma unroll
  for (int p = 0; p < kEvalPPT; ++p) {
    const int64_t j = p0 + tid + p * kEvalThreads;
    th[p] = j < m ? zt[j] : 1.0e30f;
    tl[p] = j < m ? zt[m + j] : 0.0f;
  }
  double acc64[kEvalPPT];
#pragma unroll
  for (int p = 0; p < kEvalPPT; ++p) acc64[p] = 0.0;
  const int64_t s0 = blockIdx.y * chunk;
  const int64_t s1 = s0 + chunk < n_pad ? s0 + chunk : n_pad;
  for (int64_t base = s0; base < s1; base += kEvalTile) {
    __syncthreads();
    for (int k = tid; k < kEvalTile; k += kEvalThreads) {
      sh[k] = zx[base + k];
      sl[k] = zx[n_pad + base + k];
    }
    __syncthreads();
    float sum[kEvalPPT], comp[kEvalPPT];
#pragma unroll
    for (int p = 0; p < kEvalPPT; ++p) sum[p] = comp[p] = 0.0f;
#pragma unroll 2
    for (int k = 0; k < kEvalTile; k += 4) {
      const float4 h4 = *reinterpret_cast<const float4*>(sh + k);
      const float4 l4 = *reinterpret_cast<const float4*>(sl + k);
      const float hs[4] = {h4.x, h4.y, h4.z, h4.w};
      const float ls[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
      for (int p = 0; p < kEvalPPT; ++p) {
        float e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float d = __fadd_rn(__fsub_rn(th[p], hs[q]), __fsub_rn(tl[p], ls[q]));
          e[q] = ex2_neg(__fmul_rn(d, d));
        }
        const float g4 = __fadd_rn(__fadd_rn(e[0], e[1]), __fadd_rn(e[2], e[3]));
        const float y = __fsub_rn(g4, comp[p]);
        const float t = __fadd_rn(sum[p], y);
        comp[p] = __fsub_rn(__fsub_rn(t, sum[p]), y);
        sum[p] = t;
      }
    }
#pragma unroll
    for (int p = 0; p < kEvalPPT; ++p)
      acc64[p] += static_cast<double>(sum[p]) - static_cast<double>(comp[p]);
  }
#pragma unroll
  for (int p = 0; p < kEvalPPT; ++p) {
    const int64_t j = p0 + tid + p * kEvalThreads;
    if (j < m) part[blockIdx.y * m + j] = acc64[p];
  }
}

__global__ void __launch_bounds__(kEvalThreads) eval_pairs64_kernel(const double* __restrict__ zx,
                                                                    const double* __restrict__ zt,
                                                                    int64_t n_pad, int64_t m,
                                                                    int64_t chunk, double half_inv_h2,
                                                                    double* part) {
  __shared__ __align__(16) double sx[kEvalTile];
  const int tid = threadIdx.x;
  const int64_t p0 = blockIdx.x * static_cast<int64_t>(kEvalPoints);
  double tz[kEvalPPT], acc[kEvalPPT];
#pragma unroll
  for (int p = 0; p < kEvalPPT; ++p) {
    const int64_t j = p0 + tid + p * kEvalThreads;
    tz[p] = j < m ? zt[j] : 1.0e30;
    acc[p] = 0.0;
  }
  const int64_t s0 = blockIdx.y * chunk;
  const int64_t s1 = s0 + chunk < n_pad ? s0 + chunk : n_pad;
  for (int64_t base = s0; base < s1; base += kEvalTile) {
    __syncthreads();
    for (int k = tid; k < kEvalTile; k += kEvalThreads) sx[k] = zx[base + k];
    __syncthreads();
    for (int k = 0; k < kEvalTile; ++k) {
      const double xk = sx[k];
#pragma unroll
      for (int p = 0; p < kEvalPPT; ++p) {
        const double d = tz[p] - xk;
        acc[p] += exp(-(d * d) * half_inv_h2);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < kEvalPPT; ++p) {
    const int64_t j = p0 + tid + p * kEvalThreads;
    if (j < m) part[blockIdx.y * m + j] = acc[p];
  }
}

// out[j] = (sum over chunks, in chunk order) * norm; NaN for every point if the
// prescale flagged a value.
__global__ void eval_reduce_kernel(const double* part, int64_t chunks, int64_t m, double norm,
                                   const int* flag, double* out) {
  const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (j >= m) return;
  double s = 0.0;
  for (int64_t c = 0; c < chunks; ++c) s += part[c * m + j];
  out[j] = *flag ? CUDART_NAN : s * norm;
}

struct EvalBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct EvalWorkspace {
  std::mutex mu;
  EvalBuf x, tmp, t, z, part, counts, meta, out;
};

std::mutex g_eval_mu;
std::map<std::pair<int, cudaStream_t>, std::unique_ptr<EvalWorkspace>> g_eval_ws;

#define KDE_EVAL_CU(call)                                                                       \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return set_err(e_ == cudaErrorMemoryAllocation ? KDE_ERR_OOM : KDE_ERR_CUDA,              \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

kde_status grow(EvalWorkspace& W, EvalBuf& b, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return KDE_OK;
  if (b.p) {
    KDE_EVAL_CU(cudaStreamSynchronize(s));
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  const size_t want = bytes + bytes / 4;
  KDE_EVAL_CU(cudaMalloc(&b.p, want));
  b.cap = want;
  (void)W;
  return KDE_OK;
}

}  // namespace

void eval_release_all() {
  std::lock_guard<std::mutex> lk(g_eval_mu);
  for (auto& kv : g_eval_ws) {
    std::lock_guard<std::mutex> wl(kv.second->mu);
    for (EvalBuf* b : {&kv.second->x, &kv.second->tmp, &kv.second->t, &kv.second->z, &kv.second->part,
                       &kv.second->counts, &kv.second->meta, &kv.second->out}) {
      if (b->p) cudaFree(b->p);
      b->p = nullptr;
      b->cap = 0;
    }
  }
  g_eval_ws.clear();
}

}  // namespace kde

using namespace kde;

extern "C" kde_status kde_eval(const double* x, int64_t n, double h, const double* t, int64_t m,
                               kde_precision prec, double* out, void* stream) {
  if (!x || !t || !out) return set_err(KDE_ERR_INVALID, "null pointer");
  if (n < 1) return set_err(KDE_ERR_INVALID, "n < 1");
  if (m < 1) return set_err(KDE_ERR_INVALID, "m < 1");
  if (!(h > 0) || !std::isfinite(h)) return set_err(KDE_ERR_INVALID, "h must be finite and > 0");
  if (prec != KDE_FP32 && prec != KDE_FP64) return set_err(KDE_ERR_INVALID, "bad precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  KDE_EVAL_CU(cudaGetDevice(&dev));
  EvalWorkspace* W = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_eval_mu);
    auto& slot = g_eval_ws[{dev, s}];
    if (!slot) slot.reset(new EvalWorkspace());
    W = slot.get();
  }
  std::lock_guard<std::mutex> lk(W->mu);

  const int64_t n_pad = (n + kEvalTile - 1) / kEvalTile * kEvalTile;
  const int64_t sblocks = (n + kSortChunk - 1) / kSortChunk;
  const int64_t point_tiles = (m + kEvalPoints - 1) / kEvalPoints;
  int per_sm = 0;
  if (prec == KDE_FP32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eval_pairs32_kernel, kEvalThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eval_pairs64_kernel, kEvalThreads, 0);
  const int64_t target = 2 * static_cast<int64_t>(std::max(per_sm, 1)) * num_sms();
  const int64_t tiles = n_pad / kEvalTile;
  const int64_t want_chunks = std::max<int64_t>(1, (target + point_tiles - 1) / point_tiles);
  const int64_t chunks_raw = std::min<int64_t>(tiles, want_chunks);
  const int64_t chunk = (tiles + chunks_raw - 1) / chunks_raw * kEvalTile;   // samples per chunk
  const int64_t chunks = (n_pad + chunk - 1) / chunk;

  kde_status st;
  const size_t zbytes = prec == KDE_FP32 ? 2 * sizeof(float) : sizeof(double);
  if ((st = grow(*W, W->x, static_cast<size_t>(n) * sizeof(double), s)) != KDE_OK) return st;
  if ((st = grow(*W, W->tmp, static_cast<size_t>(n) * sizeof(double), s)) != KDE_OK) return st;
  if ((st = grow(*W, W->t, static_cast<size_t>(m) * sizeof(double), s)) != KDE_OK) return st;
  if ((st = grow(*W, W->z, static_cast<size_t>(n_pad + m) * zbytes, s)) != KDE_OK) return st;
  if ((st = grow(*W, W->part, static_cast<size_t>(chunks * m) * sizeof(double), s)) != KDE_OK) return st;
  if ((st = grow(*W, W->counts, static_cast<size_t>(sblocks) * 256 * sizeof(uint32_t), s)) != KDE_OK) return st;
  if ((st = grow(*W, W->meta, 1024, s)) != KDE_OK) return st;
  const bool out_dev = is_device_ptr(out);
  if (!out_dev && (st = grow(*W, W->out, static_cast<size_t>(m) * sizeof(double), s)) != KDE_OK) return st;

  auto* meta = static_cast<unsigned char*>(W->meta.p);
  auto* desc = reinterpret_cast<SampleDesc*>(meta);
  auto* prefix = reinterpret_cast<int64_t*>(meta + 512);
  auto* flag = reinterpret_cast<int*>(meta + 768);
  KDE_EVAL_CU(cudaMemcpyAsync(W->x.p, x, static_cast<size_t>(n) * sizeof(double), cudaMemcpyDefault, s));
  KDE_EVAL_CU(cudaMemcpyAsync(W->t.p, t, static_cast<size_t>(m) * sizeof(double), cudaMemcpyDefault, s));
  SampleDesc d{};
  d.n = n;
  eval_setup_kernel<<<1, 1, 0, s>>>(d, sblocks, desc, prefix, flag);
  KDE_EVAL_CU(cudaGetLastError());
  SortArgs sa{};
  sa.x_is_f32 = 0;
  sa.desc = desc;
  sa.bprefix = prefix;
  sa.ids = nullptr;
  sa.m = 1;
  sa.counts = static_cast<uint32_t*>(W->counts.p);
  if (prec == KDE_FP32) KDE_EVAL_CU(launch_sort(sa, sblocks, W->x.p, W->tmp.p, s));   // for the median

  EvalArgs ea{};
  ea.xs = static_cast<const double*>(W->x.p);
  ea.n = n;
  ea.t = static_cast<const double*>(W->t.p);
  ea.m = m;
  ea.n_pad = n_pad;
  ea.prec = prec;
  ea.flag = flag;
  if (prec == KDE_FP32) {
    ea.scale = kInvSqrt2Ln2 / h;
    ea.zx = static_cast<float*>(W->z.p);
    ea.zt = ea.zx + 2 * n_pad;
  } else {
    ea.zx64 = static_cast<double*>(W->z.p);
    ea.zt64 = ea.zx64 + n_pad;
  }
  const int64_t total = n_pad + m;
  eval_prescale_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(ea);
  KDE_EVAL_CU(cudaGetLastError());
  const dim3 grid(static_cast<unsigned>(point_tiles), static_cast<unsigned>(chunks));
  double* part = static_cast<double*>(W->part.p);
  if (prec == KDE_FP32)
    eval_pairs32_kernel<<<grid, kEvalThreads, 0, s>>>(ea.zx, ea.zt, n_pad, m, chunk, part);
  else
    eval_pairs64_kernel<<<grid, kEvalThreads, 0, s>>>(ea.zx64, ea.zt64, n_pad, m, chunk, 0.5 / (h * h), part);
  KDE_EVAL_CU(cudaGetLastError());
  const double norm = 1.0 / (static_cast<double>(n) * h * std::sqrt(2.0 * kPi));
  double* dst = out_dev ? out : static_cast<double*>(W->out.p);
  eval_reduce_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(part, chunks, m, norm, flag, dst);
  KDE_EVAL_CU(cudaGetLastError());
  if (out_dev) return KDE_OK;
  int hflag = 0;
  KDE_EVAL_CU(cudaMemcpyAsync(out, dst, static_cast<size_t>(m) * sizeof(double), cudaMemcpyDeviceToHost, s));
  KDE_EVAL_CU(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  KDE_EVAL_CU(cudaStreamSynchronize(s));
  if (hflag)
    return set_err(KDE_ERR_INVALID, "a value is not finite, or (KDE_FP32) lies more than 1e7 "
                                    "bandwidths from the sample median");
  return KDE_OK;
}
