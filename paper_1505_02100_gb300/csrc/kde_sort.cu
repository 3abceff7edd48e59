// kde_sort.cu -- stable LSD radix sort of every sample's values, on the device.
//
// psi_r is a sum over all pairs, so the order of the sample does not change it
// mathematically; sorting changes how binary32 accumulates it.  With sorted
// data every tile pair holds values from two narrow ranges, so the terms one
// accumulator adds over a tile are of similar size: a run of tiny far-pair
// terms is never added one by one to a large running sum, where each would be
// rounded away -- a loss that is biased (those terms all have the sign of
// He_r at large u) and that the cancellation in the pair sum would amplify.
//
// Keys are the order-preserving integer images of the values (all 64 bits of a
// binary64, all 32 of a binary32), sorted in 8-bit digits, least significant
// first: per-block digit histogram, per-sample scan over (digit, block), stable
// scatter.  The sorted order is therefore the order of the values themselves,
// whatever order they arrived in.  Every sample is sorted independently inside
// one set of launches; passes alternate between x and a scratch area of the
// same size (desc[k].tmp_off) and end in x.
#include "kde_internal.cuh"

namespace kde {
namespace {

constexpr int kSortThreads = 256;
constexpr int kRadix = 256;

// digit of element i: 8 bits of the order-preserving image of the value
__device__ __forceinline__ uint32_t digit(const void* v, int f32, int64_t i, int shift) {
  if (f32) {
    const uint32_t b = __float_as_uint(static_cast<const float*>(v)[i]);
    const uint32_t k = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return (k >> shift) & 0xffu;
  }
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(static_cast<const double*>(v)[i]));
  const uint64_t k = (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
  return static_cast<uint32_t>(k >> shift) & 0xffu;
}

// block -> (launch-local sample, chunk) through the per-sample block prefix
__device__ __forceinline__ int64_t find_sample(const int64_t* prefix, int64_t m, int64_t b) {
  int64_t lo = 0, hi = m;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= b) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(SortArgs a, const void* src, int from_x,
                                                                 int shift) {
  __shared__ uint32_t hist[kRadix];
  const int64_t b = blockIdx.x;
  const int64_t s = find_sample(a.bprefix, a.m, b);
  const int64_t k = a.ids ? a.ids[s] : s;
  const SampleDesc& d = a.desc[k];
  const int64_t c0 = (b - a.bprefix[s]) * kSortChunk;
  const int64_t c1 = c0 + kSortChunk < d.n ? c0 + kSortChunk : d.n;
  hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t off = from_x ? d.x_off : d.tmp_off;
  for (int64_t i = c0 + threadIdx.x; i < c1; i += kSortThreads)
    atomicAdd(&hist[digit(src, a.x_is_f32, off + i, shift)], 1u);
  __syncthreads();
  a.counts[b * kRadix + threadIdx.x] = hist[threadIdx.x];
}

// One block per sample: offsets[b][digit] = (elements of the sample with a
// smaller digit) + (elements with this digit in earlier blocks).
__global__ void __launch_bounds__(kSortThreads) sort_scan_kernel(SortArgs a) {
  __shared__ uint32_t tot[kRadix];
  const int64_t s = blockIdx.x;
  const int64_t b0 = a.bprefix[s], b1 = a.bprefix[s + 1];
  const int dg = threadIdx.x;
  uint32_t t = 0;
  for (int64_t b = b0; b < b1; ++b) t += a.counts[b * kRadix + dg];
  tot[dg] = t;
  __syncthreads();
  // exclusive scan over digits (fixed order, small)
  if (dg == 0) {
    uint32_t run = 0;
    for (int i = 0; i < kRadix; ++i) {
      const uint32_t c = tot[i];
      tot[i] = run;
      run += c;
    }
  }
  __syncthreads();
  uint32_t run = tot[dg];
  for (int64_t b = b0; b < b1; ++b) {
    const uint32_t c = a.counts[b * kRadix + dg];
    a.counts[b * kRadix + dg] = run;
    run += c;
  }
}

// Stable scatter: the chunk is read in rounds of one element per thread; a
// thread's rank among equal digits counts every earlier element of the chunk
// (earlier rounds, earlier warps of this round, lower lanes of its warp).
template <typename V>
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(SortArgs a, const void* src_v, void* dst_v,
                                                                    int from_x, int shift) {
  __shared__ uint32_t base[kRadix];                       // running offset per digit
  __shared__ uint32_t wcnt[kSortThreads / 32][kRadix];    // this round: per-warp digit counts
  const V* src = static_cast<const V*>(src_v);
  V* dst = static_cast<V*>(dst_v);
  const int64_t b = blockIdx.x;
  const int64_t s = find_sample(a.bprefix, a.m, b);
  const int64_t k = a.ids ? a.ids[s] : s;
  const SampleDesc& d = a.desc[k];
  const int64_t c0 = (b - a.bprefix[s]) * kSortChunk;
  const int64_t c1 = c0 + kSortChunk < d.n ? c0 + kSortChunk : d.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t soff = from_x ? d.x_off : d.tmp_off, doff = from_x ? d.tmp_off : d.x_off;
  base[threadIdx.x] = a.counts[b * kRadix + threadIdx.x];
  for (int64_t r0 = c0; r0 < c1; r0 += kSortThreads) {
    for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = r0 + threadIdx.x;
    const bool valid = i < c1;
    const uint32_t dig = valid ? digit(src_v, a.x_is_f32, soff + i, shift) : kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const int rank_in_warp = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank_in_warp == 0) wcnt[warp][dig] = __popc(peers);
    __syncthreads();
    // per digit: exclusive scan over warps, then advance the running base
    {
      const int dd = threadIdx.x;
      uint32_t run = 0;
      for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t c = wcnt[w][dd];
        wcnt[w][dd] = run;
        run += c;
      }
      __syncthreads();
      if (valid) {
        const uint32_t pos = base[dig] + wcnt[warp][dig] + rank_in_warp;
        dst[doff + pos] = src[soff + i];
      }
      __syncthreads();
      base[dd] += run;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_sort(const SortArgs& a, int64_t total_blocks, void* x, void* tmp, cudaStream_t s) {
  if (total_blocks <= 0 || a.m <= 0) return cudaSuccess;
  const int passes = a.x_is_f32 ? 4 : 8;   // even: the sorted values end in x
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * pass;
    const int from_x = (pass % 2 == 0) ? 1 : 0;
    const void* src = from_x ? x : tmp;
    void* dst = from_x ? tmp : x;
    sort_hist_kernel<<<static_cast<unsigned>(total_blocks), kSortThreads, 0, s>>>(a, src, from_x, shift);
    sort_scan_kernel<<<static_cast<unsigned>(a.m), kSortThreads, 0, s>>>(a);
    if (a.x_is_f32)
      sort_scatter_kernel<float><<<static_cast<unsigned>(total_blocks), kSortThreads, 0, s>>>(a, src, dst, from_x, shift);
    else
      sort_scatter_kernel<double><<<static_cast<unsigned>(total_blocks), kSortThreads, 0, s>>>(a, src, dst, from_x, shift);
  }
  return cudaGetLastError();
}

}  // namespace kde
