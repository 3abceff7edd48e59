// kde_static.cu -- kde_psi_static: psi_r(g) for one sample of at most
// kStaticMaxN values, computed entirely in a scratch area that is part of the
// loaded module, so that the call itself allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// bandwidth functional:
// - A process whose framework's caching allocator already holds most of HBM.
//   A fresh cudaMalloc there fails or evicts that allocator's cache.
// - A latency-bound loop. cudaMalloc and cudaFree can synchronise the device
//   and stall every stream.
// - Code that must show a fixed, known device footprint up front.
// The regular entry points grow a per-stream workspace on demand. This one
// uses a fixed `static __device__` array instead.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's address with cudaGetSymbolAddress and caches it per device. Do that
// first call before any stream capture.
// Later calls only launch kernels and copy the result.
//
// Zero state: the init kernel of every call clears the two work counters of
// the pair kernel and every per-sample flag (done_mom, done_pairs). The last
// pair block resets the counters again. Nothing else in the scratch area is
// read before it is written within the same call.
//
// Concurrency: there is ONE scratch area per device. A host-side lock is held
// from the address lookup to the last enqueued operation, so calls from
// different host threads on the same stream run one after the other on the
// device. Calls on different streams still overlap on the device and race on
// the scratch area: callers must order them (for example, issue them all on
// one stream).
//
// Device reset: kde_shutdown forgets the cached addresses, so the first call
// after a reset (cudaDeviceReset, which reloads the module) looks the address
// up again. Call kde_shutdown before resetting the device.
#include "kde_internal.cuh"

#include <cmath>
#include <mutex>

namespace kde {
namespace {

constexpr int64_t kStaticMaxN = KDE_STATIC_MAX_N;
constexpr int64_t kMinTile = 256;                      // smallest T of any pair configuration
constexpr int64_t kMaxTiles = kStaticMaxN / kMinTile;  // 256
constexpr int64_t kMaxTilePairs = kMaxTiles * (kMaxTiles + 1) / 2;   // 32896 (one per chunk)
constexpr int64_t kMaxSortBlocks = (kStaticMaxN + kSortChunk - 1) / kSortChunk;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// byte offsets of the regions inside the scratch area
constexpr size_t kOffX = 0;                                                     // n doubles
constexpr size_t kOffY = kOffX + align256(kStaticMaxN * sizeof(double));        // n x 8 B: sort scratch, scaled values
constexpr size_t kOffCounts = kOffY + align256(kStaticMaxN * sizeof(double));   // 256 u32 per sort block
constexpr size_t kOffMslots = kOffCounts + align256(kMaxSortBlocks * 256 * sizeof(uint32_t));
constexpr size_t kOffSlots = kOffMslots + align256(kMomMaxBlocks * 5 * sizeof(double));
constexpr size_t kOffItems = kOffSlots + align256(kMaxTilePairs * sizeof(double));
constexpr size_t kOffDesc = kOffItems + align256(kMaxTilePairs * sizeof(uint64_t));
constexpr size_t kOffState = kOffDesc + align256(sizeof(SampleDesc));
constexpr size_t kOffPrefix = kOffState + align256(sizeof(SampleState));       // 3 x 2 int64
constexpr size_t kOffCounters = kOffPrefix + align256(6 * sizeof(int64_t));     // 2 u64
constexpr size_t kScratchBytes = kOffCounters + align256(2 * sizeof(unsigned long long));
static_assert(kScratchBytes < (2u << 20), "the static scratch area stays under 2 MiB");

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Writes the descriptor, the three block prefixes and the work list from
// kernel arguments, so that no host-to-device copy is needed.
__global__ void static_setup_kernel(SampleDesc d, int64_t mblocks, int64_t pblocks, int64_t sblocks,
                                    SampleDesc* desc, int64_t* prefix, uint64_t* items) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i == 0) {
    *desc = d;
    prefix[0] = 0; prefix[1] = mblocks;    // moments
    prefix[2] = 0; prefix[3] = pblocks;    // prescale
    prefix[4] = 0; prefix[5] = sblocks;    // sort
  }
  for (int64_t c = i; c < d.nchunks; c += static_cast<int64_t>(gridDim.x) * blockDim.x)
    items[c] = static_cast<uint64_t>(c);   // sample 0, chunk c
}

// Caller holds g_static_mu.
kde_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(KDE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_err(KDE_ERR_INVALID, "device ordinal out of range");
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return set_err(KDE_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_static_ptr[dev]);
  return KDE_OK;
}

#define KDE_STATIC_CU(call)                                                             \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return set_err(KDE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

// Forget the cached scratch addresses (kde_shutdown; a device reset may move
// the module).
void static_scratch_forget() {
  std::lock_guard<std::mutex> lk(g_static_mu);
  for (auto& p : g_static_ptr) p = nullptr;
}

}  // namespace kde

using namespace kde;

extern "C" kde_status kde_psi_static(const double* x, int64_t n, int r, double g, kde_precision prec,
                                     double* out, void* stream) {
  if (!x || !out) return set_err(KDE_ERR_INVALID, "null pointer");
  if (n < 2) return set_err(KDE_ERR_INVALID, "n < 2");
  if (n > kStaticMaxN)
    return set_err(KDE_ERR_INVALID, "kde_psi_static: n = " + std::to_string(n) +
                                        " exceeds the static scratch limit of " + std::to_string(kStaticMaxN) +
                                        " values; use kde_psi");
  if (r != 4 && r != 6 && r != 8 && r != 10) return set_err(KDE_ERR_INVALID, "r must be 4, 6, 8 or 10");
  if (!(g > 0) || !std::isfinite(g)) return set_err(KDE_ERR_INVALID, "g must be finite and > 0");
  if (prec != KDE_FP32 && prec != KDE_FP64 && prec != KDE_Q32) return set_err(KDE_ERR_INVALID, "bad precision");
  if (prec == KDE_Q32 && r > 6) return set_err(KDE_ERR_INVALID, "KDE_Q32 evaluates psi_4 and psi_6 only");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // held until the last operation is enqueued: same-stream calls from several
  // host threads do not interleave their launches on the one scratch area
  std::unique_lock<std::mutex> lk(g_static_mu);
  unsigned char* base = nullptr;
  kde_status st = scratch_for_current_device(&base);
  if (st != KDE_OK) return st;

  const int cfg = choose_config(prec, n);
  SampleDesc d = make_desc(prec, cfg, n, g);   // offsets all 0: one sample
  if (d.nchunks > kMaxTilePairs || d.mblocks > kMomMaxBlocks)
    return set_err(KDE_ERR_INVALID, "tiling exceeds the static scratch layout");
  const int64_t mblocks = d.mblocks;
  const int64_t pblocks = (n + kPrescaleThreads - 1) / kPrescaleThreads;
  const int64_t sblocks = (n + kSortChunk - 1) / kSortChunk;

  void* xs = base + kOffX;
  void* ys = base + kOffY;
  auto* desc = reinterpret_cast<SampleDesc*>(base + kOffDesc);
  auto* state = reinterpret_cast<SampleState*>(base + kOffState);
  auto* prefix = reinterpret_cast<int64_t*>(base + kOffPrefix);
  auto* items = reinterpret_cast<uint64_t*>(base + kOffItems);
  auto* counters = reinterpret_cast<unsigned long long*>(base + kOffCounters);

  KDE_STATIC_CU(cudaMemcpyAsync(xs, x, static_cast<size_t>(n) * sizeof(double), cudaMemcpyDefault, s));
  const int setup_blocks = static_cast<int>(std::min<int64_t>((d.nchunks + 255) / 256, 1024));
  static_setup_kernel<<<setup_blocks > 0 ? setup_blocks : 1, 256, 0, s>>>(d, mblocks, pblocks, sblocks, desc,
                                                                          prefix, items);
  KDE_STATIC_CU(cudaGetLastError());
  KDE_STATIC_CU(launch_init(desc, state, 1, counters, 2, s));

  SortArgs sa{};
  sa.x_is_f32 = 0;
  sa.desc = desc;
  sa.bprefix = prefix + 4;
  sa.ids = nullptr;
  sa.m = 1;
  sa.counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
  KDE_STATIC_CU(launch_sort(sa, sblocks, xs, ys, s));

  MomentsArgs ma{};
  ma.x = xs;
  ma.x_is_f32 = 0;
  ma.desc = desc;
  ma.state = state;
  ma.mprefix = prefix;
  ma.ids = nullptr;
  ma.m = 1;
  ma.mslots = reinterpret_cast<double*>(base + kOffMslots);
  KDE_STATIC_CU(launch_moments(ma, mblocks, s));

  PrescaleArgs pr{};
  pr.x = xs;
  pr.x_is_f32 = 0;
  pr.desc = desc;
  pr.state = state;
  pr.bprefix = prefix + 2;
  pr.ids = nullptr;
  pr.m = 1;
  pr.y = ys;
  KDE_STATIC_CU(launch_prescale(pr, pblocks, s));

  PairArgs pa{};
  pa.y = ys;
  pa.desc = desc;
  pa.state = state;
  pa.items = items;
  pa.n_items = d.nchunks;
  pa.slots = reinterpret_cast<double*>(base + kOffSlots);
  pa.counters = counters;
  pa.r = r;
  pa.chain = 0;
  const int64_t resident = static_cast<int64_t>(pair_blocks_per_sm(prec, cfg)) * num_sms();
  const int grid = static_cast<int>(std::min<int64_t>(resident, d.nchunks));
  KDE_STATIC_CU(launch_pairs(prec, cfg, pa, grid, s));

  if (is_device_ptr(out)) {
    KDE_STATIC_CU(cudaMemcpyAsync(out, &state->psi_out, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return KDE_OK;
  }
  double psi = 0.0;
  int32_t status = 0;
  KDE_STATIC_CU(cudaMemcpyAsync(&psi, &state->psi_out, sizeof(double), cudaMemcpyDeviceToHost, s));
  KDE_STATIC_CU(cudaMemcpyAsync(&status, &state->res.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  lk.unlock();
  KDE_STATIC_CU(cudaStreamSynchronize(s));
  *out = psi;
  if (status != KDE_OK) return set_err(static_cast<kde_status>(status), "psi failed on device");
  return KDE_OK;
}
