// kde_internal.cuh -- data layout shared by the kernels and the host runtime of
// libkde.  Nothing here is part of the public ABI (include/kde.h).
//
// Layout in HBM for one launch over m samples (m = 1 for a single call):
//   x          the samples back to back (binary64 or binary32), staged by the
//              library; sample k is x[desc[k].x_off .. desc[k].x_off + n_k)
//   desc[m]    SampleDesc: tiling of each sample (written by the host)
//   state[m]   SampleState: every scalar of Algorithm 1 plus the counters the
//              "last CTA finishes the sample" pattern uses (written on device)
//   mslots     5 doubles per moments block: (count, mean, M2, min, max)
//   slots      1 double per chunk of tile pairs: the chunk's pair sum
//   items      the work-list of the persistent pair kernel: (sample << 32) | chunk
//   counters   2 x u64 per pair launch: next work item, CTAs that have exited
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/kde.h"

namespace kde {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Moments: elements per block is max(kMomMinChunk, ceil(n / kMomMaxBlocks))
// rounded up to a multiple of the block size, so a sample never needs more than
// kMomMaxBlocks blocks and the final merge fits one block.
constexpr int kMomThreads = 256;
constexpr int64_t kMomMinChunk = 4096;
constexpr int64_t kMomMaxBlocks = 256;

// Pair kernel: a sample's tile pairs are cut into chunks of as few tile pairs
// as keep the count under kMaxChunks (one tile pair each up to n ~ 1.4M at T = 512).
constexpr int64_t kMaxChunks = int64_t(1) << 22;

// Pair-kernel value representation.  The binary64 path holds u-units
// z = (X - median) / g.  The binary32 path holds a float2 (y, residual) with
// residual = M + z 2^F - y and y = M + round(z * 2^F) with
// M = 1.5 * 2^23: every value within 2^(22-F) bandwidths of the mean lies in
// the binade [2^23, 2^24), so y_i - y_j is EXACT (Sterbenz) and only the
// element-wise rounding (unbiased, first-order cancelling) remains.  The
// window is centred on the sample median and F is chosen per sample and per
// psi so that it holds everything between the 0.1% and 99.9% quantiles (read
// off the sorted sample; robust to outliers, which stay exact in their own
// binades and only ever meet far-away partners).
constexpr double kYBias = 12582912.0;          // 1.5 * 2^23
constexpr int kFMin = 4, kFMax = 21;           // 2^(-6F) must stay a normal binary32
// Padding (ragged last tile) and overflow limits, in u-units.
constexpr double kPadMargin = 1000.0;         // |u| >= 1000 against padding: the term vanishes
constexpr double kFp32RangeLimit = 1.0e30;    // max|u| 2^F beyond this: not representable
constexpr double kFp64RangeLimit = 1.0e45;
constexpr double kQ32ZLimit = 536870912.0;      // Q32.32: |z| < 2^29 keeps differences in int64

struct SampleDesc {
  int64_t x_off, n;
  int64_t nt;        // tiles of side T: ceil(n / T)
  int64_t ntp;       // tile pairs I <= J: nt (nt + 1) / 2
  int64_t chunk;     // tile pairs per chunk
  int64_t nchunks;   // ceil(ntp / chunk)
  int64_t slot_off;  // first slot of this sample
  int64_t mchunk;    // elements per moments block
  int64_t mblocks;   // moments blocks of this sample
  int64_t mslot_off; // offset (in doubles) of this sample's moments slots
  int64_t y_off;     // offset (in elements of the pair type) of this sample's scaled values
  int64_t tmp_off;   // offset (in elements of x's type) of the sort's scratch area
  double g_fixed;    // > 0: stand-alone psi_r(g) at this g; else Algorithm 1 (g1 from Step III)
  int32_t prec;      // kde_precision of this sample's pair terms
  int32_t cfg;       // pair-kernel tile configuration
  int32_t stages;    // plug-in stages l (2: Algorithm 1); unused for a stand-alone psi_r(g)
  int32_t reserved;
};

struct SampleState {
  kde_result res;      // mean, sigma, psi8, g1, psi6, g2, psi4, h, status
  double xmin, xmax;
  double center;       // median of the sample: origin of the scaled values
  double qlo, qhi;     // 0.1% and 99.9% quantiles of the sample
  double g_cur;        // bandwidth of the psi being evaluated next
  double scale;        // binary32: 2^F / g_cur (grid units); binary64: 1 / g_cur (u-units);
                       // scaled value = (X - center) * scale
  double pad_lo, pad_hi; // padding values for rows / columns, same units as the scaled values
  double psi_out;      // stand-alone psi_r(g) (kde_psi)
  int32_t F;           // binary32 grid exponent
  int32_t reserved;
  uint32_t done_mom;   // moments blocks finished (reset by the last one)
  uint32_t done_pairs; // chunks finished (reset by the last one)
  unsigned long long skipped[2];   // unique pairs in far tile pairs not evaluated: psi6, psi4
  kde_stage_result sres;           // l-stage results (psi_r, pilots) as the plug-in proceeds
};

struct MomentsArgs {
  const void* x;
  int x_is_f32;
  const SampleDesc* desc;
  SampleState* state;
  const int64_t* mprefix;  // m + 1 prefix sums of the launch's samples' mblocks
  const int32_t* ids;      // launch-local sample -> index into desc/state (NULL: identity)
  int64_t m;
  double* mslots;
};

struct PrescaleArgs {
  const void* x;
  int x_is_f32;
  const SampleDesc* desc;
  const SampleState* state;
  const int64_t* bprefix;  // m + 1 prefix sums of the launch's samples' blocks
  const int32_t* ids;      // launch-local sample -> index into desc/state (NULL: identity)
  int64_t m;
  void* y;                 // float (binary32 samples) or double (binary64 samples)
};

struct PairArgs {
  const void* y;           // scaled values (see above), per sample at desc[k].y_off
  const SampleDesc* desc;
  SampleState* state;
  const uint64_t* items;
  int64_t n_items;
  double* slots;
  unsigned long long* counters;
  int r;                   // 4, 6, 8 or 10
  int chain;               // 1: plug-in chain (r > 4 -> next pilot, r = 4 -> Step VII)
};

constexpr int kPrescaleThreads = 256;

// Device radix sort of every sample's values (see kde_sort.cu).
constexpr int64_t kSortChunk = 4096;          // elements per sort block
struct SortArgs {
  int x_is_f32;
  const SampleDesc* desc;
  const int64_t* bprefix;  // m + 1 prefix sums of the launch's samples' sort blocks
  const int32_t* ids;      // launch-local sample -> index into desc (NULL: identity)
  int64_t m;
  uint32_t* counts;        // 256 per sort block
};

// Tile configurations of the pair kernel.  T = threads * rows per thread.
struct PairConfig {
  int threads, rows;
  int tile() const { return threads * rows; }
};

int pair_config_count(int prec);
PairConfig pair_config(int prec, int cfg);
cudaError_t launch_init(const SampleDesc* desc, SampleState* state, int64_t m,
                        unsigned long long* counters, int n_counters, cudaStream_t s);
cudaError_t launch_moments(const MomentsArgs& a, int64_t total_blocks, cudaStream_t s);
cudaError_t launch_prescale(const PrescaleArgs& a, int64_t total_blocks, cudaStream_t s);
// Sorts each sample's values in x in place (tmp: scratch of the same size).
cudaError_t launch_sort(const SortArgs& a, int64_t total_blocks, void* x, void* tmp, cudaStream_t s);
cudaError_t launch_pairs(int prec, int cfg, const PairArgs& a, int grid, cudaStream_t s);
cudaError_t launch_stage_results(SampleState* state, int64_t m, cudaStream_t s);
// Resident CTAs per SM of a pair configuration (occupancy query, cached).
int pair_blocks_per_sm(int prec, int cfg);

// host runtime helpers (kde_api.cu)
kde_status set_err(kde_status s, const std::string& m);
bool is_device_ptr(const void* p);
int num_sms();
// kde_psi_static: forget the cached per-device scratch addresses (kde_shutdown).
void static_scratch_forget();
int choose_config(int prec, int64_t n);    // tuner's force, environment, tuned table, built-in rule
int default_config(int prec, int64_t n);   // the built-in rule
SampleDesc make_desc(int prec, int cfg, int64_t n, double g_fixed);
void drop_workspace(cudaStream_t stream);
void eval_release_all();                     // kde_eval.cu: free the density-estimate workspaces

// tile-configuration autotuner (kde_tune.cu)
extern thread_local int t_tune_force_cfg;    // >= 0 only while the tuner times that configuration
int tuned_config(int prec, int64_t n);       // tuned choice for the current device, or -1

}  // namespace kde
