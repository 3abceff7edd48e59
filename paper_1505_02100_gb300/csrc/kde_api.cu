// kde_api.cu -- host runtime and C ABI of libkde (declared in include/kde.h).
//
// A call becomes a "batch plan": one SampleDesc per sample (its tiling), and
// per tile configuration a work-list of (sample, chunk) items sorted by cost,
// largest first.  The plan's launches -- init, moments, pairs r=6, pairs r=4
// (Algorithm 1) or one pairs launch (stand-alone psi_r) -- are captured once
// into a CUDA graph per plan shape and replayed on the caller's stream.
//
// Device memory lives in per-(device, stream) workspaces that only grow.  Calls
// on one stream share a workspace, which stream order makes safe; calls on
// different streams never share one.
#include "kde_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

namespace kde {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

thread_local std::string t_err;

kde_status set_err(kde_status s, const std::string& m) {
  t_err = m;
  return s;
}

#define KDE_CU(call)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return set_err(e_ == cudaErrorMemoryAllocation ? KDE_ERR_OOM : KDE_ERR_CUDA,    \
                     std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// tiling
// ---------------------------------------------------------------------------

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return (v && *v) ? std::atoi(v) : dflt;
}

// Tile configuration for a sample of n values.  It depends only on n (and an
// explicit override), so a sample gets the same tiling -- and bitwise the same
// result -- alone, in a batch or in the server.
int choose_config(int prec, int64_t n) {
  const int count = pair_config_count(prec);
  if (t_tune_force_cfg >= 0 && t_tune_force_cfg < count) return t_tune_force_cfg;   // the tuner is timing it
  const int forced = env_int(prec == KDE_FP32 ? "KDE_FP32_TILE_CONFIG" : "KDE_FP64_TILE_CONFIG", -1);
  if (forced >= 0 && forced < count) return forced;
  const int tuned = tuned_config(prec, n);
  if (tuned >= 0 && tuned < count) return tuned;
  return default_config(prec, n);
}

int default_config(int prec, int64_t n) {
  if (prec == KDE_FP32) return n <= 16384 ? 3 : 0;   // T = 256 for small n, else T = 512
  return 0;                                          // T = 256
}

SampleDesc make_desc(int prec, int cfg, int64_t n, double g_fixed) {
  SampleDesc d{};
  d.n = n;
  d.g_fixed = g_fixed;
  d.prec = prec;
  d.cfg = cfg;
  d.stages = 2;
  if (n < 2) return d;
  const int64_t T = pair_config(prec, cfg).tile();
  d.nt = (n + T - 1) / T;
  d.ntp = d.nt * (d.nt + 1) / 2;
  d.chunk = std::max<int64_t>(1, (d.ntp + kMaxChunks - 1) / kMaxChunks);
  d.nchunks = (d.ntp + d.chunk - 1) / d.chunk;
  int64_t mc = std::max<int64_t>(kMomMinChunk, (n + kMomMaxBlocks - 1) / kMomMaxBlocks);
  mc = (mc + kMomThreads - 1) / kMomThreads * kMomThreads;
  d.mchunk = mc;
  d.mblocks = (n + mc - 1) / mc;
  return d;
}

enum Mode { kPlugin = 0 };   // or the order r of a stand-alone psi_r(g)

struct Group {
  int cfg = 0;
  std::vector<uint64_t> items;
  int64_t item_off = 0;
  int grid = 0;
};

struct BatchPlan {
  int prec = KDE_FP32;
  int mode = kPlugin;
  int stages = 2;                 // plug-in stages (2: Algorithm 1)
  int x_f32 = 0;
  std::vector<SampleDesc> desc;
  std::vector<int64_t> mprefix;
  std::vector<int64_t> bprefix;   // prescale blocks per sample, prefix sums
  std::vector<int64_t> sprefix;   // sort blocks per sample, prefix sums
  std::vector<Group> groups;
  int64_t total_x = 0, total_slots = 0, total_mslots = 0, total_items = 0;
  uint64_t key = 0;

  int n_pair_launches() const {
    return static_cast<int>(groups.size()) * (mode == kPlugin ? stages : 1);
  }
};

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

int num_sms() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

// ns[k] sample sizes; offsets into the packed x are cumulative.
void build_plan(BatchPlan& P, int prec, int mode, int x_f32, const int64_t* ns, int64_t m,
                double g_fixed, int stages = 2) {
  P.prec = prec;
  P.mode = mode;
  P.stages = stages;
  P.x_f32 = x_f32;
  P.desc.resize(m);
  P.mprefix.assign(m + 1, 0);
  P.bprefix.assign(m + 1, 0);
  P.sprefix.assign(m + 1, 0);
  std::map<int, std::vector<int64_t>> by_cfg;
  int64_t x_off = 0, slot_off = 0, mslot_off = 0;
  for (int64_t k = 0; k < m; ++k) {
    const int cfg = choose_config(prec, ns[k]);
    SampleDesc d = make_desc(prec, cfg, ns[k], g_fixed);
    d.stages = stages;
    d.x_off = x_off;
    d.y_off = x_off;
    d.tmp_off = x_off;   // the sort's scratch is the y buffer, same offsets
    d.slot_off = slot_off;
    d.mslot_off = mslot_off;
    x_off += std::max<int64_t>(ns[k], 0);
    slot_off += d.nchunks;
    mslot_off += d.mblocks * 5;
    P.mprefix[k + 1] = P.mprefix[k] + d.mblocks;
    P.bprefix[k + 1] = P.bprefix[k] + (d.n >= 2 ? (d.n + kPrescaleThreads - 1) / kPrescaleThreads : 0);
    P.sprefix[k + 1] = P.sprefix[k] + (d.n >= 2 ? (d.n + kSortChunk - 1) / kSortChunk : 0);
    P.desc[k] = d;
    if (d.nchunks > 0) by_cfg[cfg].push_back(k);
  }
  P.total_x = x_off;
  P.total_slots = slot_off;
  P.total_mslots = mslot_off;
  P.groups.clear();
  const int sms = num_sms();
  int64_t item_off = 0;
  for (auto& kv : by_cfg) {
    Group g;
    g.cfg = kv.first;
    struct It { int64_t cost, k, c; };
    std::vector<It> its;
    for (int64_t k : kv.second) {
      const SampleDesc& d = P.desc[k];
      for (int64_t c = 0; c < d.nchunks; ++c)
        its.push_back({std::min(d.chunk, d.ntp - c * d.chunk), k, c});
    }
    // largest chunks first, ties in (sample, chunk) order: the order only
    // balances the load, it never changes which slot a chunk writes
    std::stable_sort(its.begin(), its.end(),
                     [](const It& a, const It& b) { return a.cost > b.cost; });
    g.items.reserve(its.size());
    for (const It& t : its) g.items.push_back((static_cast<uint64_t>(t.k) << 32) | static_cast<uint64_t>(t.c));
    g.item_off = item_off;
    item_off += static_cast<int64_t>(g.items.size());
    const int64_t resident = static_cast<int64_t>(pair_blocks_per_sm(prec, g.cfg)) * sms;
    g.grid = static_cast<int>(std::min<int64_t>(resident, static_cast<int64_t>(g.items.size())));
    P.groups.push_back(std::move(g));
  }
  P.total_items = item_off;
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, &prec, sizeof prec);
  h = fnv(h, &mode, sizeof mode);
  h = fnv(h, &stages, sizeof stages);
  h = fnv(h, &x_f32, sizeof x_f32);
  h = fnv(h, &m, sizeof m);
  h = fnv(h, &g_fixed, sizeof g_fixed);
  h = fnv(h, ns, sizeof(int64_t) * static_cast<size_t>(m));
  for (const SampleDesc& d : P.desc) h = fnv(h, &d.cfg, sizeof d.cfg);
  P.key = h;
}

// What build_plan's result depends on: its arguments and each sample's tile
// configuration (the autotuner or KDE_*_TILE_CONFIG may change that between
// calls).  The device is fixed per workspace.
struct PlanArgs {
  int prec = -1, mode = 0, x_f32 = 0, stages = 0;
  double g_fixed = 0.0;
  std::vector<int64_t> ns;
  std::vector<int> cfgs;

  void set(int prec_, int mode_, int x_f32_, const int64_t* ns_, int64_t m, double g_, int stages_) {
    prec = prec_;
    mode = mode_;
    x_f32 = x_f32_;
    stages = stages_;
    g_fixed = g_;
    ns.assign(ns_, ns_ + m);
    cfgs.resize(static_cast<size_t>(m));
    for (int64_t k = 0; k < m; ++k) cfgs[k] = choose_config(prec_, ns_[k]);
  }
  bool operator==(const PlanArgs& o) const {
    return prec == o.prec && mode == o.mode && x_f32 == o.x_f32 && stages == o.stages &&
           std::memcmp(&g_fixed, &o.g_fixed, sizeof g_fixed) == 0 && ns == o.ns && cfgs == o.cfgs;
  }
};

// ---------------------------------------------------------------------------
// workspaces
// ---------------------------------------------------------------------------

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct Workspace {
  int device = 0;
  cudaStream_t stream = nullptr;       // the caller's stream this workspace serves
  cudaStream_t cap_stream = nullptr;   // private stream used only for graph capture
  std::mutex mu;
  DevBuf x, y, desc, state, mprefix, bprefix, sprefix, scounts, mslots, slots, items, counters;
  uint64_t meta_key = 0;
  struct GraphEntry {
    cudaGraphExec_t exec;
    int launches;   // kernel launches it replays
  };
  std::unordered_map<uint64_t, GraphEntry> graphs;
  int last_launches = 0;   // kernel launches of the last run on this workspace
  int64_t last_m = 0;      // samples of the last run on this workspace
  cudaEvent_t prof[5] = {};   // before init, after prescale r=6, after pairs r=6, after prescale r=4, after pairs r=4
  bool prof_valid = false;
  // The plan of the last call and the arguments it was built from (plan_for).
  BatchPlan plan;
  PlanArgs plan_args;
  bool plan_set = false;

  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
  void release() {
    if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
    drop_graphs();
    for (DevBuf* b : {&x, &y, &desc, &state, &mprefix, &bprefix, &sprefix, &scounts, &mslots, &slots, &items, &counters}) {
      if (b->p) cudaFree(b->p);
      b->p = nullptr;
      b->cap = 0;
    }
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    for (cudaEvent_t& e : prof) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    prof_valid = false;
    meta_key = 0;
    plan_set = false;
  }
};

std::atomic<int> g_profile{0};

struct Registry {
  std::mutex mu;
  std::map<std::pair<int, cudaStream_t>, std::unique_ptr<Workspace>> ws;
};

Registry& registry() {
  static Registry* r = new Registry();   // never destroyed: CUDA may be gone at exit
  return *r;
}

kde_status get_workspace(cudaStream_t stream, Workspace** out) {
  int dev = 0;
  KDE_CU(cudaGetDevice(&dev));
  Registry& R = registry();
  std::lock_guard<std::mutex> lk(R.mu);
  auto& slot = R.ws[{dev, stream}];
  if (!slot) {
    slot.reset(new Workspace());
    slot->device = dev;
    slot->stream = stream;
  }
  *out = slot.get();
  return KDE_OK;
}

// Release and forget the workspace of (current device, stream).
void drop_workspace(cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  Registry& R = registry();
  std::lock_guard<std::mutex> lk(R.mu);
  auto it = R.ws.find({dev, stream});
  if (it == R.ws.end()) return;
  {
    std::lock_guard<std::mutex> wl(it->second->mu);
    it->second->release();
  }
  R.ws.erase(it);
}

// Grow `b` to at least `bytes`.  Growing frees the old buffer, so in-flight
// work on the stream is waited for and every captured graph is dropped.
kde_status ensure(Workspace& W, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return KDE_OK;
  if (b.p) {
    if (W.stream) cudaStreamSynchronize(W.stream); else cudaDeviceSynchronize();
    W.drop_graphs();
    W.meta_key = 0;
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  const size_t want = bytes + bytes / 4;
  KDE_CU(cudaMalloc(&b.p, want));
  b.cap = want;
  W.drop_graphs();
  W.meta_key = 0;
  return KDE_OK;
}

// The plan for these arguments, built only when they differ from the last
// call's on this workspace.  Building it is O(tile pairs) host work -- the
// work-list of 524,800 items at n = 2^20, sorted by cost, ~10 ms -- during which
// the GPU would idle between back-to-back calls.  Call with W.mu held; the
// reference stays valid until the next plan_for on W.
const BatchPlan& plan_for(Workspace& W, int prec, int mode, int x_f32, const int64_t* ns, int64_t m,
                          double g_fixed, int stages = 2) {
  PlanArgs a;
  a.set(prec, mode, x_f32, ns, m, g_fixed, stages);
  if (!W.plan_set || !(a == W.plan_args)) {
    build_plan(W.plan, prec, mode, x_f32, ns, m, g_fixed, stages);
    W.plan_args = std::move(a);
    W.plan_set = true;
  }
  return W.plan;
}

kde_status reserve(Workspace& W, const BatchPlan& P) {
  const size_t xb = static_cast<size_t>(P.total_x) * (P.x_f32 ? sizeof(float) : sizeof(double));
  const size_t m = P.desc.size();
  kde_status s;
  if ((s = ensure(W, W.x, xb)) != KDE_OK) return s;
  // y doubles as the sort's scratch, so it holds 8 bytes per element
  if ((s = ensure(W, W.y, static_cast<size_t>(P.total_x) * sizeof(double))) != KDE_OK) return s;
  if ((s = ensure(W, W.bprefix, (m + 1) * sizeof(int64_t))) != KDE_OK) return s;
  if ((s = ensure(W, W.sprefix, (m + 1) * sizeof(int64_t))) != KDE_OK) return s;
  if ((s = ensure(W, W.scounts, static_cast<size_t>(P.sprefix[m]) * 256 * sizeof(uint32_t))) != KDE_OK) return s;
  if ((s = ensure(W, W.desc, m * sizeof(SampleDesc))) != KDE_OK) return s;
  if ((s = ensure(W, W.state, m * sizeof(SampleState))) != KDE_OK) return s;
  if ((s = ensure(W, W.mprefix, (m + 1) * sizeof(int64_t))) != KDE_OK) return s;
  if ((s = ensure(W, W.mslots, static_cast<size_t>(P.total_mslots) * sizeof(double))) != KDE_OK) return s;
  if ((s = ensure(W, W.slots, static_cast<size_t>(P.total_slots) * sizeof(double))) != KDE_OK) return s;
  if ((s = ensure(W, W.items, static_cast<size_t>(P.total_items) * sizeof(uint64_t))) != KDE_OK) return s;
  if ((s = ensure(W, W.counters, static_cast<size_t>(2 * P.n_pair_launches() + 2) * sizeof(unsigned long long))) != KDE_OK) return s;
  return KDE_OK;
}

// Record a profiling event; under stream capture it becomes an event-record
// node of the graph (external), so every replay records it.
cudaError_t prof_record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &cs);
  if (err != cudaSuccess) return err;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

// The launches of one plan, on stream s: init, sort, moments (Steps I-III),
// then per psi a prescale and the pair kernel(s) (Steps IV-V, then VI-VII).
kde_status enqueue(Workspace& W, const BatchPlan& P, cudaStream_t s) {
  const int64_t m = static_cast<int64_t>(P.desc.size());
  const int n_counters = 2 * P.n_pair_launches();
  auto* desc = static_cast<const SampleDesc*>(W.desc.p);
  auto* state = static_cast<SampleState*>(W.state.p);
  auto* counters = static_cast<unsigned long long*>(W.counters.p);
  const bool prof = g_profile.load() != 0;
  int launches = 0;
  if (prof) KDE_CU(prof_record(W.prof[0], s));
  KDE_CU(launch_init(desc, state, m, counters, n_counters, s));
  launches += m > 0 ? 1 : 0;
  SortArgs sa{};
  sa.x_is_f32 = P.x_f32;
  sa.desc = desc;
  sa.bprefix = static_cast<const int64_t*>(W.sprefix.p);
  sa.ids = nullptr;
  sa.m = m;
  sa.counts = static_cast<uint32_t*>(W.scounts.p);
  KDE_CU(launch_sort(sa, P.sprefix[m], W.x.p, W.y.p, s));
  if (P.sprefix[m] > 0 && m > 0) launches += 3 * (P.x_f32 ? 4 : 8);   // histogram, scan, scatter per pass
  MomentsArgs ma{};
  ma.x = W.x.p;
  ma.x_is_f32 = P.x_f32;
  ma.desc = desc;
  ma.state = state;
  ma.mprefix = static_cast<const int64_t*>(W.mprefix.p);
  ma.ids = nullptr;
  ma.m = m;
  ma.mslots = static_cast<double*>(W.mslots.p);
  KDE_CU(launch_moments(ma, P.mprefix[m], s));
  launches += P.mprefix[m] > 0 ? 1 : 0;
  PrescaleArgs pr{};
  pr.x = W.x.p;
  pr.x_is_f32 = P.x_f32;
  pr.desc = desc;
  pr.state = state;
  pr.bprefix = static_cast<const int64_t*>(W.bprefix.p);
  pr.ids = nullptr;
  pr.m = m;
  pr.y = W.y.p;
  std::vector<int> orders;   // the plug-in's estimated orders, top first
  if (P.mode == kPlugin)
    for (int r = 2 * P.stages + 2; r >= 4; r -= 2) orders.push_back(r);
  else
    orders = {P.mode};
  int L = 0;
  for (size_t o = 0; o < orders.size(); ++o) {
    const int r = orders[o];
    KDE_CU(launch_prescale(pr, P.bprefix[m], s));
    launches += P.bprefix[m] > 0 ? 1 : 0;
    const bool first = o == 0, last = o + 1 == orders.size();
    if (prof && first) KDE_CU(prof_record(W.prof[1], s));
    if (prof && last && !first) KDE_CU(prof_record(W.prof[3], s));
    for (const Group& g : P.groups) {
      PairArgs pa{};
      pa.y = W.y.p;
      pa.desc = desc;
      pa.state = state;
      pa.items = static_cast<const uint64_t*>(W.items.p) + g.item_off;
      pa.n_items = static_cast<int64_t>(g.items.size());
      pa.slots = static_cast<double*>(W.slots.p);
      pa.counters = counters + 2 * L;
      pa.r = r;
      pa.chain = P.mode == kPlugin ? 1 : 0;
      KDE_CU(launch_pairs(P.prec, g.cfg, pa, g.grid, s));
      launches += g.grid > 0 ? 1 : 0;
      ++L;
    }
    if (prof && first) KDE_CU(prof_record(W.prof[2], s));
    if (prof && last && !first) KDE_CU(prof_record(W.prof[4], s));
  }
  if (P.mode == kPlugin) {
    KDE_CU(launch_stage_results(state, m, s));
    launches += m > 0 ? 1 : 0;
  }
  if (prof && orders.size() == 1) {
    KDE_CU(prof_record(W.prof[3], s));
    KDE_CU(prof_record(W.prof[4], s));
  }
  W.prof_valid = prof;
  W.last_launches = launches;
  return KDE_OK;
}

bool graphs_enabled() { return env_int("KDE_NO_GRAPH", 0) == 0; }

// Stage x, upload the plan's metadata if it changed, run the plan.
kde_status run_plan(Workspace& W, const BatchPlan& P, const void* x, bool x_dev, cudaStream_t s) {
  kde_status st = reserve(W, P);
  if (st != KDE_OK) return st;
  const size_t xb = static_cast<size_t>(P.total_x) * (P.x_f32 ? sizeof(float) : sizeof(double));
  if (xb) KDE_CU(cudaMemcpyAsync(W.x.p, x, xb, x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (W.meta_key != P.key) {
    std::vector<uint64_t> items(static_cast<size_t>(P.total_items));
    for (const Group& g : P.groups)
      std::copy(g.items.begin(), g.items.end(), items.begin() + g.item_off);
    // pageable sources: the copies are staged before cudaMemcpyAsync returns
    KDE_CU(cudaMemcpyAsync(W.desc.p, P.desc.data(), P.desc.size() * sizeof(SampleDesc), cudaMemcpyHostToDevice, s));
    KDE_CU(cudaMemcpyAsync(W.mprefix.p, P.mprefix.data(), P.mprefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    KDE_CU(cudaMemcpyAsync(W.bprefix.p, P.bprefix.data(), P.bprefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    KDE_CU(cudaMemcpyAsync(W.sprefix.p, P.sprefix.data(), P.sprefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (!items.empty())
      KDE_CU(cudaMemcpyAsync(W.items.p, items.data(), items.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    W.meta_key = P.key;
  }
  if (g_profile.load()) {
    for (cudaEvent_t& e : W.prof)
      if (!e) KDE_CU(cudaEventCreate(&e));
  }
  W.last_m = static_cast<int64_t>(P.desc.size());
  if (!graphs_enabled()) return enqueue(W, P, s);
  const uint64_t gkey = P.key ^ (g_profile.load() ? 0x9E3779B97F4A7C15ull : 0ull);
  auto it = W.graphs.find(gkey);
  if (it == W.graphs.end()) {
    if (W.graphs.size() >= 64) W.drop_graphs();
    if (!W.cap_stream) KDE_CU(cudaStreamCreateWithFlags(&W.cap_stream, cudaStreamNonBlocking));
    KDE_CU(cudaStreamBeginCapture(W.cap_stream, cudaStreamCaptureModeThreadLocal));
    kde_status es = enqueue(W, P, W.cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(W.cap_stream, &graph);
    if (es != KDE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return es;
    }
    if (ce != cudaSuccess) return set_err(KDE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return set_err(KDE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    it = W.graphs.emplace(gkey, Workspace::GraphEntry{exec, W.last_launches}).first;
  }
  KDE_CU(cudaGraphLaunch(it->second.exec, s));
  W.last_launches = it->second.launches;
  return KDE_OK;
}

kde_status copy_results(Workspace& W, int64_t m, kde_result* out, bool out_dev, cudaStream_t s) {
  KDE_CU(cudaMemcpy2DAsync(out, sizeof(kde_result), W.state.p, sizeof(SampleState), sizeof(kde_result),
                           static_cast<size_t>(m), out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (!out_dev) KDE_CU(cudaStreamSynchronize(s));
  return KDE_OK;
}

// ---------------------------------------------------------------------------
// entry points (C++ side)
// ---------------------------------------------------------------------------

kde_status plugin_one(const void* x, int x_f32, int64_t n, kde_precision prec, kde_result* out,
                      void* stream) {
  if (!x || !out) return set_err(KDE_ERR_INVALID, "null pointer");
  if (n < 2) return set_err(KDE_ERR_INVALID, "n < 2");
  if (prec != KDE_FP32 && prec != KDE_FP64 && prec != KDE_Q32) return set_err(KDE_ERR_INVALID, "bad precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace* W = nullptr;
  kde_status st = get_workspace(s, &W);
  if (st != KDE_OK) return st;
  std::lock_guard<std::mutex> lk(W->mu);
  const BatchPlan& P = plan_for(*W, prec, kPlugin, x_f32, &n, 1, 0.0);
  if ((st = run_plan(*W, P, x, is_device_ptr(x), s)) != KDE_OK) return st;
  const bool out_dev = is_device_ptr(out);
  if ((st = copy_results(*W, 1, out, out_dev, s)) != KDE_OK) return st;
  if (!out_dev && out->status != KDE_OK) {
    static const char* msg[] = {"", "invalid input", "zero standard deviation", "psi6 >= 0 or psi4 <= 0"};
    return set_err(static_cast<kde_status>(out->status),
                   out->status < 4 ? msg[out->status] : "error");
  }
  return KDE_OK;
}

kde_status plugin_stages_one(const double* x, int64_t n, int stages, kde_precision prec,
                             kde_stage_result* out, void* stream) {
  if (!x || !out) return set_err(KDE_ERR_INVALID, "null pointer");
  if (n < 2) return set_err(KDE_ERR_INVALID, "n < 2");
  if (stages < 1 || stages > 4) return set_err(KDE_ERR_INVALID, "stages must be 1..4");
  if (prec != KDE_FP32 && prec != KDE_FP64 && prec != KDE_Q32) return set_err(KDE_ERR_INVALID, "bad precision");
  if (prec == KDE_Q32 && stages > 2) return set_err(KDE_ERR_INVALID, "KDE_Q32 evaluates psi_4 and psi_6 only");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace* W = nullptr;
  kde_status st = get_workspace(s, &W);
  if (st != KDE_OK) return st;
  std::lock_guard<std::mutex> lk(W->mu);
  const BatchPlan& P = plan_for(*W, prec, kPlugin, 0, &n, 1, 0.0, stages);
  if ((st = run_plan(*W, P, x, is_device_ptr(x), s)) != KDE_OK) return st;
  const bool out_dev = is_device_ptr(out);
  const auto* src = &static_cast<const SampleState*>(W->state.p)->sres;
  KDE_CU(cudaMemcpyAsync(out, src, sizeof(kde_stage_result),
                         out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (out_dev) return KDE_OK;
  KDE_CU(cudaStreamSynchronize(s));
  if (out->status != KDE_OK) return set_err(static_cast<kde_status>(out->status), "plug-in failed on device");
  return KDE_OK;
}

kde_status psi_check(const double* x, int64_t n, int r, double g, kde_precision prec, Workspace** Wout,
                     cudaStream_t s) {
  if (!x) return set_err(KDE_ERR_INVALID, "null pointer");
  if (n < 2) return set_err(KDE_ERR_INVALID, "n < 2");
  if (r != 4 && r != 6 && r != 8 && r != 10) return set_err(KDE_ERR_INVALID, "r must be 4, 6, 8 or 10");
  if (!(g > 0) || !std::isfinite(g)) return set_err(KDE_ERR_INVALID, "g must be finite and > 0");
  if (prec != KDE_FP32 && prec != KDE_FP64 && prec != KDE_Q32) return set_err(KDE_ERR_INVALID, "bad precision");
  if (prec == KDE_Q32 && r > 6) return set_err(KDE_ERR_INVALID, "KDE_Q32 evaluates psi_4 and psi_6 only");
  return get_workspace(s, Wout);
}

}  // namespace kde

using namespace kde;

extern "C" {

kde_status kde_psi(const double* x, int64_t n, int r, double g, kde_precision prec, double* out,
                   void* stream) {
  if (!out) return set_err(KDE_ERR_INVALID, "null pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace* W = nullptr;
  kde_status st = psi_check(x, n, r, g, prec, &W, s);
  if (st != KDE_OK) return st;
  std::lock_guard<std::mutex> lk(W->mu);
  const BatchPlan& P = plan_for(*W, prec, r, 0, &n, 1, g);
  if ((st = run_plan(*W, P, x, is_device_ptr(x), s)) != KDE_OK) return st;
  const auto* dst = static_cast<const SampleState*>(W->state.p);
  if (is_device_ptr(out)) {
    KDE_CU(cudaMemcpyAsync(out, &dst->psi_out, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return KDE_OK;
  }
  SampleState h{};
  KDE_CU(cudaMemcpyAsync(&h, dst, sizeof(SampleState), cudaMemcpyDeviceToHost, s));
  KDE_CU(cudaStreamSynchronize(s));
  *out = h.psi_out;
  if (h.res.status != KDE_OK) return set_err(static_cast<kde_status>(h.res.status), "psi failed on device");
  return KDE_OK;
}

kde_status kde_psi_slots(const double* x, int64_t n, int r, double g, kde_precision prec,
                         double* slots, int64_t cap, int64_t* info) {
  if (!info) return set_err(KDE_ERR_INVALID, "null info");
  Workspace* W = nullptr;
  kde_status st = psi_check(x, n, r, g, prec, &W, nullptr);
  if (st != KDE_OK) return st;
  std::lock_guard<std::mutex> lk(W->mu);
  const BatchPlan& P = plan_for(*W, prec, r, 0, &n, 1, g);
  const SampleDesc& d = P.desc[0];
  info[0] = pair_config(prec, P.groups[0].cfg).tile();
  info[1] = d.chunk;
  info[2] = d.ntp;
  info[3] = d.nchunks;
  if (!slots) return KDE_OK;
  if (cap < d.nchunks) return set_err(KDE_ERR_INVALID, "slot capacity too small");
  if ((st = run_plan(*W, P, x, is_device_ptr(x), nullptr)) != KDE_OK) return st;
  KDE_CU(cudaMemcpy(slots, W->slots.p, static_cast<size_t>(d.nchunks) * sizeof(double), cudaMemcpyDeviceToHost));
  return KDE_OK;
}

kde_status kde_plugin_h_stages(const double* x, int64_t n, int stages, kde_precision prec,
                               kde_stage_result* out, void* stream) {
  return plugin_stages_one(x, n, stages, prec, out, stream);
}

kde_status kde_plugin_h(const double* x, int64_t n, kde_precision prec, kde_result* out, void* stream) {
  return plugin_one(x, 0, n, prec, out, stream);
}

kde_status kde_plugin_h_f32(const float* x, int64_t n, kde_precision prec, kde_result* out, void* stream) {
  return plugin_one(x, 1, n, prec, out, stream);
}

kde_status kde_plugin_h_batch(const double* x_packed, const int64_t* offsets, int64_t m,
                              kde_precision prec, kde_result* out, void* stream) {
  if (!x_packed || !offsets || !out) return set_err(KDE_ERR_INVALID, "null pointer");
  if (m < 1) return set_err(KDE_ERR_INVALID, "m < 1");
  if (prec != KDE_FP32 && prec != KDE_FP64 && prec != KDE_Q32) return set_err(KDE_ERR_INVALID, "bad precision");
  if (offsets[0] != 0) return set_err(KDE_ERR_INVALID, "offsets[0] must be 0");
  std::vector<int64_t> ns(static_cast<size_t>(m));
  for (int64_t k = 0; k < m; ++k) {
    ns[k] = offsets[k + 1] - offsets[k];
    if (ns[k] < 0) return set_err(KDE_ERR_INVALID, "offsets must not decrease");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Workspace* W = nullptr;
  kde_status st = get_workspace(s, &W);
  if (st != KDE_OK) return st;
  std::lock_guard<std::mutex> lk(W->mu);
  const BatchPlan& P = plan_for(*W, prec, kPlugin, 0, ns.data(), m, 0.0);
  if ((st = run_plan(*W, P, x_packed, is_device_ptr(x_packed), s)) != KDE_OK) return st;
  return copy_results(*W, m, out, is_device_ptr(out), s);
}

kde_status kde_profile_enable(int on) {
  g_profile.store(on ? 1 : 0);
  return KDE_OK;
}

kde_status kde_profile_last(void* stream, double* ms, int cap) {
  if (!ms || cap < 4) return set_err(KDE_ERR_INVALID, "need room for 4 durations");
  for (int i = 4; i < cap && i < 7; ++i) ms[i] = 0.0;
  Workspace* W = nullptr;
  kde_status st = get_workspace(static_cast<cudaStream_t>(stream), &W);
  if (st != KDE_OK) return st;
  std::lock_guard<std::mutex> lk(W->mu);
  if (!W->prof_valid) return set_err(KDE_ERR_INVALID, "no profiled run on this stream");
  KDE_CU(cudaEventSynchronize(W->prof[4]));
  for (int i = 0; i < 4; ++i) {
    float v = 0.0f;
    KDE_CU(cudaEventElapsedTime(&v, W->prof[i], W->prof[i + 1]));
    ms[i] = v;
  }
  if (cap >= 5) ms[4] = W->last_launches;
  if (cap >= 7) {
    // unique pairs the pair kernels skipped (far tile pairs), summed over the samples
    std::vector<SampleState> h(static_cast<size_t>(W->last_m));
    if (!h.empty())
      KDE_CU(cudaMemcpy(h.data(), W->state.p, h.size() * sizeof(SampleState), cudaMemcpyDeviceToHost));
    double s6 = 0.0, s4 = 0.0;
    for (const SampleState& q : h) {
      s6 += static_cast<double>(q.skipped[0]);
      s4 += static_cast<double>(q.skipped[1]);
    }
    ms[5] = s6;
    ms[6] = s4;
  }
  return KDE_OK;
}

const char* kde_last_error(void) { return t_err.c_str(); }

const char* kde_version(void) { return "libkde 0.1 (sm_103a)"; }

void kde_shutdown(void) {
  Registry& R = registry();
  std::lock_guard<std::mutex> lk(R.mu);
  for (auto& kv : R.ws) {
    std::lock_guard<std::mutex> wl(kv.second->mu);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(kv.second->device);
    kv.second->release();
    cudaSetDevice(prev);
  }
  R.ws.clear();
  eval_release_all();
  static_scratch_forget();
}

}  // extern "C"
