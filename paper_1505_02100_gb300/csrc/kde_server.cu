// kde_server.cu -- continuous batching of bandwidth-selection requests
// (kde_server_* in include/kde.h).
//
// One host thread owns the device.  Requests wait in a FIFO queue until a
// request slot and room in the device arena (one cudaMalloc made at creation,
// carved by a first-fit allocator) are free; then their samples are copied to
// the arena and they are "admitted".  The thread then runs ticks: each tick is
// one moments launch, one pair launch with r = 6 and one with r = 4 per
// (precision, tile configuration), over work items taken from every admitted
// request -- smallest remaining work first, the oldest request always served
// -- until the tick's budget of pair evaluations is spent.  Stream order makes a
// request's moments, psi6 chunks and psi4 chunks correct within one tick, so
// small requests finish in the tick they join, while large ones progress a
// budget slice per tick beside them.  Up to two ticks are in flight; a
// request's result is copied back with the tick that runs its last chunk.
//
// Per-sample results and summation order are those of kde_plugin_h_f32: the
// tiling depends only on n and every chunk writes its own slot.
#include "kde_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace kde {
namespace {

int64_t now_ns(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, capacity) with coalescing of freed ranges.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) { free_[0] = cap; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes ? bytes : 1, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes ? bytes : 1, 256);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t capacity() const { return cap_; }
  size_t used() const { return used_; }

 private:
  size_t cap_, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Req {
  uint64_t ticket = 0;
  int64_t n = 0;
  int prec = KDE_FP32;
  int cfg = 0;
  std::vector<float> x;
  SampleDesc d{};
  int slot = -1;
  size_t off_x = 0, off_y = 0, off_s = 0, off_m = 0, b_x = 0, b_y = 0, b_s = 0, b_m = 0;
  int phase = 0;            // 0 moments, 1 psi6 chunks, 2 psi4 chunks, 3 all scheduled
  int64_t next_chunk = 0;
  double cost_per_pair = 1.0;
  bool finished = false;
  kde_result res{};
  kde_request_times times{};

  size_t footprint() const {
    return align_up(b_x, 256) + align_up(b_y, 256) + align_up(b_s, 256) + align_up(b_m, 256);
  }
  double chunk_cost(int64_t c) const {
    const double T = static_cast<double>(pair_config(prec, cfg).tile());
    return static_cast<double>(std::min(d.chunk, d.ntp - c * d.chunk)) * T * T * cost_per_pair;
  }
  double remaining() const {
    double r = 0.0;
    const double full = static_cast<double>(d.ntp);
    const double T = static_cast<double>(pair_config(prec, cfg).tile());
    if (phase <= 1) r += (full - static_cast<double>(phase == 1 ? next_chunk * d.chunk : 0)) * T * T;
    if (phase <= 2) r += (full - static_cast<double>(phase == 2 ? next_chunk * d.chunk : 0)) * T * T;
    return r * cost_per_pair;
  }
};

struct TickBufs {
  void* h = nullptr;        // pinned host: upload area, then result area
  void* d = nullptr;        // device: uploaded work-lists
  size_t cap = 0;
  cudaEvent_t start = nullptr, done = nullptr;
  std::vector<std::shared_ptr<Req>> finishing;
  double scheduled_cost = 0.0;
  bool in_flight = false;
};

}  // namespace

struct ServerImpl {
  kde_server_config cfg{};
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::vector<std::shared_ptr<Req>> admitted;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> by_ticket;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::thread worker;
  // device state (touched by the worker thread only, after create)
  cudaStream_t stream = nullptr;
  char* arena_d = nullptr;
  std::unique_ptr<Arena> arena;
  SampleDesc* desc_d = nullptr;
  SampleState* state_d = nullptr;
  unsigned long long* counters_d = nullptr;
  uint32_t* sort_counts_d = nullptr;   // radix-sort digit counts (grown on demand)
  size_t sort_counts_cap = 0;
  std::vector<int> free_slots;
  TickBufs ticks[2];
  int tick_next = 0;
  double rate_per_ms = 4.0e9;   // FP32 pair evaluations per device ms (EWMA)
  double min_budget = 1.0e9;     // pair evaluations that fill every SM (set in init)
  kde_status fatal = KDE_OK;

  static constexpr int kMaxGroups = 16;
  static constexpr double kFp64Cost = 40.0;   // an FP64 pair costs this many FP32 pairs

  kde_status init() {
    cudaError_t e = cudaSetDevice(cfg.device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&arena_d, cfg.hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&desc_d, sizeof(SampleDesc) * cfg.max_inflight);
    if (e == cudaSuccess) e = cudaMalloc(&state_d, sizeof(SampleState) * cfg.max_inflight);
    if (e == cudaSuccess) e = cudaMalloc(&counters_d, sizeof(unsigned long long) * 4 * kMaxGroups);
    for (auto& t : ticks) {
      if (e == cudaSuccess) e = cudaEventCreate(&t.start);
      if (e == cudaSuccess) e = cudaEventCreate(&t.done);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(e == cudaErrorMemoryAllocation ? KDE_ERR_OOM : KDE_ERR_CUDA,
                     std::string("server init: ") + cudaGetErrorString(e));
    }
    arena.reset(new Arena(cfg.hbm_budget_bytes));
    // a tick never schedules less than ~32 tile pairs of side 512 per SM, so
    // launch overhead stays small next to the work even when the rate
    // estimate is off
    min_budget = static_cast<double>(num_sms()) * 32.0 * 512.0 * 512.0;
    for (int i = cfg.max_inflight - 1; i >= 0; --i) free_slots.push_back(i);
    return KDE_OK;
  }

  void destroy_device() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& t : ticks) {
      if (t.h) cudaFreeHost(t.h);
      if (t.d) cudaFree(t.d);
      if (t.start) cudaEventDestroy(t.start);
      if (t.done) cudaEventDestroy(t.done);
    }
    if (arena_d) cudaFree(arena_d);
    if (sort_counts_d) cudaFree(sort_counts_d);
    if (desc_d) cudaFree(desc_d);
    if (state_d) cudaFree(state_d);
    if (counters_d) cudaFree(counters_d);
    if (stream) cudaStreamDestroy(stream);
  }

  // plan a request: tiling and device footprint
  void plan(Req& r) {
    r.cfg = choose_config(r.prec, r.n);
    r.d = make_desc(r.prec, r.cfg, r.n, 0.0);
    r.b_x = sizeof(float) * static_cast<size_t>(r.n);
    r.b_y = sizeof(double) * static_cast<size_t>(r.n);   // float2 (binary32) or double (binary64)
    r.b_s = sizeof(double) * static_cast<size_t>(r.d.nchunks);
    r.b_m = sizeof(double) * 5 * static_cast<size_t>(r.d.mblocks);
    r.cost_per_pair = r.prec == KDE_FP64 ? kFp64Cost : 1.0;
  }

  // worker thread: move queued requests onto the device while room remains
  bool admit_locked(std::vector<std::shared_ptr<Req>>& fresh) {
    while (!queue.empty() && !free_slots.empty()) {
      auto r = queue.front();
      size_t o[4];
      const size_t sz[4] = {r->b_x, r->b_y, r->b_s, r->b_m};
      int got = 0;
      while (got < 4 && arena->alloc(sz[got], &o[got])) ++got;
      if (got < 4) {
        for (int i = 0; i < got; ++i) arena->release(o[i], sz[i]);
        break;
      }
      queue.pop_front();
      r->off_x = o[0]; r->off_y = o[1]; r->off_s = o[2]; r->off_m = o[3];
      r->slot = free_slots.back();
      free_slots.pop_back();
      r->d.x_off = static_cast<int64_t>(r->off_x / sizeof(float));
      r->d.y_off = static_cast<int64_t>(r->off_y / 8);   // float2 or double elements
      r->d.tmp_off = static_cast<int64_t>(r->off_y / sizeof(float));   // sort scratch: the y region
      r->d.slot_off = static_cast<int64_t>(r->off_s / sizeof(double));
      r->d.mslot_off = static_cast<int64_t>(r->off_m / sizeof(double));
      r->times.t_admit_ns = now_ns(t0);
      admitted.push_back(r);
      fresh.push_back(r);
    }
    return !fresh.empty();
  }

  kde_status upload_fresh(const std::vector<std::shared_ptr<Req>>& fresh) {
    for (auto& r : fresh) {
      cudaError_t e = cudaMemcpyAsync(arena_d + r->off_x, r->x.data(), r->b_x, cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(desc_d + r->slot, &r->d, sizeof(SampleDesc), cudaMemcpyHostToDevice, stream);
      SampleState s0{};
      const double q = std::nan("");
      s0.res.mean = s0.res.sigma = s0.res.psi8 = s0.res.g1 = s0.res.psi6 = s0.res.g2 = s0.res.psi4 = s0.res.h = q;
      s0.res.status = KDE_OK;
      s0.xmin = s0.xmax = s0.g_cur = s0.scale = s0.pad_lo = s0.pad_hi = s0.psi_out = q;
      s0.center = s0.qlo = s0.qhi = q;
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(state_d + r->slot, &s0, sizeof(SampleState), cudaMemcpyHostToDevice, stream);
      if (e != cudaSuccess) return set_err(KDE_ERR_CUDA, std::string("server upload: ") + cudaGetErrorString(e));
      std::vector<float>().swap(r->x);   // pageable copies are staged before return
    }
    return KDE_OK;
  }

  // Build and launch one tick into ticks[tick_next].  Returns false if there was no work.
  bool launch_tick_locked(kde_status* err) {
    std::vector<std::shared_ptr<Req>> order;
    for (auto& r : admitted)
      if (r->phase < 3) order.push_back(r);
    if (order.empty()) return false;
    const double target_ms = cfg.tick_target_ms > 0 ? cfg.tick_target_ms : 2.0;
    double budget = std::max(min_budget, target_ms * rate_per_ms);
    // The oldest admitted request is served first but with at most a quarter
    // of the budget (no starvation, no monopoly); the others go smallest
    // remaining work first; whatever budget is left returns to the oldest.
    std::stable_sort(order.begin() + 1, order.end(),
                     [](const std::shared_ptr<Req>& a, const std::shared_ptr<Req>& b) {
                       return a->remaining() < b->remaining();
                     });
    std::vector<int32_t> mom_ids, pre_ids[2];
    std::vector<int64_t> mom_prefix{0}, sort_prefix{0}, pre_prefix[2] = {{0}, {0}};
    std::map<std::pair<int, int>, std::vector<uint64_t>> items6, items4;
    TickBufs& tb = ticks[tick_next];
    tb.finishing.clear();
    double spent = 0.0;
    auto grant = [&](Req& r, double cap) {
      if (r.phase == 0) {
        mom_ids.push_back(r.slot);
        mom_prefix.push_back(mom_prefix.back() + r.d.mblocks);
        sort_prefix.push_back(sort_prefix.back() + (r.n + kSortChunk - 1) / kSortChunk);
        r.phase = 1;
        r.next_chunk = 0;
      }
      double used = 0.0;
      for (int ph = 1; ph <= 2 && used < cap; ++ph) {
        if (r.phase != ph) continue;
        auto& dst = (ph == 1 ? items6 : items4)[{r.prec, r.cfg}];
        while (r.next_chunk < r.d.nchunks && used < cap) {
          if (r.next_chunk == 0) {   // first chunk of this psi: scale the sample first
            pre_ids[ph - 1].push_back(r.slot);
            pre_prefix[ph - 1].push_back(pre_prefix[ph - 1].back() +
                                         (r.n + kPrescaleThreads - 1) / kPrescaleThreads);
          }
          const double c = r.chunk_cost(r.next_chunk);
          dst.push_back((static_cast<uint64_t>(r.slot) << 32) | static_cast<uint64_t>(r.next_chunk));
          used += c;
          ++r.next_chunk;
        }
        if (r.next_chunk == r.d.nchunks) {
          r.phase = ph + 1;
          r.next_chunk = 0;
        }
      }
      return used;
    };
    double left = budget;
    left -= grant(*order[0], 0.25 * budget);
    for (size_t i = 1; i < order.size() && left > 0.0; ++i) left -= grant(*order[i], left);
    if (left > 0.0) left -= grant(*order[0], left);
    spent = budget - left;
    for (auto& r : order)
      if (r->phase == 3 && std::find(tb.finishing.begin(), tb.finishing.end(), r) == tb.finishing.end())
        tb.finishing.push_back(r);
    // upload layout: [mom_prefix][mom_ids][pre6 prefix][pre6 ids][pre4 prefix][pre4 ids]
    //                [items6 groups][items4 groups], each 16-byte aligned
    size_t bytes = align_up(mom_prefix.size() * 8, 16) + align_up(mom_ids.size() * 4, 16) +
                   align_up(sort_prefix.size() * 8, 16);
    for (int q = 0; q < 2; ++q)
      bytes += align_up(pre_prefix[q].size() * 8, 16) + align_up(pre_ids[q].size() * 4, 16);
    for (auto& kv : items6) bytes += align_up(kv.second.size() * 8, 16);
    for (auto& kv : items4) bytes += align_up(kv.second.size() * 8, 16);
    const size_t res_bytes = tb.finishing.size() * sizeof(SampleState);
    const size_t need = std::max(bytes, res_bytes) + 64;
    if (tb.cap < need) {
      if (tb.h) cudaFreeHost(tb.h);
      if (tb.d) cudaFree(tb.d);
      tb.h = tb.d = nullptr;
      tb.cap = 0;
      const size_t c = align_up(need * 2, 4096);
      if (cudaMallocHost(&tb.h, c) != cudaSuccess || cudaMalloc(&tb.d, c) != cudaSuccess) {
        cudaGetLastError();
        *err = set_err(KDE_ERR_OOM, "server tick buffers");
        return false;
      }
      tb.cap = c;
    }
    char* h = static_cast<char*>(tb.h);
    char* d = static_cast<char*>(tb.d);
    size_t o = 0;
    auto put = [&](const void* src, size_t n) {
      const size_t at = o;
      if (n) std::memcpy(h + o, src, n);
      o += align_up(n, 16);
      return at;
    };
    const size_t o_prefix = put(mom_prefix.data(), mom_prefix.size() * 8);
    const size_t o_ids = put(mom_ids.data(), mom_ids.size() * 4);
    const size_t o_sp = put(sort_prefix.data(), sort_prefix.size() * 8);
    size_t o_pp[2], o_pi[2];
    for (int q = 0; q < 2; ++q) {
      o_pp[q] = put(pre_prefix[q].data(), pre_prefix[q].size() * 8);
      o_pi[q] = put(pre_ids[q].data(), pre_ids[q].size() * 4);
    }
    std::vector<std::pair<std::pair<int, int>, std::pair<size_t, size_t>>> g6, g4;
    for (auto& kv : items6) g6.push_back({kv.first, {put(kv.second.data(), kv.second.size() * 8), kv.second.size()}});
    for (auto& kv : items4) g4.push_back({kv.first, {put(kv.second.data(), kv.second.size() * 8), kv.second.size()}});
    cudaError_t e = cudaEventRecord(tb.start, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, o, cudaMemcpyHostToDevice, stream);
    const int n_launch = static_cast<int>(g6.size() + g4.size());
    if (e == cudaSuccess)
      e = cudaMemsetAsync(counters_d, 0, sizeof(unsigned long long) * 2 * std::max(n_launch, 1), stream);
    if (e == cudaSuccess && !mom_ids.empty()) {
      // sort the new requests' samples (device order = value order), then moments
      const size_t need_counts = static_cast<size_t>(sort_prefix.back()) * 256;
      if (need_counts > sort_counts_cap) {
        cudaStreamSynchronize(stream);   // earlier ticks may still read the old buffer
        if (sort_counts_d) cudaFree(sort_counts_d);
        sort_counts_d = nullptr;
        sort_counts_cap = 0;
        e = cudaMalloc(&sort_counts_d, sizeof(uint32_t) * need_counts * 2);
        if (e == cudaSuccess) sort_counts_cap = need_counts * 2;
      }
      if (e == cudaSuccess) {
        SortArgs sa{};
        sa.x_is_f32 = 1;
        sa.desc = desc_d;
        sa.bprefix = reinterpret_cast<const int64_t*>(d + o_sp);
        sa.ids = reinterpret_cast<const int32_t*>(d + o_ids);
        sa.m = static_cast<int64_t>(mom_ids.size());
        sa.counts = sort_counts_d;
        e = launch_sort(sa, sort_prefix.back(), arena_d, arena_d, stream);
      }
    }
    if (e == cudaSuccess && !mom_ids.empty()) {
      MomentsArgs ma{};
      ma.x = arena_d;
      ma.x_is_f32 = 1;
      ma.desc = desc_d;
      ma.state = state_d;
      ma.mprefix = reinterpret_cast<const int64_t*>(d + o_prefix);
      ma.ids = reinterpret_cast<const int32_t*>(d + o_ids);
      ma.m = static_cast<int64_t>(mom_ids.size());
      ma.mslots = reinterpret_cast<double*>(arena_d);
      e = launch_moments(ma, mom_prefix.back(), stream);
    }
    int L = 0;
    const int sms = num_sms();
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
      if (!pre_ids[pass].empty()) {
        PrescaleArgs pr{};
        pr.x = arena_d;
        pr.x_is_f32 = 1;
        pr.desc = desc_d;
        pr.state = state_d;
        pr.bprefix = reinterpret_cast<const int64_t*>(d + o_pp[pass]);
        pr.ids = reinterpret_cast<const int32_t*>(d + o_pi[pass]);
        pr.m = static_cast<int64_t>(pre_ids[pass].size());
        pr.y = arena_d;
        e = launch_prescale(pr, pre_prefix[pass].back(), stream);
        if (e != cudaSuccess) break;
      }
      for (auto& g : (pass == 0 ? g6 : g4)) {
        PairArgs pa{};
        pa.y = arena_d;
        pa.desc = desc_d;
        pa.state = state_d;
        pa.items = reinterpret_cast<const uint64_t*>(d + g.second.first);
        pa.n_items = static_cast<int64_t>(g.second.second);
        pa.slots = reinterpret_cast<double*>(arena_d);
        pa.counters = counters_d + 2 * L;
        pa.r = pass == 0 ? 6 : 4;
        pa.chain = 1;
        const int prec = g.first.first, cf = g.first.second;
        const int64_t resident = static_cast<int64_t>(pair_blocks_per_sm(prec, cf)) * sms;
        const int grid = static_cast<int>(std::min<int64_t>(resident, pa.n_items));
        e = launch_pairs(prec, cf, pa, grid, stream);
        ++L;
        if (e != cudaSuccess) break;
      }
    }
    // results of requests whose last chunk runs in this tick
    for (size_t i = 0; i < tb.finishing.size() && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(h + i * sizeof(SampleState), state_d + tb.finishing[i]->slot, sizeof(SampleState),
                          cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaEventRecord(tb.done, stream);
    if (e != cudaSuccess) {
      *err = set_err(KDE_ERR_CUDA, std::string("server tick: ") + cudaGetErrorString(e));
      return false;
    }
    tb.scheduled_cost = spent;
    tb.in_flight = true;
    tick_next ^= 1;
    return true;
  }

  // Wait for tick t, hand out its finished requests, update the rate estimate.
  void complete_tick(TickBufs& tb) {
    cudaEventSynchronize(tb.done);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, tb.start, tb.done);
    // learn the device rate only from ticks that carried a full budget
    if (ms > 0.05f && tb.scheduled_cost >= min_budget) {
      const double r = std::min(1.0e11, std::max(1.0e8, tb.scheduled_cost / ms));
      rate_per_ms = 0.7 * rate_per_ms + 0.3 * r;
    }
    std::lock_guard<std::mutex> lk(mu);
    const char* h = static_cast<const char*>(tb.h);
    const int64_t t = now_ns(t0);
    for (size_t i = 0; i < tb.finishing.size(); ++i) {
      auto& r = tb.finishing[i];
      SampleState s;
      std::memcpy(&s, h + i * sizeof(SampleState), sizeof s);
      r->res = s.res;
      r->times.status = s.res.status;
      r->times.t_done_ns = t;
      r->times.skipped6 = s.skipped[0];
      r->times.skipped4 = s.skipped[1];
      r->finished = true;
      arena->release(r->off_x, r->b_x);
      arena->release(r->off_y, r->b_y);
      arena->release(r->off_s, r->b_s);
      arena->release(r->off_m, r->b_m);
      free_slots.push_back(r->slot);
      admitted.erase(std::find(admitted.begin(), admitted.end(), r));
    }
    tb.finishing.clear();
    tb.in_flight = false;
    cv_done.notify_all();
  }

  void run() {
    cudaSetDevice(cfg.device);
    for (;;) {
      std::vector<std::shared_ptr<Req>> fresh;
      kde_status err = KDE_OK;
      bool launched = false;
      {
        std::unique_lock<std::mutex> lk(mu);
        const bool any_flight = ticks[0].in_flight || ticks[1].in_flight;
        if (!any_flight) {
          cv_work.wait(lk, [&] {
            bool work = !queue.empty() && !free_slots.empty();
            for (auto& r : admitted) work = work || r->phase < 3;
            return work || (stopping && queue.empty() && admitted.empty());
          });
          if (stopping && queue.empty() && admitted.empty()) break;
        }
        admit_locked(fresh);
      }
      if (!fresh.empty()) err = upload_fresh(fresh);
      TickBufs& nxt = ticks[tick_next];
      if (err == KDE_OK && nxt.in_flight) complete_tick(nxt);   // keep at most two ticks in flight
      if (err == KDE_OK) {
        std::lock_guard<std::mutex> lk(mu);
        launched = launch_tick_locked(&err);
      }
      if (err != KDE_OK) {
        fail_all(err);
        break;
      }
      if (!launched) {
        // nothing new to launch: retire the oldest tick in flight, if any
        TickBufs& a = ticks[tick_next];
        TickBufs& b = ticks[tick_next ^ 1];
        if (a.in_flight) complete_tick(a);
        else if (b.in_flight) complete_tick(b);
      }
    }
    for (auto& t : ticks)
      if (t.in_flight) complete_tick(t);
  }

  void fail_all(kde_status err) {
    cudaStreamSynchronize(stream);
    std::lock_guard<std::mutex> lk(mu);
    fatal = err;
    auto mark = [&](const std::shared_ptr<Req>& r) {
      r->res.status = err;
      r->times.status = err;
      r->times.t_done_ns = now_ns(t0);
      r->finished = true;
    };
    for (auto& r : admitted) mark(r);
    for (auto& r : queue) mark(r);
    admitted.clear();
    queue.clear();
    for (auto& t : ticks) { t.in_flight = false; t.finishing.clear(); }
    cv_done.notify_all();
  }
};

}  // namespace kde

struct kde_server {
  kde::ServerImpl impl;
};

using namespace kde;

extern "C" {

kde_status kde_server_create(const kde_server_config* cfg, kde_server** out) {
  if (!cfg || !out) return set_err(KDE_ERR_INVALID, "null pointer");
  if (cfg->max_inflight < 1 || cfg->hbm_budget_bytes < (1u << 20))
    return set_err(KDE_ERR_INVALID, "max_inflight >= 1 and hbm_budget_bytes >= 1 MiB required");
  int prev = 0;
  cudaGetDevice(&prev);
  auto* s = new kde_server();
  s->impl.cfg = *cfg;
  kde_status st = s->impl.init();
  cudaSetDevice(prev);
  if (st != KDE_OK) {
    s->impl.destroy_device();
    delete s;
    return st;
  }
  s->impl.worker = std::thread([s] { s->impl.run(); });
  *out = s;
  return KDE_OK;
}

kde_status kde_server_submit(kde_server* s, const float* x, int64_t n, kde_precision prec, uint64_t* ticket) {
  if (!s || !x || !ticket) return set_err(KDE_ERR_INVALID, "null pointer");
  if (n < 2) return set_err(KDE_ERR_INVALID, "n < 2");
  if (prec != KDE_FP32 && prec != KDE_FP64) return set_err(KDE_ERR_INVALID, "bad precision");
  if (is_device_ptr(x)) return set_err(KDE_ERR_INVALID, "server requests take host memory");
  auto r = std::make_shared<Req>();
  r->n = n;
  r->prec = prec;
  s->impl.plan(*r);
  if (r->footprint() > s->impl.cfg.hbm_budget_bytes) return set_err(KDE_ERR_BUSY, "request exceeds the server's HBM budget");
  r->x.assign(x, x + n);
  std::lock_guard<std::mutex> lk(s->impl.mu);
  if (s->impl.stopping) return set_err(KDE_ERR_BUSY, "server is shutting down");
  if (s->impl.fatal != KDE_OK) return set_err(s->impl.fatal, "server failed");
  r->ticket = s->impl.next_ticket++;
  r->times.n = n;
  r->times.precision = prec;
  r->times.t_submit_ns = now_ns(s->impl.t0);
  s->impl.queue.push_back(r);
  s->impl.by_ticket[r->ticket] = r;
  *ticket = r->ticket;
  s->impl.cv_work.notify_one();
  return KDE_OK;
}

kde_status kde_server_poll(kde_server* s, uint64_t ticket, int32_t timeout_ms, kde_result* out,
                           kde_request_times* times) {
  if (!s || !out) return set_err(KDE_ERR_INVALID, "null pointer");
  std::unique_lock<std::mutex> lk(s->impl.mu);
  auto it = s->impl.by_ticket.find(ticket);
  if (it == s->impl.by_ticket.end()) return set_err(KDE_ERR_INVALID, "unknown ticket");
  auto r = it->second;
  auto pred = [&] { return r->finished; };
  if (timeout_ms < 0) s->impl.cv_done.wait(lk, pred);
  else if (!s->impl.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return set_err(KDE_ERR_TIMEOUT, "request not finished");
  *out = r->res;
  if (times) *times = r->times;
  s->impl.by_ticket.erase(it);
  return KDE_OK;
}

void kde_server_destroy(kde_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->impl.mu);
    s->impl.stopping = true;
  }
  s->impl.cv_work.notify_all();
  if (s->impl.worker.joinable()) s->impl.worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->impl.cfg.device);
  s->impl.destroy_device();
  cudaSetDevice(prev);
  delete s;
}

}  // extern "C"
