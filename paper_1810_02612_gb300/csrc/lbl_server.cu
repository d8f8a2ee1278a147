// Serving loop with continuous batching (lbl_server_*): resident roadmaps,
// admission by device memory, and batches formed from whatever has been
// admitted whenever an execution lane is free, so requests that arrive while
// others run join the next batch and overlap on the device.  Each batch is the
// batched launch pair of lbl_batch (frame transforms, then labels with the
// fused monitors) over per-roadmap work units precomputed at creation.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lbl_internal.cuh"

namespace {

using lbl::BatchItem;
using lbl::BatchTable;
using lbl::FrameItem;
using lbl::FrameTable;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over one device arena (offsets only; host side).
class Arena {
 public:
  void init(size_t size) {
    size_ = size;
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = align_up(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes ? bytes : 1);
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
  size_t size() const { return size_; }
  size_t used() const { return used_; }

 private:
  size_t size_ = 0, used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Resident {
  lbl_roadmap rm = nullptr;
  lbl_monitor mon = nullptr;
  int32_t P = 0;
  bool quad = false;        // label through the roadmap's quadtree form
  int64_t *part = nullptr;  // units + 1 entries
  int64_t units = 0;
};

enum ReqState { kPending = 0, kAdmitted = 1, kRunning = 2, kDone = 3, kFailed = 4 };

struct Request {
  int res = 0;
  lbl_grid world{};
  const uint8_t *h_planes = nullptr;
  lbl_pose pose{};
  uint64_t *h_L = nullptr, *h_next = nullptr;
  uint16_t *h_viol = nullptr;
  int64_t t_arrival = 0, t_done = 0;
  int state = kPending;
  int status = LBL_OK;
  size_t off = 0, bytes = 0;
  uint8_t *d_planes = nullptr;
  uint64_t *d_O = nullptr, *d_pyr = nullptr, *d_L = nullptr, *d_next = nullptr;
  uint16_t *d_viol = nullptr;
};

struct Lane {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  unsigned long long *counter = nullptr;
  std::vector<int64_t> reqs;
  bool busy = false;
};

}  // namespace

struct lbl_server_s {
  int device = 0;
  int num_sms = 1;
  int ctas = 1;
  int depth = 8;  // groups in flight per warp of the label launch (12 when every resident is quadtree)
  int max_batch = lbl::kMaxBatch;
  std::vector<Resident> res;
  uint8_t *arena_base = nullptr;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> pending, ready;
  std::unordered_map<int64_t, Request> reqs;
  std::vector<Lane> lanes;
  int64_t next_id = 1;
  bool stop = false;
  int fatal = LBL_OK;
  std::thread th;
  // statistics
  int64_t n_batches = 0, n_done = 0, max_batch_seen = 0;
};

namespace {

size_t request_bytes(const lbl_server_s &S, const Request &r) {
  const Resident &R = S.res[r.res];
  const lbl::Roadmap &rm = *R.rm;
  size_t b = align_up(static_cast<size_t>(R.P) * lbl::grid_cells(r.world));
  b += align_up(static_cast<size_t>(rm.cells) * 8);
  if (R.quad) b += align_up(static_cast<size_t>(rm.pyr_words) * 8);
  b += align_up(static_cast<size_t>(rm.E) * 8);
  if (R.mon) b += align_up(static_cast<size_t>(rm.E) * 8) + align_up(static_cast<size_t>(rm.E) * 2);
  return b;
}

void carve(lbl_server_s &S, Request &r) {
  const Resident &R = S.res[r.res];
  const lbl::Roadmap &rm = *R.rm;
  uint8_t *p = S.arena_base + r.off;
  r.d_planes = p;
  p += align_up(static_cast<size_t>(R.P) * lbl::grid_cells(r.world));
  r.d_O = reinterpret_cast<uint64_t *>(p);
  p += align_up(static_cast<size_t>(rm.cells) * 8);
  if (R.quad) {
    r.d_pyr = reinterpret_cast<uint64_t *>(p);
    p += align_up(static_cast<size_t>(rm.pyr_words) * 8);
  }
  r.d_L = reinterpret_cast<uint64_t *>(p);
  p += align_up(static_cast<size_t>(rm.E) * 8);
  if (R.mon) {
    r.d_next = reinterpret_cast<uint64_t *>(p);
    p += align_up(static_cast<size_t>(rm.E) * 8);
    r.d_viol = reinterpret_cast<uint16_t *>(p);
  }
}

// Enqueue one batch on a lane (called without the lock held; the lane and its
// requests belong to the scheduler thread until completion).
cudaError_t launch_group(lbl_server_s &S, Lane &lane, std::vector<Request *> &group) {
  BatchTable tab{};
  FrameTable ftab{};
  lbl::PyrTable ptab{};
  int64_t unit0 = 0, cell0 = 0, block0 = 0;
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < group.size() && e == cudaSuccess; ++i) {
    Request &r = *group[i];
    const Resident &R = S.res[r.res];
    const lbl::Roadmap &rm = *R.rm;
    const size_t plane_bytes = static_cast<size_t>(R.P) * lbl::grid_cells(r.world);
    if (plane_bytes) e = cudaMemcpyAsync(r.d_planes, r.h_planes, plane_bytes, cudaMemcpyHostToDevice, lane.s);
    lbl::FrameMap m{};
    lbl::frame_map(r.world, rm.agent, r.pose, &m);  // checked at submit
    ftab.items[i] = lbl::frame_item(m, r.world, rm.agent, r.d_planes, R.P, r.d_O, cell0);
    cell0 += rm.cells;
    BatchItem &it = tab.items[i];
    it = BatchItem{};
    it.rowptr = R.quad ? rm.qd_rowptr : rm.rowptr;
    it.colidx = R.quad ? rm.qd_idx : rm.colidx;
    it.perm = R.quad ? rm.qd_perm : nullptr;
    it.part = R.part;
    it.O = r.d_O;
    if (R.quad) {  // gather from the request's pyramid, built after its transform
      lbl::PyrItem &pi = ptab.items[ptab.n++];
      pi = lbl::PyrItem{};
      pi.O = r.d_O;
      pi.pyr = r.d_pyr;
      pi.cells = rm.cells;
      pi.block0 = block0;
      pi.off = rm.qd_off;
      pi.tiled_w = rm.qd_tiled_w;
      block0 += (rm.cells + lbl::kThreads - 1) / lbl::kThreads;
      it.O = r.d_pyr;
    }
    it.L = r.d_L;
    it.next = r.d_next;
    it.viol = r.d_viol;
    it.mask = R.P >= 64 ? ~0ull : ((1ull << R.P) - 1ull);
    it.warp0 = unit0;
    it.warps = rm.E > 0 ? R.units : 0;
    if (R.mon) {
      it.T = R.mon->T;
      it.V = R.mon->V;
      it.m = R.mon->m;
      for (int j = 0; j < 8; ++j) it.rel[j] = R.mon->rel[j];
    }
    unit0 += it.warps;
  }
  tab.n = ftab.n = static_cast<int32_t>(group.size());
  tab.depth = S.depth;
  tab.total = unit0;
  ftab.total = cell0;
  ptab.total = block0;
  for (size_t i = 0; i < group.size(); ++i) {
    const Resident &R = S.res[group[i]->res];
    const int64_t ent = R.quad ? R.rm->n_qd : R.rm->nnz;
    if (ent >= lbl::kNarrowLimit || R.rm->E >= lbl::kNarrowLimit) tab.wide = 1;
  }
  if (e == cudaSuccess) e = lbl::launch_frame_batch(ftab, S.num_sms, lane.s);
  if (e == cudaSuccess) e = lbl::launch_quad_pyramid_batch(ptab, lane.s);
  if (e == cudaSuccess) e = lbl::launch_label_batch(tab, lane.counter, S.num_sms, S.ctas, lane.s);
  for (size_t i = 0; i < group.size() && e == cudaSuccess; ++i) {
    Request &r = *group[i];
    const Resident &R = S.res[r.res];
    const int64_t E = R.rm->E;
    if (E == 0) continue;
    e = cudaMemcpyAsync(r.h_L, r.d_L, E * 8, cudaMemcpyDeviceToHost, lane.s);
    if (e == cudaSuccess && R.mon && r.h_next)
      e = cudaMemcpyAsync(r.h_next, r.d_next, E * 8, cudaMemcpyDeviceToHost, lane.s);
    if (e == cudaSuccess && R.mon && r.h_viol)
      e = cudaMemcpyAsync(r.h_viol, r.d_viol, E * 2, cudaMemcpyDeviceToHost, lane.s);
  }
  if (e == cudaSuccess) e = cudaEventRecord(lane.done, lane.s);
  return e;
}

void scheduler(lbl_server_s *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    bool progress = false;
    // completions
    for (Lane &lane : S->lanes) {
      if (!lane.busy) continue;
      const cudaError_t q = cudaEventQuery(lane.done);
      if (q == cudaErrorNotReady) continue;
      const int64_t t = now_ns();
      for (int64_t id : lane.reqs) {
        Request &r = S->reqs[id];
        r.t_done = t;
        r.state = q == cudaSuccess ? kDone : kFailed;
        r.status = q == cudaSuccess ? LBL_OK : LBL_ECUDA;
        S->arena.release(r.off, r.bytes);
        ++S->n_done;
      }
      if (q != cudaSuccess) S->fatal = LBL_ECUDA;
      lane.reqs.clear();
      lane.busy = false;
      progress = true;
      S->cv_done.notify_all();
    }
    // admission by memory, first come first served
    while (!S->pending.empty()) {
      Request &r = S->reqs[S->pending.front()];
      size_t off = 0;
      if (!S->arena.alloc(r.bytes, &off)) break;
      r.off = off;
      carve(*S, r);
      r.state = kAdmitted;
      S->ready.push_back(S->pending.front());
      S->pending.pop_front();
      progress = true;
    }
    // continuous batching: a free lane takes everything admitted so far
    for (Lane &lane : S->lanes) {
      if (lane.busy || S->ready.empty()) continue;
      std::vector<Request *> group;
      while (!S->ready.empty() && static_cast<int>(group.size()) < S->max_batch) {
        const int64_t id = S->ready.front();
        S->ready.pop_front();
        Request &r = S->reqs[id];
        r.state = kRunning;
        lane.reqs.push_back(id);
        group.push_back(&r);
      }
      lane.busy = true;
      ++S->n_batches;
      S->max_batch_seen = std::max<int64_t>(S->max_batch_seen, static_cast<int64_t>(group.size()));
      lk.unlock();
      const cudaError_t e = launch_group(*S, lane, group);
      lk.lock();
      if (e != cudaSuccess) {
        S->fatal = LBL_ECUDA;
        for (int64_t id : lane.reqs) {
          Request &r = S->reqs[id];
          r.state = kFailed;
          r.status = LBL_ECUDA;
          r.t_done = now_ns();
          S->arena.release(r.off, r.bytes);
        }
        lane.reqs.clear();
        lane.busy = false;
        S->cv_done.notify_all();
      }
      progress = true;
    }
    if (!progress) {
      bool any_busy = false;
      for (const Lane &lane : S->lanes) any_busy |= lane.busy;
      // short naps while work is on the device, longer ones when idle
      S->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 10 : 200));
    }
  }
}

}  // namespace

extern "C" {

int lbl_server_create(int32_t n, const lbl_roadmap *rms, const int32_t *n_props, const lbl_monitor *mons,
                      int32_t lanes, int32_t max_batch, int64_t mem_budget, lbl_server *out) {
  lbl::set_error("%s", "");
  if (!out) {
    lbl::set_error("server create: out is NULL");
    return LBL_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || !rms || !n_props || lanes < 1 || lanes > 16 || max_batch < 1 || max_batch > lbl::kMaxBatch ||
      mem_budget < 1) {
    lbl::set_error("server create: need n >= 1 roadmaps, 1 <= lanes <= 16, 1 <= max_batch <= %d and a positive "
                   "memory budget", lbl::kMaxBatch);
    return LBL_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lbl::cuda_fail(e, "server create: cudaGetDevice");
  for (int i = 0; i < n; ++i)
    if (!rms[i] || rms[i]->device != dev || n_props[i] < 0 || n_props[i] > 64 ||
        (mons && mons[i] && mons[i]->device != dev)) {
      lbl::set_error("server create: roadmap %d missing, on another device, or n_props outside 0..64", i);
      return LBL_EINVAL;
    }
  lbl_server_s *S = new (std::nothrow) lbl_server_s();
  if (!S) {
    lbl::set_error("server create: out of host memory");
    return LBL_ENOMEM;
  }
  S->device = dev;
  S->num_sms = rms[0]->num_sms;
  S->ctas = lbl::batch_ctas_per_sm(8);
  S->max_batch = max_batch;
  S->res.resize(n);
  // fixed work-unit size: 32k nonzero-equivalents (a unit takes a warp ~10 us)
  constexpr double kUnitCost = 32768.0;
  auto cleanup = [&](int code) {
    cudaStreamSynchronize(nullptr);  // the partitions were made there
    for (Resident &R : S->res) lbl::obj_free_now(R.part);
    for (Lane &l : S->lanes) {
      if (l.s) cudaStreamDestroy(l.s);
      if (l.done) cudaEventDestroy(l.done);
      lbl::obj_free_now(l.counter);
    }
    lbl::obj_free_now(S->arena_base);
    delete S;
    return code;
  };
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    Resident &R = S->res[i];
    R.rm = rms[i];
    R.mon = mons ? mons[i] : nullptr;
    R.P = n_props[i];
    const lbl::Roadmap &rm = *R.rm;
    R.quad = rm.has_qd && rm.E > 0;
    const double cost = static_cast<double>((R.quad ? rm.n_qd : rm.nnz) + lbl::kEdgeCost * rm.E);
    R.units = rm.E > 0 ? std::min<int64_t>(rm.E, std::max<int64_t>(1, static_cast<int64_t>(std::ceil(cost / kUnitCost))))
                       : 0;
    e = lbl::obj_alloc(&R.part, static_cast<size_t>(R.units + 1), nullptr);
    if (e == cudaSuccess)
      e = lbl::launch_partition_into(R.quad ? rm.qd_rowptr : rm.rowptr, rm.E, R.units, R.part, nullptr);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  bool all_quad = true;
  for (const Resident &R : S->res) all_quad = all_quad && (R.quad || R.rm->E == 0);
  S->depth = all_quad ? lbl::kQuadDepth : 8;
  S->ctas = lbl::batch_ctas_per_sm(S->depth);
  if (e == cudaSuccess) e = lbl::obj_alloc(&S->arena_base, static_cast<size_t>(mem_budget), nullptr);
  if (e != cudaSuccess) return cleanup(lbl::cuda_fail(e, "server create: resident state"));
  S->arena.init(static_cast<size_t>(mem_budget));
  S->lanes.resize(lanes);
  for (Lane &l : S->lanes) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = lbl::obj_alloc(&l.counter, 1, nullptr);
  }
  if (e != cudaSuccess) return cleanup(lbl::cuda_fail(e, "server create: lanes"));
  try {
    S->th = std::thread(scheduler, S);
  } catch (...) {
    lbl::set_error("server create: cannot start the scheduler thread");
    return cleanup(LBL_ENOMEM);
  }
  *out = S;
  return LBL_OK;
}

int lbl_server_submit(lbl_server S, int32_t roadmap, const lbl_grid *world, const uint8_t *h_planes, lbl_pose pose,
                      uint64_t *h_L, uint64_t *h_next, uint16_t *h_viol, int64_t arrival_ns, int64_t *ticket) {
  lbl::set_error("%s", "");
  if (!S || !ticket || roadmap < 0 || roadmap >= static_cast<int32_t>(S->res.size()) || !world) {
    lbl::set_error("server submit: bad server, ticket, roadmap index or world grid");
    return LBL_EINVAL;
  }
  const Resident &R = S->res[roadmap];
  if (world->w < 1 || world->h < 1 || world->w > 32768 || world->h > 32768 || world->d > 32768 ||
      !(world->res > 0) || (world->d > 1 && !(world->tres > 0)) || (R.P > 0 && !h_planes) || (R.rm->E > 0 && !h_L)) {
    lbl::set_error("server submit: bad world grid or missing host buffer");
    return LBL_EINVAL;
  }
  lbl::FrameMap m;
  if (!lbl::frame_map(*world, R.rm->agent, pose, &m)) return LBL_EINVAL;
  Request r;
  r.res = roadmap;
  r.world = *world;
  r.h_planes = h_planes;
  r.pose = pose;
  r.h_L = h_L;
  r.h_next = h_next;
  r.h_viol = h_viol;
  r.t_arrival = arrival_ns > 0 ? arrival_ns : now_ns();
  r.bytes = request_bytes(*S, r);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->fatal != LBL_OK) {
    lbl::set_error("server submit: the server stopped after a CUDA error");
    return S->fatal;
  }
  if (align_up(r.bytes) > S->arena.size()) {
    lbl::set_error("server submit: request needs %zu bytes, more than the server's memory budget %zu", r.bytes,
                   S->arena.size());
    return LBL_ENOMEM;
  }
  const int64_t id = S->next_id++;
  S->reqs.emplace(id, r);
  S->pending.push_back(id);
  *ticket = id;
  S->cv_work.notify_one();
  return LBL_OK;
}

int lbl_server_wait(lbl_server S, int64_t ticket, int64_t timeout_ms, int64_t *latency_ns) {
  lbl::set_error("%s", "");
  if (!S) {
    lbl::set_error("server wait: NULL server");
    return LBL_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    lbl::set_error("server wait: unknown ticket %lld", static_cast<long long>(ticket));
    return LBL_EINVAL;
  }
  const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] {
    const int st = S->reqs[ticket].state;
    return st == kDone || st == kFailed;
  });
  if (!ok) {
    lbl::set_error("server wait: ticket %lld not complete after %lld ms", static_cast<long long>(ticket),
                   static_cast<long long>(timeout_ms));
    return LBL_ETIMEOUT;
  }
  Request r = S->reqs[ticket];
  S->reqs.erase(ticket);
  if (latency_ns) *latency_ns = r.t_done - r.t_arrival;
  if (r.status != LBL_OK) lbl::set_error("server wait: the batch of ticket %lld failed", static_cast<long long>(ticket));
  return r.status;
}

int lbl_server_stats(lbl_server S, int64_t *batches, int64_t *completed, int64_t *max_batch, int64_t *arena_used) {
  lbl::set_error("%s", "");
  if (!S) {
    lbl::set_error("server stats: NULL server");
    return LBL_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (batches) *batches = S->n_batches;
  if (completed) *completed = S->n_done;
  if (max_batch) *max_batch = S->max_batch_seen;
  if (arena_used) *arena_used = static_cast<int64_t>(S->arena.used());
  return LBL_OK;
}

int lbl_server_free(lbl_server S) {
  lbl::set_error("%s", "");
  if (!S) return LBL_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  // the server's work is all on its own lanes: wait for those alone, then free
  // its memory in stream order (no device-wide synchronisation)
  for (Lane &l : S->lanes) cudaStreamSynchronize(l.s);
  for (Resident &R : S->res) lbl::obj_free_now(R.part);
  for (Lane &l : S->lanes) {
    cudaStreamDestroy(l.s);
    cudaEventDestroy(l.done);
    lbl::obj_free_now(l.counter);
  }
  lbl::obj_free_now(S->arena_base);
  delete S;
  return LBL_OK;
}

}  // extern "C"
