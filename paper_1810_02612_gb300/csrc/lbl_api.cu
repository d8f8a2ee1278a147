// C ABI of liblbl (declared in include/lbl.h): argument checks, roadmap and
// monitor handles with their device memory, frame transforms and labeling
// dispatch.  Batches live in lbl_batch.cu, sessions in lbl_session.cu, the
// server in lbl_server.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "lbl_internal.cuh"

namespace lbl {

namespace {
thread_local std::string g_err;
constexpr int kDefaultPipeline = LBL_PIPE_REGISTERS;  // measured fastest on GB300

int resolve_lpe(const Roadmap &rm, const lbl_config *cfg) {
  int lpe = cfg ? cfg->lanes_per_edge : 0;
  if (lpe == 4 || lpe == 8 || lpe == 16 || lpe == 32) return lpe;
  const double avg = rm.E ? static_cast<double>(rm.nnz) / static_cast<double>(rm.E) : 0.0;
  lpe = 4;
  while (lpe < 32 && lpe * 16 < avg) lpe *= 2;
  return lpe;
}

}  // namespace

int device_sms(int dev) {
  static int cache[64] = {0};
  if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  if (dev >= 0 && dev < 64) cache[dev] = n;
  return n;
}

bool valid_grid(const lbl_grid *g, const char *name, bool need_order) {
  if (!g) {
    set_error("%s: grid pointer is NULL", name);
    return false;
  }
  const int64_t d = grid_depth(*g);
  if (g->w < 1 || g->h < 1 || g->w > 32768 || g->h > 32768 || d > 32768 ||
      static_cast<int64_t>(g->w) * g->h * d > 2147483647LL) {
    set_error("%s: grid size %d x %d x %lld outside 1..32768 per side / 2^31-1 cells", name, g->w, g->h,
              static_cast<long long>(d));
    return false;
  }
  if (!(g->res > 0.0) || !std::isfinite(g->res) || !std::isfinite(g->x0) || !std::isfinite(g->y0)) {
    set_error("%s: resolution must be positive and the corner finite", name);
    return false;
  }
  if (d > 1 && (!(g->tres > 0.0) || !std::isfinite(g->tres) || !std::isfinite(g->t0))) {
    set_error("%s: a time-augmented grid needs a positive slab length and a finite start", name);
    return false;
  }
  if (need_order) {
    if (g->order != LBL_ORDER_ROWMAJOR && g->order != LBL_ORDER_MORTON) {
      set_error("%s: unknown cell order %d", name, g->order);
      return false;
    }
    if (g->order == LBL_ORDER_MORTON && (g->w != g->h || (d > 1 && d != g->w) || (g->w & (g->w - 1)) != 0)) {
      set_error("%s: z-order needs a cube (or square) power-of-two grid (got %d x %d x %lld)", name, g->w, g->h,
                static_cast<long long>(d));
      return false;
    }
  }
  return true;
}

bool same_device(int dev) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    set_error("cudaGetDevice failed");
    return false;
  }
  if (cur != dev) {
    set_error("handle belongs to device %d but device %d is current", dev, cur);
    return false;
  }
  return true;
}

// One stream per device on which objects' memory is released (created on first
// use, kept for the life of the process).
cudaStream_t release_stream(int device) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (device < 0 || device >= 64) return nullptr;
  if (!streams[device] && cudaStreamCreateWithFlags(&streams[device], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    streams[device] = nullptr;
  }
  return streams[device];
}

void UseLog::note(cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return;  // e.g. the legacy stream while another stream captures
  }
  if (cap != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lock(mu);
  cudaEvent_t e = nullptr;
  for (auto &u : ev)
    if (u.first == s) e = u.second;
  if (!e) {
    if (ev.size() >= 16) {  // many streams: wait for the oldest uses here rather than keep every event
      for (auto &u : ev) {
        cudaEventSynchronize(u.second);
        cudaEventDestroy(u.second);
      }
      ev.clear();
    }
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      cudaStreamSynchronize(s);  // no event: make the use complete now instead
      return;
    }
    ev.emplace_back(s, e);
  }
  cudaEventRecord(e, s);
}

void UseLog::release(int device, const std::vector<void *> &ptrs) {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != device) cudaSetDevice(device);
  cudaStream_t rs = release_stream(device);
  {
    std::lock_guard<std::mutex> lock(mu);
    for (auto &u : ev) {
      if (!rs || cudaStreamWaitEvent(rs, u.second, 0) != cudaSuccess) cudaEventSynchronize(u.second);
      cudaEventDestroy(u.second);
    }
    ev.clear();
  }
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, rs);  // rs NULL: the legacy stream, after the host waits above
  cudaGetLastError();
  if (cur >= 0 && cur != device) cudaSetDevice(cur);
}

void free_roadmap(Roadmap *rm) {
  if (!rm) return;
  rm->uses->release(rm->device, {rm->rowptr, rm->colidx, rm->bt_rowptr, rm->bt_block, rm->bt_mask, rm->planes,
                                 rm->part, rm->err, rm->sec_rowptr, rm->sec, rm->sec_part, rm->qd_rowptr,
                                 rm->qd_perm, rm->qd_idx, rm->qd_part, rm->pyr, rm->mma_perm, rm->mma_tptr,
                                 rm->mma_tblk, rm->mma_bits, rm->mma_b});
  delete rm;
}


// perm[a..b) = a..b-1 ordered by key (stable): LSD radix sort, two 16-bit digits.
void sort_range_by_key(const uint32_t *key, int64_t a, int64_t b, int32_t *perm) {
  const int64_t n = b - a;
  if (n <= 0) return;
  std::vector<int32_t> tmp(static_cast<size_t>(n));
  int32_t *src = perm + a, *dst = tmp.data();
  for (int64_t i = 0; i < n; ++i) src[i] = static_cast<int32_t>(a + i);
  std::vector<int64_t> count(65537);
  for (int shift = 0; shift < 32; shift += 16) {
    std::fill(count.begin(), count.end(), 0);
    for (int64_t i = 0; i < n; ++i) ++count[((key[src[i]] >> shift) & 0xFFFFu) + 1];
    for (int d = 0; d < 65536; ++d) count[d + 1] += count[d];
    for (int64_t i = 0; i < n; ++i) dst[count[(key[src[i]] >> shift) & 0xFFFFu]++] = src[i];
    std::swap(src, dst);
  }
  // two passes: the sorted order is back in perm + a
}

// Q32.32 coefficients of (ix, iy) -> continuous world-cell coordinates:
//   u = a00*ix + a01*iy + b0,  v = a10*ix + a11*iy + b1,
// from world point q = (X, Y) + R(theta) * centre(ix, iy) (Sec. 5, eq. 13).
// The double expressions are evaluated exactly as written (the library is built
// without floating-point contraction) and each is rounded half to even.
bool frame_map(const lbl_grid &W, const lbl_grid &A, const lbl_pose &p, FrameMap *out) {
  if (!std::isfinite(p.x) || !std::isfinite(p.y) || !std::isfinite(p.theta) || !std::isfinite(p.t)) {
    set_error("frame transform: pose must be finite");
    return false;
  }
  if (grid_depth(W) > 1 && grid_depth(A) <= 1) {
    set_error("frame transform: a time-augmented world needs a time-augmented agent grid");
    return false;
  }
  const double c = std::cos(p.theta);
  const double s = std::sin(p.theta);
  const double k = A.res / W.res;
  const double a00 = c * k;
  const double a01 = -(s * k);
  const double a10 = s * k;
  const double a11 = c * k;
  const double xa = A.x0 + 0.5 * A.res;
  const double ya = A.y0 + 0.5 * A.res;
  const double b0 = ((p.x + ((c * xa) - (s * ya))) - W.x0) / W.res;
  const double b1 = ((p.y + ((s * xa) + (c * ya))) - W.y0) / W.res;
  // |a| <= 2^14 and |b| <= 2^28 keep a*ix + a*iy + b (ix, iy < 2^15) inside int64
  const double lim_a = 16384.0, lim_b = 268435456.0;
  if (!(std::fabs(a00) <= lim_a && std::fabs(a01) <= lim_a && std::fabs(b0) <= lim_b && std::fabs(b1) <= lim_b)) {
    set_error("frame transform: pose or resolution ratio out of the fixed-point range");
    return false;
  }
  auto q = [](double v) { return static_cast<int64_t>(std::nearbyint(v * 4294967296.0)); };
  out->A00 = q(a00);
  out->A01 = q(a01);
  out->B0 = q(b0);
  out->A10 = q(a10);
  out->A11 = q(a11);
  out->B1 = q(b1);
  out->At = out->Bt = 0;
  if (grid_depth(W) > 1) {
    // slab it of the agent (centre t0 + (it + 1/2) tres after the query time)
    // -> continuous world slab coordinate, the time shift of eq. 13
    const double at = A.tres / W.tres;
    const double ta = A.t0 + 0.5 * A.tres;
    const double bt = ((p.t + ta) - W.t0) / W.tres;
    if (!(std::fabs(at) <= lim_a && std::fabs(bt) <= lim_b)) {
      set_error("frame transform: query time or slab ratio out of the fixed-point range");
      return false;
    }
    out->At = q(at);
    out->Bt = q(bt);
  }
  return true;
}

FrameItem frame_item(const FrameMap &m, const lbl_grid &W, const lbl_grid &A, const uint8_t *planes, int32_t P,
                     uint64_t *O, int64_t cell0) {
  FrameItem f{m.A00, m.A01, m.B0, m.A10, m.A11, m.B1, m.At, m.Bt, planes, O, grid_cells(W), cell0,
              W.w, W.h, grid_depth(W), A.w, A.h, grid_depth(A), P, A.order};
  return f;
}

void set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

void clear_error() { g_err.clear(); }

int cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LBL_ENOMEM : LBL_ECUDA;
}

}  // namespace lbl

using namespace lbl;


namespace lbl {


// A roadmap with device arrays for its CSR (rowptr int64[E+1], colidx padded
// to whole 16-byte vectors plus one, the padding zeroed); contents to be
// filled by the caller before roadmap_finish.
int roadmap_new(const lbl_grid &agent, int64_t n_edges, int64_t nnz, lbl_roadmap_s **out) {
  lbl_roadmap_s *rm = new (std::nothrow) lbl_roadmap_s();
  if (!rm) {
    set_error("roadmap: out of host memory");
    return LBL_ENOMEM;
  }
  cudaError_t e = cudaGetDevice(&rm->device);
  if (e != cudaSuccess) {
    delete rm;
    return cuda_fail(e, "roadmap: cudaGetDevice");
  }
  rm->num_sms = device_sms(rm->device);
  rm->agent = agent;
  rm->E = n_edges;
  rm->nnz = nnz;
  rm->cells = grid_cells(agent);
  const int64_t padded = ((nnz + 3) / 4) * 4 + 4;
  if ((e = obj_alloc(&rm->rowptr, static_cast<size_t>(n_edges + 1), &rm->bytes)) != cudaSuccess ||
      (e = obj_alloc(&rm->colidx, static_cast<size_t>(padded), &rm->bytes)) != cudaSuccess ||
      (e = cudaMemset(rm->colidx + nnz, 0, sizeof(int32_t) * (padded - nnz))) != cudaSuccess) {
    free_roadmap(rm);
    return cuda_fail(e, "roadmap: CSR arrays");
  }
  *out = rm;
  return LBL_OK;
}

// Check the CSR on the device and derive what the kernels need (edge
// partition, optional block and sector forms); synchronises `st`.  Frees the
// roadmap on failure.
int roadmap_finish(lbl_roadmap_s *rm, uint32_t flags, cudaStream_t st) {
  const int64_t n_edges = rm->E, nnz = rm->nnz;
  unsigned long long *d_bad = nullptr;
  int32_t *d_cnt = nullptr;
  cudaError_t e = cudaSuccess;
  auto fail = [&](int code) {
    cudaStreamSynchronize(st);
    cudaFree(d_bad);
    cudaFree(d_cnt);
    free_roadmap(rm);
    return code;
  };
  // row pointer end points
  int64_t ends[2] = {0, 0};
  if ((e = cudaMemcpyAsync(&ends[0], rm->rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&ends[1], rm->rowptr + n_edges, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(cuda_fail(e, "roadmap: read row pointer"));
  if (ends[0] != 0 || ends[1] != nnz) {
    set_error("roadmap: rowptr[0] = %lld and rowptr[E] = %lld, expected 0 and nnz = %lld",
              static_cast<long long>(ends[0]), static_cast<long long>(ends[1]), static_cast<long long>(nnz));
    return fail(LBL_EINVAL);
  }
  const bool want_bt = flags & LBL_UPLOAD_BITTILE;
  if ((e = obj_alloc(&rm->err, 1, &rm->bytes)) != cudaSuccess ||
      (e = cudaMemsetAsync(rm->err, 0, sizeof(int), st)) != cudaSuccess)
    return fail(cuda_fail(e, "roadmap: error flag"));
  if ((e = dev_alloc(&d_bad, 1, nullptr)) != cudaSuccess) return fail(cuda_fail(e, "roadmap: scratch"));
  if (want_bt && (e = dev_alloc(&d_cnt, static_cast<size_t>(n_edges), nullptr)) != cudaSuccess)
    return fail(cuda_fail(e, "roadmap: block counts"));
  if ((e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st)) != cudaSuccess ||
      (e = launch_scan_rows(rm->rowptr, rm->colidx, n_edges, nnz, rm->cells, d_bad, d_cnt, st)) != cudaSuccess)
    return fail(cuda_fail(e, "roadmap: row check"));
  unsigned long long bad = 0;
  if ((e = cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(cuda_fail(e, "roadmap: row check"));
  if (bad) {
    set_error("roadmap: %llu malformed rows (row pointer decreasing or out of range, or column indices "
              "not strictly increasing inside [0, %lld))",
              bad, static_cast<long long>(rm->cells));
    return fail(LBL_EINVAL);
  }
  if (n_edges > 0) {
    // edge partition of the streaming CSR kernel, for its default grid
    rm->part_cap = static_cast<int64_t>(rm->num_sms) * kMaxCtasPerSm * (kThreads / 32) + 1;
    if ((e = obj_alloc(&rm->part, static_cast<size_t>(rm->part_cap), &rm->bytes)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: partition"));
    rm->part_ctas = stream_ctas_per_sm(8);
    if ((e = launch_partition(*rm, rm->part_ctas, st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: partition"));
  }
  if (want_bt) {
    std::vector<int32_t> cnt(static_cast<size_t>(n_edges));
    std::vector<int64_t> brow(static_cast<size_t>(n_edges + 1));
    if (n_edges &&
        ((e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * n_edges, cudaMemcpyDeviceToHost, st)) !=
             cudaSuccess ||
         (e = cudaStreamSynchronize(st)) != cudaSuccess))
      return fail(cuda_fail(e, "roadmap: block counts"));
    brow[0] = 0;
    for (int64_t i = 0; i < n_edges; ++i) brow[i + 1] = brow[i] + cnt[i];
    rm->n_bt = brow[n_edges];
    rm->n_blocks = (rm->cells + 63) / 64;
    if ((e = obj_alloc(&rm->bt_rowptr, static_cast<size_t>(n_edges + 1), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->bt_block, static_cast<size_t>(rm->n_bt), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->bt_mask, static_cast<size_t>(rm->n_bt), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->planes, static_cast<size_t>(rm->n_blocks * 64), &rm->bytes)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: block form"));
    if ((e = cudaMemcpyAsync(rm->bt_rowptr, brow.data(), sizeof(int64_t) * (n_edges + 1), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = launch_bt_fill(rm->rowptr, rm->colidx, n_edges, rm->bt_rowptr, rm->bt_block, rm->bt_mask, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: block form"));
    rm->has_bt = true;
  }
  if ((flags & LBL_UPLOAD_SECTOR) && n_edges > 0) {
    if (rm->cells > (1LL << 30)) {
      set_error("roadmap: the sector form needs at most 2^30 cells");
      return fail(LBL_EINVAL);
    }
    std::vector<int32_t> cnt(static_cast<size_t>(n_edges));
    std::vector<int64_t> srow(static_cast<size_t>(n_edges + 1));
    int32_t *d_sc = nullptr;
    if ((e = dev_alloc(&d_sc, static_cast<size_t>(n_edges), nullptr)) != cudaSuccess ||
        (e = launch_sector_count(rm->rowptr, rm->colidx, n_edges, d_sc, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(cnt.data(), d_sc, sizeof(int32_t) * n_edges, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      cudaFree(d_sc);
      return fail(cuda_fail(e, "roadmap: sector form"));
    }
    cudaFree(d_sc);
    srow[0] = 0;
    for (int64_t i = 0; i < n_edges; ++i) srow[i + 1] = srow[i] + cnt[i];
    rm->n_sec = srow[n_edges];
    if ((e = obj_alloc(&rm->sec_rowptr, static_cast<size_t>(n_edges + 1), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->sec, static_cast<size_t>(rm->n_sec), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->sec_part, static_cast<size_t>(rm->part_cap), &rm->bytes)) != cudaSuccess ||
        (e = cudaMemcpyAsync(rm->sec_rowptr, srow.data(), sizeof(int64_t) * (n_edges + 1), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = launch_sector_fill(rm->rowptr, rm->colidx, n_edges, rm->sec_rowptr, rm->sec, st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: sector form"));
    rm->sec_part_ctas = sector_ctas_per_sm(4);
    const int64_t W = static_cast<int64_t>(rm->num_sms) * rm->sec_part_ctas * (kThreads / 32);
    if ((e = launch_partition_into(rm->sec_rowptr, n_edges, W, rm->sec_part, st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: sector partition"));
    rm->has_sec = true;
  }
  if ((flags & LBL_UPLOAD_QUAD) && n_edges > 0) {
    if (rm->cells >= (1LL << 30)) {
      set_error("roadmap: the quadtree form needs fewer than 2^30 cells");
      return fail(LBL_EINVAL);
    }
    // pyramid layout: level k has floor(cells / 4^k) words
    int64_t words = 0;
    for (int k = 0; k <= kQuadLevels; ++k) {
      rm->qd_off.at[k] = words;
      words += rm->cells >> (2 * k);
    }
    rm->pyr_words = words;
    // row-major 2-D grids whose sides are multiples of 16 take the tiled order
    // (square blocks); other row-major grids keep runs of a grid row
    if (rm->agent.order == LBL_ORDER_ROWMAJOR && grid_depth(rm->agent) == 1 && rm->agent.w % 16 == 0 &&
        rm->agent.h % 16 == 0)
      rm->qd_tiled_w = rm->agent.w;
    if (n_edges > 1 && n_edges < (1LL << 31) && !(flags & LBL_UPLOAD_KEEP_ORDER) && grid_depth(rm->agent) == 1) {
      // locality order: inside each of kOrderRanges edge ranges, rows by the z-order of
      // their middle cell's (x, y); time-augmented grids keep the caller's
      // order, which measured faster than every key tried there
      std::vector<uint32_t> key(static_cast<size_t>(n_edges));
      uint32_t *d_key = nullptr;
      if ((e = dev_alloc(&d_key, static_cast<size_t>(n_edges), nullptr)) != cudaSuccess ||
          (e = launch_row_keys(rm->rowptr, rm->colidx, n_edges, rm->agent.order, rm->agent.w, d_key, st)) !=
              cudaSuccess ||
          (e = cudaMemcpyAsync(key.data(), d_key, sizeof(uint32_t) * n_edges, cudaMemcpyDeviceToHost, st)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        cudaFree(d_key);
        return fail(cuda_fail(e, "roadmap: quadtree order"));
      }
      cudaFree(d_key);
      std::vector<int32_t> perm(static_cast<size_t>(n_edges));
      for (int c = 0; c < kOrderRanges; ++c)
        sort_range_by_key(key.data(), n_edges * c / kOrderRanges, n_edges * (c + 1) / kOrderRanges, perm.data());
      if ((e = obj_alloc(&rm->qd_perm, static_cast<size_t>(n_edges), &rm->bytes)) != cudaSuccess ||
          (e = cudaMemcpyAsync(rm->qd_perm, perm.data(), sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, st)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(cuda_fail(e, "roadmap: quadtree order"));
    }
    std::vector<int32_t> cnt(static_cast<size_t>(n_edges));
    std::vector<int64_t> drow(static_cast<size_t>(n_edges + 1));
    int32_t *d_dc = nullptr;
    if ((e = dev_alloc(&d_dc, static_cast<size_t>(n_edges), nullptr)) != cudaSuccess ||
        (e = launch_quad_count(rm->rowptr, rm->colidx, n_edges, rm->qd_perm, rm->qd_tiled_w, d_dc, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(cnt.data(), d_dc, sizeof(int32_t) * n_edges, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      cudaFree(d_dc);
      return fail(cuda_fail(e, "roadmap: quadtree form"));
    }
    cudaFree(d_dc);
    drow[0] = 0;
    for (int64_t i = 0; i < n_edges; ++i) drow[i + 1] = drow[i] + cnt[i];
    rm->n_qd = drow[n_edges];
    if ((e = obj_alloc(&rm->qd_rowptr, static_cast<size_t>(n_edges + 1), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->qd_idx, static_cast<size_t>(rm->n_qd + 4), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->qd_part, static_cast<size_t>(rm->part_cap), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->pyr, static_cast<size_t>(words), &rm->bytes)) != cudaSuccess ||
        (e = cudaMemcpyAsync(rm->qd_rowptr, drow.data(), sizeof(int64_t) * (n_edges + 1), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = launch_quad_fill(rm->rowptr, rm->colidx, n_edges, rm->qd_perm, rm->qd_tiled_w, rm->qd_off, rm->qd_rowptr,
                              rm->qd_idx,
                              st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: quadtree form"));
    rm->qd_part_ctas = stream_ctas_per_sm(kQuadDepth);
    const int64_t W = static_cast<int64_t>(rm->num_sms) * rm->qd_part_ctas * (kThreads / 32);
    if ((e = launch_partition_into(rm->qd_rowptr, n_edges, W, rm->qd_part, st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: quadtree partition"));
    rm->has_qd = true;
  }
  if ((flags & LBL_UPLOAD_MMA) && n_edges > 0) {
    if (rm->cells > (int64_t{1} << 22) || n_edges >= (int64_t{1} << 31)) {
      set_error("roadmap: the tensor-core form needs at most 2^22 cells and fewer than 2^31 edges");
      return fail(LBL_EINVAL);
    }
    rm->mma_nkb = static_cast<int32_t>((rm->cells + 127) / 128);
    rm->mma_T = (n_edges + 127) / 128;
    // tiles of 128 edges in locality order: the whole roadmap sorted by the
    // z-order of each row's middle cell
    std::vector<uint32_t> key(static_cast<size_t>(n_edges));
    std::vector<int32_t> perm(static_cast<size_t>(n_edges));
    uint32_t *d_key = nullptr;
    if ((e = dev_alloc(&d_key, static_cast<size_t>(n_edges), nullptr)) != cudaSuccess ||
        (e = launch_row_keys(rm->rowptr, rm->colidx, n_edges, rm->agent.order, rm->agent.w, d_key, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(key.data(), d_key, sizeof(uint32_t) * n_edges, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      cudaFree(d_key);
      return fail(cuda_fail(e, "roadmap: tensor-core form order"));
    }
    cudaFree(d_key);
    sort_range_by_key(key.data(), 0, n_edges, perm.data());
    std::vector<int64_t> cnt(static_cast<size_t>(rm->mma_T)), tptr(static_cast<size_t>(rm->mma_T + 1));
    int64_t *d_cnt64 = nullptr;
    if ((e = obj_alloc(&rm->mma_perm, static_cast<size_t>(n_edges), &rm->bytes)) != cudaSuccess ||
        (e = cudaMemcpyAsync(rm->mma_perm, perm.data(), sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = dev_alloc(&d_cnt64, static_cast<size_t>(rm->mma_T), nullptr)) != cudaSuccess ||
        (e = launch_mma_count(rm->rowptr, rm->colidx, rm->mma_perm, n_edges, rm->mma_nkb, d_cnt64, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(cnt.data(), d_cnt64, sizeof(int64_t) * rm->mma_T, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      cudaFree(d_cnt64);
      return fail(cuda_fail(e, "roadmap: tensor-core form"));
    }
    cudaFree(d_cnt64);
    tptr[0] = 0;
    for (int64_t t = 0; t < rm->mma_T; ++t) tptr[t + 1] = tptr[t] + cnt[t];
    rm->n_mma = tptr[rm->mma_T];
    if ((e = obj_alloc(&rm->mma_tptr, static_cast<size_t>(rm->mma_T + 1), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->mma_tblk, static_cast<size_t>(rm->n_mma), &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->mma_bits, static_cast<size_t>(rm->n_mma) * 128 * 4, &rm->bytes)) != cudaSuccess ||
        (e = obj_alloc(&rm->mma_b, static_cast<size_t>(rm->mma_nkb) * 64 * 128, &rm->bytes)) != cudaSuccess ||
        (e = cudaMemcpyAsync(rm->mma_tptr, tptr.data(), sizeof(int64_t) * (rm->mma_T + 1), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemsetAsync(rm->mma_bits, 0, sizeof(uint32_t) * 128 * 4 * static_cast<size_t>(rm->n_mma), st)) !=
            cudaSuccess ||
        (e = launch_mma_fill(rm->rowptr, rm->colidx, rm->mma_perm, n_edges, rm->mma_nkb, rm->mma_tptr, rm->mma_tblk,
                             rm->mma_bits, st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: tensor-core form"));
    rm->has_mma = true;
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(cuda_fail(e, "roadmap"));
  cudaFree(d_bad);
  cudaFree(d_cnt);
  return LBL_OK;
}

}  // namespace lbl

namespace lbl {

int transform_pyramid(const lbl_grid *world, const void *d_words, int32_t n_props, lbl_pose pose, const Roadmap &rm,
                      uint64_t *d_O, void *pyr, cudaStream_t st) {
  const lbl_grid *agent = &rm.agent;
  if (!valid_grid(world, "frame transform (world)", false)) return LBL_EINVAL;
  if (n_props < 0 || n_props > 64) {
    set_error("frame transform (pyramid): n_props = %d outside 0..64", n_props);
    return LBL_EINVAL;
  }
  // z-order grids, and row-major grids in the tiled order, build the pyramid
  // inside the transform and need no O
  const bool one_launch = agent->order == LBL_ORDER_MORTON || rm.qd_tiled_w > 0;
  if (!d_words || (!d_O && !one_launch)) {
    set_error("frame transform (pyramid): NULL buffer (row-major agent grids need O unless their sides are "
              "multiples of 16)");
    return LBL_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_words) % static_cast<uintptr_t>(packed_word_bytes(n_props)) ||
      reinterpret_cast<uintptr_t>(d_O) % 8u) {
    set_error("frame transform (pyramid): words or O not aligned to their width");
    return LBL_EINVAL;
  }
  FrameMap m;
  if (!frame_map(*world, *agent, pose, &m)) return LBL_EINVAL;
  FrameItem f = frame_item(m, *world, *agent, nullptr, n_props, d_O, 0);
  f.words = d_words;
  f.word_bytes = packed_word_bytes(n_props);
  f.wmask = n_props >= 64 ? ~0ull : ((1ull << n_props) - 1ull);
  const int wb = quad_word_bytes(rm, n_props);
  cudaError_t e;
  if (one_launch) {
    e = launch_frame_transform_pyramid(f, rm.qd_off, wb, pyr, rm.qd_tiled_w, st);
  } else {  // other row-major grids: the pyramid's blocks are row runs, not the transform's tiles
    e = launch_frame_transform(f, st);
    if (e == cudaSuccess) e = launch_quad_pyramid(rm, d_O, wb, pyr, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "frame transform (pyramid): launch");
  return LBL_OK;
}

}  // namespace lbl

extern "C" {

const char *lbl_last_error(void) { return g_err.c_str(); }

int lbl_version(void) { return 10100; }

int lbl_roadmap_upload(const lbl_grid *agent, const int64_t *rowptr, const int32_t *colidx, int64_t n_edges,
                       int64_t nnz, uint32_t flags, lbl_stream s, lbl_roadmap *out) {
  g_err.clear();
  if (!out) {
    set_error("roadmap upload: out is NULL");
    return LBL_EINVAL;
  }
  *out = nullptr;
  if (!valid_grid(agent, "roadmap upload", true)) return LBL_EINVAL;
  if (n_edges < 0 || nnz < 0 || nnz > 2147483647LL * 4) {
    set_error("roadmap upload: negative or oversized n_edges/nnz");
    return LBL_EINVAL;
  }
  if (!rowptr || (nnz > 0 && !colidx)) {
    set_error("roadmap upload: rowptr/colidx is NULL");
    return LBL_EINVAL;
  }
  if (flags & ~(LBL_UPLOAD_DEVICE_PTRS | LBL_UPLOAD_BITTILE | LBL_UPLOAD_SECTOR | LBL_UPLOAD_QUAD |
                LBL_UPLOAD_KEEP_ORDER | LBL_UPLOAD_MMA)) {
    set_error("roadmap upload: unknown flags 0x%x", flags);
    return LBL_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  lbl_roadmap_s *rm = nullptr;
  int rc = roadmap_new(*agent, n_edges, nnz, &rm);
  if (rc != LBL_OK) return rc;
  const cudaMemcpyKind kind = (flags & LBL_UPLOAD_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(rm->rowptr, rowptr, sizeof(int64_t) * (n_edges + 1), kind, st);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(rm->colidx, colidx, sizeof(int32_t) * nnz, kind, st);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(st);
    free_roadmap(rm);
    return cuda_fail(e, "roadmap upload: copy");
  }
  rc = roadmap_finish(rm, flags, st);
  if (rc == LBL_OK) *out = rm;
  return rc;
}

int lbl_roadmap_free(lbl_roadmap rm) {
  g_err.clear();
  if (!rm) return LBL_OK;
  free_roadmap(rm);  // released in stream order after the roadmap's last logged use
  return LBL_OK;
}

int lbl_roadmap_set_wait_limit(lbl_roadmap rm, int64_t limit_ns) {
  g_err.clear();
  if (!rm || limit_ns < 0 || limit_ns > 60000000000LL) {
    set_error("roadmap wait limit: NULL roadmap or a limit outside 0..60e9 ns");
    return LBL_EINVAL;
  }
  rm->wait_ns = limit_ns;
  return LBL_OK;
}

int lbl_roadmap_form_info(lbl_roadmap rm, int32_t algo, int64_t *entries, int64_t *tiles) {
  g_err.clear();
  if (!rm) {
    set_error("roadmap form info: NULL roadmap");
    return LBL_EINVAL;
  }
  int64_t n = 0, t = 0;
  switch (algo) {
    case LBL_ALGO_CSR: n = rm->nnz; break;
    case LBL_ALGO_BITTILE: n = rm->has_bt ? rm->n_bt : 0; break;
    case LBL_ALGO_SECTOR: n = rm->has_sec ? rm->n_sec : 0; break;
    case LBL_ALGO_QUAD: n = rm->has_qd ? rm->n_qd : 0; break;
    case LBL_ALGO_MMA:
      n = rm->has_mma ? rm->n_mma : 0;
      t = rm->has_mma ? rm->mma_T : 0;
      break;
    default:
      set_error("roadmap form info: unknown algo %d", algo);
      return LBL_EINVAL;
  }
  if (entries) *entries = n;
  if (tiles) *tiles = t;
  return LBL_OK;
}

int lbl_roadmap_info(lbl_roadmap rm, int64_t *n_edges, int64_t *nnz, int64_t *n_block_entries,
                     int64_t *n_sector_entries, int64_t *n_qdadic_entries, int64_t *device_bytes) {
  g_err.clear();
  if (!rm) {
    set_error("roadmap info: NULL roadmap");
    return LBL_EINVAL;
  }
  if (n_edges) *n_edges = rm->E;
  if (nnz) *nnz = rm->nnz;
  if (n_block_entries) *n_block_entries = rm->n_bt;
  if (n_sector_entries) *n_sector_entries = rm->n_sec;
  if (n_qdadic_entries) *n_qdadic_entries = rm->n_qd;
  if (device_bytes) *device_bytes = rm->bytes;
  return LBL_OK;
}

int lbl_roadmap_rows(lbl_roadmap rm, int64_t *d_rowptr, int32_t *d_colidx, lbl_stream s) {
  g_err.clear();
  if (!rm || !d_rowptr || (rm->nnz > 0 && !d_colidx)) {
    set_error("roadmap rows: NULL roadmap or buffer");
    return LBL_EINVAL;
  }
  if (!same_device(rm->device)) return LBL_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  cudaError_t e = cudaMemcpyAsync(d_rowptr, rm->rowptr, sizeof(int64_t) * (rm->E + 1), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && rm->nnz > 0)
    e = cudaMemcpyAsync(d_colidx, rm->colidx, sizeof(int32_t) * rm->nnz, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "roadmap rows");
  rm->uses->note(st);
  return LBL_OK;
}

int lbl_roadmap_status(lbl_roadmap rm, lbl_stream s) {
  g_err.clear();
  if (!rm) {
    set_error("roadmap status: NULL roadmap");
    return LBL_EINVAL;
  }
  if (!same_device(rm->device)) return LBL_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  int flag = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&flag, rm->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && flag) e = cudaMemset(rm->err, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "roadmap status");
  if (flag) {
    set_error("a labeling kernel gave up waiting for its index stream; its labels are incomplete");
    return LBL_ETIMEOUT;
  }
  return LBL_OK;
}

int lbl_frame_transform(const lbl_grid *world, const uint8_t *d_planes, int32_t n_props, lbl_pose pose,
                        const lbl_grid *agent, uint64_t *d_O, lbl_stream s) {
  g_err.clear();
  if (!valid_grid(world, "frame transform (world)", false) || !valid_grid(agent, "frame transform (agent)", true))
    return LBL_EINVAL;
  if (n_props < 0 || n_props > 64) {
    set_error("frame transform: n_props = %d outside 0..64", n_props);
    return LBL_EINVAL;
  }
  if (!d_O || (n_props > 0 && !d_planes)) {
    set_error("frame transform: NULL buffer");
    return LBL_EINVAL;
  }
  FrameMap m;
  if (!frame_map(*world, *agent, pose, &m)) return LBL_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "frame transform: cudaGetDevice");
  e = launch_frame_transform(frame_item(m, *world, *agent, d_planes, n_props, d_O, 0), reinterpret_cast<cudaStream_t>(s));
  if (e != cudaSuccess) return cuda_fail(e, "frame transform: launch");
  return LBL_OK;
}

int lbl_pack_planes(const lbl_grid *world, const uint8_t *d_planes, int32_t n_props, void *d_words,
                    lbl_stream s) {
  g_err.clear();
  if (!valid_grid(world, "pack planes (world)", false)) return LBL_EINVAL;
  if (n_props < 0 || n_props > 64) {
    set_error("pack planes: n_props = %d outside 0..64", n_props);
    return LBL_EINVAL;
  }
  if (!d_words || (n_props > 0 && !d_planes)) {
    set_error("pack planes: NULL buffer");
    return LBL_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_words) % static_cast<uintptr_t>(packed_word_bytes(n_props))) {
    set_error("pack planes: words not aligned to their %d-byte width", packed_word_bytes(n_props));
    return LBL_EINVAL;
  }
  const PackItem it{d_planes, d_words, grid_cells(*world), n_props, packed_word_bytes(n_props)};
  cudaError_t e = launch_pack_planes(it, reinterpret_cast<cudaStream_t>(s));
  if (e != cudaSuccess) return cuda_fail(e, "pack planes: launch");
  return LBL_OK;
}

int lbl_frame_transform_words(const lbl_grid *world, const void *d_words, int32_t n_props, lbl_pose pose,
                              const lbl_grid *agent, uint64_t *d_O, lbl_stream s) {
  g_err.clear();
  if (!valid_grid(world, "frame transform (world)", false) || !valid_grid(agent, "frame transform (agent)", true))
    return LBL_EINVAL;
  if (n_props < 0 || n_props > 64) {
    set_error("frame transform: n_props = %d outside 0..64", n_props);
    return LBL_EINVAL;
  }
  if (!d_O || !d_words) {
    set_error("frame transform: NULL buffer");
    return LBL_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_words) % static_cast<uintptr_t>(packed_word_bytes(n_props)) ||
      reinterpret_cast<uintptr_t>(d_O) % 8u) {
    set_error("frame transform: words or O not aligned to their width");
    return LBL_EINVAL;
  }
  FrameMap m;
  if (!frame_map(*world, *agent, pose, &m)) return LBL_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "frame transform: cudaGetDevice");
  FrameItem f = frame_item(m, *world, *agent, nullptr, n_props, d_O, 0);
  f.words = d_words;
  f.word_bytes = packed_word_bytes(n_props);
  f.wmask = n_props >= 64 ? ~0ull : ((1ull << n_props) - 1ull);
  e = launch_frame_transform(f, reinterpret_cast<cudaStream_t>(s));
  if (e != cudaSuccess) return cuda_fail(e, "frame transform: launch");
  return LBL_OK;
}

int lbl_frame_transform_pyramid(lbl_roadmap rm, const lbl_grid *world, const void *d_words, int32_t n_props,
                                lbl_pose pose, uint64_t *d_O, lbl_stream s) {
  g_err.clear();
  if (!rm) {
    set_error("frame transform (pyramid): NULL roadmap");
    return LBL_EINVAL;
  }
  if (!same_device(rm->device)) return LBL_EINVAL;
  if (rm->E > 0 && !rm->has_qd) {
    set_error("frame transform (pyramid): the roadmap has no quadtree form (LBL_UPLOAD_QUAD)");
    return LBL_EUNSUPPORTED;
  }
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  if (rm->E == 0) {  // no rows, no pyramid: the transform alone, if O is wanted
    if (!d_O) return valid_grid(world, "frame transform (world)", false) ? LBL_OK : LBL_EINVAL;
    return lbl_frame_transform_words(world, d_words, n_props, pose, &rm->agent, d_O, s);
  }
  const int rc = transform_pyramid(world, d_words, n_props, pose, *rm, d_O, rm->pyr, st);
  if (rc != LBL_OK) return rc;
  rm->pyr_built_bytes = quad_word_bytes(*rm, n_props);
  rm->uses->note(st);
  return LBL_OK;
}

int lbl_label_pyramid(lbl_roadmap rm, int32_t n_props, uint64_t *d_L, lbl_monitor mon, uint64_t *d_next,
                      uint16_t *d_viol, const lbl_config *cfg, lbl_stream s) {
  g_err.clear();
  if (!rm) {
    set_error("label (pyramid): NULL roadmap");
    return LBL_EINVAL;
  }
  if (n_props < 0 || n_props > 64) {
    set_error("label (pyramid): n_props = %d outside 0..64", n_props);
    return LBL_EINVAL;
  }
  if (rm->E > 0 && !d_L) {
    set_error("label (pyramid): NULL L");
    return LBL_EINVAL;
  }
  if (mon && rm->E > 0 && (!d_next || !d_viol)) {
    set_error("label (pyramid): monitor given but next/viol is NULL");
    return LBL_EINVAL;
  }
  if (!same_device(rm->device)) return LBL_EINVAL;
  if (mon && mon->device != rm->device) {
    set_error("label (pyramid): monitor and roadmap live on different devices");
    return LBL_EINVAL;
  }
  const int algo = cfg ? cfg->algo : LBL_ALGO_AUTO;
  if (algo != LBL_ALGO_AUTO && algo != LBL_ALGO_QUAD) {
    set_error("label (pyramid): labels from the pyramid are the quadtree form (algo %d asked)", algo);
    return LBL_EINVAL;
  }
  if (rm->E == 0) return LBL_OK;
  if (rm->pyr_built_bytes == 0 || rm->pyr_built_bytes != quad_word_bytes(*rm, n_props)) {
    set_error("label (pyramid): no pyramid for %d propositions on this roadmap (lbl_frame_transform_pyramid first)",
              n_props);
    return LBL_EINVAL;
  }
  lbl_config tuned_cfg;
  if (algo == LBL_ALGO_AUTO) {  // the measured quadtree configuration, else the form's defaults
    cfg = nullptr;
    if (rm->tuned_valid[n_props] && rm->tuned[n_props].algo == LBL_ALGO_QUAD) {
      tuned_cfg = rm->tuned[n_props];
      cfg = &tuned_cfg;
    }
  }
  MonitorTables t{};
  if (mon) t = tables_of(*mon, d_next, d_viol);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  const int rc = quad_label(rm, nullptr, n_props, d_L, mon ? &t : nullptr, cfg, st);
  if (rc != LBL_OK) return rc;
  rm->uses->note(st);
  if (mon) mon->uses->note(st);
  return LBL_OK;
}

int lbl_monitor_create(int32_t n_states, int32_t m, const uint8_t *relbits, const uint8_t *delta, int32_t reject,
                       lbl_monitor *out) {
  g_err.clear();
  if (!out) {
    set_error("monitor create: out is NULL");
    return LBL_EINVAL;
  }
  *out = nullptr;
  if (n_states < 1 || n_states > 16 || m < 0 || m > 8 || reject < -1 || reject >= n_states) {
    set_error("monitor create: need 1 <= n_states <= 16, 0 <= m <= 8, -1 <= reject < n_states");
    return LBL_EINVAL;
  }
  if (!delta || (m > 0 && !relbits)) {
    set_error("monitor create: NULL table");
    return LBL_EINVAL;
  }
  for (int j = 0; j < m; ++j)
    if (relbits[j] >= 64) {
      set_error("monitor create: relbits[%d] = %d >= 64", j, relbits[j]);
      return LBL_EINVAL;
    }
  const int letters = 1 << m;
  for (int i = 0; i < n_states * letters; ++i)
    if (delta[i] >= n_states) {
      set_error("monitor create: delta[%d] = %d is not a state", i, delta[i]);
      return LBL_EINVAL;
    }
  lbl_monitor_s *mon = new (std::nothrow) lbl_monitor_s();
  if (!mon) {
    set_error("monitor create: out of host memory");
    return LBL_ENOMEM;
  }
  mon->n_states = n_states;
  mon->m = m;
  mon->reject = reject;
  for (int j = 0; j < m; ++j) mon->rel[j] = relbits[j];
  // Per letter: the next state of every monitor state packed in 4-bit fields,
  // and which of those next states is the reject state.
  for (int letter = 0; letter < letters; ++letter) {
    uint64_t t = 0;
    uint16_t v = 0;
    for (int q = 0; q < n_states; ++q) {
      const uint32_t nq = delta[q * letters + letter];
      t |= static_cast<uint64_t>(nq) << (4 * q);
      if (static_cast<int32_t>(nq) == reject) v |= static_cast<uint16_t>(1u << q);
    }
    mon->hT[letter] = t;
    mon->hV[letter] = v;
  }
  cudaError_t e = cudaGetDevice(&mon->device);
  if (e == cudaSuccess) e = obj_alloc(&mon->T, 256, nullptr);
  if (e == cudaSuccess) e = obj_alloc(&mon->V, 256, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(mon->T, mon->hT, sizeof(mon->hT), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(mon->V, mon->hV, sizeof(mon->hV), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    mon->uses->release(mon->device, {mon->T, mon->V});
    delete mon;
    return cuda_fail(e, "monitor create");
  }
  *out = mon;
  return LBL_OK;
}

int lbl_monitor_free(lbl_monitor mon) {
  g_err.clear();
  if (!mon) return LBL_OK;
  mon->uses->release(mon->device, {mon->T, mon->V});  // after the monitor's last logged use
  delete mon;
  return LBL_OK;
}

}  // extern "C"

namespace lbl {

MonitorTables tables_of(const Monitor &mon, uint64_t *next, uint16_t *viol) {
  MonitorTables t{};
  t.T = mon.T;
  t.V = mon.V;
  t.next = next;
  t.viol = viol;
  t.m = mon.m;
  for (int j = 0; j < 8; ++j) t.rel[j] = mon.rel[j];
  return t;
}

}  // namespace lbl

extern "C" {

int lbl_monitor_step(lbl_monitor mon, const uint64_t *d_L, int64_t n, uint64_t *d_next, uint16_t *d_viol,
                     lbl_stream s) {
  g_err.clear();
  if (!mon || n < 0 || (n > 0 && (!d_L || !d_next || !d_viol))) {
    set_error("monitor step: NULL monitor/buffer or negative n");
    return LBL_EINVAL;
  }
  if (!same_device(mon->device)) return LBL_EINVAL;
  MonitorTables t = tables_of(*mon, d_next, d_viol);
  cudaError_t e = launch_monitor_step(t, d_L, n, device_sms(mon->device), reinterpret_cast<cudaStream_t>(s));
  if (e != cudaSuccess) return cuda_fail(e, "monitor step: launch");
  mon->uses->note(reinterpret_cast<cudaStream_t>(s));
  return LBL_OK;
}

}  // extern "C"

namespace lbl {

// The quadtree form's launch (lbl_label, lbl_label_pyramid): the partition
// for the requested grid, the pyramid of d_O (none when d_O is NULL: the rows
// gather from the pyramid the frame transform built), then the stream over
// the quadtree rows.
int quad_label(lbl_roadmap rm, const uint64_t *d_O, int32_t n_props, uint64_t *d_L, const MonitorTables *mt,
               const lbl_config *cfg, cudaStream_t st) {
  const int ctas = cfg ? cfg->ctas_per_sm : 0;
  const int qpipe = cfg ? cfg->pipeline : 0;
  if (qpipe != 0 && qpipe != LBL_PIPE_REGISTERS && qpipe != LBL_PIPE_FRONT) {
    set_error("label: pipeline %d does not apply to the quadtree form", qpipe);
    return LBL_EINVAL;
  }
  const int depth = (cfg && cfg->depth) ? cfg->depth : kQuadDepth;
  cudaError_t e;
  if (rm->E > 0) {
    const int occ = stream_ctas_per_sm(depth);
    const int want = ctas > 0 ? std::min(ctas, occ) : occ;
    if (want != rm->qd_part_ctas) {
      const int64_t W = static_cast<int64_t>(rm->num_sms) * want * (kThreads / 32);
      if ((e = launch_partition_into(rm->qd_rowptr, rm->E, W, rm->qd_part, st)) != cudaSuccess)
        return cuda_fail(e, "label: quadtree partition");
      rm->qd_part_ctas = want;
    }
  }
  // pipeline: 0 = the moving front on large roadmaps (by size), LBL_PIPE_FRONT
  // = the front whatever the size, anything else = the per-warp stream
  const int fchunk = qpipe == 0 ? -1 : qpipe == LBL_PIPE_FRONT ? std::max(front_chunk_for(rm->E, rm->num_sms), 8) : 0;
  e = launch_label_quad(*rm, d_O, n_props, d_L, mt, depth, st, fchunk);
  if (e != cudaSuccess) return cuda_fail(e, "label: launch");
  if (d_O && rm->E > 0) rm->pyr_built_bytes = quad_word_bytes(*rm, n_props);
  return LBL_OK;
}

int label_impl(lbl_roadmap rm, const uint64_t *d_O, int32_t n_props, uint64_t *d_L, lbl_monitor mon,
               uint64_t *d_next, uint16_t *d_viol, const lbl_config *cfg, cudaStream_t st) {
  if (!rm) {
    set_error("label: NULL roadmap");
    return LBL_EINVAL;
  }
  if (n_props < 0 || n_props > 64) {
    set_error("label: n_props = %d outside 0..64", n_props);
    return LBL_EINVAL;
  }
  if (rm->E > 0 && (!d_O || !d_L)) {
    set_error("label: NULL O or L");
    return LBL_EINVAL;
  }
  if (mon && rm->E > 0 && (!d_next || !d_viol)) {
    set_error("label: monitor given but next/viol is NULL");
    return LBL_EINVAL;
  }
  if (!same_device(rm->device)) return LBL_EINVAL;
  if (mon && mon->device != rm->device) {
    set_error("label: monitor and roadmap live on different devices");
    return LBL_EINVAL;
  }
  int algo = cfg ? cfg->algo : LBL_ALGO_AUTO;
  if (algo < LBL_ALGO_AUTO || algo > LBL_ALGO_MMA) {
    set_error("label: unknown algo %d", algo);
    return LBL_EINVAL;
  }
  if (algo == LBL_ALGO_BITTILE && !rm->has_bt) {
    set_error("label: LBL_ALGO_BITTILE needs a roadmap uploaded with LBL_UPLOAD_BITTILE");
    return LBL_EUNSUPPORTED;
  }
  if (algo == LBL_ALGO_SECTOR && !rm->has_sec) {
    set_error("label: LBL_ALGO_SECTOR needs a roadmap uploaded with LBL_UPLOAD_SECTOR");
    return LBL_EUNSUPPORTED;
  }
  if (algo == LBL_ALGO_QUAD && !rm->has_qd) {
    set_error("label: LBL_ALGO_QUAD needs a roadmap uploaded with LBL_UPLOAD_QUAD");
    return LBL_EUNSUPPORTED;
  }
  if (algo == LBL_ALGO_MMA && !rm->has_mma) {
    set_error("label: LBL_ALGO_MMA needs a roadmap uploaded with LBL_UPLOAD_MMA");
    return LBL_EUNSUPPORTED;
  }
  if (algo == LBL_ALGO_SECTOR && rm->E > 0 && (reinterpret_cast<uintptr_t>(d_O) & 31u)) {
    set_error("label: LBL_ALGO_SECTOR needs O 32-byte aligned");
    return LBL_EINVAL;
  }
  lbl_config tuned_cfg;
  if (algo == LBL_ALGO_AUTO && rm->tuned_valid[n_props]) {
    tuned_cfg = rm->tuned[n_props];  // measured by lbl_roadmap_autotune
    cfg = &tuned_cfg;
    algo = tuned_cfg.algo;
  }
  if (algo == LBL_ALGO_AUTO)
    algo = rm->has_qd ? LBL_ALGO_QUAD : (rm->has_bt && n_props <= 8) ? LBL_ALGO_BITTILE : LBL_ALGO_CSR;
  int ee = cfg ? cfg->early_exit : -1;
  const bool early = ee > 0;  // measured: the per-step OR-reduce costs more than it saves
  const int ctas = cfg ? cfg->ctas_per_sm : 0;
  const int lpe = cfg ? cfg->lanes_per_edge : 0;
  MonitorTables t{};
  if (mon) t = tables_of(*mon, d_next, d_viol);
  cudaError_t e;
  if (algo == LBL_ALGO_MMA) {
    e = launch_label_mma(*rm, d_O, n_props, d_L, mon ? &t : nullptr, st);
  } else if (algo == LBL_ALGO_BITTILE) {
    e = launch_label_bittile(*rm, d_O, n_props, d_L, mon ? &t : nullptr, early, ctas, st);
  } else if (algo == LBL_ALGO_SECTOR) {
    const int depth = (cfg && cfg->depth == 8) ? 8 : 4;
    if (rm->E > 0) {
      const int occ = sector_ctas_per_sm(depth);
      const int want = ctas > 0 ? std::min(ctas, occ) : occ;
      if (want != rm->sec_part_ctas) {
        const int64_t W = static_cast<int64_t>(rm->num_sms) * want * (kThreads / 32);
        if ((e = launch_partition_into(rm->sec_rowptr, rm->E, W, rm->sec_part, st)) != cudaSuccess)
          return cuda_fail(e, "label: sector partition");
        rm->sec_part_ctas = want;
      }
    }
    e = launch_label_sector(*rm, d_O, n_props, d_L, mon ? &t : nullptr, depth, st);
  } else if (algo == LBL_ALGO_QUAD) {
    const int rc = quad_label(rm, d_O, n_props, d_L, mon ? &t : nullptr, cfg, st);
    if (rc != LBL_OK) return rc;
    e = cudaSuccess;
  } else if (early || lpe > 0) {
    // lanes-per-edge form (one edge per lane group; supports early exit)
    e = launch_label_csr(*rm, d_O, n_props, d_L, mon ? &t : nullptr, resolve_lpe(*rm, cfg), early, ctas, st);
  } else {
    // streaming form over the edge partition; re-partition for a new grid
    int pipe = cfg ? cfg->pipeline : 0;
    if (pipe < 0 || pipe > LBL_PIPE_ASYNC) {
      set_error("label: unknown pipeline %d", pipe);
      return LBL_EINVAL;
    }
    if (pipe == 0) pipe = kDefaultPipeline;
    const int depth = cfg ? cfg->depth : 0;
    if (rm->E > 0) {
      const int occ = pipe == LBL_PIPE_BULK ? tma_ctas_per_sm()
                      : pipe == LBL_PIPE_ASYNC ? async_ctas_per_sm()
                                               : stream_ctas_per_sm(depth);
      const int want = ctas > 0 ? std::min(ctas, occ) : occ;
      if (want != rm->part_ctas) {
        if ((e = launch_partition(*rm, want, st)) != cudaSuccess) return cuda_fail(e, "label: partition");
        rm->part_ctas = want;
      }
    }
    const MonitorTables *mt = mon ? &t : nullptr;
    e = pipe == LBL_PIPE_BULK    ? launch_label_tma(*rm, d_O, n_props, d_L, mt, st)
        : pipe == LBL_PIPE_ASYNC ? launch_label_async(*rm, d_O, n_props, d_L, mt, st)
                                 : launch_label_stream(*rm, d_O, n_props, d_L, mt, depth, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "label: launch");
  rm->uses->note(st);
  if (mon) mon->uses->note(st);
  return LBL_OK;
}

}  // namespace lbl

extern "C" {

int lbl_label(lbl_roadmap rm, const uint64_t *d_O, int32_t n_props, uint64_t *d_L, lbl_monitor mon, uint64_t *d_next,
              uint16_t *d_viol, const lbl_config *cfg, lbl_stream s) {
  g_err.clear();
  return label_impl(rm, d_O, n_props, d_L, mon, d_next, d_viol, cfg, reinterpret_cast<cudaStream_t>(s));
}

int lbl_roadmap_autotune(lbl_roadmap rm, const uint64_t *d_O, int32_t n_props, lbl_monitor mon, uint64_t *d_L,
                         uint64_t *d_next, uint16_t *d_viol, int32_t reps, lbl_config *chosen, lbl_stream s) {
  g_err.clear();
  if (!rm || n_props < 0 || n_props > 64 || reps < 1 || reps > 1000) {
    set_error("autotune: need a roadmap, 0 <= n_props <= 64 and 1 <= reps <= 1000");
    return LBL_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  std::vector<lbl_config> cand;
  for (int depth : {8, 12, 16}) cand.push_back(lbl_config{LBL_ALGO_CSR, 0, 0, 0, LBL_PIPE_REGISTERS, depth});
  for (int pipe : {LBL_PIPE_BULK, LBL_PIPE_ASYNC}) cand.push_back(lbl_config{LBL_ALGO_CSR, 0, 0, 0, pipe, 0});
  for (int lpe : {8, 16, 32}) cand.push_back(lbl_config{LBL_ALGO_CSR, lpe, 0, 0, 0, 0});
  if (rm->has_bt) cand.push_back(lbl_config{LBL_ALGO_BITTILE, 0, 0, 0, 0, 0});
  if (rm->has_sec && !(reinterpret_cast<uintptr_t>(d_O) & 31u))
    for (int depth : {4, 8}) cand.push_back(lbl_config{LBL_ALGO_SECTOR, 0, 0, 0, 0, depth});
  if (rm->has_qd) {
    for (int depth : {8, 12}) cand.push_back(lbl_config{LBL_ALGO_QUAD, 0, 0, 0, LBL_PIPE_REGISTERS, depth});
    cand.push_back(lbl_config{LBL_ALGO_QUAD, 0, 0, 0, LBL_PIPE_FRONT, 8});
  }
  if (rm->has_mma) cand.push_back(lbl_config{LBL_ALGO_MMA, 0, 0, 0, 0, 0});
  cudaEvent_t t0, t1;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e != cudaSuccess) return cuda_fail(e, "autotune: events");
  float best = 0.f;
  int best_i = -1, rc = LBL_OK;
  for (size_t i = 0; i < cand.size() && rc == LBL_OK; ++i) {
    rc = label_impl(rm, d_O, n_props, d_L, mon, d_next, d_viol, &cand[i], st);  // warm-up, re-partition
    if (rc != LBL_OK) break;
    e = cudaEventRecord(t0, st);
    for (int r = 0; r < reps && rc == LBL_OK && e == cudaSuccess; ++r)
      rc = label_impl(rm, d_O, n_props, d_L, mon, d_next, d_viol, &cand[i], st);
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e != cudaSuccess) break;
    if (best_i < 0 || ms < best) {
      best = ms;
      best_i = static_cast<int>(i);
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (rc != LBL_OK) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "autotune: timing");
  rm->tuned[n_props] = cand[best_i];
  rm->tuned_valid[n_props] = true;
  if (chosen) *chosen = cand[best_i];
  return LBL_OK;
}

}  // extern "C"
