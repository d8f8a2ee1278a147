// C ABI of liblbl (declared in include/lbl.h): argument checks, handles,
// device memory of roadmaps and sessions, and kernel dispatch.
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

template <typename T>
cudaError_t dev_alloc(T **p, size_t count, int64_t *bytes) {
  const size_t b = count * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), b ? b : 16);
  if (e == cudaSuccess && bytes) *bytes += static_cast<int64_t>(b);
  return e;
}

void free_roadmap(Roadmap *rm) {
  if (!rm) return;
  cudaFree(rm->rowptr);
  cudaFree(rm->colidx);
  cudaFree(rm->bt_rowptr);
  cudaFree(rm->bt_block);
  cudaFree(rm->bt_mask);
  cudaFree(rm->planes);
  cudaFree(rm->part);
  cudaFree(rm->err);
  cudaFree(rm->sec_rowptr);
  cudaFree(rm->sec);
  cudaFree(rm->sec_part);
  cudaFree(rm->qd_rowptr);
  cudaFree(rm->qd_perm);
  cudaFree(rm->qd_idx);
  cudaFree(rm->qd_part);
  cudaFree(rm->pyr);
  delete rm;
}

int resolve_lpe(const Roadmap &rm, const lbl_config *cfg) {
  int lpe = cfg ? cfg->lanes_per_edge : 0;
  if (lpe == 4 || lpe == 8 || lpe == 16 || lpe == 32) return lpe;
  const double avg = rm.E ? static_cast<double>(rm.nnz) / static_cast<double>(rm.E) : 0.0;
  lpe = 4;
  while (lpe < 32 && lpe * 16 < avg) lpe *= 2;
  return lpe;
}

}  // namespace

// Q32.32 coefficients of (ix, iy) -> continuous world-cell coordinates:
//   u = a00*ix + a01*iy + b0,  v = a10*ix + a11*iy + b1,
// from world point q = (X, Y) + R(theta) * centre(ix, iy) (Sec. 5, eq. 13).
// The double expressions are evaluated exactly as written (the library is built
// without floating-point contraction) and each is rounded half to even.
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

int cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LBL_ENOMEM : LBL_ECUDA;
}

}  // namespace lbl

using namespace lbl;
struct lbl_batch_s {
  int device = 0;
  int num_sms = 1;
  int32_t n = 0;
  std::vector<lbl_roadmap> rms;
  std::vector<int32_t> P;
  std::vector<lbl_monitor> mons;
  int64_t *part = nullptr;  // every item's partition, concatenated
  unsigned long long *counter = nullptr;  // next work unit of each class's label launch
  int ctas = 1;
  // items grouped by gathered word width (class c = 1, 2, 4, 8 bytes); item i
  // is entry slot[i] of tabs[cls[i]]
  BatchTable tabs[kWordClasses]{};
  std::vector<int> cls, slot;
  FrameTable ftab{};
  // items whose roadmap has the quadtree form label from their own pyramid
  uint64_t *pyr = nullptr;      // every such item's pyramid, concatenated
  std::vector<int> pyr_slot;    // item -> entry of ptab, or -1
  PyrTable ptab{};
  // frames whose world has at most kPackedWorldRatio times the agent's cells
  // are packed (one launch) and transformed from 64-bit words; the words
  // buffer grows on demand, and a replaced buffer is kept until the batch is
  // freed so graphs captured before still see live memory
  PackTable pktab{};
  uint64_t *words = nullptr;
  int64_t words_cap = 0;
  std::vector<uint64_t *> retired;
  bool frames_set = false;
};

struct lbl_session_s {
  int device = 0;
  lbl_roadmap rm = nullptr;
  lbl_monitor mon = nullptr;
  lbl_grid world{};
  int32_t P = 0;
  lbl_config cfg{};
  bool has_cfg = false;
  uint8_t *planes = nullptr;
  uint64_t *O = nullptr, *L = nullptr, *next = nullptr;
  uint16_t *viol = nullptr;
  // Two plane buffers, filled on `cin` in turn: frame i+1's planes go to the
  // device while frame i is transformed and labeled.  ev_in[k]: slot k filled;
  // ev_free[k]: the transform that read slot k is done.
  uint8_t *slot[2] = {nullptr, nullptr};
  cudaStream_t cin = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  int64_t frame = 0;
  // The session's kernels run on `cc`, and its outputs go to one of two device
  // buffer sets in turn, so frame i+1 computes while frame i's results are
  // still being copied out; ev_out[k]: output set k copied to the host.
  cudaStream_t cc = nullptr;
  uint64_t *Ls[2] = {nullptr, nullptr}, *Ns[2] = {nullptr, nullptr};
  uint16_t *Vs[2] = {nullptr, nullptr};
  cudaEvent_t ev_out[2] = {nullptr, nullptr};
  uint64_t *pyr = nullptr;  // the session's own quadtree pyramid (chunked quadtree sessions)
  // Packed world words: the planes are packed (one coalesced pass) and the
  // transform gathers one word per agent cell.  Used for planes of at least
  // kPackedMinPlaneBytes on a world of at most kPackedWorldRatio times the
  // agent's cells, so packing reads little the transform would not.
  uint8_t *words = nullptr;
  // Chunked labeling: the edges in kSessionChunks ranges, each labeled by the
  // whole grid; a range's results go to the host on `cs` while the next range
  // is labeled.  Used with the default form (quadtree, else streaming CSR).
  bool chunked = false;
  bool quad = false;
  int depth = 8, ctas = 0;
  int64_t edge0[lbl::kSessionChunks + 1] = {0};
  int64_t *cpart = nullptr;  // kSessionChunks partitions of warps + 1 entries
  int64_t warps = 0;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[lbl::kSessionChunks + 1] = {nullptr};
};

namespace lbl {

bool valid_grid_public(const lbl_grid *g, const char *name, bool need_order) {
  return valid_grid(g, name, need_order);
}
int device_sms_public(int dev) { return device_sms(dev); }
void free_roadmap_public(lbl_roadmap_s *rm) { free_roadmap(rm); }

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
  if ((e = dev_alloc(&rm->rowptr, static_cast<size_t>(n_edges + 1), &rm->bytes)) != cudaSuccess ||
      (e = dev_alloc(&rm->colidx, static_cast<size_t>(padded), &rm->bytes)) != cudaSuccess ||
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
  if ((e = dev_alloc(&rm->err, 1, &rm->bytes)) != cudaSuccess ||
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
    if ((e = dev_alloc(&rm->part, static_cast<size_t>(rm->part_cap), &rm->bytes)) != cudaSuccess)
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
    if ((e = dev_alloc(&rm->bt_rowptr, static_cast<size_t>(n_edges + 1), &rm->bytes)) != cudaSuccess ||
        (e = dev_alloc(&rm->bt_block, static_cast<size_t>(rm->n_bt), &rm->bytes)) != cudaSuccess ||
        (e = dev_alloc(&rm->bt_mask, static_cast<size_t>(rm->n_bt), &rm->bytes)) != cudaSuccess ||
        (e = dev_alloc(&rm->planes, static_cast<size_t>(rm->n_blocks * 64), &rm->bytes)) != cudaSuccess)
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
    if ((e = dev_alloc(&rm->sec_rowptr, static_cast<size_t>(n_edges + 1), &rm->bytes)) != cudaSuccess ||
        (e = dev_alloc(&rm->sec, static_cast<size_t>(rm->n_sec), &rm->bytes)) != cudaSuccess ||
        (e = dev_alloc(&rm->sec_part, static_cast<size_t>(rm->part_cap), &rm->bytes)) != cudaSuccess ||
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
    if (n_edges > 1 && n_edges < (1LL << 31) && !(flags & LBL_UPLOAD_KEEP_ORDER) && grid_depth(rm->agent) == 1) {
      // locality order: inside each session edge range, rows by the z-order of
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
      for (int c = 0; c < kSessionChunks; ++c)
        sort_range_by_key(key.data(), n_edges * c / kSessionChunks, n_edges * (c + 1) / kSessionChunks, perm.data());
      if ((e = dev_alloc(&rm->qd_perm, static_cast<size_t>(n_edges), &rm->bytes)) != cudaSuccess ||
          (e = cudaMemcpyAsync(rm->qd_perm, perm.data(), sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, st)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(cuda_fail(e, "roadmap: quadtree order"));
    }
    std::vector<int32_t> cnt(static_cast<size_t>(n_edges));
    std::vector<int64_t> drow(static_cast<size_t>(n_edges + 1));
    int32_t *d_dc = nullptr;
    if ((e = dev_alloc(&d_dc, static_cast<size_t>(n_edges), nullptr)) != cudaSuccess ||
        (e = launch_quad_count(rm->rowptr, rm->colidx, n_edges, rm->qd_perm, d_dc, st)) != cudaSuccess ||
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
    if ((e = dev_alloc(&rm->qd_rowptr, static_cast<size_t>(n_edges + 1), &rm->bytes)) != cudaSuccess ||
        (e = dev_alloc(&rm->qd_idx, static_cast<size_t>(rm->n_qd + 4), &rm->bytes)) != cudaSuccess ||
        (e = dev_alloc(&rm->qd_part, static_cast<size_t>(rm->part_cap), &rm->bytes)) != cudaSuccess ||
        (e = dev_alloc(&rm->pyr, static_cast<size_t>(words), &rm->bytes)) != cudaSuccess ||
        (e = cudaMemcpyAsync(rm->qd_rowptr, drow.data(), sizeof(int64_t) * (n_edges + 1), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = launch_quad_fill(rm->rowptr, rm->colidx, n_edges, rm->qd_perm, rm->qd_off, rm->qd_rowptr, rm->qd_idx,
                              st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: quadtree form"));
    rm->qd_part_ctas = stream_ctas_per_sm(kQuadDepth);
    const int64_t W = static_cast<int64_t>(rm->num_sms) * rm->qd_part_ctas * (kThreads / 32);
    if ((e = launch_partition_into(rm->qd_rowptr, n_edges, W, rm->qd_part, st)) != cudaSuccess)
      return fail(cuda_fail(e, "roadmap: quadtree partition"));
    rm->has_qd = true;
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(cuda_fail(e, "roadmap"));
  cudaFree(d_bad);
  cudaFree(d_cnt);
  return LBL_OK;
}

}  // namespace lbl

extern "C" {

const char *lbl_last_error(void) { return g_err.c_str(); }

int lbl_version(void) { return 10000; }

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
                LBL_UPLOAD_KEEP_ORDER)) {
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
  cudaDeviceSynchronize();
  free_roadmap(rm);
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
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&mon->T), sizeof(mon->hT));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&mon->V), sizeof(mon->hV));
  if (e == cudaSuccess) e = cudaMemcpy(mon->T, mon->hT, sizeof(mon->hT), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(mon->V, mon->hV, sizeof(mon->hV), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(mon->T);
    cudaFree(mon->V);
    delete mon;
    return cuda_fail(e, "monitor create");
  }
  *out = mon;
  return LBL_OK;
}

int lbl_monitor_free(lbl_monitor mon) {
  g_err.clear();
  if (!mon) return LBL_OK;
  cudaDeviceSynchronize();
  cudaFree(mon->T);
  cudaFree(mon->V);
  delete mon;
  return LBL_OK;
}

static MonitorTables tables_of(const Monitor &mon, uint64_t *next, uint16_t *viol) {
  MonitorTables t{};
  t.T = mon.T;
  t.V = mon.V;
  t.next = next;
  t.viol = viol;
  t.m = mon.m;
  for (int j = 0; j < 8; ++j) t.rel[j] = mon.rel[j];
  return t;
}

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
  return LBL_OK;
}

static int label_impl(lbl_roadmap rm, const uint64_t *d_O, int32_t n_props, uint64_t *d_L, lbl_monitor mon,
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
  if (algo < LBL_ALGO_AUTO || algo > LBL_ALGO_QUAD) {
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
  if (algo == LBL_ALGO_BITTILE) {
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
    const int depth = (cfg && cfg->depth) ? cfg->depth : kQuadDepth;
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
    e = launch_label_quad(*rm, d_O, n_props, d_L, mon ? &t : nullptr, depth, st);
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
  return LBL_OK;
}

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
  if (rm->has_qd)
    for (int depth : {8, 12}) cand.push_back(lbl_config{LBL_ALGO_QUAD, 0, 0, 0, 0, depth});
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

int lbl_batch_create(int32_t n, const lbl_roadmap *rms, const int32_t *n_props, const lbl_monitor *mons,
                     int32_t ctas_per_sm, lbl_batch *out) {
  g_err.clear();
  if (!out) {
    set_error("batch create: out is NULL");
    return LBL_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || n > kMaxBatch || !rms || !n_props) {
    set_error("batch create: need 1 <= n <= %d roadmaps and their proposition counts", kMaxBatch);
    return LBL_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    if (!rms[i] || n_props[i] < 0 || n_props[i] > 64) {
      set_error("batch create: item %d has no roadmap or n_props outside 0..64", i);
      return LBL_EINVAL;
    }
    if (rms[i]->device != rms[0]->device || (mons && mons[i] && mons[i]->device != rms[0]->device)) {
      set_error("batch create: items live on different devices");
      return LBL_EINVAL;
    }
  }
  if (!same_device(rms[0]->device)) return LBL_EINVAL;
  lbl_batch_s *b = new (std::nothrow) lbl_batch_s();
  if (!b) {
    set_error("batch create: out of host memory");
    return LBL_ENOMEM;
  }
  b->device = rms[0]->device;
  b->num_sms = rms[0]->num_sms;
  b->n = n;
  b->rms.assign(rms, rms + n);
  b->P.assign(n_props, n_props + n);
  b->mons.assign(n, nullptr);
  if (mons) b->mons.assign(mons, mons + n);
  // The persistent grid's warps take work units from a counter; items are
  // cut into units of about equal cost (nonzeros + kEdgeCost per edge),
  // kUnitsPerWarp per warp overall, at least one per item with edges.
  bool all_quad = true;
  for (int i = 0; i < n; ++i) all_quad = all_quad && (rms[i]->has_qd || rms[i]->E == 0);
  const int depth = all_quad ? kQuadDepth : 8;
  for (BatchTable &t : b->tabs) t.depth = depth;
  const int occ = batch_ctas_per_sm(depth);
  const int ctas = ctas_per_sm > 0 ? std::min<int>(ctas_per_sm, occ) : occ;
  b->ctas = ctas;
  constexpr int64_t kUnitsPerWarp = 8;
  const int64_t units_target = static_cast<int64_t>(b->num_sms) * ctas * (kThreads / 32) * kUnitsPerWarp;
  // entries streamed per item: quadtree entries when the roadmap has them;
  // word width of its gathers (items of one width share a launch)
  auto entries = [](const Roadmap &r) { return r.has_qd ? r.n_qd : r.nnz; };
  auto width = [&](int i) { return rms[i]->has_qd && rms[i]->E > 0 ? quad_word_bytes(*rms[i], n_props[i]) : 8; };
  // every class's launch gets about kUnitsPerWarp units per warp of its own
  double total[kWordClasses] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) total[word_class(width(i))] += static_cast<double>(entries(*rms[i]) + kEdgeCost * rms[i]->E);
  std::vector<int64_t> W(n), off(n + 1, 0);
  int64_t pyr_words = 0;
  for (int i = 0; i < n; ++i)
    if (rms[i]->has_qd && rms[i]->E > 0) pyr_words += rms[i]->pyr_words;
  for (int i = 0; i < n; ++i) {
    const Roadmap &r = *rms[i];
    W[i] = 0;
    if (r.E > 0) {
      const double c = static_cast<double>(entries(r) + kEdgeCost * r.E);
      const double unit_cost = total[word_class(width(i))] / static_cast<double>(units_target);
      W[i] = std::max<int64_t>(1, static_cast<int64_t>(std::ceil(c / unit_cost)));
      W[i] = std::min<int64_t>(W[i], r.E);  // never more units than edges
    }
    off[i + 1] = off[i] + W[i] + 1;
  }
  cudaError_t e = dev_alloc(&b->part, static_cast<size_t>(off[n]), nullptr);
  if (e == cudaSuccess) e = dev_alloc(&b->counter, kWordClasses, nullptr);
  if (e == cudaSuccess && pyr_words > 0) e = dev_alloc(&b->pyr, static_cast<size_t>(pyr_words), nullptr);
  b->pyr_slot.assign(n, -1);
  b->cls.assign(n, kWordClasses - 1);
  b->slot.assign(n, 0);
  int64_t pyr0 = 0, block0 = 0;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const Roadmap &r = *rms[i];
    const bool quad = r.has_qd && r.E > 0;
    const int wb = width(i);
    e = launch_partition_into(quad ? r.qd_rowptr : r.rowptr, r.E, W[i], b->part + off[i], nullptr);
    BatchTable &tb = b->tabs[word_class(wb)];
    b->cls[i] = word_class(wb);
    b->slot[i] = tb.n;
    tb.word_bytes = wb;
    BatchItem &it = tb.items[tb.n++];
    it = BatchItem{};
    it.rowptr = quad ? r.qd_rowptr : r.rowptr;
    it.colidx = quad ? r.qd_idx : r.colidx;
    it.perm = quad ? r.qd_perm : nullptr;
    it.part = b->part + off[i];
    if (quad) {  // labels gather from the item's pyramid, built from its O at the label stage
      PyrItem &pi = b->ptab.items[b->ptab.n];
      pi = PyrItem{};
      pi.pyr = b->pyr + pyr0;
      pi.cells = r.cells;
      pi.block0 = block0;
      pi.off = r.qd_off;
      pi.word_bytes = wb;
      it.O = pi.pyr;
      b->pyr_slot[i] = b->ptab.n++;
      pyr0 += r.pyr_words;
      block0 += (r.cells + kThreads - 1) / kThreads;
    }
    it.mask = n_props[i] >= 64 ? ~0ull : ((1ull << n_props[i]) - 1ull);
    it.warp0 = tb.total;  // work units of this class's launch
    it.warps = W[i];
    if (b->mons[i]) {
      const Monitor &m = *b->mons[i];
      it.T = m.T;
      it.V = m.V;
      it.m = m.m;
      for (int j = 0; j < 8; ++j) it.rel[j] = m.rel[j];
    }
    tb.total += W[i];
    if (entries(r) >= kNarrowLimit || r.E >= kNarrowLimit) tb.wide = 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e != cudaSuccess) {
    cudaFree(b->part);
    cudaFree(b->counter);
    cudaFree(b->pyr);
    delete b;
    return cuda_fail(e, "batch create: partitions");
  }
  b->ptab.total = block0;
  b->ftab.n = n;
  *out = b;
  return LBL_OK;
}

int lbl_batch_set_frames(lbl_batch b, const lbl_frame *frames) {
  g_err.clear();
  if (!b || !frames) {
    set_error("batch frames: NULL batch or frames");
    return LBL_EINVAL;
  }
  int64_t cell0 = 0;
  for (int i = 0; i < b->n; ++i) {
    const lbl_frame &f = frames[i];
    const Roadmap &r = *b->rms[i];
    const int32_t P = b->P[i];
    if (!valid_grid(&f.world, "batch frames (world)", false)) return LBL_EINVAL;
    if ((P > 0 && !f.d_planes) || !f.d_O || (r.E > 0 && !f.d_L) ||
        (b->mons[i] && r.E > 0 && (!f.d_next || !f.d_viol))) {
      set_error("batch frames: frame %d is missing a buffer", i);
      return LBL_EINVAL;
    }
    FrameMap m;
    if (!frame_map(f.world, r.agent, f.pose, &m)) return LBL_EINVAL;
    b->ftab.items[i] = frame_item(m, f.world, r.agent, f.d_planes, P, f.d_O, cell0);
    cell0 += r.cells;
    BatchItem &it = b->tabs[b->cls[i]].items[b->slot[i]];
    if (b->pyr_slot[i] >= 0)
      b->ptab.items[b->pyr_slot[i]].O = f.d_O;  // the item gathers from its pyramid
    else
      it.O = f.d_O;
    it.L = f.d_L;
    it.next = f.d_next;
    it.viol = f.d_viol;
  }
  b->ftab.total = cell0;
  // packed frames: 64-bit words at 4-word aligned offsets (vector stores)
  int64_t need = 0;
  std::vector<int64_t> woff(b->n, -1);
  for (int i = 0; i < b->n; ++i) {
    const int64_t wc = grid_cells(frames[i].world);
    if (b->P[i] > 0 && wc > 0 && wc <= kPackedWorldRatio * b->rms[i]->cells) {
      woff[i] = need;
      need += (wc + 3) / 4 * 4;
    }
  }
  if (need > b->words_cap) {
    uint64_t *w = nullptr;
    cudaError_t e = dev_alloc(&w, static_cast<size_t>(need), nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "batch frames: packed words");
    if (b->words) b->retired.push_back(b->words);
    b->words = w;
    b->words_cap = need;
  }
  PackTable &pt = b->pktab;
  pt.n = 0;
  pt.lane0[0] = 0;
  for (int i = 0; i < b->n; ++i) {
    FrameItem &fi = b->ftab.items[i];
    fi.words = nullptr;
    if (woff[i] < 0) continue;
    const int32_t P = b->P[i];
    const PackItem it{frames[i].d_planes, b->words + woff[i], grid_cells(frames[i].world), P, 8};
    pt.items[pt.n] = it;
    pt.vec[pt.n] = pack_vec_ok(it) ? 1 : 0;
    pt.lane0[pt.n + 1] = pt.lane0[pt.n] + (it.cells + 3) / 4;
    ++pt.n;
    fi.words = it.words;
    fi.word_bytes = 8;
    fi.wmask = P >= 64 ? ~0ull : ((1ull << P) - 1ull);
  }
  b->frames_set = true;
  return LBL_OK;
}

int lbl_batch_launch(lbl_batch b, uint32_t stages, lbl_stream s) {
  g_err.clear();
  if (!b || !b->frames_set || (stages & ~(LBL_STAGE_TRANSFORM | LBL_STAGE_LABEL))) {
    set_error("batch launch: NULL batch, no frames set, or unknown stages");
    return LBL_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  cudaError_t e = cudaSuccess;
  if (stages & LBL_STAGE_TRANSFORM) {
    e = launch_pack_batch(b->pktab, st);
    if (e == cudaSuccess) e = launch_frame_batch(b->ftab, b->num_sms, st);
  }
  if (e == cudaSuccess && (stages & LBL_STAGE_LABEL)) {
    e = launch_quad_pyramid_batch(b->ptab, st);
    for (int c = 0; c < kWordClasses && e == cudaSuccess; ++c)
      if (b->tabs[c].n > 0) e = launch_label_batch(b->tabs[c], b->counter + c, b->num_sms, b->ctas, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return LBL_OK;
}

int lbl_batch_free(lbl_batch b) {
  g_err.clear();
  if (!b) return LBL_OK;
  cudaDeviceSynchronize();
  cudaFree(b->part);
  cudaFree(b->counter);
  cudaFree(b->pyr);
  cudaFree(b->words);
  for (uint64_t *w : b->retired) cudaFree(w);
  delete b;
  return LBL_OK;
}

int lbl_session_create(lbl_roadmap rm, const lbl_grid *world, int32_t n_props, lbl_monitor mon,
                       const lbl_config *cfg, lbl_session *out) {
  g_err.clear();
  if (!out) {
    set_error("session create: out is NULL");
    return LBL_EINVAL;
  }
  *out = nullptr;
  if (!rm) {
    set_error("session create: NULL roadmap");
    return LBL_EINVAL;
  }
  if (!valid_grid(world, "session create (world)", false)) return LBL_EINVAL;
  if (n_props < 0 || n_props > 64) {
    set_error("session create: n_props = %d outside 0..64", n_props);
    return LBL_EINVAL;
  }
  if (!same_device(rm->device)) return LBL_EINVAL;
  lbl_session_s *ss = new (std::nothrow) lbl_session_s();
  if (!ss) {
    set_error("session create: out of host memory");
    return LBL_ENOMEM;
  }
  ss->device = rm->device;
  ss->rm = rm;
  ss->mon = mon;
  ss->world = *world;
  ss->P = n_props;
  if (cfg) {
    ss->cfg = *cfg;
    ss->has_cfg = true;
  }
  const size_t plane_bytes = static_cast<size_t>(n_props) * grid_cells(*world);
  cudaError_t e = dev_alloc(&ss->planes, 2 * plane_bytes, nullptr);
  ss->slot[0] = ss->planes;
  ss->slot[1] = ss->planes + plane_bytes;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ss->cin, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&ss->ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss->ev_free[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = dev_alloc(&ss->O, static_cast<size_t>(rm->cells), nullptr);
  if (e == cudaSuccess && static_cast<int64_t>(plane_bytes) >= kPackedMinPlaneBytes &&
      grid_cells(*world) <= kPackedWorldRatio * rm->cells)
    e = dev_alloc(&ss->words, static_cast<size_t>(grid_cells(*world)) * packed_word_bytes(n_props), nullptr);
  if (e == cudaSuccess) e = dev_alloc(&ss->L, static_cast<size_t>(2 * rm->E), nullptr);
  if (e == cudaSuccess && mon) e = dev_alloc(&ss->next, static_cast<size_t>(2 * rm->E), nullptr);
  if (e == cudaSuccess && mon) e = dev_alloc(&ss->viol, static_cast<size_t>(2 * rm->E), nullptr);
  for (int k = 0; k < 2; ++k) {
    ss->Ls[k] = ss->L ? ss->L + k * rm->E : nullptr;
    ss->Ns[k] = ss->next ? ss->next + k * rm->E : nullptr;
    ss->Vs[k] = ss->viol ? ss->viol + k * rm->E : nullptr;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ss->cc, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ss->ev_out[k], cudaEventDisableTiming);

  // Chunked labeling when the configuration resolves to a register-pipelined
  // stream (quadtree, or CSR without lane groups, early exit or copy rings) on
  // a roadmap big enough to pay.
  lbl_config c{};
  if (cfg) c = *cfg;
  if (c.algo == LBL_ALGO_AUTO && rm->tuned_valid[n_props]) c = rm->tuned[n_props];
  if (c.algo == LBL_ALGO_AUTO)  // as lbl_label resolves it
    c.algo = rm->has_qd ? LBL_ALGO_QUAD : (rm->has_bt && n_props <= 8) ? LBL_ALGO_BITTILE : LBL_ALGO_CSR;
  const bool stream_form = (c.algo == LBL_ALGO_QUAD && rm->has_qd) ||
                           (c.algo == LBL_ALGO_CSR && c.lanes_per_edge == 0 && c.early_exit <= 0 &&
                            (c.pipeline == 0 || c.pipeline == LBL_PIPE_REGISTERS));
  if (e == cudaSuccess && stream_form && rm->E >= kSessionChunkMinEdges) {
    ss->chunked = true;
    ss->quad = c.algo == LBL_ALGO_QUAD;
    if (ss->quad) e = dev_alloc(&ss->pyr, static_cast<size_t>(rm->pyr_words), nullptr);
    ss->depth = c.depth ? c.depth : (ss->quad ? kQuadDepth : 8);
    const int occ = stream_ctas_per_sm(ss->depth);
    ss->ctas = c.ctas_per_sm > 0 ? std::min(c.ctas_per_sm, occ) : occ;
    ss->warps = static_cast<int64_t>(rm->num_sms) * ss->ctas * (kThreads / 32);
    for (int c = 0; c <= kSessionChunks; ++c) ss->edge0[c] = rm->E * c / kSessionChunks;
    const int64_t *rows = ss->quad ? rm->qd_rowptr : rm->rowptr;
    e = dev_alloc(&ss->cpart, static_cast<size_t>(kSessionChunks * (ss->warps + 1)), nullptr);
    for (int c = 0; c < kSessionChunks && e == cudaSuccess; ++c)
      e = launch_partition_into(rows + ss->edge0[c], ss->edge0[c + 1] - ss->edge0[c], ss->warps,
                                ss->cpart + c * (ss->warps + 1), nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ss->cs, cudaStreamNonBlocking);
  for (int c = 0; c <= kSessionChunks && e == cudaSuccess; ++c)
    e = cudaEventCreateWithFlags(&ss->ev[c], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    lbl_session_free(ss);
    return cuda_fail(e, "session create");
  }
  *out = ss;
  return LBL_OK;
}

int lbl_session_run(lbl_session ss, const uint8_t *h_planes, lbl_pose pose, uint64_t *h_L, uint64_t *h_next,
                    uint16_t *h_viol, lbl_stream s) {
  g_err.clear();
  if (!ss) {
    set_error("session run: NULL session");
    return LBL_EINVAL;
  }
  const Roadmap &rm = *ss->rm;
  if ((ss->P > 0 && !h_planes) || (rm.E > 0 && !h_L)) {
    set_error("session run: NULL host buffer");
    return LBL_EINVAL;
  }
  if (!same_device(ss->device)) return LBL_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  // A chunked session touches only its own device memory (planes, O,
  // pyramid, partitions, outputs) besides the roadmap's read-only rows, so
  // its kernels run on its own stream `cc` and frame i+1 computes while frame
  // i's results are still being copied out.  Other sessions label through
  // lbl_label (roadmap-owned working memory), ordered on the caller's stream.
  cudaStream_t cc = ss->chunked ? ss->cc : st;
  const size_t plane_bytes = static_cast<size_t>(ss->P) * grid_cells(ss->world);
  const int k = static_cast<int>(ss->frame & 1);  // plane slot and output set of this frame
  uint64_t *dL = ss->Ls[k], *dN = ss->Ns[k];
  uint16_t *dV = ss->Vs[k];
  // planes in on `cin` once slot k is no longer read
  cudaError_t e = cudaStreamWaitEvent(ss->cin, ss->ev_free[k], 0);
  if (e == cudaSuccess && plane_bytes)
    e = cudaMemcpyAsync(ss->slot[k], h_planes, plane_bytes, cudaMemcpyHostToDevice, ss->cin);
  if (e == cudaSuccess) e = cudaEventRecord(ss->ev_in[k], ss->cin);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cc, ss->ev_in[k], 0);
  if (e != cudaSuccess) return cuda_fail(e, "session run: copy planes");
  int rc = LBL_OK;
  if (ss->words) {
    const PackItem it{ss->slot[k], ss->words, grid_cells(ss->world), ss->P, packed_word_bytes(ss->P)};
    if ((e = launch_pack_planes(it, cc)) != cudaSuccess) return cuda_fail(e, "session run: pack planes");
    rc = lbl_frame_transform_words(&ss->world, ss->words, ss->P, pose, &rm.agent, ss->O, reinterpret_cast<lbl_stream>(cc));
  } else {
    rc = lbl_frame_transform(&ss->world, ss->slot[k], ss->P, pose, &rm.agent, ss->O, reinterpret_cast<lbl_stream>(cc));
  }
  if (rc != LBL_OK) return rc;
  if ((e = cudaEventRecord(ss->ev_free[k], cc)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(cc, ss->ev_out[k], 0)) != cudaSuccess)  // output set k copied out (frame i-2)
    return cuda_fail(e, "session run: event");
  ++ss->frame;
  auto copy_out = [&](int64_t e0, int64_t n) {
    cudaError_t r = cudaMemcpyAsync(h_L + e0, dL + e0, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, ss->cs);
    if (r == cudaSuccess && ss->mon && h_next)
      r = cudaMemcpyAsync(h_next + e0, dN + e0, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, ss->cs);
    if (r == cudaSuccess && ss->mon && h_viol)
      r = cudaMemcpyAsync(h_viol + e0, dV + e0, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost, ss->cs);
    return r;
  };
  if (ss->chunked) {
    const void *base = ss->O;
    int wb = 8;
    if (ss->quad) {
      wb = quad_word_bytes(rm, ss->P);
      if ((e = launch_quad_pyramid(rm, ss->O, wb, ss->pyr, cc)) != cudaSuccess)
        return cuda_fail(e, "session run: pyramid");
      base = ss->pyr;
    }
    for (int c = 0; c < kSessionChunks; ++c) {
      const int64_t e0 = ss->edge0[c], n = ss->edge0[c + 1] - e0;
      if (n == 0) continue;
      // quadtree rows in locality order write to the caller's edges of the
      // same range: the outputs are addressed from their start, not from e0
      const int32_t *perm = ss->quad && rm.qd_perm ? rm.qd_perm + e0 : nullptr;
      const int64_t o0 = perm ? 0 : e0;
      const StreamRows r{(ss->quad ? rm.qd_rowptr : rm.rowptr) + e0, ss->quad ? rm.qd_idx : rm.colidx,
                         ss->cpart + c * (ss->warps + 1), ss->ctas, n, ss->quad ? rm.n_qd : rm.nnz, perm};
      MonitorTables t{};
      if (ss->mon) t = tables_of(*ss->mon, dN + o0, dV + o0);
      e = launch_label_rows(r, base, wb, ss->P, dL + o0, ss->mon ? &t : nullptr, ss->depth, rm.num_sms, cc);
      if (e == cudaSuccess) e = cudaEventRecord(ss->ev[c], cc);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->cs, ss->ev[c], 0);
      if (e == cudaSuccess) e = copy_out(e0, n);
      if (e != cudaSuccess) return cuda_fail(e, "session run: chunk");
    }
  } else {
    rc = label_impl(ss->rm, ss->O, ss->P, dL, ss->mon, dN, dV, ss->has_cfg ? &ss->cfg : nullptr, cc);
    if (rc != LBL_OK) return rc;
    if ((e = cudaEventRecord(ss->ev[0], cc)) != cudaSuccess || (e = cudaStreamWaitEvent(ss->cs, ss->ev[0], 0)) != cudaSuccess ||
        (rm.E > 0 && (e = copy_out(0, rm.E)) != cudaSuccess))
      return cuda_fail(e, "session run: copy results");
  }
  // output set k is free again once its copies land; the caller's stream sees
  // the whole frame (copies in, kernels, copies out) before its next work
  if ((e = cudaEventRecord(ss->ev_out[k], ss->cs)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, ss->ev_out[k], 0)) != cudaSuccess)
    return cuda_fail(e, "session run: join");
  return LBL_OK;
}

int lbl_session_free(lbl_session ss) {
  g_err.clear();
  if (!ss) return LBL_OK;
  cudaDeviceSynchronize();
  cudaFree(ss->planes);
  cudaFree(ss->O);
  cudaFree(ss->L);
  cudaFree(ss->next);
  cudaFree(ss->viol);
  cudaFree(ss->cpart);
  if (ss->cs) cudaStreamDestroy(ss->cs);
  if (ss->cin) cudaStreamDestroy(ss->cin);
  if (ss->cc) cudaStreamDestroy(ss->cc);
  for (int k = 0; k < 2; ++k)
    if (ss->ev_out[k]) cudaEventDestroy(ss->ev_out[k]);
  cudaFree(ss->pyr);
  cudaFree(ss->words);
  for (cudaEvent_t ev : ss->ev)
    if (ev) cudaEventDestroy(ev);
  for (int k = 0; k < 2; ++k) {
    if (ss->ev_in[k]) cudaEventDestroy(ss->ev_in[k]);
    if (ss->ev_free[k]) cudaEventDestroy(ss->ev_free[k]);
  }
  delete ss;
  return LBL_OK;
}

}  // extern "C"
