// Roadmap rows built on the device (lbl_roadmap_rasterize): the swept set of
// eq. 7 with a closed disc footprint (eq. 5), discretised by cell centres as in
// Sec. 4.1.  Membership is a distance test; to take it exactly as the CPU
// definition does, the arc geometry (which needs sin/cos) is computed on the
// host, and every decision near the footprint boundary is evaluated in fp64
// with explicitly rounded operations in a fixed order.  Cells far from the
// boundary are screened in fp32 (1 mm margin), which decides almost all.
#include <cmath>
#include <vector>

#include "lbl_internal.cuh"

namespace lbl {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kMargin = 1e-3f;  // fp32 screen: undecided within 1 mm of the radius

struct RArc {
  double g[12];     // straight {1, x, y, cos, sin, len}; circle {0, cx, cy, R, sgn, u0, u1, end, class}
  double ax, ay;    // start point
  int32_t i0, i1, j0, j1;  // candidate cell box (inclusive), empty if i0 > i1
  int32_t exact;    // 1 = decide every cell in fp64 (large radii of curvature)
  int32_t pad;
};

// --- host: geometry exactly as the CPU definition computes it --------------
void arc_geometry(const double *a, double *g) {
  const double x = a[0], y = a[1], th = a[2], k = a[3], len = a[4];
  for (int i = 0; i < 12; ++i) g[i] = 0.0;
  if (std::fabs(k) < 1e-9 || !(len > 0.0)) {  // a segment, or a zero-length arc: its start point
    g[0] = 1.0;
    g[1] = x;
    g[2] = y;
    g[3] = std::cos(th);
    g[4] = std::sin(th);
    g[5] = len;
    return;
  }
  const double inv = 1.0 / k;
  const double sg = k > 0 ? 1.0 : -1.0;
  const double cx = x - inv * std::sin(th);
  const double cy = y + inv * std::cos(th);
  const double th1 = th + k * len;
  const double sweep = std::fabs(k * len);
  g[0] = 0.0;
  g[1] = cx;
  g[2] = cy;
  g[3] = std::fabs(inv);
  g[4] = sg;
  g[5] = sg * std::sin(th);
  g[6] = -sg * std::cos(th);
  g[7] = sg * std::sin(th1);
  g[8] = -sg * std::cos(th1);
  g[9] = cx + inv * std::sin(th1);
  g[10] = cy - inv * std::cos(th1);
  g[11] = sweep >= 2.0 * M_PI ? 2.0 : (sweep > M_PI ? 1.0 : 0.0);
}

bool in_sector(const double *g, double wx, double wy) {
  if (g[11] == 2.0) return true;
  if (g[11] == 0.0)
    return g[4] * (g[5] * wy - g[6] * wx) >= 0.0 && g[4] * (wx * g[8] - wy * g[7]) >= 0.0;
  return !(g[4] * (g[7] * wy - g[8] * wx) > 0.0 && g[4] * (wx * g[6] - wy * g[5]) > 0.0);
}

// Conservative candidate box: the arc's extent (end points and the circle's
// axis-extreme points inside the sweep) grown by radius + one cell.
void arc_box(const RArc &r, const double *a, const lbl_grid &G, double radius, RArc *out) {
  const double *g = r.g;
  double lx = a[0], hx = a[0], ly = a[1], hy = a[1];
  auto add = [&](double x, double y) {
    lx = std::fmin(lx, x);
    hx = std::fmax(hx, x);
    ly = std::fmin(ly, y);
    hy = std::fmax(hy, y);
  };
  if (g[0] == 1.0) {
    add(a[0] + g[5] * g[3], a[1] + g[5] * g[4]);
  } else {
    add(g[9], g[10]);
    const double R = g[3];
    const double ex[4][2] = {{R, 0.0}, {0.0, R}, {-R, 0.0}, {0.0, -R}};
    for (auto &p : ex)
      if (in_sector(g, p[0], p[1])) add(g[1] + p[0], g[2] + p[1]);
  }
  const double m = radius + G.res + 1e-6;
  auto cell = [&](double v, double o) { return std::floor((v - o) / G.res); };
  const double i0 = cell(lx - m, G.x0), i1 = cell(hx + m, G.x0), j0 = cell(ly - m, G.y0), j1 = cell(hy + m, G.y0);
  out->i0 = static_cast<int32_t>(std::fmax(0.0, i0));
  out->i1 = static_cast<int32_t>(std::fmin(G.w - 1.0, i1));
  out->j0 = static_cast<int32_t>(std::fmax(0.0, j0));
  out->j1 = static_cast<int32_t>(std::fmin(G.h - 1.0, j1));
  if (i1 < 0 || j1 < 0 || i0 > G.w - 1 || j0 > G.h - 1) out->i0 = 1, out->i1 = 0;  // empty
  out->exact = (g[0] == 0.0 && g[3] > 100.0) ? 1 : 0;
}

// --- device -----------------------------------------------------------------
// The distance of the CPU definition, operation by operation, correctly rounded.
__device__ __forceinline__ double dist64(const RArc &r, double px, double py) {
  const double *g = r.g;
  if (g[0] == 1.0) {
    double t = __dadd_rn(__dmul_rn(__dsub_rn(px, g[1]), g[3]), __dmul_rn(__dsub_rn(py, g[2]), g[4]));
    if (t < 0.0) t = 0.0;
    if (t > g[5]) t = g[5];
    const double ex = __dsub_rn(__dsub_rn(px, g[1]), __dmul_rn(t, g[3]));
    const double ey = __dsub_rn(__dsub_rn(py, g[2]), __dmul_rn(t, g[4]));
    return __dsqrt_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
  }
  const double wx = __dsub_rn(px, g[1]), wy = __dsub_rn(py, g[2]);
  const double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy)));
  bool inside = true;
  if (g[11] != 2.0 && rho > 0.0) {
    if (g[11] == 0.0) {
      const double c0 = __dmul_rn(g[4], __dsub_rn(__dmul_rn(g[5], wy), __dmul_rn(g[6], wx)));
      const double c1 = __dmul_rn(g[4], __dsub_rn(__dmul_rn(wx, g[8]), __dmul_rn(wy, g[7])));
      inside = c0 >= 0.0 && c1 >= 0.0;
    } else {
      const double c0 = __dmul_rn(g[4], __dsub_rn(__dmul_rn(g[7], wy), __dmul_rn(g[8], wx)));
      const double c1 = __dmul_rn(g[4], __dsub_rn(__dmul_rn(wx, g[6]), __dmul_rn(wy, g[5])));
      inside = !(c0 > 0.0 && c1 > 0.0);
    }
  }
  if (inside) return fabs(__dsub_rn(rho, g[3]));
  const double ax = __dsub_rn(px, r.ax), ay = __dsub_rn(py, r.ay);
  const double bx = __dsub_rn(px, g[9]), by = __dsub_rn(py, g[10]);
  const double d0 = __dsqrt_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)));
  const double d1 = __dsqrt_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)));
  return d0 < d1 ? d0 : d1;
}

// fp32 screen of the same distance in coordinates relative to the start point.
struct Arc32 {
  bool straight;
  int cls;
  float dx, dy, len, cx, cy, R, sg, u0x, u0y, u1x, u1y, bx, by;
};

__device__ __forceinline__ Arc32 to32(const RArc &r) {
  const double *g = r.g;
  Arc32 f{};
  f.straight = g[0] == 1.0;
  if (f.straight) {
    f.dx = static_cast<float>(g[3]);
    f.dy = static_cast<float>(g[4]);
    f.len = static_cast<float>(g[5]);
  } else {
    f.cx = static_cast<float>(g[1] - r.ax);
    f.cy = static_cast<float>(g[2] - r.ay);
    f.R = static_cast<float>(g[3]);
    f.sg = static_cast<float>(g[4]);
    f.u0x = static_cast<float>(g[5]);
    f.u0y = static_cast<float>(g[6]);
    f.u1x = static_cast<float>(g[7]);
    f.u1y = static_cast<float>(g[8]);
    f.bx = static_cast<float>(g[9] - r.ax);
    f.by = static_cast<float>(g[10] - r.ay);
    f.cls = static_cast<int>(g[11]);
  }
  return f;
}

// Explicitly rounded fp32 operations: the count and fill passes evaluate the
// screen identically, never contracted.
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }

__device__ __forceinline__ float dist32(const Arc32 &f, float px, float py) {
  if (f.straight) {
    const float t = fminf(fmaxf(fa(fm(px, f.dx), fm(py, f.dy)), 0.f), f.len);
    const float ex = fs(px, fm(t, f.dx)), ey = fs(py, fm(t, f.dy));
    return __fsqrt_rn(fa(fm(ex, ex), fm(ey, ey)));
  }
  const float wx = fs(px, f.cx), wy = fs(py, f.cy);
  const float rho = __fsqrt_rn(fa(fm(wx, wx), fm(wy, wy)));
  bool inside = true;
  if (f.cls != 2) {
    if (f.cls == 0)
      inside = fm(f.sg, fs(fm(f.u0x, wy), fm(f.u0y, wx))) >= 0.f && fm(f.sg, fs(fm(wx, f.u1y), fm(wy, f.u1x))) >= 0.f;
    else
      inside = !(fm(f.sg, fs(fm(f.u1x, wy), fm(f.u1y, wx))) > 0.f && fm(f.sg, fs(fm(wx, f.u0y), fm(wy, f.u0x))) > 0.f);
  }
  if (inside) return fabsf(fs(rho, f.R));
  const float d0 = __fsqrt_rn(fa(fm(px, px), fm(py, py)));
  const float qx = fs(px, f.bx), qy = fs(py, f.by);
  const float d1 = __fsqrt_rn(fa(fm(qx, qx), fm(qy, qy)));
  return fminf(d0, d1);
}

struct RGrid {
  int32_t w, h, morton;
  double res, x0, y0, radius;
};

__device__ __forceinline__ bool member(const RArc &r, const Arc32 &f, const RGrid &G, int ix, int iy) {
  const double cx = __dadd_rn(G.x0, __dmul_rn(static_cast<double>(ix) + 0.5, G.res));
  const double cy = __dadd_rn(G.y0, __dmul_rn(static_cast<double>(iy) + 0.5, G.res));
  if (!r.exact) {
    const float d = dist32(f, static_cast<float>(cx - r.ax), static_cast<float>(cy - r.ay));
    const float rr = static_cast<float>(G.radius);
    if (d < rr - kMargin) return true;
    if (d > rr + kMargin) return false;
  }
  return dist64(r, cx, cy) <= G.radius;
}

__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return static_cast<uint32_t>(x);
}

// One warp per arc.  Cells are visited in increasing cell index, so each row
// comes out sorted: row-major scans rows of the candidate box 32 columns at a
// time; z-order walks the 32-code blocks (4 x 8 cells) between the box's
// corner codes, each lane rejecting one block against the box and the fp32
// distance bound, then tests the surviving blocks' cells.
template <bool FILL>
__global__ void __launch_bounds__(256) k_raster(const RArc *__restrict__ arcs, int64_t E, RGrid G,
                                                int64_t *__restrict__ counts, const int64_t *__restrict__ rowptr,
                                                int32_t *__restrict__ colidx) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t e = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; e < E; e += nw) {
    const RArc r = arcs[e];
    const Arc32 f = to32(r);
    int64_t n = 0;
    int64_t out = FILL ? rowptr[e] : 0;
    const int64_t end = FILL ? rowptr[e + 1] : 0;  // writes never pass the counted row
    if (r.i0 <= r.i1 && r.j0 <= r.j1) {
      if (!G.morton) {
        for (int j = r.j0; j <= r.j1; ++j)
          for (int ib = r.i0; ib <= r.i1; ib += 32) {
            const int ix = ib + lane;
            const bool in = ix <= r.i1 && member(r, f, G, ix, j);
            const unsigned m = __ballot_sync(kFull, in);
            if (FILL && in && out + __popc(m & lt) < end) colidx[out + __popc(m & lt)] = j * G.w + ix;
            out += __popc(m);
            n += __popc(m);
          }
      } else {
        const uint32_t lo = (spread_bits(r.i0) << 1 | spread_bits(r.j0)) >> 5;
        const uint32_t hi = (spread_bits(r.i1) << 1 | spread_bits(r.j1)) >> 5;
        const float rr = static_cast<float>(G.radius);
        const float hd = static_cast<float>(G.res) * 4.5f;  // half diagonal of a 4 x 8 block, rounded up
        for (uint32_t b0 = lo; b0 <= hi; b0 += 32) {
          const uint32_t b = b0 + lane;
          bool keep = false;
          if (b <= hi) {
            const uint64_t code = static_cast<uint64_t>(b) << 5;
            const int bx = static_cast<int>(gather_even_bits(code >> 1));
            const int by = static_cast<int>(gather_even_bits(code));
            keep = bx + 3 >= r.i0 && bx <= r.i1 && by + 7 >= r.j0 && by <= r.j1;
            if (keep && !r.exact) {
              const double cx = G.x0 + (bx + 2.0) * G.res, cy = G.y0 + (by + 4.0) * G.res;
              keep = dist32(f, static_cast<float>(cx - r.ax), static_cast<float>(cy - r.ay)) <= rr + hd + kMargin;
            }
          }
          unsigned todo = __ballot_sync(kFull, keep);
          while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint64_t code = (static_cast<uint64_t>(b0 + l) << 5) + lane;
            const int ix = static_cast<int>(gather_even_bits(code >> 1));
            const int iy = static_cast<int>(gather_even_bits(code));
            const bool in = ix >= r.i0 && ix <= r.i1 && iy >= r.j0 && iy <= r.j1 && member(r, f, G, ix, iy);
            const unsigned m = __ballot_sync(kFull, in);
            if (FILL && in && out + __popc(m & lt) < end) colidx[out + __popc(m & lt)] = static_cast<int32_t>(code);
            out += __popc(m);
            n += __popc(m);
          }
          if (b0 > 0xFFFFFFFFu - 32) break;
        }
      }
    }
    if (!FILL && lane == 0) counts[e] = n;
  }
}

}  // namespace
}  // namespace lbl

using namespace lbl;

extern "C" int lbl_roadmap_rasterize(const lbl_grid *agent, const double *h_arcs, int64_t n_edges, double radius,
                                     uint32_t flags, lbl_stream s, lbl_roadmap *out) {
  set_error("%s", "");
  if (!out) {
    set_error("rasterize: out is NULL");
    return LBL_EINVAL;
  }
  *out = nullptr;
  if (!valid_grid(agent, "rasterize", true)) return LBL_EINVAL;
  if (grid_depth(*agent) > 1) {
    set_error("rasterize: time-augmented grids are not rasterised on the device (upload their rows)");
    return LBL_EUNSUPPORTED;
  }
  if (n_edges < 0 || (n_edges > 0 && !h_arcs) || !(radius > 0.0) || !std::isfinite(radius)) {
    set_error("rasterize: need n_edges >= 0, arcs and a positive radius");
    return LBL_EINVAL;
  }
  if (flags & ~(LBL_UPLOAD_BITTILE | LBL_UPLOAD_SECTOR | LBL_UPLOAD_QUAD | LBL_UPLOAD_KEEP_ORDER)) {
    set_error("rasterize: unknown flags 0x%x", flags);
    return LBL_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  std::vector<RArc> arcs(static_cast<size_t>(n_edges));
  for (int64_t e = 0; e < n_edges; ++e) {
    const double *a = h_arcs + 5 * e;
    for (int i = 0; i < 5; ++i)
      if (!std::isfinite(a[i]) || (i == 4 && a[i] < 0)) {
        set_error("rasterize: arc %lld is not finite or has a negative length", static_cast<long long>(e));
        return LBL_EINVAL;
      }
    RArc &r = arcs[e];
    arc_geometry(a, r.g);
    r.ax = a[0];
    r.ay = a[1];
    arc_box(r, a, *agent, radius, &r);
  }
  const RGrid G{agent->w, agent->h, agent->order == LBL_ORDER_MORTON, agent->res, agent->x0, agent->y0, radius};
  RArc *d_arcs = nullptr;
  int64_t *d_counts = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&d_arcs), sizeof(RArc) * (n_edges ? n_edges : 1));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&d_counts), sizeof(int64_t) * (n_edges + 1));
  if (e == cudaSuccess && n_edges)
    e = cudaMemcpyAsync(d_arcs, arcs.data(), sizeof(RArc) * n_edges, cudaMemcpyHostToDevice, st);
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  const int64_t warps = n_edges;
  int64_t blocks = (warps + 7) / 8;
  const int64_t cap = static_cast<int64_t>(device_sms(dev)) * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (e == cudaSuccess && n_edges) {
    k_raster<false><<<static_cast<unsigned>(blocks), 256, 0, st>>>(d_arcs, n_edges, G, d_counts, nullptr, nullptr);
    e = cudaGetLastError();
  }
  std::vector<int64_t> rowptr(static_cast<size_t>(n_edges + 1), 0);
  if (e == cudaSuccess && n_edges)
    e = cudaMemcpyAsync(rowptr.data() + 1, d_counts, sizeof(int64_t) * n_edges, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(d_arcs);
    cudaFree(d_counts);
    return cuda_fail(e, "rasterize: count");
  }
  for (int64_t i = 0; i < n_edges; ++i) rowptr[i + 1] += rowptr[i];
  const int64_t nnz = rowptr[n_edges];
  if (nnz > 2147483647LL * 4) {
    cudaFree(d_arcs);
    cudaFree(d_counts);
    set_error("rasterize: %lld swept cells exceed the roadmap limit", static_cast<long long>(nnz));
    return LBL_EINVAL;
  }
  lbl_roadmap_s *rm = nullptr;
  int rc = roadmap_new(*agent, n_edges, nnz, &rm);
  if (rc != LBL_OK) {
    cudaFree(d_arcs);
    cudaFree(d_counts);
    return rc;
  }
  e = cudaMemcpyAsync(rm->rowptr, rowptr.data(), sizeof(int64_t) * (n_edges + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_edges) {
    k_raster<true><<<static_cast<unsigned>(blocks), 256, 0, st>>>(d_arcs, n_edges, G, nullptr, rm->rowptr,
                                                                   rm->colidx);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_arcs);
  cudaFree(d_counts);
  if (e != cudaSuccess) {
    free_roadmap(rm);
    return cuda_fail(e, "rasterize: fill");
  }
  rc = roadmap_finish(rm, flags, st);
  if (rc == LBL_OK) *out = rm;
  return rc;
}
