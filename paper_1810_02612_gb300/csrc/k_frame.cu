// Frame transform (equivariant re-use of the roadmap, Sec. 5 / eq. 13) and the
// stand-alone safety-monitor step (Sec. 3.2).
#include "lbl_internal.cuh"

namespace lbl {
namespace {

template <int WB> struct WordOf;
template <> struct WordOf<1> { using T = uint8_t; };
template <> struct WordOf<2> { using T = uint16_t; };
template <> struct WordOf<4> { using T = uint32_t; };
template <> struct WordOf<8> { using T = uint64_t; };

// Plane bytes a thread has in flight in the byte-gather transform: with 16
// rather than 8 the small grids, whose few threads wait on each batch in turn,
// transform faster (driving 9.1 -> 8.4 us; 32 is no better; large grids unchanged).
constexpr int kPlaneBatch = 16;

// Grids have at most 32768 cells a side and fewer than 2^31 cells (checked on
// the host), so cell indices and coordinates are 32-bit throughout.

// Every third / every second bit of a z-order index, packed: the inverse of
// the 3-D / 2-D bit interleave for one coordinate.
__device__ __forceinline__ uint32_t third_bits(uint32_t v) {
  v &= 0x49249249u;
  v = (v | (v >> 2)) & 0xC30C30C3u;
  v = (v | (v >> 4)) & 0x0F00F00Fu;
  v = (v | (v >> 8)) & 0xFF0000FFu;
  return (v | (v >> 16)) & 0x000007FFu;
}
__device__ __forceinline__ uint32_t even_bits(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  return (v | (v >> 8)) & 0x0000FFFFu;
}

// Coordinates (ix, iy, it) of agent cell idx of frame f in the grid's order.
__device__ __forceinline__ void agent_coords(const FrameItem &f, uint32_t idx, uint32_t &ix, uint32_t &iy,
                                             uint32_t &it) {
  it = 0;
  if (f.order == LBL_ORDER_MORTON) {
    if (f.ad > 1) {
      ix = third_bits(idx >> 2);
      iy = third_bits(idx >> 1);
      it = third_bits(idx);
    } else {
      ix = even_bits(idx >> 1);
      iy = even_bits(idx);
    }
  } else {
    const uint32_t aw = static_cast<uint32_t>(f.aw), plane = aw * static_cast<uint32_t>(f.ah);
    it = idx / plane;
    const uint32_t r = idx - it * plane;
    iy = r / aw;
    ix = r - iy * aw;
  }
}

// Word of world cell c (row-major, time slabs outermost) of frame f: WB = 0
// reads the P planes, WB = 1, 2, 4 or 8 reads packed words that wide.
template <int WB>
__device__ __forceinline__ uint64_t cell_word(const FrameItem &f, uint32_t c) {
  uint64_t word = 0;
  if constexpr (WB > 0) {
    word = static_cast<uint64_t>(__ldg(static_cast<const typename WordOf<WB>::T *>(f.words) + c)) & f.wmask;
  } else {
    const uint8_t *p = f.planes + c;
    int q = 0;
    for (; q + kPlaneBatch <= f.P; q += kPlaneBatch) {
      uint8_t b[kPlaneBatch];
#pragma unroll
      for (int j = 0; j < kPlaneBatch; ++j) b[j] = __ldg(p + (q + j) * f.plane_cells);
#pragma unroll
      for (int j = 0; j < kPlaneBatch; ++j) word |= static_cast<uint64_t>(b[j] != 0) << (q + j);
    }
    for (; q + 8 <= f.P; q += 8) {
      uint8_t b[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = __ldg(p + (q + j) * f.plane_cells);
#pragma unroll
      for (int j = 0; j < 8; ++j) word |= static_cast<uint64_t>(b[j] != 0) << (q + j);
    }
    for (; q < f.P; ++q) word |= static_cast<uint64_t>(__ldg(p + q * f.plane_cells) != 0) << q;
  }
  return word;
}

// World word of agent cell (ix, iy, it) of frame f (2-D or time-augmented).
// The world cell is the floor (arithmetic shift) of exact Q32.32 affine maps
// of (ix, iy) and of the slab it; coordinates zero-extend to 64 bits.
template <int WB>
__device__ __forceinline__ uint64_t world_word(const FrameItem &f, uint32_t ix, uint32_t iy, uint32_t it) {
  const int64_t x = ix, y = iy;
  const int64_t wx = (f.A00 * x + f.A01 * y + f.B0) >> 32;
  const int64_t wy = (f.A10 * x + f.A11 * y + f.B1) >> 32;
  const int64_t wt = f.wd > 1 ? ((f.At * static_cast<int64_t>(it) + f.Bt) >> 32) : 0;  // a 2-D world is static
  if (wx >= 0 && wx < f.ww && wy >= 0 && wy < f.wh && wt >= 0 && wt < f.wd) {
    const uint32_t c = (static_cast<uint32_t>(wt) * static_cast<uint32_t>(f.wh) + static_cast<uint32_t>(wy)) *
                           static_cast<uint32_t>(f.ww) +
                       static_cast<uint32_t>(wx);
    return cell_word<WB>(f, c);
  }
  return 0;
}

template <int WB>
__device__ __forceinline__ uint64_t frame_word(const FrameItem &f, uint32_t idx) {
  uint32_t ix, iy, it;
  agent_coords(f, idx, ix, iy, it);
  return world_word<WB>(f, ix, iy, it);
}

// z-order grids: a thread per agent cell in cell order (a warp's 32 cells are
// a 4 x 8 tile and its O stores coalesce).
template <int WB>
__global__ void __launch_bounds__(256) k_frame_z(const __grid_constant__ FrameItem f, uint32_t n) {
  pdl_wait();
  pdl_trigger();
  const uint32_t idx = blockIdx.x * 256u + threadIdx.x;
  if (idx < n) f.O[idx] = frame_word<WB>(f, idx);
}

// z-order grids with the quadtree pyramid: a CTA's 256 cells are one block
// of the pyramid's top level, so the words each thread computes go to O (when
// asked for) and to the pyramid's level 0, and the CTA ORs levels 1-4 from the
// same registers: no O re-read and no pyramid launch before the labels.
// On a row-major 2-D grid in the quadtree form's tiled order (tiled_w > 0) a
// CTA is one 16 x 16 tile: its words go to the tile's cells of the row-major O
// and, in the tile's z-order, to the pyramid.
template <int WB, typename T>
__global__ void __launch_bounds__(256) k_frame_z_pyramid(const __grid_constant__ FrameItem f, uint32_t n,
                                                         const __grid_constant__ QuadOffsets off, T *__restrict__ pyr,
                                                         int32_t tiled_w) {
  __shared__ uint64_t wsum[kThreads / 32];
  pdl_wait();
  pdl_trigger();
  const uint32_t idx = blockIdx.x * 256u + threadIdx.x;
  uint64_t v = 0;
  if (tiled_w > 0) {  // n is a multiple of 256: every thread has a cell
    uint32_t ix, iy;
    tiled_cell(tiled_w, blockIdx.x, threadIdx.x, ix, iy);
    v = world_word<WB>(f, ix, iy, 0);
    if (f.O) f.O[iy * static_cast<uint32_t>(f.aw) + ix] = v;
  } else if (idx < n) {
    v = frame_word<WB>(f, idx);
    if (f.O) f.O[idx] = v;
  }
  quad_pyramid_of<T>(v, n, off, pyr, blockIdx.x, wsum);
}

// Row-major grids: a warp per 8 x 4 tile of one slab (grid: x tiles / 8, y
// tiles, slabs), so under any rotation a warp's world reads stay within a few
// rows (a warp along one row would read a rotated line of up to 32 world
// rows); the tile's O stores are four 64-byte runs.
template <int WB>
__global__ void __launch_bounds__(256) k_frame_tiles(const __grid_constant__ FrameItem f) {
  pdl_wait();
  pdl_trigger();
  const uint32_t xt = blockIdx.x * 8u + (threadIdx.x >> 5), lane = threadIdx.x & 31u;
  const uint32_t ix = 8u * xt + (lane & 7u), iy = 4u * blockIdx.y + (lane >> 3), it = blockIdx.z;
  if (ix >= static_cast<uint32_t>(f.aw) || iy >= static_cast<uint32_t>(f.ah)) return;
  f.O[(it * static_cast<uint32_t>(f.ah) + iy) * static_cast<uint32_t>(f.aw) + ix] = world_word<WB>(f, ix, iy, it);
}

// Batched frame transform: thread per (frame, agent cell) over all frames'
// cells; the frame is found by binary search over the items' first cells.
__global__ void __launch_bounds__(256) k_frame_batch(const __grid_constant__ FrameTable tab) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t gidx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; gidx < tab.total;
       gidx += stride) {
    int lo = 0, hi = tab.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (tab.items[mid].cell0 <= gidx)
        lo = mid;
      else
        hi = mid - 1;
    }
    const FrameItem &f = tab.items[lo];
    const uint32_t idx = static_cast<uint32_t>(gidx - f.cell0);
    f.O[idx] = f.words ? frame_word<8>(f, idx) : frame_word<0>(f, idx);  // packed items: 64-bit words
  }
}

// Packing: a lane per four consecutive world cells.  For each plane the lane
// reads its cells' four bytes (one 4-byte load when the planes allow it), so a
// warp reads a whole 128-byte line of a plane per load instruction and NB
// planes are in flight per lane.  "byte != 0" becomes bit 7 of each byte
// without carries between bytes, and the plane loop is unrolled so the bit
// moves to position p of the cell's word by constant shifts.  Each lane stores
// its four words as one vector (two for 8-byte words) when VEC holds.
template <int WB, bool VEC>
__device__ __forceinline__ void pack_lane(const PackItem &it, int64_t lane) {
  using T = typename WordOf<WB>::T;
  constexpr int NB = WB == 8 || WB == 4 ? 32 : 8 * WB;  // planes per batch of loads
  constexpr int PMAX = 8 * WB;
  const int64_t c0 = 4 * lane;
  if (c0 >= it.cells) return;
  uint32_t lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
#pragma unroll
  for (int b = 0; b < PMAX / NB; ++b) {
    if (b * NB >= it.P) break;
    uint32_t v[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int p = b * NB + i;
      uint32_t x = 0;
      if (p < it.P) {
        const uint8_t *pl = it.planes + p * it.cells + c0;
        if (VEC) {
          x = __ldg(reinterpret_cast<const uint32_t *>(pl));
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c0 + j < it.cells) x |= static_cast<uint32_t>(__ldg(pl + j)) << (8 * j);
        }
      }
      v[i] = x;
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const uint32_t x = v[i];
      const uint32_t nz = (((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
      const int p = b * NB + i;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t bit = (nz >> (8 * k + 7)) & 1u;
        if (p < 32)
          lo[k] |= bit << p;
        else
          hi[k] |= bit << (p - 32);
      }
    }
  }
  T *w = static_cast<T *>(it.words) + c0;
  if (VEC) {
    if constexpr (WB == 8) {
      reinterpret_cast<uint4 *>(w)[0] = make_uint4(lo[0], hi[0], lo[1], hi[1]);
      reinterpret_cast<uint4 *>(w)[1] = make_uint4(lo[2], hi[2], lo[3], hi[3]);
    } else if constexpr (WB == 4) {
      *reinterpret_cast<uint4 *>(w) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    } else if constexpr (WB == 2) {
      *reinterpret_cast<uint2 *>(w) = make_uint2(lo[0] | (lo[1] << 16), lo[2] | (lo[3] << 16));
    } else {
      *reinterpret_cast<uint32_t *>(w) = lo[0] | (lo[1] << 8) | (lo[2] << 16) | (lo[3] << 24);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (c0 + k < it.cells) w[k] = static_cast<T>(lo[k] | (static_cast<uint64_t>(hi[k]) << 32));
  }
}

template <int WB, bool VEC>
__global__ void __launch_bounds__(256) k_pack_planes(const __grid_constant__ PackItem it) {
  pdl_wait();
  pdl_trigger();
  pack_lane<WB, VEC>(it, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
}

// Batched packing: the item of a lane by binary search over the items' first
// lanes; every item packs into 64-bit words.
__global__ void __launch_bounds__(256) k_pack_batch(const __grid_constant__ PackTable tab) {
  const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= tab.lane0[tab.n]) return;
  int lo = 0, hi = tab.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (tab.lane0[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  if (tab.vec[lo])
    pack_lane<8, true>(tab.items[lo], g - tab.lane0[lo]);
  else
    pack_lane<8, false>(tab.items[lo], g - tab.lane0[lo]);
}

// letter = sum_j bit(L, rel[j]) << j ; next/viol from the per-letter tables.
__global__ void __launch_bounds__(256) k_monitor_step(MonitorTables mon, const uint64_t *__restrict__ L, int64_t n) {
  __shared__ uint64_t sT[256];
  __shared__ uint16_t sV[256];
  const int letters = 1 << mon.m;
  for (int i = threadIdx.x; i < letters; i += blockDim.x) {
    sT[i] = mon.T[i];
    sV[i] = mon.V[i];
  }
  __syncthreads();
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t w = L[i];
    uint32_t letter = 0;
    for (int j = 0; j < mon.m; ++j) letter |= static_cast<uint32_t>((w >> mon.rel[j]) & 1u) << j;
    mon.next[i] = sT[letter];
    mon.viol[i] = sV[letter];
  }
}

}  // namespace

template <int WB>
static void transform_launch(const FrameItem &f, cudaStream_t s) {
  const uint32_t n = static_cast<uint32_t>(f.aw) * static_cast<uint32_t>(f.ah) * static_cast<uint32_t>(f.ad);
  if (f.order == LBL_ORDER_MORTON) {
    pdl_launch(k_frame_z<WB>, dim3((n + 255u) / 256u), dim3(256), s, f, n);
  } else {  // at most 32768 / 4 tile rows and 32768 slabs: within the grid's y and z limits
    const dim3 grid((static_cast<unsigned>(f.aw) + 63u) / 64u, (static_cast<unsigned>(f.ah) + 3u) / 4u,
                    static_cast<unsigned>(f.ad));
    pdl_launch(k_frame_tiles<WB>, grid, dim3(256), s, f);
  }
}

cudaError_t launch_frame_transform(const FrameItem &f, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(f.aw) * f.ah * f.ad;
  if (n == 0) return cudaSuccess;
  if (n >= (1ll << 31) || f.plane_cells >= (1ll << 31)) return cudaErrorInvalidValue;  // grids are checked on the host
  switch (f.words ? f.word_bytes : 0) {
    case 0: transform_launch<0>(f, s); break;
    case 1: transform_launch<1>(f, s); break;
    case 2: transform_launch<2>(f, s); break;
    case 4: transform_launch<4>(f, s); break;
    case 8: transform_launch<8>(f, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int WB, typename T>
static cudaError_t transform_pyramid_launch(const FrameItem &f, const QuadOffsets &off, void *pyr, int32_t tiled_w,
                                            cudaStream_t s) {
  const uint32_t n = static_cast<uint32_t>(f.aw) * static_cast<uint32_t>(f.ah) * static_cast<uint32_t>(f.ad);
  return pdl_launch(k_frame_z_pyramid<WB, T>, dim3((n + 255u) / 256u), dim3(256), s, f, n, off, static_cast<T *>(pyr),
                    tiled_w);
}

template <int WB>
static cudaError_t transform_pyramid_width(const FrameItem &f, const QuadOffsets &off, int pyr_bytes, void *pyr,
                                           int32_t tiled_w, cudaStream_t s) {
  using W = typename WordOf<WB>::T;
  if (pyr_bytes == WB) return transform_pyramid_launch<WB, W>(f, off, pyr, tiled_w, s);
  if (pyr_bytes == 8) return transform_pyramid_launch<WB, uint64_t>(f, off, pyr, tiled_w, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_frame_transform_pyramid(const FrameItem &f, const QuadOffsets &off, int pyr_bytes, void *pyr,
                                           int32_t tiled_w, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(f.aw) * f.ah * f.ad;
  if (n == 0) return cudaSuccess;
  if (n >= (1ll << 31) || f.plane_cells >= (1ll << 31)) return cudaErrorInvalidValue;  // grids are checked on the host
  if (!f.words) return cudaErrorInvalidValue;
  if (tiled_w > 0) {  // a row-major 2-D grid of whole 16 x 16 tiles
    if (f.order != LBL_ORDER_ROWMAJOR || f.ad != 1 || f.aw != tiled_w || f.aw % 16 || f.ah % 16)
      return cudaErrorInvalidValue;
  } else if (f.order != LBL_ORDER_MORTON) {
    return cudaErrorInvalidValue;
  }
  cudaError_t e;
  switch (f.word_bytes) {
    case 1: e = transform_pyramid_width<1>(f, off, pyr_bytes, pyr, tiled_w, s); break;
    case 2: e = transform_pyramid_width<2>(f, off, pyr_bytes, pyr, tiled_w, s); break;
    case 4: e = transform_pyramid_width<4>(f, off, pyr_bytes, pyr, tiled_w, s); break;
    case 8: e = transform_pyramid_width<8>(f, off, pyr_bytes, pyr, tiled_w, s); break;
    default: return cudaErrorInvalidValue;
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int WB>
static void pack_launch(const PackItem &it, bool vec, unsigned blocks, cudaStream_t s) {
  if (vec)
    pdl_launch(k_pack_planes<WB, true>, dim3(blocks), dim3(256), s, it);
  else
    pdl_launch(k_pack_planes<WB, false>, dim3(blocks), dim3(256), s, it);
}

// vector loads and stores: 4-byte aligned planes, whole lanes, words aligned to the lane's store
bool pack_vec_ok(const PackItem &it) {
  const uintptr_t store_align = it.word_bytes >= 4 ? 16 : 4 * static_cast<uintptr_t>(it.word_bytes);
  return (reinterpret_cast<uintptr_t>(it.planes) & 3u) == 0 && it.cells % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(it.words) & (store_align - 1)) == 0;
}

cudaError_t launch_pack_planes(const PackItem &it, cudaStream_t s) {
  const int64_t lanes = (it.cells + 3) / 4;
  if (lanes == 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((lanes + 255) / 256);
  const bool vec = pack_vec_ok(it);
  switch (it.word_bytes) {
    case 1: pack_launch<1>(it, vec, blocks, s); break;
    case 2: pack_launch<2>(it, vec, blocks, s); break;
    case 4: pack_launch<4>(it, vec, blocks, s); break;
    case 8: pack_launch<8>(it, vec, blocks, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pack_batch(const PackTable &tab, cudaStream_t s) {
  if (tab.n == 0 || tab.lane0[tab.n] == 0) return cudaSuccess;
  k_pack_batch<<<static_cast<unsigned>((tab.lane0[tab.n] + 255) / 256), 256, 0, s>>>(tab);
  return cudaGetLastError();
}

cudaError_t launch_frame_batch(const FrameTable &tab, int num_sms, cudaStream_t s) {
  if (tab.total == 0) return cudaSuccess;
  (void)num_sms;  // a thread per cell: each thread's gathers are its only latency, no serial grid stride
  int64_t blocks = (tab.total + 255) / 256;
  if (blocks > 2147483647LL) blocks = 2147483647LL;
  k_frame_batch<<<static_cast<unsigned>(blocks), 256, 0, s>>>(tab);
  return cudaGetLastError();
}

cudaError_t launch_monitor_step(const MonitorTables &mon, const uint64_t *L, int64_t n, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  if (blocks > cap) blocks = cap;
  k_monitor_step<<<static_cast<unsigned>(blocks), 256, 0, s>>>(mon, L, n);
  return cudaGetLastError();
}

}  // namespace lbl
