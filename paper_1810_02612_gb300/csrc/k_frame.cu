// Frame transform (equivariant re-use of the roadmap, Sec. 5 / eq. 13) and the
// stand-alone safety-monitor step (Sec. 3.2).
#include "lbl_internal.cuh"

namespace lbl {
namespace {

// Even-position bits of v packed into the low half: the inverse of the
// z-order interleave for one coordinate (Sec. 4.1).
__device__ __forceinline__ uint32_t gather_even_bits(uint64_t v) {
  v &= 0x5555555555555555ull;
  v = (v | (v >> 1)) & 0x3333333333333333ull;
  v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  v = (v | (v >> 4)) & 0x00FF00FF00FF00FFull;
  v = (v | (v >> 8)) & 0x0000FFFF0000FFFFull;
  v = (v | (v >> 16)) & 0x00000000FFFFFFFFull;
  return static_cast<uint32_t>(v);
}

struct FrameArgs {
  FrameMap map;
  const uint8_t *planes;
  uint64_t *O;
  int64_t plane_cells;  // ww * wh
  int32_t ww, wh, aw, ah, P, order;
};

// One thread per agent cell, in output (cell-order) index so the O stores are
// coalesced.  The world cell is the floor of an exact Q32.32 affine map of
// (ix, iy); P byte gathers build the proposition word.
__global__ void __launch_bounds__(256) k_frame_transform(FrameArgs a) {
  const int64_t n = static_cast<int64_t>(a.aw) * a.ah;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < n; idx += stride) {
    int64_t ix, iy;
    if (a.order == LBL_ORDER_MORTON) {
      ix = gather_even_bits(static_cast<uint64_t>(idx) >> 1);
      iy = gather_even_bits(static_cast<uint64_t>(idx));
    } else {
      iy = idx / a.aw;
      ix = idx - iy * a.aw;
    }
    const int64_t u = a.map.A00 * ix + a.map.A01 * iy + a.map.B0;
    const int64_t v = a.map.A10 * ix + a.map.A11 * iy + a.map.B1;
    const int64_t wx = u >> 32;  // arithmetic shift: floor for negative values too
    const int64_t wy = v >> 32;
    uint64_t word = 0;
    if (wx >= 0 && wx < a.ww && wy >= 0 && wy < a.wh) {
      const uint8_t *p = a.planes + wy * a.ww + wx;
      int q = 0;
      for (; q + 8 <= a.P; q += 8) {
        uint8_t b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = __ldg(p + (q + j) * a.plane_cells);
#pragma unroll
        for (int j = 0; j < 8; ++j) word |= static_cast<uint64_t>(b[j] != 0) << (q + j);
      }
      for (; q < a.P; ++q) word |= static_cast<uint64_t>(__ldg(p + q * a.plane_cells) != 0) << q;
    }
    a.O[idx] = word;
  }
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
    const int64_t idx = gidx - f.cell0;
    int64_t ix, iy;
    if (f.order == LBL_ORDER_MORTON) {
      ix = gather_even_bits(static_cast<uint64_t>(idx) >> 1);
      iy = gather_even_bits(static_cast<uint64_t>(idx));
    } else {
      iy = idx / f.aw;
      ix = idx - iy * f.aw;
    }
    const int64_t u = f.A00 * ix + f.A01 * iy + f.B0;
    const int64_t v = f.A10 * ix + f.A11 * iy + f.B1;
    const int64_t wx = u >> 32;
    const int64_t wy = v >> 32;
    uint64_t word = 0;
    if (wx >= 0 && wx < f.ww && wy >= 0 && wy < f.wh) {
      const uint8_t *p = f.planes + wy * f.ww + wx;
      for (int q = 0; q < f.P; ++q) word |= static_cast<uint64_t>(__ldg(p + q * f.plane_cells) != 0) << q;
    }
    f.O[idx] = word;
  }
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

cudaError_t launch_frame_transform(const FrameMap &m, const uint8_t *planes, int32_t ww, int32_t wh, int32_t P,
                                   int32_t aw, int32_t ah, int32_t order, uint64_t *O, int num_sms, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(aw) * ah;
  if (n == 0) return cudaSuccess;
  FrameArgs a{m, planes, O, static_cast<int64_t>(ww) * wh, ww, wh, aw, ah, P, order};
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  if (blocks > cap) blocks = cap;
  k_frame_transform<<<static_cast<unsigned>(blocks), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_frame_batch(const FrameTable &tab, int num_sms, cudaStream_t s) {
  if (tab.total == 0) return cudaSuccess;
  int64_t blocks = (tab.total + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  if (blocks > cap) blocks = cap;
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
