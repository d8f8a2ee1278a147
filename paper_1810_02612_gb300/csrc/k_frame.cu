// Frame transform (equivariant re-use of the roadmap, Sec. 5 / eq. 13) and the
// stand-alone safety-monitor step (Sec. 3.2).
#include "lbl_internal.cuh"

namespace lbl {
namespace {

// Every third bit of v (positions 0, 3, ..., 60) packed into the low 21 bits:
// the inverse of the 3-D z-order interleave for one coordinate.
__device__ __forceinline__ uint32_t gather_third_bits(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v | (v >> 2)) & 0x10C30C30C30C30C3ull;
  v = (v | (v >> 4)) & 0x100F00F00F00F00Full;
  v = (v | (v >> 8)) & 0x001F0000FF0000FFull;
  v = (v | (v >> 16)) & 0x001F00000000FFFFull;
  v = (v | (v >> 32)) & 0x00000000001FFFFFull;
  return static_cast<uint32_t>(v);
}

// World word of agent cell idx of frame f (2-D or time-augmented).  The world
// cell is the floor of exact Q32.32 affine maps of (ix, iy) and of the slab it.
__device__ __forceinline__ uint64_t frame_word(const FrameItem &f, int64_t idx) {
  int64_t ix, iy, it = 0;
  if (f.ad > 1) {
    if (f.order == LBL_ORDER_MORTON) {
      ix = gather_third_bits(static_cast<uint64_t>(idx) >> 2);
      iy = gather_third_bits(static_cast<uint64_t>(idx) >> 1);
      it = gather_third_bits(static_cast<uint64_t>(idx));
    } else {
      const int64_t plane = static_cast<int64_t>(f.aw) * f.ah;
      it = idx / plane;
      const int64_t r = idx - it * plane;
      iy = r / f.aw;
      ix = r - iy * f.aw;
    }
  } else if (f.order == LBL_ORDER_MORTON) {
    ix = gather_even_bits(static_cast<uint64_t>(idx) >> 1);
    iy = gather_even_bits(static_cast<uint64_t>(idx));
  } else {
    iy = idx / f.aw;
    ix = idx - iy * f.aw;
  }
  const int64_t wx = (f.A00 * ix + f.A01 * iy + f.B0) >> 32;  // arithmetic shift: floor
  const int64_t wy = (f.A10 * ix + f.A11 * iy + f.B1) >> 32;
  const int64_t wt = f.wd > 1 ? ((f.At * it + f.Bt) >> 32) : 0;  // a 2-D world is static in time
  uint64_t word = 0;
  if (wx >= 0 && wx < f.ww && wy >= 0 && wy < f.wh && wt >= 0 && wt < f.wd && f.words) {
    word = __ldg(f.words + (wt * f.wh + wy) * f.ww + wx) & f.wmask;
  } else if (wx >= 0 && wx < f.ww && wy >= 0 && wy < f.wh && wt >= 0 && wt < f.wd) {
    const uint8_t *p = f.planes + (wt * f.wh + wy) * f.ww + wx;
    int q = 0;
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

// One thread per agent cell, in output (cell-order) index so the O stores are
// coalesced.
__global__ void __launch_bounds__(256) k_frame_transform(const __grid_constant__ FrameItem f) {
  const int64_t n = static_cast<int64_t>(f.aw) * f.ah * f.ad;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < n; idx += stride)
    f.O[idx] = frame_word(f, idx);
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
    f.O[idx] = frame_word(f, idx);
  }
}

// Packing: lane quad (4 consecutive lanes) per group of four world cells;
// lane q of the quad reads planes q, q+4, q+8, ... of the group (4 bytes at a
// time when the planes are 4-byte aligned and the cell count divisible by 4),
// so all of a lane's loads are in flight at once; the quad ORs its partial
// words by two shuffles and lane j stores the word of cell 4g + j.
// `t` is the global lane index; lanes past the last group only shuffle.
__device__ __forceinline__ void pack_quad(const PackItem &it, int64_t t, bool valid) {
  const int q = static_cast<int>(t & 3);
  const int64_t g = t >> 2;
  const int64_t c0 = 4 * g;
  uint64_t w[4] = {0, 0, 0, 0};
  if (valid) {
    const bool vec = ((reinterpret_cast<uintptr_t>(it.planes) | static_cast<uintptr_t>(it.cells)) & 3u) == 0;
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int p = q + 4 * i;
      uint32_t x = 0;
      if (p < it.P) {
        const uint8_t *pl = it.planes + p * it.cells;
        if (vec) {
          x = __ldg(reinterpret_cast<const uint32_t *>(pl + c0));
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (c0 + j < it.cells) x |= static_cast<uint32_t>(__ldg(pl + c0 + j)) << (8 * j);
        }
      }
      v[i] = x;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int p = q + 4 * i;
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] |= static_cast<uint64_t>((v[i] >> (8 * j)) & 0xFFu ? 1u : 0u) << p;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    w[j] |= __shfl_xor_sync(0xffffffffu, w[j], 1);
    w[j] |= __shfl_xor_sync(0xffffffffu, w[j], 2);
  }
  if (valid && c0 + q < it.cells) it.words[c0 + q] = q == 0 ? w[0] : q == 1 ? w[1] : q == 2 ? w[2] : w[3];
}

__global__ void __launch_bounds__(256) k_pack_planes(const __grid_constant__ PackItem it) {
  const int64_t lanes = 4 * ((it.cells + 3) / 4);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  // the loop bound is tested on the warp's first lane, so whole warps iterate together
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t - (threadIdx.x & 31) < lanes;
       t += stride)
    pack_quad(it, t, t < lanes);
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

cudaError_t launch_frame_transform(const FrameItem &f, int num_sms, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(f.aw) * f.ah * f.ad;
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  if (blocks > cap) blocks = cap;
  k_frame_transform<<<static_cast<unsigned>(blocks), 256, 0, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_pack_planes(const PackItem &it, int num_sms, cudaStream_t s) {
  const int64_t lanes = 4 * ((it.cells + 3) / 4);
  if (lanes == 0) return cudaSuccess;
  int64_t blocks = (lanes + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms) * 8;
  if (blocks > cap) blocks = cap;
  k_pack_planes<<<static_cast<unsigned>(blocks), 256, 0, s>>>(it);
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
