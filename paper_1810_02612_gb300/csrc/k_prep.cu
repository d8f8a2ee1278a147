// Roadmap preparation at upload time: row checks and the 64-cell block form of
// the trajectory matrix (derived once, Sec. 4.3's dense bit-packed variant).
#include "lbl_internal.cuh"

namespace lbl {
namespace {

// One thread per row.  A row is bad unless 0 <= rowptr[e] <= rowptr[e+1] <= nnz
// and its indices are strictly increasing inside [0, cells).  The row pointer is
// checked before any column index is read, so every access stays inside the
// arrays.  bt_count[e] (optional) = number of distinct 64-cell blocks of row e.
__global__ void __launch_bounds__(256) k_scan_rows(const int64_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colidx, int64_t E, int64_t nnz,
                                                   int64_t cells, unsigned long long *n_bad, int32_t *bt_count) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int64_t beg = rowptr[e], end = rowptr[e + 1];
    bool bad = !(beg >= 0 && beg <= end && end <= nnz);
    int32_t blocks = 0;
    if (!bad) {
      int64_t prev = -1, prev_block = -1;
      for (int64_t k = beg; k < end; ++k) {
        const int64_t c = colidx[k];
        if (c < 0 || c >= cells || c <= prev) {
          bad = true;
          break;
        }
        if ((c >> 6) != prev_block) {
          ++blocks;
          prev_block = c >> 6;
        }
        prev = c;
      }
    }
    if (bad) atomicAdd(n_bad, 1ull);
    if (bt_count) bt_count[e] = bad ? 0 : blocks;
  }
}

// One thread per row: write the (block, mask) entries of row e at bt_rowptr[e].
__global__ void __launch_bounds__(256) k_bt_fill(const int64_t *__restrict__ rowptr,
                                                 const int32_t *__restrict__ colidx, int64_t E,
                                                 const int64_t *__restrict__ bt_rowptr, uint32_t *__restrict__ bt_block,
                                                 uint64_t *__restrict__ bt_mask) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    int64_t out = bt_rowptr[e];
    int64_t cur = -1;
    uint64_t m = 0;
    for (int64_t k = rowptr[e]; k < rowptr[e + 1]; ++k) {
      const int64_t c = colidx[k];
      const int64_t b = c >> 6;
      if (b != cur) {
        if (cur >= 0) {
          bt_block[out] = static_cast<uint32_t>(cur);
          bt_mask[out] = m;
          ++out;
        }
        cur = b;
        m = 0;
      }
      m |= 1ull << (c & 63);
    }
    if (cur >= 0) {
      bt_block[out] = static_cast<uint32_t>(cur);
      bt_mask[out] = m;
    }
  }
}

// Sector form: per row, the number of distinct 4-cell sectors (count) and the
// entries (sector << 4) | cell mask (fill), rows already checked.
__global__ void __launch_bounds__(256) k_sector_count(const int64_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ colidx, int64_t E,
                                                      int32_t *__restrict__ count) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    int32_t n = 0;
    int64_t prev = -1;
    for (int64_t k = rowptr[e]; k < rowptr[e + 1]; ++k) {
      const int64_t sct = colidx[k] >> 2;
      n += sct != prev;
      prev = sct;
    }
    count[e] = n;
  }
}

__global__ void __launch_bounds__(256) k_sector_fill(const int64_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ colidx, int64_t E,
                                                     const int64_t *__restrict__ srow, int32_t *__restrict__ sec) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    int64_t out = srow[e];
    int64_t cur = -1;
    uint32_t m = 0;
    for (int64_t k = rowptr[e]; k < rowptr[e + 1]; ++k) {
      const int64_t c = colidx[k];
      if ((c >> 2) != cur) {
        if (cur >= 0) sec[out++] = static_cast<int32_t>((static_cast<uint32_t>(cur) << 4) | m);
        cur = c >> 2;
        m = 0;
      }
      m |= 1u << (c & 3);
    }
    if (cur >= 0) sec[out] = static_cast<int32_t>((static_cast<uint32_t>(cur) << 4) | m);
  }
}

// Quadtree form: a row (strictly increasing cells) is cut greedily from its
// first cell into blocks of 4^j consecutive cells starting at a multiple of
// 4^j, each as large as the row allows (j <= kQuadLevels).  In z-order such a
// block is a 2^j x 2^j square of the quadtree; in row-major order an aligned
// run.  Level of the block that starts at entry k (cell c) of a row ending at
// `end`.
__device__ __forceinline__ int quad_level(const int32_t *__restrict__ colidx, int64_t k, int64_t end, int64_t c) {
  int j = 0;
  while (j < kQuadLevels) {
    const int64_t n = 4LL << (2 * j);  // the next larger block
    if ((c & (n - 1)) != 0 || k + n > end || colidx[k + n - 1] != c + n - 1) break;
    ++j;
  }
  return j;
}

// Bits 0..15 of v spread to the even positions 0, 2, ..., 30.
__device__ __forceinline__ uint32_t spread_even(uint32_t v) {
  v &= 0x0000FFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  return (v | (v << 1)) & 0x55555555u;
}

// Locality key of row e of a 2-D grid: the z-order index of its middle cell's
// (x, y) (the cell index itself on a z-order grid; 0 for an empty row).
__global__ void __launch_bounds__(256) k_row_keys(const int64_t *__restrict__ rowptr,
                                                  const int32_t *__restrict__ colidx, int64_t E, int32_t order,
                                                  int32_t w, uint32_t *__restrict__ key) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int64_t beg = rowptr[e], n = rowptr[e + 1] - beg;
    uint32_t k = 0;
    if (n > 0) {
      const uint32_t c = static_cast<uint32_t>(colidx[beg + n / 2]);
      if (order == LBL_ORDER_MORTON) {
        k = c;
      } else {
        const uint32_t y = c / static_cast<uint32_t>(w), x = c - y * static_cast<uint32_t>(w);
        k = (spread_even(x) << 1) | spread_even(y);
      }
    }
    key[e] = k;
  }
}

// Quadtree row e is built from CSR row rowmap[e] (rowmap NULL: row e).
__global__ void __launch_bounds__(256) k_quad_count(const int64_t *__restrict__ rowptr,
                                                    const int32_t *__restrict__ colidx, int64_t E,
                                                    const int32_t *__restrict__ rowmap, int32_t *__restrict__ count) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int64_t src = rowmap ? rowmap[e] : e;
    const int64_t end = rowptr[src + 1];
    int32_t n = 0;
    for (int64_t k = rowptr[src]; k < end; ++n) k += 1LL << (2 * quad_level(colidx, k, end, colidx[k]));
    count[e] = n;
  }
}

// Entries of a row are written level by level (level 0 first), ascending
// inside a level, i.e. ascending pyramid index: neighbouring lanes then
// gather neighbouring words of one level.
__global__ void __launch_bounds__(256) k_quad_fill(const int64_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colidx, int64_t E,
                                                   const int32_t *__restrict__ rowmap, QuadOffsets off,
                                                   const int64_t *__restrict__ qrow, int32_t *__restrict__ idx) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int64_t src = rowmap ? rowmap[e] : e;
    const int64_t beg = rowptr[src], end = rowptr[src + 1];
    int64_t out = qrow[e];
    for (int lev = 0; lev <= kQuadLevels; ++lev) {
      for (int64_t k = beg; k < end;) {
        const int64_t c = colidx[k];
        const int j = quad_level(colidx, k, end, c);
        if (j == lev) idx[out++] = static_cast<int32_t>(off.at[j] + (c >> (2 * j)));
        k += 1LL << (2 * j);
      }
    }
  }
}

unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 65535LL * 8) b = 65535LL * 8;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_sector_count(const int64_t *rowptr, const int32_t *colidx, int64_t E, int32_t *count,
                                cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_sector_count<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, count);
  return cudaGetLastError();
}

cudaError_t launch_sector_fill(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int64_t *srow,
                               int32_t *sec, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_sector_fill<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, srow, sec);
  return cudaGetLastError();
}

cudaError_t launch_scan_rows(const int64_t *rowptr, const int32_t *colidx, int64_t E, int64_t nnz, int64_t cells,
                             unsigned long long *n_bad, int32_t *bt_count, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_scan_rows<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, nnz, cells, n_bad, bt_count);
  return cudaGetLastError();
}

cudaError_t launch_bt_fill(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int64_t *bt_rowptr,
                           uint32_t *bt_block, uint64_t *bt_mask, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_bt_fill<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, bt_rowptr, bt_block, bt_mask);
  return cudaGetLastError();
}

}  // namespace lbl

namespace lbl {

cudaError_t launch_row_keys(const int64_t *rowptr, const int32_t *colidx, int64_t E, int32_t order, int32_t w,
                            uint32_t *key, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_row_keys<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, order, w, key);
  return cudaGetLastError();
}

cudaError_t launch_quad_count(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int32_t *rowmap,
                              int32_t *count, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_quad_count<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, rowmap, count);
  return cudaGetLastError();
}

cudaError_t launch_quad_fill(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int32_t *rowmap,
                             QuadOffsets off, const int64_t *qrow, int32_t *idx, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_quad_fill<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, rowmap, off, qrow, idx);
  return cudaGetLastError();
}

}  // namespace lbl
