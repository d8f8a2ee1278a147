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

// Tiled order of a row-major 2-D grid whose sides are multiples of 16 (the
// quadtree form's order there): 16 x 16 tiles in row-major order, cells in
// z-order inside a tile (bit i of the tile-local x -> bit 2i+1, of y -> bit
// 2i).  Its aligned blocks of 4^j cells are 2^j x 2^j squares, where the
// row-major order's are runs of one grid row (the 2^21-cell 2-D frame: 113
// instead of 176 entries and 32 instead of 77 distinct 32-byte pyramid sectors
// per row).
__device__ __forceinline__ uint32_t tile_z(uint32_t lx, uint32_t ly) {
  return (spread_even(lx) << 1) | spread_even(ly);
}

// Maximal aligned blocks of one tile, given its cells as a 256-bit mask over
// tile-local z indices; the tile's first cell has tiled index `base`.  Counts
// the blocks of every level (lev < 0) or writes those of level `lev` to out,
// ascending; returns how many.
__device__ __forceinline__ int tile_blocks(const uint64_t (&m)[4], int64_t base, int lev, const QuadOffsets &off,
                                           int32_t *__restrict__ out) {
  int n = 0;
  auto put = [&](int j, int64_t first) {
    if (lev < 0) {
      ++n;
    } else if (j == lev) {
      out[n++] = static_cast<int32_t>(off.at[j] + (first >> (2 * j)));
    }
  };
  if ((m[0] & m[1] & m[2] & m[3]) == ~0ull) {
    put(4, base);
    return n;
  }
  for (int q = 0; q < 4; ++q) {
    const uint64_t word = m[q];
    const int64_t qb = base + 64 * q;
    if (word == ~0ull) {
      put(3, qb);
      continue;
    }
    for (int g = 0; g < 4; ++g) {
      const uint32_t g16 = static_cast<uint32_t>(word >> (16 * g)) & 0xFFFFu;
      const int64_t gb = qb + 16 * g;
      if (g16 == 0xFFFFu) {
        put(2, gb);
        continue;
      }
      for (int nb = 0; nb < 4 && (g16 >> (4 * nb)); ++nb) {
        const uint32_t nib = (g16 >> (4 * nb)) & 0xFu;
        const int64_t nbb = gb + 4 * nb;
        if (nib == 0xFu) {
          put(1, nbb);
        } else {
          for (int b = 0; b < 4; ++b)
            if ((nib >> b) & 1u) put(0, nbb + b);
        }
      }
    }
  }
  return n;
}

// The quadtree entries of one row (strictly increasing row-major cells of a
// grid w cells wide) in the tiled order: band by band (16 grid rows), a
// cursor per grid row of the band, tiles of the band in ascending x, each
// tile's cells gathered into a 256-bit mask and cut into maximal squares.
// Counts every level (lev < 0) or writes level `lev`; returns how many.
__device__ int64_t tiled_row(const int32_t *__restrict__ colidx, int64_t beg, int64_t end, int32_t w, int lev,
                             const QuadOffsets &off, int32_t *__restrict__ out) {
  const uint32_t uw = static_cast<uint32_t>(w), tw = uw >> 4;
  int64_t n = 0, s = beg;
  int64_t cur[16], lim[16];
  while (s < end) {
    const uint32_t band = (static_cast<uint32_t>(colidx[s]) / uw) >> 4;
    int64_t k = s;
    for (uint32_t r = 0; r < 16; ++r) {  // grid row 16 * band + r: entries [cur[r], lim[r])
      cur[r] = k;
      while (k < end && static_cast<uint32_t>(colidx[k]) / uw == 16 * band + r) ++k;
      lim[r] = k;
    }
    s = k;
    for (;;) {
      uint32_t tx = ~0u;  // the leftmost tile of the band with cells left
      for (int r = 0; r < 16; ++r)
        if (cur[r] < lim[r]) tx = min(tx, (static_cast<uint32_t>(colidx[cur[r]]) % uw) >> 4);
      if (tx == ~0u) break;
      uint64_t m[4] = {0ull, 0ull, 0ull, 0ull};
      for (uint32_t r = 0; r < 16; ++r) {
        while (cur[r] < lim[r]) {
          const uint32_t x = static_cast<uint32_t>(colidx[cur[r]]) % uw;
          if ((x >> 4) != tx) break;
          const uint32_t z = tile_z(x & 15u, r);
          m[z >> 6] |= 1ull << (z & 63u);
          ++cur[r];
        }
      }
      n += tile_blocks(m, (static_cast<int64_t>(band) * tw + tx) * 256, lev, off, out ? out + n : nullptr);
    }
  }
  return n;
}

// Quadtree row e is built from CSR row rowmap[e] (rowmap NULL: row e);
// tiled_w > 0: in the tiled order of a row-major grid tiled_w cells wide.
__global__ void __launch_bounds__(256) k_quad_count(const int64_t *__restrict__ rowptr,
                                                    const int32_t *__restrict__ colidx, int64_t E,
                                                    const int32_t *__restrict__ rowmap, int32_t tiled_w,
                                                    int32_t *__restrict__ count) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const QuadOffsets none{};
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int64_t src = rowmap ? rowmap[e] : e;
    const int64_t end = rowptr[src + 1];
    int32_t n = 0;
    if (tiled_w > 0) {
      n = static_cast<int32_t>(tiled_row(colidx, rowptr[src], end, tiled_w, -1, none, nullptr));
    } else {
      for (int64_t k = rowptr[src]; k < end; ++n) k += 1LL << (2 * quad_level(colidx, k, end, colidx[k]));
    }
    count[e] = n;
  }
}

// Entries of a row are written level by level (level 0 first), ascending
// inside a level, i.e. ascending pyramid index: neighbouring lanes then
// gather neighbouring words of one level.
__global__ void __launch_bounds__(256) k_quad_fill(const int64_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colidx, int64_t E,
                                                   const int32_t *__restrict__ rowmap, int32_t tiled_w,
                                                   QuadOffsets off, const int64_t *__restrict__ qrow,
                                                   int32_t *__restrict__ idx) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += stride) {
    const int64_t src = rowmap ? rowmap[e] : e;
    const int64_t beg = rowptr[src], end = rowptr[src + 1];
    int64_t out = qrow[e];
    if (tiled_w > 0) {
      for (int lev = 0; lev <= kQuadLevels; ++lev) out += tiled_row(colidx, beg, end, tiled_w, lev, off, idx + out);
      continue;
    }
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
                              int32_t tiled_w, int32_t *count, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_quad_count<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, rowmap, tiled_w, count);
  return cudaGetLastError();
}

cudaError_t launch_quad_fill(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int32_t *rowmap,
                             int32_t tiled_w, QuadOffsets off, const int64_t *qrow, int32_t *idx, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  k_quad_fill<<<blocks_for(E), 256, 0, s>>>(rowptr, colidx, E, rowmap, tiled_w, off, qrow, idx);
  return cudaGetLastError();
}

}  // namespace lbl
