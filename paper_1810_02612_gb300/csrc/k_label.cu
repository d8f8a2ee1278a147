// Labeling kernels: the Boolean product L = M.P of eq. 10 (Sec. 4.2-4.3).
//
// k_label_csr   gather-OR over CSR rows (the sparse form of Sec. 4.3): lanes of
//               a group stream an edge's column indices with 16-byte loads that
//               bypass L1, gather the proposition words of those cells (O is a
//               few MiB and stays in L2/L1) and OR them; the group then ORs its
//               lanes together.  Optional early exit once every proposition is
//               set (the early termination of Sec. 5).
// k_label_bt    the dense bit-packed form: each edge is a list of 64-cell
//               blocks with a cell mask; proposition p is hit iff
//               (mask AND plane[block][p]) != 0.  Lanes own propositions, so
//               each block costs P plane words instead of one index per cell.
// Both optionally feed the label through the safety monitor (Sec. 3.2) before
// it leaves the register file.
#include <algorithm>

#include "lbl_internal.cuh"

namespace lbl {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int4 ld_stream_v4(const int32_t *p) {
  int4 r;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

__device__ __forceinline__ uint64_t or_xor(uint64_t v, int off) { return v | __shfl_xor_sync(kFull, v, off); }

struct EpiSmem {
  uint64_t T[256];
  uint16_t V[256];
};

__device__ __forceinline__ void load_tables(const MonitorTables &mon, EpiSmem &sm) {
  const int letters = 1 << mon.m;
  for (int i = threadIdx.x; i < letters; i += blockDim.x) {
    sm.T[i] = mon.T[i];
    sm.V[i] = mon.V[i];
  }
  __syncthreads();
}

__device__ __forceinline__ void epilogue(const MonitorTables &mon, const EpiSmem &sm, int64_t e, uint64_t w) {
  uint32_t letter = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (j < mon.m) letter |= static_cast<uint32_t>((w >> mon.rel[j]) & 1u) << j;
  mon.next[e] = sm.T[letter];
  mon.viol[e] = sm.V[letter];
}

// LPE lanes per edge (32/LPE edges per warp at a time); U steps of 4*LPE
// indices per group in flight.
template <int LPE, int U, bool EPI, bool EARLY>
__global__ void __launch_bounds__(kThreads) k_label_csr(const int64_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ colidx,
                                                        const uint64_t *__restrict__ O, int64_t E, uint64_t mask,
                                                        uint64_t *__restrict__ L, MonitorTables mon) {
  constexpr int G = 32 / LPE;
  constexpr int SPAN = 4 * LPE;
  __shared__ EpiSmem sm;
  if (EPI) load_tables(mon, sm);
  const int lane = threadIdx.x & 31;
  const int g = lane / LPE;
  const int gl = lane % LPE;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * kThreads) >> 5;
  for (int64_t base_e = warp * G; base_e < E; base_e += nwarps * G) {
    const int64_t e = base_e + g;
    int64_t beg = 0, end = 0;
    if (e < E) {
      beg = __ldg(rowptr + e);
      end = __ldg(rowptr + e + 1);
    }
    const int64_t a = beg & ~static_cast<int64_t>(3);  // 16-byte aligned start
    int64_t lim = end;                                   // loads stop here
    const uint32_t steps = static_cast<uint32_t>((end - a + SPAN - 1) / SPAN);
    const uint32_t nsteps = __reduce_max_sync(kFull, steps);
    uint64_t acc = 0;
    for (uint32_t s = 0; s < nsteps; s += U) {
      int4 v[U];
      int64_t idx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        idx[u] = a + static_cast<int64_t>(s + u) * SPAN + 4 * gl;
        v[u] = idx[u] < lim ? ld_stream_v4(colidx + idx[u]) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t c[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t k = idx[u] + j;
          if (k >= beg && k < lim) acc |= __ldg(O + c[j]);
        }
      }
      if (EARLY) {
        uint64_t r = acc;
#pragma unroll
        for (int off = LPE / 2; off > 0; off >>= 1) r = or_xor(r, off);
        const bool full = (r & mask) == mask;
        if (full) lim = 0;
        if (__all_sync(kFull, full || s + U >= steps)) break;
      }
    }
#pragma unroll
    for (int off = LPE / 2; off > 0; off >>= 1) acc = or_xor(acc, off);
    if (gl == 0 && e < E) {
      acc &= mask;
      L[e] = acc;
      if (EPI) epilogue(mon, sm, e, acc);
    }
  }
}

// Bit-plane re-layout of O for the block form: one warp per 64-cell block.
__global__ void __launch_bounds__(kThreads) k_planes(const uint64_t *__restrict__ O, int64_t cells, int64_t n_blocks,
                                                     int32_t P, uint64_t *__restrict__ planes) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * kThreads) >> 5;
  for (int64_t b = warp; b < n_blocks; b += nwarps) {
    const int64_t c0 = b * 64 + lane, c1 = c0 + 32;
    const uint64_t w0 = c0 < cells ? O[c0] : 0;
    const uint64_t w1 = c1 < cells ? O[c1] : 0;
    uint64_t mine0 = 0, mine1 = 0;  // planes lane and lane + 32
    for (int q = 0; q < P; ++q) {
      const uint64_t lo = __ballot_sync(kFull, (w0 >> q) & 1u);
      const uint64_t hi = __ballot_sync(kFull, (w1 >> q) & 1u);
      const uint64_t plane = lo | (hi << 32);
      if (q == lane) mine0 = plane;
      if (q == lane + 32) mine1 = plane;
    }
    uint64_t *dst = planes + b * P;
    if (lane < P) dst[lane] = mine0;
    if (lane + 32 < P) dst[lane + 32] = mine1;
  }
}

// LPB lanes per block entry (a power of two >= min(P, 32)); 32/LPB entries per
// step; lane owns propositions q = lane % LPB + k * LPB.
template <int LPB, bool EPI, bool EARLY>
__global__ void __launch_bounds__(kThreads) k_label_bt(const int64_t *__restrict__ brow,
                                                       const uint32_t *__restrict__ bblock,
                                                       const uint64_t *__restrict__ bmask,
                                                       const uint64_t *__restrict__ planes, int32_t P, int64_t E,
                                                       uint64_t mask, uint64_t *__restrict__ L, MonitorTables mon) {
  constexpr int EPS = 32 / LPB;
  __shared__ EpiSmem sm;
  if (EPI) load_tables(mon, sm);
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPB;
  const int pl = lane % LPB;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * kThreads) >> 5;
  for (int64_t e = warp; e < E; e += nwarps) {
    const int64_t beg = __ldg(brow + e), end = __ldg(brow + e + 1);
    uint64_t word = 0;
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
      const int64_t k = k0 + lane;
      uint32_t b = 0;
      uint64_t m = 0;
      if (k < end) {
        b = __ldg(bblock + k);
        m = __ldg(bmask + k);
      }
      const int n = static_cast<int>(end - k0 < 32 ? end - k0 : 32);
      for (int j = 0; j < n; j += EPS) {
        const int src = j + sub;
        const uint32_t bj = __shfl_sync(kFull, b, src);
        const uint64_t mj = __shfl_sync(kFull, m, src);
        if (mj) {
          const uint64_t *pp = planes + static_cast<int64_t>(bj) * P;
          for (int q = pl; q < P; q += LPB)
            if (__ldg(pp + q) & mj) word |= 1ull << q;
        }
      }
      if (EARLY) {
        uint64_t r = word;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r = or_xor(r, off);
        if ((r & mask) == mask) break;  // warp-uniform: r is the same in every lane
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) word = or_xor(word, off);
    if (lane == 0) {
      word &= mask;
      L[e] = word;
      if (EPI) epilogue(mon, sm, e, word);
    }
  }
}

template <typename Kernel>
int occupancy(Kernel k) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, 0) != cudaSuccess || occ < 1) occ = 1;
  return occ;
}

int64_t grid_size(int occ, int num_sms, int ctas_per_sm, int64_t warps_needed) {
  if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
  int64_t g = static_cast<int64_t>(num_sms) * occ;
  const int64_t need = (warps_needed + (kThreads / 32) - 1) / (kThreads / 32);
  if (need < g) g = need;
  return g < 1 ? 1 : g;
}

template <int LPE, int U, bool EPI, bool EARLY>
cudaError_t run_csr(const Roadmap &rm, const uint64_t *O, uint64_t mask, uint64_t *L, const MonitorTables &mon,
                    int ctas_per_sm, cudaStream_t s) {
  auto k = k_label_csr<LPE, U, EPI, EARLY>;
  static const int occ = occupancy(k);
  const int64_t warps = (rm.E + (32 / LPE) - 1) / (32 / LPE);
  const int64_t g = grid_size(occ, rm.num_sms, ctas_per_sm, warps);
  k<<<static_cast<unsigned>(g), kThreads, 0, s>>>(rm.rowptr, rm.colidx, O, rm.E, mask, L, mon);
  return cudaGetLastError();
}

template <int LPE, bool EPI, bool EARLY>
cudaError_t pick_u(const Roadmap &rm, const uint64_t *O, uint64_t mask, uint64_t *L, const MonitorTables &mon,
                   int ctas_per_sm, cudaStream_t s) {
  return run_csr<LPE, 2, EPI, EARLY>(rm, O, mask, L, mon, ctas_per_sm, s);
}

template <bool EPI, bool EARLY>
cudaError_t pick_lpe(int lpe, const Roadmap &rm, const uint64_t *O, uint64_t mask, uint64_t *L,
                     const MonitorTables &mon, int ctas_per_sm, cudaStream_t s) {
  switch (lpe) {
    case 4: return pick_u<4, EPI, EARLY>(rm, O, mask, L, mon, ctas_per_sm, s);
    case 8: return pick_u<8, EPI, EARLY>(rm, O, mask, L, mon, ctas_per_sm, s);
    case 16: return pick_u<16, EPI, EARLY>(rm, O, mask, L, mon, ctas_per_sm, s);
    default: return pick_u<32, EPI, EARLY>(rm, O, mask, L, mon, ctas_per_sm, s);
  }
}

template <int LPB, bool EPI, bool EARLY>
cudaError_t run_bt(const Roadmap &rm, int32_t P, uint64_t mask, uint64_t *L, const MonitorTables &mon,
                   int ctas_per_sm, cudaStream_t s) {
  auto k = k_label_bt<LPB, EPI, EARLY>;
  static const int occ = occupancy(k);
  const int64_t g = grid_size(occ, rm.num_sms, ctas_per_sm, rm.E);
  k<<<static_cast<unsigned>(g), kThreads, 0, s>>>(rm.bt_rowptr, rm.bt_block, rm.bt_mask, rm.planes, P, rm.E, mask,
                                                  L, mon);
  return cudaGetLastError();
}

template <bool EPI, bool EARLY>
cudaError_t pick_lpb(int32_t P, const Roadmap &rm, uint64_t mask, uint64_t *L, const MonitorTables &mon,
                     int ctas_per_sm, cudaStream_t s) {
  if (P <= 1) return run_bt<1, EPI, EARLY>(rm, P, mask, L, mon, ctas_per_sm, s);
  if (P <= 2) return run_bt<2, EPI, EARLY>(rm, P, mask, L, mon, ctas_per_sm, s);
  if (P <= 4) return run_bt<4, EPI, EARLY>(rm, P, mask, L, mon, ctas_per_sm, s);
  if (P <= 8) return run_bt<8, EPI, EARLY>(rm, P, mask, L, mon, ctas_per_sm, s);
  if (P <= 16) return run_bt<16, EPI, EARLY>(rm, P, mask, L, mon, ctas_per_sm, s);
  return run_bt<32, EPI, EARLY>(rm, P, mask, L, mon, ctas_per_sm, s);
}

uint64_t prop_mask(int32_t P) { return P >= 64 ? ~0ull : ((1ull << P) - 1ull); }

}  // namespace

cudaError_t launch_label_csr(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L, const MonitorTables *mon,
                             int lanes_per_edge, bool early_exit, int ctas_per_sm, cudaStream_t s) {
  if (rm.E == 0) return cudaSuccess;
  const uint64_t mask = prop_mask(P);
  MonitorTables none{};
  const MonitorTables &mt = mon ? *mon : none;
  if (mon) {
    if (early_exit) return pick_lpe<true, true>(lanes_per_edge, rm, O, mask, L, mt, ctas_per_sm, s);
    return pick_lpe<true, false>(lanes_per_edge, rm, O, mask, L, mt, ctas_per_sm, s);
  }
  if (early_exit) return pick_lpe<false, true>(lanes_per_edge, rm, O, mask, L, mt, ctas_per_sm, s);
  return pick_lpe<false, false>(lanes_per_edge, rm, O, mask, L, mt, ctas_per_sm, s);
}

cudaError_t launch_label_bittile(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                                 const MonitorTables *mon, bool early_exit, int ctas_per_sm, cudaStream_t s) {
  if (rm.E == 0) return cudaSuccess;
  if (rm.n_blocks > 0 && P > 0) {
    static const int occ = occupancy(k_planes);
    const int64_t g = grid_size(occ, rm.num_sms, 0, rm.n_blocks);
    k_planes<<<static_cast<unsigned>(g), kThreads, 0, s>>>(O, rm.cells, rm.n_blocks, P, rm.planes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const uint64_t mask = prop_mask(P);
  MonitorTables none{};
  const MonitorTables &mt = mon ? *mon : none;
  if (mon) {
    if (early_exit) return pick_lpb<true, true>(P, rm, mask, L, mt, ctas_per_sm, s);
    return pick_lpb<true, false>(P, rm, mask, L, mt, ctas_per_sm, s);
  }
  if (early_exit) return pick_lpb<false, true>(P, rm, mask, L, mt, ctas_per_sm, s);
  return pick_lpb<false, false>(P, rm, mask, L, mt, ctas_per_sm, s);
}

}  // namespace lbl
