// Labeling kernels: the Boolean product L = M.P of eq. 10 (Sec. 4.2-4.3).
//
// k_label_csr   gather-OR over CSR rows (the sparse form of Sec. 4.3): the lanes
//               of a group read consecutive column indices of an edge (loads
//               that bypass L1 and are evicted first from L2), gather the
//               proposition words of those cells (O is a few MiB and stays in
//               L2/L1) and OR them; the group then ORs its lanes together.
//               Optional early exit once every proposition is set (the early
//               termination of Sec. 5).
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

__device__ __forceinline__ uint64_t or_xor(uint64_t v, int off) { return v | __shfl_xor_sync(kFull, v, off); }

// OR of v over the whole warp, in every lane: one redux.sync per 32-bit half.
__device__ __forceinline__ uint64_t warp_or(uint64_t v) {
  const uint32_t lo = __reduce_or_sync(kFull, static_cast<uint32_t>(v));
  const uint32_t hi = __reduce_or_sync(kFull, static_cast<uint32_t>(v >> 32));
  return (static_cast<uint64_t>(hi) << 32) | lo;
}

// Index load that bypasses L1 and asks L2 to evict the line first: the column
// indices are streamed exactly once, O should keep its L2 residency.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ int32_t ld_stream(const int32_t *p, uint64_t pol) {
  int32_t r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
  return r;
}

// LPE lanes per edge (32/LPE edges per warp at a time).  Lane gl of a group
// handles elements a + s*LPE + gl, so one gather instruction of the group reads
// LPE consecutive entries of the (z-order sorted) row: neighbouring cells,
// few distinct sectors.  U steps are in flight, and the indices of the next U
// steps are requested before the current gathers are consumed.
template <int LPE, int U, bool EPI, bool EARLY>
__global__ void __launch_bounds__(kThreads) k_label_csr(const int64_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ colidx,
                                                        const uint64_t *__restrict__ O, int64_t E, uint64_t mask,
                                                        uint64_t *__restrict__ L, MonitorTables mon) {
  constexpr int G = 32 / LPE;
  __shared__ EpiSmem sm;
  if (EPI) load_tables(mon, sm);
  const uint64_t pol = evict_first_policy();
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
    const int64_t a = beg & ~static_cast<int64_t>(LPE - 1);  // LPE*4-byte aligned start
    int64_t lim = end;
    const uint32_t steps = static_cast<uint32_t>((end - a + LPE - 1) / LPE);
    const uint32_t nsteps = __reduce_max_sync(kFull, steps);
    uint64_t acc = 0;
    int32_t nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = a + static_cast<int64_t>(u) * LPE + gl;
      nxt[u] = (k >= beg && k < lim) ? ld_stream(colidx + k, pol) : -1;
    }
    for (uint32_t s = 0; s < nsteps; s += U) {
      int32_t cur[U];
#pragma unroll
      for (int u = 0; u < U; ++u) cur[u] = nxt[u];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = a + static_cast<int64_t>(s + U + u) * LPE + gl;
        nxt[u] = (k >= beg && k < lim) ? ld_stream(colidx + k, pol) : -1;
      }
      uint64_t w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) w[u] = cur[u] >= 0 ? __ldg(O + cur[u]) : 0ull;
#pragma unroll
      for (int u = 0; u < U; ++u) acc |= w[u];
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

// Streaming form of the gather-OR.  A warp owns the contiguous edge range
// [e_beg, e_end) (balanced by nonzeros plus a per-edge cost when the roadmap
// is uploaded), so its column indices are one contiguous stream: lane l reads
// entry g + l of each 32-entry group, the loads of the next U groups are in
// flight while the current gathers are consumed, and edge boundaries never
// stall the stream.  A boundary inside a group (some valid lane with k >= end
// of the current edge) flushes the current edge: its lanes' words are ORed in,
// the warp reduces, lane 0 hands the label to `emit`, and the next edge starts.
// Empty edges are flushed the same way with nothing ORed in.
// Gather for the CSR and quadtree streams: entry = index of a word, -1 = no
// entry.  Words are uint64 proposition words, or narrower pyramid words when
// every proposition fits (the label's bits >= P are masked anyway).
template <typename T>
struct WordGather {
  const T *__restrict__ O;
  static constexpr int32_t kNone = -1;
  __device__ __forceinline__ uint64_t full(int32_t c) const { return static_cast<uint64_t>(__ldg(O + c)); }
  __device__ __forceinline__ uint64_t masked(int32_t c) const {
    return c >= 0 ? static_cast<uint64_t>(__ldg(O + c)) : 0ull;
  }
};
using CsrGather = WordGather<uint64_t>;

// Positions inside a warp's range are kept relative to its first entry `a`
// and first edge in `Off` (int32_t whenever the range allows it: fewer
// registers and cheaper boundary tests, so more warps fit per SM).  The U
// gathers of a group are issued before the indices of the next group are
// requested, so one register per lane and group holds both.
template <int U, typename Off, typename Gather, typename Emit>
__device__ __forceinline__ void stream_body(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                            const Gather gather, int64_t e_beg, int64_t e_end, int64_t p0, int64_t p1,
                                            uint64_t pol, int lane, Emit emit) {
  constexpr int GS = 32 * U;
  const int64_t a = p0 & ~static_cast<int64_t>(31);
  const Off n_e = static_cast<Off>(e_end - e_beg);
  const Off n_rel = static_cast<Off>(p1 - a);
  const int head = static_cast<int>(p0 - a);
  const int64_t *rpb = rowptr + e_beg + 1;  // rpb[i] = end of edge e_beg + i
  // window of edge ends: lane i holds the end of edge (win + i), relative to a
  Off win = 0;
  Off rp = lane < n_e ? static_cast<Off>(__ldg(rpb + lane) - a) : Off(0);
  Off cur = 0;
  Off stop = __shfl_sync(kFull, rp, 0);
  uint64_t acc = 0;
  uint64_t mine = 0;  // lane i keeps the label of edge (win + i) until its window is complete

  // Close the current edge: every lane gets the OR of the warp, the edge's
  // lane keeps it; a complete window of 32 labels leaves in one coalesced
  // store, each lane running the epilogue for its own edge.
  auto flush = [&]() {
    const uint64_t r = warp_or(acc);
    if (lane == static_cast<int>(cur - win)) mine = r;
    acc = 0;
    ++cur;
    if (cur - win == 32) {
      emit(e_beg + win + lane, mine);
      win = cur;
      if (cur < n_e) rp = win + lane < n_e ? static_cast<Off>(__ldg(rpb + win + lane) - a) : Off(0);
    }
    if (cur < n_e) stop = __shfl_sync(kFull, rp, static_cast<int>(cur - win));
  };

  // Lane l's entry of group g is base[g + l]; whether a group crosses the end
  // of the current edge is a warp-uniform test on scalars, so the common case
  // (no boundary) only ORs.
  const int32_t *base = colidx + a + lane;
  int32_t idx[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const Off off = 32 * u + lane;
    idx[u] = (off >= head && off < n_rel) ? ld_stream(base + 32 * u, pol) : Gather::kNone;
  }
  for (Off g = 0; g < n_rel; g += GS) {
    uint64_t wv[U];
    if ((g > 0 || head == 0) && g + GS <= n_rel) {  // every entry valid
#pragma unroll
      for (int u = 0; u < U; ++u) wv[u] = gather.full(idx[u]);
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) wv[u] = gather.masked(idx[u]);
    }
    const Off ns = g + GS;  // next group
    const Off rem = n_rel - ns;
    if (rem >= GS) {
#pragma unroll
      for (int u = 0; u < U; ++u) idx[u] = ld_stream(base + ns + 32 * u, pol);
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) idx[u] = (32 * u + lane < rem) ? ld_stream(base + ns + 32 * u, pol) : Gather::kNone;
    }
    const Off grp_end = min(ns, n_rel);
    if (grp_end <= stop) {
#pragma unroll
      for (int u = 0; u < U; ++u) acc |= wv[u];
      continue;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const Off k = g + 32 * u + lane;
      const Off sub_end = min(static_cast<Off>(g + 32 * (u + 1)), n_rel);
      while (sub_end > stop) {  // some valid entry of this 32-group is past the current edge
        if (k < stop) {
          acc |= wv[u];
          wv[u] = 0;
        }
        flush();
      }
      acc |= wv[u];
    }
  }
  while (cur < n_e) flush();
  if (lane < static_cast<int>(cur - win)) emit(e_beg + win + lane, mine);  // the last, partial window
}

// A warp's range: `Off` is int32_t when the whole roadmap has fewer than
// kNarrowLimit nonzeros and edges (so every range fits), int64_t otherwise.

template <int U, typename Off, typename Gather, typename Emit>
__device__ __forceinline__ void stream_range(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                             const Gather gather, int64_t e_beg, int64_t e_end, uint64_t pol,
                                             int lane, Emit emit) {
  const int64_t p0 = __ldg(rowptr + e_beg), p1 = __ldg(rowptr + e_end);
  stream_body<U, Off>(rowptr, colidx, gather, e_beg, e_end, p0, p1, pol, lane, emit);
}

// Resident CTAs per SM each streaming variant is compiled for: deeper
// pipelines hold more entries in flight per warp and get more registers.
template <int U>
constexpr int stream_min_blocks() {
  return U <= 8 ? 4 : (U <= 12 ? 3 : 2);
}

template <int U, bool EPI, typename Off, typename T = uint64_t>
__global__ void __launch_bounds__(kThreads, stream_min_blocks<U>()) k_label_stream(const int64_t *__restrict__ rowptr,
                                                           const int32_t *__restrict__ colidx,
                                                           const T *__restrict__ O,
                                                           const int64_t *__restrict__ part, uint64_t mask,
                                                           uint64_t *__restrict__ L, MonitorTables mon,
                                                           const int32_t *__restrict__ perm) {
  __shared__ EpiSmem sm;
  if (EPI) load_tables(mon, sm);
  const uint64_t pol = evict_first_policy();
  const int lane = threadIdx.x & 31;
  const int64_t w = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t e_beg = __ldg(part + w), e_end = __ldg(part + w + 1);
  if (e_beg >= e_end) return;  // warp-uniform
  stream_range<U, Off>(rowptr, colidx, WordGather<T>{O}, e_beg, e_end, pol, lane, [&](int64_t e, uint64_t r) {
    r &= mask;
    const int64_t o = perm ? static_cast<int64_t>(__ldg(perm + e)) : e;  // the caller's edge
    L[o] = r;
    if (EPI) epilogue(mon, sm, o, r);
  });
}

// Moving-front form of the streaming gather-OR (quadtree rows in locality
// order, large roadmaps): one CTA of kFrontWarps warps per SM owns the edges
// its SM's warps would own in the stream partition (a contiguous range), cut
// into chunks of `chunk` edges; the warps take chunks in order from a
// shared-memory counter.  The warps of an SM then label neighbouring edges at
// the same time, so the pyramid words their rows share are gathered while
// they are still in the SM's L1 (1M-edge workload: gather misses per edge
// 33 -> 19 sectors).  Each chunk is streamed by stream_range as a range of
// its own.  The last `tail` edges of the range come in chunks of `small`
// edges, so the warps' last chunks end closer together (1M-edge call 0.2608
// -> 0.2586 ms, 2^21-cell paper frame 0.2626 -> 0.2566 ms with the last 512
// edges in chunks of 8).
//
// With pf_bytes > 0, the warp that takes a chunk asks L2 for the first
// pf_bytes of the index stream that follows it (one bulk prefetch by lane 0,
// no registers held): the warp that takes the next chunk, typically within a
// microsecond, then finds its first index groups in L2 instead of waiting on
// DRAM.  Measured on the 1M-edge call (64-bit pyramid words, chunks of 24 edges
// of ~23 KB of indices): no prefetch 0.2539 ms, 2 / 4 / 6 / 8 / 10 / 12 / 16 KB
// 0.2536 / 0.2507 / 0.2484 / 0.2469 / 0.2460 / 0.2463 / 0.2485 ms; the chunk's
// own entries instead 0.2650 ms.  The 2^21-cell 2-D frame (1-byte words, rows
// in the tiled order and sorted for locality): 0.1560 ms without, 2 / 4 / 8 /
// 10 / 12 / 16 / 24 KB 0.1557 / 0.1535 / 0.1517 / 0.1513 / 0.1509 / 0.1514 /
// 0.1518 ms.  The (x, y, tau) frame, whose rows keep the caller's order (the
// chunks of a CTA are not neighbours in space): 0.3035 ms without, 4 / 8 KB
// 0.3095 / 0.3065 ms.  So the front prefetches only rows the library put in
// locality order.  The same warp also asks L2 for the next chunk's
// entries of the row order (`perm`, read when a window of labels is written
// out): 1M-edge call 0.2464 -> 0.2459 ms, paper frame unchanged.  (The
// next chunk's last row pointer, likewise: no change, 0.2457 ms.)
constexpr int kFrontWarps = 32;
constexpr int kFrontTailChunk = 8;
constexpr int kFrontPrefetchBytes = 10240;
template <int U, bool EPI, typename T>
__global__ void __launch_bounds__(kFrontWarps * 32, 1) k_label_front(const int64_t *__restrict__ rowptr,
                                                                    const int32_t *__restrict__ idx,
                                                                    const T *__restrict__ O,
                                                                    const int64_t *__restrict__ part, int stride,
                                                                    int chunk, int tail, int small, uint64_t mask,
                                                                    uint64_t *__restrict__ L, MonitorTables mon,
                                                                    const int32_t *__restrict__ perm, int pf_bytes,
                                                                    int64_t idx_bytes) {
  __shared__ EpiSmem sm;
  __shared__ int next_chunk;
  // The monitor tables are written once, when the monitor is created, so
  // they are loaded before waiting for the kernel before (the frame
  // transform), while its last CTAs run.
  if (threadIdx.x == 0) next_chunk = 0;
  if (EPI)
    load_tables(mon, sm);  // contains __syncthreads
  else
    __syncthreads();
  pdl_wait();
  const uint64_t pol = evict_first_policy();
  const int lane = threadIdx.x & 31;
  const int64_t r0 = __ldg(part + static_cast<int64_t>(blockIdx.x) * stride);
  const int64_t r1 = __ldg(part + static_cast<int64_t>(blockIdx.x + 1) * stride);
  const int64_t rb = r1 - min(r1 - r0, static_cast<int64_t>(tail));  // [rb, r1): chunks of `small` edges
  const int64_t nbig = (rb - r0 + chunk - 1) / chunk;
  for (;;) {
    int c = 0;
    if (lane == 0) c = atomicAdd(&next_chunk, 1);
    c = __shfl_sync(kFull, c, 0);
    int64_t e_beg, e_end;
    if (c < nbig) {
      e_beg = r0 + static_cast<int64_t>(c) * chunk;
      e_end = min(rb, e_beg + chunk);
    } else {
      e_beg = rb + (static_cast<int64_t>(c) - nbig) * small;
      e_end = min(r1, e_beg + small);
    }
    if (e_beg >= r1) return;  // warp-uniform
    const int64_t p0 = __ldg(rowptr + e_beg), p1 = __ldg(rowptr + e_end);
    if (perm && lane < 2) {  // the next chunk's caller-order indices into L2 (its first and last)
      const int32_t *q = perm + min(e_end + lane * (e_end - e_beg), r1 - 1);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
    }
    if (pf_bytes > 0 && lane == 0) {  // the start of the next chunk's index stream into L2
      const int64_t a = (p1 * 4 + 15) & ~static_cast<int64_t>(15);
      const int64_t b = min(p1 * 4 + pf_bytes, idx_bytes) & ~static_cast<int64_t>(15);
      if (b > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const char *>(idx) + a),
                     "r"(static_cast<uint32_t>(b - a))
                     : "memory");
    }
    stream_body<U, int32_t>(rowptr, idx, WordGather<T>{O}, e_beg, e_end, p0, p1, pol, lane,
                            [&](int64_t e, uint64_t r) {
                              r &= mask;
                              const int64_t o = perm ? static_cast<int64_t>(__ldg(perm + e)) : e;  // the caller's edge
                              L[o] = r;
                              if (EPI) epilogue(mon, sm, o, r);
                            });
  }
}

// Sector form (compressed A at L2-sector granularity): an entry is
// (sector << 4) | mask, sector = 4 consecutive cells of O (32 bytes), mask
// bit i = cell 4*sector + i is in the row; 0 = no entry (a real entry has a
// non-empty mask).  A lane fetches its whole sector with one 256-bit load and
// ORs the words its mask selects; the stream, partition and boundary logic
// are the CSR stream's, over entries instead of cells.
struct SectorGather {
  const uint64_t *__restrict__ O;  // 32-byte aligned
  int64_t cells;
  static constexpr int32_t kNone = 0;
  __device__ __forceinline__ uint64_t pick(uint32_t v) const {
    const int64_t c0 = static_cast<int64_t>(v >> 4) * 4;
    const uint32_t m = v & 15u;
    uint64_t a, b, c, d;
    if (c0 + 4 <= cells) {
      asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(O + c0));
    } else {  // the grid's last, partial sector: only the cells that exist
      a = __ldg(O + c0);
      b = c0 + 1 < cells ? __ldg(O + c0 + 1) : 0ull;
      c = c0 + 2 < cells ? __ldg(O + c0 + 2) : 0ull;
      d = 0ull;
    }
    return ((m & 1u) ? a : 0ull) | ((m & 2u) ? b : 0ull) | ((m & 4u) ? c : 0ull) | ((m & 8u) ? d : 0ull);
  }
  __device__ __forceinline__ uint64_t full(int32_t v) const { return pick(static_cast<uint32_t>(v)); }
  __device__ __forceinline__ uint64_t masked(int32_t v) const { return v ? pick(static_cast<uint32_t>(v)) : 0ull; }
};

template <int U, bool EPI, typename Off>
__global__ void __launch_bounds__(kThreads, stream_min_blocks<2 * U>()) k_label_sector(const int64_t *__restrict__ srow,
                                                           const int32_t *__restrict__ sec,
                                                           const uint64_t *__restrict__ O, int64_t cells,
                                                           const int64_t *__restrict__ part, uint64_t mask,
                                                           uint64_t *__restrict__ L, MonitorTables mon) {
  __shared__ EpiSmem sm;
  if (EPI) load_tables(mon, sm);
  const uint64_t pol = evict_first_policy();
  const int lane = threadIdx.x & 31;
  const int64_t w = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t e_beg = __ldg(part + w), e_end = __ldg(part + w + 1);
  if (e_beg >= e_end) return;  // warp-uniform
  stream_range<U, Off>(srow, sec, SectorGather{O, cells}, e_beg, e_end, pol, lane, [&](int64_t e, uint64_t r) {
    r &= mask;
    L[e] = r;
    if (EPI) epilogue(mon, sm, e, r);
  });
}

// Batched streaming labels: many roadmaps (one frame each) in one launch.  The
// batch plan cut item i into `units` nonzero-balanced edge ranges (unit ids
// [unit0_i, unit0_i + units_i), in item order).  Warps take units from a
// global counter (zeroed before the launch), so the load stays balanced and
// only the few items being worked on keep their O words hot in L2.  Monitor
// tables, if any, are read through L1.
template <int U, typename Off, typename W = uint64_t>
__global__ void __launch_bounds__(kThreads, stream_min_blocks<U>()) k_label_batch(const __grid_constant__ BatchTable tab,
                                                          unsigned long long *__restrict__ next_unit) {
  const uint64_t pol = evict_first_policy();
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(next_unit, 1ull);
    u = __shfl_sync(kFull, u, 0);
    if (u >= static_cast<unsigned long long>(tab.total)) return;
    const int64_t unit = static_cast<int64_t>(u);
    int lo = 0, hi = tab.n - 1;  // last item with unit0 <= unit
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (tab.items[mid].warp0 <= unit)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BatchItem *it = tab.items + lo;  // in the constant bank
    const int64_t lu = unit - it->warp0;
    if (lu >= it->warps) continue;
    const int64_t *part = it->part;
    const int64_t e_beg = __ldg(part + lu), e_end = __ldg(part + lu + 1);
    if (e_beg >= e_end) continue;
    stream_range<U, Off>(it->rowptr, it->colidx, WordGather<W>{static_cast<const W *>(it->O)}, e_beg, e_end, pol,
                         lane, [&](int64_t e, uint64_t r) {
      r &= it->mask;
      const int32_t *perm = it->perm;
      const int64_t o = perm ? static_cast<int64_t>(__ldg(perm + e)) : e;  // the caller's edge
      it->L[o] = r;
      const uint64_t *T = it->T;
      if (T) {
        uint32_t letter = 0;
        const int m = it->m;
        for (int j = 0; j < m; ++j) letter |= static_cast<uint32_t>((r >> it->rel[j]) & 1u) << j;
        it->next[o] = __ldg(T + letter);
        it->viol[o] = __ldg(it->V + letter);
      }
    });
  }
}

// Quadtree pyramid of O (quad_pyramid_of): one CTA per 256-cell block of the
// top level, each thread loading the word of its cell.
// In the tiled order (tiled_w > 0) the CTA's block is one 16 x 16 tile, read
// from the row-major O.
template <typename T>
__device__ __forceinline__ void quad_pyramid_block(const uint64_t *__restrict__ O, int64_t cells,
                                                   const QuadOffsets &off, T *__restrict__ pyr, int64_t blk,
                                                   uint64_t *wsum, int32_t tiled_w) {
  const int64_t i = blk * kThreads + threadIdx.x;
  int64_t src = i;
  if (tiled_w > 0) {
    uint32_t x, y;
    tiled_cell(tiled_w, blk, threadIdx.x, x, y);
    src = static_cast<int64_t>(y) * tiled_w + x;
  }
  quad_pyramid_of<T>(i < cells ? __ldg(O + src) : 0ull, cells, off, pyr, blk, wsum);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_quad_pyramid(const uint64_t *__restrict__ O, int64_t cells,
                                                           QuadOffsets off, T *__restrict__ pyr, int32_t tiled_w) {
  __shared__ uint64_t wsum[kThreads / 32];
  pdl_wait();
  pdl_trigger();
  quad_pyramid_block<T>(O, cells, off, pyr, blockIdx.x, wsum, tiled_w);
}

// The same for many frames in one launch: CTA b finds its item (the last with
// block0 <= b) and builds that item's top-level block b - block0.
__global__ void __launch_bounds__(kThreads) k_quad_pyramid_batch(const __grid_constant__ PyrTable tab) {
  __shared__ uint64_t wsum[kThreads / 32];
  const int64_t b = blockIdx.x;
  int lo = 0, hi = tab.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (tab.items[mid].block0 <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  const PyrItem &it = tab.items[lo];
  const int64_t blk = b - it.block0;
  switch (it.word_bytes) {  // CTA-uniform
    case 1:
      quad_pyramid_block<uint8_t>(it.O, it.cells, it.off, static_cast<uint8_t *>(it.pyr), blk, wsum, it.tiled_w);
      break;
    case 2:
      quad_pyramid_block<uint16_t>(it.O, it.cells, it.off, static_cast<uint16_t *>(it.pyr), blk, wsum, it.tiled_w);
      break;
    case 4:
      quad_pyramid_block<uint32_t>(it.O, it.cells, it.off, static_cast<uint32_t *>(it.pyr), blk, wsum, it.tiled_w);
      break;
    default:
      quad_pyramid_block<uint64_t>(it.O, it.cells, it.off, static_cast<uint64_t *>(it.pyr), blk, wsum, it.tiled_w);
  }
}

// ---------------------------------------------------------------------------
// Bulk-copy (TMA engine) form of the streaming gather-OR.  Same partition and
// boundary logic as k_label_stream, but each warp's index stream is moved by
// cp.async.bulk into a per-warp ring of kStages shared-memory chunks of
// kChunk indices, one mbarrier per chunk.  Lane 0 issues the copies; every
// lane reads its entries from shared memory (consecutive, conflict free) and
// issues kChunk/32 independent gathers.  The index stream therefore never
// waits on gathers and needs no registers for prefetching.
constexpr int kStages = 6;
constexpr int kChunk = 256;                   // indices per chunk (1 KiB)
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound on the drain after a wait gave up

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(bar))),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  // potentially blocking: the thread is suspended until the phase completes or
  // a system-dependent time limit passes
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(bar))), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(bar))), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity, by every lane of the warp
// (each lane's own acquire makes the copied bytes visible to it).  The timer
// is read only when a try_wait returns without the phase.  False after
// limit_ns; a limit of 0 only tests the phase once, without waiting.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, int lane, uint64_t limit_ns) {
  if (limit_ns == 0) return __all_sync(kFull, mbar_test_wait(bar, parity));
  bool ok = mbar_try_wait(bar, parity);
  if (__all_sync(kFull, ok)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    if (!ok) ok = mbar_try_wait(bar, parity);
    if (__all_sync(kFull, ok)) return true;
    const uint64_t t = __shfl_sync(kFull, global_ns(), 0);
    if (t - t0 > limit_ns) return false;
  }
  return false;
}

// cp.async.bulk of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol) {
  const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(bar));
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
      "l"(src), "r"(bytes), "r"(b), "l"(pol)
      : "memory");
}

template <bool EPI>
__global__ void __launch_bounds__(kThreads, 4) k_label_tma(const int64_t *__restrict__ rowptr,
                                                           const int32_t *__restrict__ colidx,
                                                           const uint64_t *__restrict__ O,
                                                           const int64_t *__restrict__ part, uint64_t mask,
                                                           uint64_t *__restrict__ L, MonitorTables mon,
                                                           int *__restrict__ err, uint64_t wait_ns) {
  constexpr int W = kThreads / 32;
  constexpr int J = kChunk / 32;
  __shared__ __align__(128) int32_t ring[W][kStages][kChunk];
  __shared__ __align__(8) uint64_t bars[W][kStages];
  __shared__ EpiSmem sm;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  if (lane == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(&bars[wid][st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (EPI) load_tables(mon, sm);  // contains __syncthreads
  __syncwarp();
  const uint64_t pol = evict_first_policy();
  const int64_t w = static_cast<int64_t>(blockIdx.x) * W + wid;
  const int64_t e_beg = __ldg(part + w), e_end = __ldg(part + w + 1);
  if (e_beg >= e_end) return;  // warp-uniform
  int64_t win = e_beg;
  int64_t rp = win + lane < e_end ? __ldg(rowptr + win + lane + 1) : 0;
  int64_t cur = e_beg;
  int64_t stop = __shfl_sync(kFull, rp, 0);
  const int64_t p0 = __ldg(rowptr + e_beg), p1 = __ldg(rowptr + e_end);
  const int64_t a4 = p0 & ~static_cast<int64_t>(3);        // 16-byte aligned start
  const int64_t end4 = (p1 + 3) & ~static_cast<int64_t>(3);  // inside the padded allocation
  const int64_t n_chunks = (end4 - a4 + kChunk - 1) / kChunk;
  uint64_t acc = 0;

  auto flush = [&]() {
    uint64_t r = warp_or(acc);
    if (lane == 0) {
      r &= mask;
      L[cur] = r;
      if (EPI) epilogue(mon, sm, cur, r);
    }
    acc = 0;
    ++cur;
    if (cur < e_end) {
      if (cur - win == 32) {
        win = cur;
        rp = win + lane < e_end ? __ldg(rowptr + win + lane + 1) : 0;
      }
      stop = __shfl_sync(kFull, rp, static_cast<int>(cur - win));
    }
  };
  auto issue = [&](int64_t i) {  // lane 0 only
    const int64_t start = a4 + i * kChunk;
    const int64_t n = end4 - start < kChunk ? end4 - start : kChunk;
    bulk_load(ring[wid][i % kStages], colidx + start, static_cast<uint32_t>(n * 4), &bars[wid][i % kStages], pol);
  };

  if (lane == 0)
    for (int64_t i = 0; i < kStages && i < n_chunks; ++i) issue(i);
  for (int64_t i = 0; i < n_chunks; ++i) {
    const int st = static_cast<int>(i % kStages);
    if (!warp_wait(&bars[wid][st], static_cast<uint32_t>((i / kStages) & 1), lane, wait_ns)) {
      // give up: record it, let the copies still in flight (chunks i to
      // i + kStages - 1) land, leave
      if (lane == 0) {
        atomicExch(err, 1);
        for (int64_t j = i; j < n_chunks && j < i + kStages; ++j) {
          const uint64_t t0 = global_ns();
          while (!mbar_try_wait(&bars[wid][j % kStages], static_cast<uint32_t>((j / kStages) & 1)) &&
                 global_ns() - t0 < kWaitNs) {
          }
        }
      }
      __syncwarp();
      return;
    }
    const int64_t cb = a4 + i * kChunk;  // global index of ring entry 0
    const int64_t lo64 = p0 - cb, hi64 = p1 - cb;
    const int lo = lo64 < 0 ? 0 : static_cast<int>(lo64);
    const int hi = hi64 > kChunk ? kChunk : static_cast<int>(hi64);
    uint64_t wv[J];
    if (lo == 0 && hi == kChunk) {  // every entry of the chunk is valid
#pragma unroll
      for (int j = 0; j < J; ++j) wv[j] = __ldg(O + ring[wid][st][32 * j + lane]);
    } else {
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int off = 32 * j + lane;
        const int32_t c = (off >= lo && off < hi) ? ring[wid][st][off] : -1;
        wv[j] = c >= 0 ? __ldg(O + c) : 0ull;
      }
    }
    if (min(cb + kChunk, p1) <= stop) {
#pragma unroll
      for (int j = 0; j < J; ++j) acc |= wv[j];
    } else {
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int64_t k = cb + 32 * j + lane;
        const int64_t sub_end = min(cb + 32 * (j + 1), p1);
        while (sub_end > stop) {
          if (k < stop) {
            acc |= wv[j];
            wv[j] = 0;
          }
          flush();
        }
        acc |= wv[j];
      }
    }
    __syncwarp();  // every lane is done with this chunk's shared memory
    if (lane == 0 && i + kStages < n_chunks) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(i + kStages);
    }
  }
  while (cur < e_end) flush();
}

// ---------------------------------------------------------------------------
// Asynchronous-copy form of the streaming gather-OR: every lane copies 2 x 16
// bytes (8 indices) of the warp's index stream into a per-warp shared-memory
// ring with cp.async, one commit group per 256-index stage, kAsyncStages - 1
// stages ahead of the 8 gathers per lane of the stage being consumed.
// Waiting is cp.async.wait_group (the warp is descheduled, nothing polls), and
// indices in flight occupy shared memory instead of registers.
constexpr int kAsyncStages = 4;
constexpr int kAsyncStage = 256;  // indices per stage: 32 lanes x 2 x 16 bytes

__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src), "r"(src_bytes)
               : "memory");
}

template <bool EPI>
__global__ void __launch_bounds__(kThreads, 4) k_label_async(const int64_t *__restrict__ rowptr,
                                                             const int32_t *__restrict__ colidx,
                                                             const uint64_t *__restrict__ O,
                                                             const int64_t *__restrict__ part, uint64_t mask,
                                                             uint64_t *__restrict__ L, MonitorTables mon) {
  constexpr int W = kThreads / 32;
  constexpr int J = kAsyncStage / 32;
  __shared__ __align__(128) int32_t ring[W][kAsyncStages][kAsyncStage];
  __shared__ EpiSmem sm;
  if (EPI) load_tables(mon, sm);
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int64_t w = static_cast<int64_t>(blockIdx.x) * W + wid;
  const int64_t e_beg = __ldg(part + w), e_end = __ldg(part + w + 1);
  if (e_beg >= e_end) return;  // warp-uniform
  int64_t win = e_beg;
  int64_t rp = win + lane < e_end ? __ldg(rowptr + win + lane + 1) : 0;
  int64_t cur = e_beg;
  int64_t stop = __shfl_sync(kFull, rp, 0);
  const int64_t p0 = __ldg(rowptr + e_beg), p1 = __ldg(rowptr + e_end);
  const int64_t a4 = p0 & ~static_cast<int64_t>(3);        // 16-byte aligned start
  const int64_t end4 = (p1 + 3) & ~static_cast<int64_t>(3);  // inside the padded allocation
  const int64_t n_st = (end4 - a4 + kAsyncStage - 1) / kAsyncStage;
  uint64_t acc = 0;

  auto flush = [&]() {
    uint64_t r = warp_or(acc);
    if (lane == 0) {
      r &= mask;
      L[cur] = r;
      if (EPI) epilogue(mon, sm, cur, r);
    }
    acc = 0;
    ++cur;
    if (cur < e_end) {
      if (cur - win == 32) {
        win = cur;
        rp = win + lane < e_end ? __ldg(rowptr + win + lane + 1) : 0;
      }
      stop = __shfl_sync(kFull, rp, static_cast<int>(cur - win));
    }
  };
  // stage i: lane copies indices [a4 + 256 i + 128 h + 4 lane, +4), h = 0, 1,
  // when they start before end4 (zero-filled otherwise)
  auto issue = [&](int64_t i) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t src = a4 + i * kAsyncStage + 128 * h + 4 * lane;
      const bool in = i < n_st && src < end4;
      cp_async16(&ring[wid][i % kAsyncStages][128 * h + 4 * lane], colidx + (in ? src : a4), in ? 16u : 0u);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  for (int64_t i = 0; i < kAsyncStages - 1; ++i) issue(i);
  for (int64_t i = 0; i < n_st; ++i) {
    issue(i + kAsyncStages - 1);  // always one group per iteration, possibly empty
    asm volatile("cp.async.wait_group %0;" ::"n"(kAsyncStages - 1) : "memory");
    __syncwarp();  // every lane's part of stage i has landed
    const int st = static_cast<int>(i % kAsyncStages);
    const int64_t cb = a4 + i * kAsyncStage;
    uint64_t wv[J];
    if (cb >= p0 && cb + kAsyncStage <= p1) {
#pragma unroll
      for (int j = 0; j < J; ++j) wv[j] = __ldg(O + ring[wid][st][32 * j + lane]);
    } else {
      const int64_t lo64 = p0 - cb, hi64 = p1 - cb;
      const int lo = lo64 < 0 ? 0 : static_cast<int>(lo64);
      const int hi = hi64 > kAsyncStage ? kAsyncStage : static_cast<int>(hi64);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int off = 32 * j + lane;
        wv[j] = (off >= lo && off < hi) ? __ldg(O + ring[wid][st][off]) : 0ull;
      }
    }
    if (min(cb + kAsyncStage, p1) <= stop) {
#pragma unroll
      for (int j = 0; j < J; ++j) acc |= wv[j];
    } else {
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int64_t k = cb + 32 * j + lane;
        const int64_t sub_end = min(cb + 32 * (j + 1), p1);
        while (sub_end > stop) {
          if (k < stop) {
            acc |= wv[j];
            wv[j] = 0;
          }
          flush();
        }
        acc |= wv[j];
      }
    }
    __syncwarp();  // stage i is free before any lane refills it
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  while (cur < e_end) flush();
}

// Edge partition of the streaming kernel: part[w] = first edge e with
// (rowptr[e] - rowptr[0]) + edge_cost * e >= w * total / W
// (total = rowptr[E] - rowptr[0] + edge_cost * E; rowptr may be a slice of a
// roadmap's row pointer, so it need not start at 0).
__global__ void k_partition(const int64_t *__restrict__ rowptr, int64_t E, int64_t W, int64_t edge_cost,
                            int64_t *__restrict__ part) {
  const int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w > W) return;
  const int64_t r0 = rowptr[0];
  const int64_t total = rowptr[E] - r0 + edge_cost * E;
  const int64_t target = w == W ? total : total / W * w + (total % W) * w / W;
  int64_t lo = 0, hi = E;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (rowptr[mid] - r0 + edge_cost * mid < target)
      lo = mid + 1;
    else
      hi = mid;
  }
  part[w] = lo;
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
// step; lane owns propositions q = lane % LPB + t * LPB (t < 2 only when LPB is
// 32 and P > 32).  Each lane keeps one hit flag per owned proposition; the
// entry loop is unrolled so several entries' plane loads are in flight.
template <int LPB, bool EPI, bool EARLY>
__global__ void __launch_bounds__(kThreads) k_label_bt(const int64_t *__restrict__ brow,
                                                       const uint32_t *__restrict__ bblock,
                                                       const uint64_t *__restrict__ bmask,
                                                       const uint64_t *__restrict__ planes, int32_t P, int64_t E,
                                                       uint64_t mask, uint64_t *__restrict__ L, MonitorTables mon) {
  constexpr int EPS = 32 / LPB;
  constexpr int T = LPB == 32 ? 2 : 1;
  __shared__ EpiSmem sm;
  if (EPI) load_tables(mon, sm);
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPB;
  const int pl = lane % LPB;
  bool owns[T];
#pragma unroll
  for (int t = 0; t < T; ++t) owns[t] = pl + t * LPB < P;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * kThreads) >> 5;
  for (int64_t e = warp; e < E; e += nwarps) {
    const int64_t beg = __ldg(brow + e), end = __ldg(brow + e + 1);
    bool hit[T];
#pragma unroll
    for (int t = 0; t < T; ++t) hit[t] = false;
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
      const int64_t k = k0 + lane;
      uint32_t b = 0;
      uint64_t m = 0;
      if (k < end) {
        b = __ldg(bblock + k);
        m = __ldg(bmask + k);
      }
      const int n = static_cast<int>(end - k0 < 32 ? end - k0 : 32);
#pragma unroll 4
      for (int j = 0; j < n; j += EPS) {
        const int src = j + sub;  // < 32; lanes past the row's end carry m = 0
        const uint32_t bj = __shfl_sync(kFull, b, src);
        const uint64_t mj = __shfl_sync(kFull, m, src);
        const uint64_t *pp = planes + static_cast<int64_t>(bj) * P + pl;
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const uint64_t v = owns[t] ? __ldg(pp + t * LPB) : 0ull;
          hit[t] |= (v & mj) != 0;
        }
      }
      if (EARLY) {
        uint64_t r = 0;
#pragma unroll
        for (int t = 0; t < T; ++t) r |= static_cast<uint64_t>(hit[t]) << (pl + t * LPB);
        r = warp_or(r);
        if ((r & mask) == mask) break;  // warp-uniform: r is the same in every lane
      }
    }
    uint64_t word = 0;
#pragma unroll
    for (int t = 0; t < T; ++t) word |= static_cast<uint64_t>(hit[t]) << (pl + t * LPB);
    word = warp_or(word);
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
  return run_csr<LPE, 4, EPI, EARLY>(rm, O, mask, L, mon, ctas_per_sm, s);
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

int sector_ctas_per_sm(int depth) {
  static const int o4 = std::min(occupancy(k_label_sector<4, false, int32_t>), occupancy(k_label_sector<4, true, int32_t>));
  static const int o8 = std::min(occupancy(k_label_sector<8, false, int32_t>), occupancy(k_label_sector<8, true, int32_t>));
  return depth == 8 ? o8 : o4;
}

template <int U, typename Off>
void sector_launch(const Roadmap &rm, const uint64_t *O, uint64_t mask, uint64_t *L, const MonitorTables *mon,
                   cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(rm.num_sms * rm.sec_part_ctas);
  MonitorTables none{};
  if (mon)
    k_label_sector<U, true, Off><<<grid, kThreads, 0, s>>>(rm.sec_rowptr, rm.sec, O, rm.cells, rm.sec_part, mask, L,
                                                           *mon);
  else
    k_label_sector<U, false, Off><<<grid, kThreads, 0, s>>>(rm.sec_rowptr, rm.sec, O, rm.cells, rm.sec_part, mask,
                                                            L, none);
}

cudaError_t launch_label_sector(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                                const MonitorTables *mon, int depth, cudaStream_t s) {
  if (rm.E == 0) return cudaSuccess;
  const uint64_t mask = prop_mask(P);
  if (rm.n_sec >= kNarrowLimit || rm.E >= kNarrowLimit)
    sector_launch<4, int64_t>(rm, O, mask, L, mon, s);
  else if (depth == 8)
    sector_launch<8, int32_t>(rm, O, mask, L, mon, s);
  else
    sector_launch<4, int32_t>(rm, O, mask, L, mon, s);
  return cudaGetLastError();
}

int batch_ctas_per_sm(int depth) {
  static const int o8 = std::min(occupancy(k_label_batch<8, int32_t>), occupancy(k_label_batch<8, int64_t>));
  static const int o12 = occupancy(k_label_batch<12, int32_t>);
  return depth == 12 ? o12 : o8;
}

cudaError_t launch_label_batch(const BatchTable &tab, unsigned long long *counter, int num_sms, int ctas_per_sm,
                               cudaStream_t s) {
  if (tab.total == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const unsigned grid = static_cast<unsigned>(num_sms * ctas_per_sm);
  const int wb = tab.word_bytes ? tab.word_bytes : 8;
  if (tab.wide) {
    if (wb != 8) return cudaErrorInvalidValue;
    k_label_batch<8, int64_t><<<grid, kThreads, 0, s>>>(tab, counter);
  } else if (tab.depth == 12) {
    switch (wb) {
      case 1: k_label_batch<12, int32_t, uint8_t><<<grid, kThreads, 0, s>>>(tab, counter); break;
      case 2: k_label_batch<12, int32_t, uint16_t><<<grid, kThreads, 0, s>>>(tab, counter); break;
      case 4: k_label_batch<12, int32_t, uint32_t><<<grid, kThreads, 0, s>>>(tab, counter); break;
      default: k_label_batch<12, int32_t><<<grid, kThreads, 0, s>>>(tab, counter);
    }
  } else {
    switch (wb) {
      case 1: k_label_batch<8, int32_t, uint8_t><<<grid, kThreads, 0, s>>>(tab, counter); break;
      case 2: k_label_batch<8, int32_t, uint16_t><<<grid, kThreads, 0, s>>>(tab, counter); break;
      case 4: k_label_batch<8, int32_t, uint32_t><<<grid, kThreads, 0, s>>>(tab, counter); break;
      default: k_label_batch<8, int32_t><<<grid, kThreads, 0, s>>>(tab, counter);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_partition_into(const int64_t *rowptr, int64_t E, int64_t W, int64_t *part, cudaStream_t s) {
  if (E == 0 || W == 0) return cudaSuccess;
  k_partition<<<static_cast<unsigned>((W + 1 + 255) / 256), 256, 0, s>>>(rowptr, E, W, kEdgeCost, part);
  return cudaGetLastError();
}

int tma_ctas_per_sm() {
  static const int occ = std::min(occupancy(k_label_tma<false>), occupancy(k_label_tma<true>));
  return occ;
}

cudaError_t launch_label_tma(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L, const MonitorTables *mon,
                             cudaStream_t s) {
  if (rm.E == 0) return cudaSuccess;
  const uint64_t mask = prop_mask(P);
  const unsigned grid = static_cast<unsigned>(rm.num_sms * rm.part_ctas);
  MonitorTables none{};
  if (mon)
    k_label_tma<true><<<grid, kThreads, 0, s>>>(rm.rowptr, rm.colidx, O, rm.part, mask, L, *mon, rm.err,
                                                 static_cast<uint64_t>(rm.wait_ns));
  else
    k_label_tma<false><<<grid, kThreads, 0, s>>>(rm.rowptr, rm.colidx, O, rm.part, mask, L, none, rm.err,
                                                  static_cast<uint64_t>(rm.wait_ns));
  return cudaGetLastError();
}

int async_ctas_per_sm() {
  static const int occ = std::min(occupancy(k_label_async<false>), occupancy(k_label_async<true>));
  return occ;
}

cudaError_t launch_label_async(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                               const MonitorTables *mon, cudaStream_t s) {
  if (rm.E == 0) return cudaSuccess;
  const uint64_t mask = prop_mask(P);
  const unsigned grid = static_cast<unsigned>(rm.num_sms * rm.part_ctas);
  MonitorTables none{};
  if (mon)
    k_label_async<true><<<grid, kThreads, 0, s>>>(rm.rowptr, rm.colidx, O, rm.part, mask, L, *mon);
  else
    k_label_async<false><<<grid, kThreads, 0, s>>>(rm.rowptr, rm.colidx, O, rm.part, mask, L, none);
  return cudaGetLastError();
}

// The stream kernels use shared memory only for the monitor tables (2.5 KB a
// CTA).  The smallest carveout that still holds four CTAs' tables leaves the
// rest of the SM's 256 KB to L1, which serves the pyramid gathers: 1M-edge
// labeling call 0.282 vs 0.285 ms with the default carveout, 0.308 ms at a
// 25 % carveout, 0.346 ms at 50 %.
constexpr int kStreamCarveoutPct = 5;

template <int U, typename Off, typename T>
void carve_stream() {
  cudaFuncSetAttribute(k_label_stream<U, true, Off, T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       kStreamCarveoutPct);
  cudaFuncSetAttribute(k_label_stream<U, false, Off, T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       kStreamCarveoutPct);
}

template <int U>
void carve_stream_widths() {
  carve_stream<U, int32_t, uint8_t>();
  carve_stream<U, int32_t, uint16_t>();
  carve_stream<U, int32_t, uint32_t>();
  carve_stream<U, int32_t, uint64_t>();
}

// Once per process, before the first occupancy query (roadmap upload), so
// never inside a stream capture.
void configure_stream_kernels() {
  static const bool done = [] {
    carve_stream_widths<8>();
    carve_stream_widths<12>();
    carve_stream_widths<16>();
    carve_stream<8, int64_t, uint64_t>();
    cudaGetLastError();  // an attribute the device ignores is not an error of any later call
    return true;
  }();
  (void)done;
}

int stream_ctas_per_sm(int depth) {
  configure_stream_kernels();
  static const int o8 = std::min(occupancy(k_label_stream<8, false, int32_t>), occupancy(k_label_stream<8, true, int32_t>));
  static const int o12 =
      std::min(occupancy(k_label_stream<12, false, int32_t>), occupancy(k_label_stream<12, true, int32_t>));
  static const int o16 =
      std::min(occupancy(k_label_stream<16, false, int32_t>), occupancy(k_label_stream<16, true, int32_t>));
  return depth == 16 ? o16 : depth == 12 ? o12 : o8;
}

cudaError_t launch_partition(const Roadmap &rm, int ctas_per_sm, cudaStream_t s) {
  const int64_t W = static_cast<int64_t>(rm.num_sms) * ctas_per_sm * (kThreads / 32);
  if (rm.E == 0 || W + 1 > rm.part_cap) return cudaErrorInvalidValue;
  k_partition<<<static_cast<unsigned>((W + 1 + 255) / 256), 256, 0, s>>>(rm.rowptr, rm.E, W, kEdgeCost, rm.part);
  return cudaGetLastError();
}

template <int U, typename Off, typename T>
void rows_launch(const StreamRows &r, const T *base, uint64_t mask, uint64_t *L, const MonitorTables *mon,
                 int num_sms, cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(num_sms * r.part_ctas);
  MonitorTables none{};
  if (mon)
    k_label_stream<U, true, Off, T><<<grid, kThreads, 0, s>>>(r.rowptr, r.idx, base, r.part, mask, L, *mon, r.perm);
  else
    k_label_stream<U, false, Off, T><<<grid, kThreads, 0, s>>>(r.rowptr, r.idx, base, r.part, mask, L, none, r.perm);
}

// Chunk size of the moving front for a range of E edges (0: the per-warp
// stream instead).  Measured on quadtree rows in locality order (1M, 500k and
// 250k edges of the 512x512, 64-proposition workload; 1.1M edges of the
// 2^21-cell workload): 24 edges per chunk from ~6,000 edges per SM (-7 % on
// 1M edges), 16 from ~3,000 (-2 % on 500k); below that too few chunks per
// warp to balance the CTA (250k: +3 %, 100k: +20 %).
int front_chunk_for(int64_t E, int num_sms) {
  const int64_t per_sm = E / (num_sms > 0 ? num_sms : 1);
  return per_sm >= 6000 ? 24 : per_sm >= 3000 ? 16 : 0;
}

template <typename T>
void front_launch(const StreamRows &r, const T *base, uint64_t mask, uint64_t *L, const MonitorTables *mon,
                  int chunk, int num_sms, cudaStream_t s) {
  static const bool carved = [] {
    cudaFuncSetAttribute(k_label_front<8, true, T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         kStreamCarveoutPct);
    cudaFuncSetAttribute(k_label_front<8, false, T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         kStreamCarveoutPct);
    cudaGetLastError();  // an attribute the device ignores is not an error of any later call
    return true;
  }();
  (void)carved;
  const int stride = r.part_ctas * (kThreads / 32);  // partition entries (warps) per SM = per front CTA
  const unsigned grid = static_cast<unsigned>(num_sms);
  const int small = std::min(chunk, kFrontTailChunk);
  const int tail = 2 * kFrontWarps * small;
  const int pf = r.perm ? kFrontPrefetchBytes : 0;  // rows in the library's locality order
  const int64_t idx_bytes = r.entries * 4;  // prefetches stay inside the rows' entries
  MonitorTables none{};
  const dim3 g(grid), b(kFrontWarps * 32);
  if (mon)
    pdl_launch(k_label_front<8, true, T>, g, b, s, r.rowptr, r.idx, base, r.part, stride, chunk, tail, small, mask, L,
               *mon, r.perm, pf, idx_bytes);
  else
    pdl_launch(k_label_front<8, false, T>, g, b, s, r.rowptr, r.idx, base, r.part, stride, chunk, tail, small, mask,
               L, none, r.perm, pf, idx_bytes);
}

template <typename T>
void rows_launch_depth(const StreamRows &r, const T *base, uint64_t mask, uint64_t *L, const MonitorTables *mon,
                       int depth, int num_sms, cudaStream_t s) {
  // the front reads the stream partition of depth 8 (kFrontWarps warps per SM)
  const int chunk = r.front_chunk < 0 ? front_chunk_for(r.E, num_sms) : r.front_chunk;
  if (chunk > 0 && depth == 8 && r.part_ctas * (kThreads / 32) == kFrontWarps) {
    front_launch<T>(r, base, mask, L, mon, chunk, num_sms, s);
    return;
  }
  if (depth == 16)
    rows_launch<16, int32_t, T>(r, base, mask, L, mon, num_sms, s);
  else if (depth == 12)
    rows_launch<12, int32_t, T>(r, base, mask, L, mon, num_sms, s);
  else
    rows_launch<8, int32_t, T>(r, base, mask, L, mon, num_sms, s);
}

cudaError_t launch_label_rows(const StreamRows &r, const void *base, int word_bytes, int32_t P, uint64_t *L,
                              const MonitorTables *mon, int depth, int num_sms, cudaStream_t s) {
  if (r.E == 0) return cudaSuccess;
  const uint64_t mask = prop_mask(P);
  if (r.entries >= kNarrowLimit || r.E >= kNarrowLimit) {  // wide rows gather 64-bit words only
    if (word_bytes != 8) return cudaErrorInvalidValue;
    rows_launch<8, int64_t, uint64_t>(r, static_cast<const uint64_t *>(base), mask, L, mon, num_sms, s);
  } else if (word_bytes == 1) {
    rows_launch_depth(r, static_cast<const uint8_t *>(base), mask, L, mon, depth, num_sms, s);
  } else if (word_bytes == 2) {
    rows_launch_depth(r, static_cast<const uint16_t *>(base), mask, L, mon, depth, num_sms, s);
  } else if (word_bytes == 4) {
    rows_launch_depth(r, static_cast<const uint32_t *>(base), mask, L, mon, depth, num_sms, s);
  } else {
    rows_launch_depth(r, static_cast<const uint64_t *>(base), mask, L, mon, depth, num_sms, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_label_stream(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                                const MonitorTables *mon, int depth, cudaStream_t s) {
  const StreamRows r{rm.rowptr, rm.colidx, rm.part, rm.part_ctas, rm.E, rm.nnz, nullptr};
  return launch_label_rows(r, O, 8, P, L, mon, depth, rm.num_sms, s);
}

int quad_word_bytes(const Roadmap &rm, int32_t P) {
  if (rm.n_qd >= kNarrowLimit || rm.E >= kNarrowLimit) return 8;
  return P <= 8 ? 1 : P <= 16 ? 2 : P <= 32 ? 4 : 8;
}

cudaError_t launch_quad_pyramid(const Roadmap &rm, const uint64_t *O, int word_bytes, void *pyr, cudaStream_t s) {
  if (rm.cells == 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((rm.cells + kThreads - 1) / kThreads);
  const dim3 g(grid), b(kThreads);
  switch (word_bytes) {  // launched dependent on the frame transform before it
    case 1: return pdl_launch(k_quad_pyramid<uint8_t>, g, b, s, O, rm.cells, rm.qd_off, static_cast<uint8_t *>(pyr),
                              rm.qd_tiled_w);
    case 2: return pdl_launch(k_quad_pyramid<uint16_t>, g, b, s, O, rm.cells, rm.qd_off, static_cast<uint16_t *>(pyr),
                               rm.qd_tiled_w);
    case 4: return pdl_launch(k_quad_pyramid<uint32_t>, g, b, s, O, rm.cells, rm.qd_off, static_cast<uint32_t *>(pyr),
                               rm.qd_tiled_w);
    default: return pdl_launch(k_quad_pyramid<uint64_t>, g, b, s, O, rm.cells, rm.qd_off, static_cast<uint64_t *>(pyr),
                               rm.qd_tiled_w);
  }
}

cudaError_t launch_quad_pyramid_batch(const PyrTable &tab, cudaStream_t s) {
  if (tab.n == 0 || tab.total == 0) return cudaSuccess;
  k_quad_pyramid_batch<<<static_cast<unsigned>(tab.total), kThreads, 0, s>>>(tab);
  return cudaGetLastError();
}

cudaError_t launch_label_quad(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                              const MonitorTables *mon, int depth, cudaStream_t s, int front_chunk) {
  if (rm.E == 0) return cudaSuccess;
  const int wb = quad_word_bytes(rm, P);
  if (O) {
    cudaError_t e = launch_quad_pyramid(rm, O, wb, rm.pyr, s);
    if (e != cudaSuccess) return e;
  }
  StreamRows r{rm.qd_rowptr, rm.qd_idx, rm.qd_part, rm.qd_part_ctas, rm.E, rm.n_qd, rm.qd_perm};
  r.front_chunk = front_chunk;
  return launch_label_rows(r, rm.pyr, wb, P, L, mon, depth, rm.num_sms, s);
}

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
