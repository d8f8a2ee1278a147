// Dense tensor-core form of the labeling product (Sec. 4.2, eq. 8-10): with
// A the 0/1 trajectory matrix (edges x cells) and O the 0/1 proposition matrix
// (cells x propositions), the count matrix A.O has entry (e, p) > 0 exactly
// when eq. 10's OR is true.  The counts are small integers, exact in fp32, and
// 0/1 are exact in e4m3, so the product runs on the 5th-generation tensor
// cores (tcgen05.mma, kind::f8f6f4; the int8 kind is not available on sm_103a)
// with fp32 accumulators in tensor memory.
//
// Layout (derived at upload, LBL_UPLOAD_MMA): edges in locality order are cut
// into tiles of 128 (the MMA's M); the cell axis into K-blocks of 128 cells of
// the cell order.  For each tile only the K-blocks its rows touch are kept, as
// 128 x 128 bit matrices (2 KiB).  Per frame, O becomes one e4m3 matrix of N x
// 128 per K-block (N = the propositions rounded up to 16, 32 or 64).
//
// k_label_mma: one CTA of 128 threads per tile (thread r owns tile row r).
// For each touched K-block the threads expand the row bits to e4m3 bytes in
// shared memory and copy the block's B matrix beside them; one thread issues
// four MMAs (K = 32 each) that accumulate D = A.B^T in tensor memory and
// commits them to an mbarrier; after the tile's last block each thread reads
// its row of D (tcgen05.ld) and sets label bit p iff D[r][p] > 0.  Every wait
// is bounded: after 2 s the kernel records an error and stops.
#include <vector>

#include "lbl_internal.cuh"

namespace lbl {
namespace {

constexpr int kMmaM = 128;   // edges per tile
constexpr int kMmaK = 128;   // cells per K-block
constexpr int kCoreRow = 16; // bytes per core-matrix row (8 rows x 16 bytes per core matrix)
constexpr int kSbo = (kMmaK / kCoreRow) * 128;  // bytes between 8-row groups of an operand tile
constexpr int kLbo = 128;                       // bytes between K-adjacent core matrices
constexpr unsigned long long kMmaWaitNs = 2000000000ull;
// CTAs per SM of the labeling kernel: each holds 64 tensor-memory columns at
// most (6 x 64 <= 512) and ~27 KB of shared memory.
constexpr int kMmaCtasPerSm = 6;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t mma_clock_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor of tcgen05: start address, leading (K) and
// stride (8-row group) byte offsets, all >> 4; descriptor version 1 (bits
// 46-48); no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: D fp32 (bits 4-5 = 1), A and B e4m3
// (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
template <int N>
__host__ __device__ constexpr uint32_t mma_idesc() {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(kMmaM >> 4) << 24);
}

// Bounded wait for the phase of `bar` with the given parity; false after
// limit_ns (a limit of 0 tests the phase once, without waiting).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns = kMmaWaitNs) {
  if (limit_ns == 0) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
  }
  const uint64_t t0 = mma_clock_ns();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    if (ok) return true;
    if (mma_clock_ns() - t0 > limit_ns) return false;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// 16 bits of a row -> 16 e4m3 bytes (1.0 = 0x38, 0.0 = 0): a nibble spread to
// one bit per byte by a multiply that places bit i at bit 8i (no carries).
__device__ __forceinline__ uint32_t nibble_bytes(uint32_t nib) { return ((nib * 0x00204081u) & 0x01010101u) * 0x38u; }

// Mark in a shared bitmap the K-blocks touched by the rows of tile blockIdx.x
// (sorted positions 128 t + r, caller's edge perm[..]).
__device__ __forceinline__ void mark_tile_blocks(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                                                 const int32_t *__restrict__ perm, int64_t E, uint32_t *bm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int r = wid; r < kMmaM; r += nwarps) {
    const int64_t s = static_cast<int64_t>(blockIdx.x) * kMmaM + r;
    if (s >= E) break;
    const int64_t e = perm ? perm[s] : s;
    for (int64_t k = rowptr[e] + lane; k < rowptr[e + 1]; k += 32) {
      const uint32_t b = static_cast<uint32_t>(colidx[k]) / kMmaK;
      atomicOr(&bm[b >> 5], 1u << (b & 31));
    }
  }
}

__global__ void __launch_bounds__(256) k_mma_count(const int64_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ colidx,
                                                   const int32_t *__restrict__ perm, int64_t E, int32_t nkb,
                                                   int64_t *__restrict__ count) {
  extern __shared__ uint32_t bm[];
  __shared__ int part[8];
  const int nw = (nkb + 31) >> 5;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) bm[i] = 0;
  __syncthreads();
  mark_tile_blocks(rowptr, colidx, perm, E, bm);
  __syncthreads();
  int c = 0;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) c += __popc(bm[i]);
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) t += part[w];
    count[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_mma_fill(const int64_t *__restrict__ rowptr,
                                                  const int32_t *__restrict__ colidx,
                                                  const int32_t *__restrict__ perm, int64_t E, int32_t nkb,
                                                  const int64_t *__restrict__ tptr, int32_t *__restrict__ tblk,
                                                  uint32_t *__restrict__ bits) {
  extern __shared__ uint32_t sh[];
  const int nw = (nkb + 31) >> 5;
  uint32_t *bm = sh, *pre = sh + nw;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) bm[i] = 0;
  __syncthreads();
  mark_tile_blocks(rowptr, colidx, perm, E, bm);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int i = 0; i < nw; ++i) {
      pre[i] = acc;
      acc += __popc(bm[i]);
    }
  }
  __syncthreads();
  const int64_t base = tptr[blockIdx.x];
  for (int i = threadIdx.x; i < nw; i += blockDim.x) {  // the tile's K-blocks, ascending
    uint32_t w = bm[i], rank = pre[i];
    while (w) {
      const int j = __ffs(w) - 1;
      w &= w - 1;
      tblk[base + rank++] = i * 32 + j;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int r = wid; r < kMmaM; r += nwarps) {
    const int64_t s = static_cast<int64_t>(blockIdx.x) * kMmaM + r;
    if (s >= E) break;
    const int64_t e = perm ? perm[s] : s;
    for (int64_t k = rowptr[e] + lane; k < rowptr[e + 1]; k += 32) {
      const uint32_t c = static_cast<uint32_t>(colidx[k]);
      const uint32_t b = c / kMmaK, j = c % kMmaK;
      const uint32_t rank = pre[b >> 5] + __popc(bm[b >> 5] & ((1u << (b & 31)) - 1u));
      atomicOr(&bits[((base + rank) * kMmaM + r) * 4 + (j >> 5)], 1u << (j & 31));
    }
  }
}

// B of K-block kb: element (n, k) = bit n of O[128 kb + k] (0 past the grid),
// e4m3 0/1, core matrix (n/8, k/16) at (n/8)*kSbo + (k/16)*kLbo, row n%8 at
// 16 bytes each.  One thread per (kb, n, k/16): 16 bytes.
__global__ void __launch_bounds__(256) k_mma_bexpand(const uint64_t *__restrict__ O, int64_t cells, int32_t nkb,
                                                     int32_t N, uint8_t *__restrict__ B) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<int64_t>(nkb) * N * 8) return;
  const int kc = static_cast<int>(i & 7);
  const int n = static_cast<int>((i >> 3) % N);
  const int64_t kb = (i >> 3) / N;
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t c = kb * kMmaK + kc * 16 + q * 4 + j;
      const uint64_t o = c < cells ? __ldg(O + c) : 0ull;
      v |= static_cast<uint32_t>((o >> n) & 1u) << (8 * j);
    }
    w[q] = v * 0x38u;
  }
  uint8_t *dst = B + kb * (static_cast<int64_t>(N) * kMmaK) + (n / 8) * kSbo + kc * kLbo + (n % 8) * kCoreRow;
  *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

template <int N, bool EPI>
__global__ void __launch_bounds__(kMmaM, kMmaCtasPerSm) k_label_mma(const int64_t *__restrict__ tptr,
                                                        const int32_t *__restrict__ tblk,
                                                        const uint4 *__restrict__ bits, const uint8_t *__restrict__ B,
                                                        int64_t T, int64_t E, const int32_t *__restrict__ perm,
                                                        uint64_t mask, uint64_t *__restrict__ L, MonitorTables mon,
                                                        int *__restrict__ err, uint64_t wait_ns) {
  constexpr int NCOL = N < 32 ? 32 : N;  // tensor-memory columns: a power of two >= 32
  __shared__ __align__(1024) uint8_t sA[kMmaM * kMmaK];
  __shared__ __align__(1024) uint8_t sB[N * kMmaK];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ EpiSmem sm;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (EPI) load_tables(mon, sm);  // contains __syncthreads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
  uint32_t phase = 0;
  bool ok = true;
  constexpr int BV = N * kMmaK / 16 / kMmaM;  // 16-byte pieces of a B block per thread
  for (int64_t t = blockIdx.x; t < T && ok; t += gridDim.x) {
    const int64_t k0 = tptr[t], k1 = tptr[t + 1];
    // the next block's row bits and B matrix are loaded into registers while
    // the current block's MMAs run
    uint4 w = make_uint4(0, 0, 0, 0), bq[BV];
    auto fetch = [&](int64_t i) {
      w = __ldg(bits + i * kMmaM + tid);
      const uint4 *src = reinterpret_cast<const uint4 *>(B + static_cast<int64_t>(__ldg(tblk + i)) * (N * kMmaK));
#pragma unroll
      for (int j = 0; j < BV; ++j) bq[j] = __ldg(src + tid + j * kMmaM);
    };
    if (k1 > k0) fetch(k0);
    for (int64_t i = k0; i < k1; ++i) {
      // A: this thread's row bits -> 128 e4m3 bytes, 16 per core matrix
      const uint32_t words[4] = {w.x, w.y, w.z, w.w};
      uint8_t *arow = sA + (tid / 8) * kSbo + (tid % 8) * kCoreRow;
#pragma unroll
      for (int kc = 0; kc < kMmaK / 16; ++kc) {
        const uint32_t h = (words[kc >> 1] >> (16 * (kc & 1))) & 0xFFFFu;
        *reinterpret_cast<uint4 *>(arow + kc * kLbo) =
            make_uint4(nibble_bytes(h & 15u), nibble_bytes((h >> 4) & 15u), nibble_bytes((h >> 8) & 15u),
                       nibble_bytes(h >> 12));
      }
      // B: the block's matrix, already in the operand layout
#pragma unroll
      for (int j = 0; j < BV; ++j) reinterpret_cast<uint4 *>(sB)[tid + j * kMmaM] = bq[j];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy writes -> the MMA's reads
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int kk = 0; kk < kMmaK / 32; ++kk) {
          const uint64_t ad = smem_desc(a0 + kk * 2 * kLbo, kLbo, kSbo);
          const uint64_t bd = smem_desc(b0 + kk * 2 * kLbo, kLbo, kSbo);
          const uint32_t acc = (i > k0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(mma_idesc<N>()), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar))
                     : "memory");
      }
      __syncwarp();
      if (i + 1 < k1) fetch(i + 1);
      // every thread waits for the MMAs before shared memory is refilled
      ok = mbar_wait_bounded(&bar, phase & 1u, wait_ns);
      ++phase;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
    }
    if (!ok) break;
    // this thread's row of D -> label bits
    uint64_t word = 0;
    if (k1 > k0) {
#pragma unroll
      for (int c = 0; c < N; c += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) word |= static_cast<uint64_t>(r[j] != 0u) << (c + j);
      }
    }
    word &= mask;
    const int64_t s = t * kMmaM + tid;
    if (s < E) {
      const int64_t o = perm ? static_cast<int64_t>(__ldg(perm + s)) : s;  // the caller's edge
      L[o] = word;
      if (EPI) epilogue(mon, sm, o, word);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // every row read before the next tile's MMAs overwrite the accumulator
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok) {  // a wait gave up: record it, give the MMAs in flight one more bounded wait before freeing
    if (tid == 0) atomicExch(err, 1);
    mbar_wait_bounded(&bar, (phase - 1u) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
}

// Rate probe of the MMA the form uses: every CTA holds one 128 x 128 A tile
// and one N x 128 B tile of 0/1 values in shared memory (e4m3, or bf16 for
// comparison) and accumulates `reps` times their product (4 MMAs of K = 32,
// or 8 of K = 16) in tensor memory.  CTA 0 writes its accumulator to D, so
// the host can check that every count is exact.
template <int KIND, int N>
__global__ void __launch_bounds__(kMmaM, 1) k_mma_probe(const uint8_t *__restrict__ a01,
                                                        const uint8_t *__restrict__ b01, int reps,
                                                        float *__restrict__ D, int *__restrict__ err) {
  constexpr int KT = KIND == 0 ? kMmaK : kMmaK / 2;  // elements per tile row (128 bytes of K either way)
  constexpr int EB = KIND == 0 ? 1 : 2;
  constexpr int T = kCoreRow / EB;
  constexpr int KSTEP = KIND == 0 ? 32 : 16;
  constexpr int NCOL = N < 32 ? 32 : N;
  __shared__ __align__(1024) uint8_t sA[kMmaM * KT * EB];
  __shared__ __align__(1024) uint8_t sB[N * KT * EB];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < kMmaM * KT; i += kMmaM) {
    const int r = i / KT, k = i % KT;
    uint8_t *d = sA + (r / 8) * kSbo + (k / T) * kLbo + (r % 8) * kCoreRow + (k % T) * EB;
    if (KIND == 0) {
      d[0] = a01[i] ? 0x38 : 0;
    } else {
      d[0] = a01[i] ? 0x80 : 0;  // bf16 1.0 = 0x3F80, little-endian
      d[1] = a01[i] ? 0x3F : 0;
    }
  }
  for (int i = tid; i < N * KT; i += kMmaM) {
    const int n = i / KT, k = i % KT;
    uint8_t *d = sB + (n / 8) * kSbo + (k / T) * kLbo + (n % 8) * kCoreRow + (k % T) * EB;
    if (KIND == 0) {
      d[0] = b01[i] ? 0x38 : 0;
    } else {
      d[0] = b01[i] ? 0x80 : 0;
      d[1] = b01[i] ? 0x3F : 0;
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  // D fp32; A, B e4m3 (kind::f8f6f4) or bf16 (kind::f16, format 1 at bits 7-9 and 10-12); K-major
  constexpr uint32_t idesc = (1u << 4) | ((KIND == 0 ? 0u : 1u) << 7) | ((KIND == 0 ? 0u : 1u) << 10) |
                             (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(kMmaM >> 4) << 24);
  if (tid == 0) {
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    for (int rep = 0; rep < reps; ++rep) {
#pragma unroll
      for (int kk = 0; kk < KT / KSTEP; ++kk) {
        const uint64_t ad = smem_desc(a0 + kk * 2 * kLbo, kLbo, kSbo), bd = smem_desc(b0 + kk * 2 * kLbo, kLbo, kSbo);
        const uint32_t acc = (rep > 0 || kk > 0) ? 1u : 0u;
        if (KIND == 0)
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        else
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                 : "memory");
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0);
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && blockIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < N; c += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c), r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) D[tid * N + c + j] = __uint_as_float(r[j]);
    }
  }
  if (!ok) mbar_wait_bounded(&bar, 0);  // the MMAs in flight land before the memory is freed
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
}

unsigned grid_of(int64_t n, int per) { return static_cast<unsigned>((n + per - 1) / per); }

template <int N>
cudaError_t run_mma(const Roadmap &rm, uint64_t mask, uint64_t *L, const MonitorTables *mon, cudaStream_t s) {
  const int64_t g = std::min<int64_t>(rm.mma_T, static_cast<int64_t>(rm.num_sms) * kMmaCtasPerSm);
  MonitorTables none{};
  if (mon)
    k_label_mma<N, true><<<static_cast<unsigned>(g), kMmaM, 0, s>>>(
        rm.mma_tptr, rm.mma_tblk, reinterpret_cast<const uint4 *>(rm.mma_bits), rm.mma_b, rm.mma_T, rm.E,
        rm.mma_perm, mask, L, *mon, rm.err, static_cast<uint64_t>(rm.wait_ns));
  else
    k_label_mma<N, false><<<static_cast<unsigned>(g), kMmaM, 0, s>>>(
        rm.mma_tptr, rm.mma_tblk, reinterpret_cast<const uint4 *>(rm.mma_bits), rm.mma_b, rm.mma_T, rm.E,
        rm.mma_perm, mask, L, none, rm.err, static_cast<uint64_t>(rm.wait_ns));
  return cudaGetLastError();
}

}  // namespace

int mma_n_of(int32_t P) { return P <= 16 ? 16 : P <= 32 ? 32 : 64; }

cudaError_t launch_mma_count(const int64_t *rowptr, const int32_t *colidx, const int32_t *perm, int64_t E,
                             int32_t nkb, int64_t *count, cudaStream_t s) {
  const int64_t T = (E + kMmaM - 1) / kMmaM;
  if (T == 0) return cudaSuccess;
  const size_t sh = sizeof(uint32_t) * ((nkb + 31) / 32);
  k_mma_count<<<static_cast<unsigned>(T), 256, sh, s>>>(rowptr, colidx, perm, E, nkb, count);
  return cudaGetLastError();
}

cudaError_t launch_mma_fill(const int64_t *rowptr, const int32_t *colidx, const int32_t *perm, int64_t E,
                            int32_t nkb, const int64_t *tptr, int32_t *tblk, uint32_t *bits, cudaStream_t s) {
  const int64_t T = (E + kMmaM - 1) / kMmaM;
  if (T == 0) return cudaSuccess;
  const size_t sh = 2 * sizeof(uint32_t) * ((nkb + 31) / 32);
  k_mma_fill<<<static_cast<unsigned>(T), 256, sh, s>>>(rowptr, colidx, perm, E, nkb, tptr, tblk, bits);
  return cudaGetLastError();
}

cudaError_t launch_label_mma(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L, const MonitorTables *mon,
                             cudaStream_t s) {
  if (rm.E == 0) return cudaSuccess;
  const int N = mma_n_of(P);
  const int64_t work = static_cast<int64_t>(rm.mma_nkb) * N * 8;
  k_mma_bexpand<<<grid_of(work, 256), 256, 0, s>>>(O, rm.cells, rm.mma_nkb, N, rm.mma_b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint64_t mask = P >= 64 ? ~0ull : ((1ull << P) - 1ull);
  if (N == 16) return run_mma<16>(rm, mask, L, mon, s);
  if (N == 32) return run_mma<32>(rm, mask, L, mon, s);
  return run_mma<64>(rm, mask, L, mon, s);
}

}  // namespace lbl

extern "C" int lbl_mma_probe(int32_t kind, int32_t n, int32_t reps, int32_t ctas_per_sm, double *tflops,
                             int32_t *exact) {
  using namespace lbl;
  set_error("%s", "");
  if ((kind != 0 && kind != 1) || (n != 16 && n != 64 && !(kind == 0 && n == 128)) || reps < 1 || reps > 100000 ||
      ctas_per_sm < 1 || ctas_per_sm > 4 || !tflops || !exact) {
    set_error("mma probe: kind 0 (e4m3) with n 16, 64 or 128, or kind 1 (bf16) with n 16 or 64; reps 1..100000; "
              "ctas_per_sm 1..4; non-NULL outputs");
    return LBL_EINVAL;
  }
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "mma probe: device");
  const int KT = kind == 0 ? 128 : 64;
  std::vector<uint8_t> a(static_cast<size_t>(128) * KT), b(static_cast<size_t>(n) * KT);
  uint32_t x = 12345u;  // a fixed xorshift stream: about 1/5 of A and 1/3 of B set
  auto next = [&]() { x ^= x << 13; x ^= x >> 17; x ^= x << 5; return x; };
  for (auto &v : a) v = (next() % 5u) == 0u;
  for (auto &v : b) v = (next() % 3u) == 0u;
  uint8_t *da = nullptr, *db = nullptr;
  float *dD = nullptr;
  int *derr = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(da);
    cudaFree(db);
    cudaFree(dD);
    cudaFree(derr);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
  };
  if ((e = dev_alloc(&da, a.size(), nullptr)) != cudaSuccess || (e = dev_alloc(&db, b.size(), nullptr)) != cudaSuccess ||
      (e = dev_alloc(&dD, static_cast<size_t>(128) * n, nullptr)) != cudaSuccess ||
      (e = dev_alloc(&derr, 1, nullptr)) != cudaSuccess || (e = cudaMemset(derr, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaMemcpy(da, a.data(), a.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(db, b.data(), b.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "mma probe: set-up");
  }
  auto launch = [&](unsigned grid, int r) {
    if (kind == 0 && n == 16) k_mma_probe<0, 16><<<grid, kMmaM>>>(da, db, r, dD, derr);
    else if (kind == 0 && n == 64) k_mma_probe<0, 64><<<grid, kMmaM>>>(da, db, r, dD, derr);
    else if (kind == 0) k_mma_probe<0, 128><<<grid, kMmaM>>>(da, db, r, dD, derr);
    else if (n == 16) k_mma_probe<1, 16><<<grid, kMmaM>>>(da, db, r, dD, derr);
    else k_mma_probe<1, 64><<<grid, kMmaM>>>(da, db, r, dD, derr);
    return cudaGetLastError();
  };
  const unsigned grid = static_cast<unsigned>(sms * ctas_per_sm);
  float ms = 0.0f;
  if ((e = launch(1, 3)) != cudaSuccess || (e = cudaStreamSynchronize(nullptr)) != cudaSuccess ||
      (e = cudaEventRecord(t0)) != cudaSuccess || (e = launch(grid, reps)) != cudaSuccess ||
      (e = cudaEventRecord(t1)) != cudaSuccess || (e = cudaEventSynchronize(t1)) != cudaSuccess ||
      (e = cudaEventElapsedTime(&ms, t0, t1)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "mma probe: run");
  }
  std::vector<float> D(static_cast<size_t>(128) * n);
  int herr = 0;
  // the timed launch's CTA 0 overwrote D with reps x A.B^T; the check uses it
  if ((e = cudaMemcpy(D.data(), dD, sizeof(float) * D.size(), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "mma probe: read back");
  }
  bool same = herr == 0;
  for (int m = 0; m < 128 && same; ++m)
    for (int j = 0; j < n && same; ++j) {
      int c = 0;
      for (int k = 0; k < KT; ++k) c += a[static_cast<size_t>(m) * KT + k] * b[static_cast<size_t>(j) * KT + k];
      same = D[static_cast<size_t>(m) * n + j] == static_cast<float>(c) * static_cast<float>(reps);
    }
  *exact = same ? 1 : 0;
  *tflops = 2.0 * 128.0 * n * KT * static_cast<double>(reps) * grid / (static_cast<double>(ms) * 1e-3) / 1e12;
  cleanup();
  if (herr) {
    set_error("mma probe: a bounded wait gave up");
    return LBL_ETIMEOUT;
  }
  return LBL_OK;
}
