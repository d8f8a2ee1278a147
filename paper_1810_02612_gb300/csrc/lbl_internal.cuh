// Internal declarations of liblbl (not part of the C ABI).
//
// Device layouts (all in HBM, all library-owned unless noted):
//   rowptr  int64[E+1]            CSR row pointer of M (eq. 11)
//   colidx  int32[nnz + pad]      CSR column indices, padded to a multiple of 4
//                                 plus 4 so 16-byte vector loads never leave the
//                                 allocation
//   O       uint64[cells]         caller-owned proposition word per agent cell
//   bt_*                          64-cell block form of M: per edge a list of
//                                 (block id, 64-bit cell mask) entries, block b =
//                                 cells [64b, 64b+64) in the grid's cell order
//   planes  uint64[blocks][P]     bit-plane re-layout of O for the block form:
//                                 bit i of planes[b][p] = bit p of O[64b + i]
//   qd_*                          quadtree form of M: each row as the union of its
//                                 maximal blocks of 4^k consecutive cells (k <= 4)
//                                 starting at a multiple of 4^k; an entry is the
//                                 index of the block's word in the pyramid
//   pyr     uint64[~4/3 cells]    per-frame pyramid: level k, block b holds the OR
//                                 of O over cells [b 4^k, (b+1) 4^k)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbl.h"

namespace lbl {

constexpr int kThreads = 256;  // threads per CTA of every labeling kernel
constexpr int kMaxCtasPerSm = 8;  // 2048 resident threads per SM / kThreads
constexpr int64_t kEdgeCost = 32;  // partition weight of one edge, in nonzeros
// Streamed row sets with fewer entries and edges than this keep positions in
// 32-bit registers (headroom for the group arithmetic).
constexpr int64_t kNarrowLimit = (1LL << 31) - 4096;

struct MonitorTables {
  const uint64_t *T;  // T[letter]: packed next states of all monitor states
  const uint16_t *V;  // V[letter]: violation mask
  uint64_t *next;
  uint16_t *viol;
  int32_t m;
  uint8_t rel[8];
};

// The fused safety-monitor epilogue (Sec. 3.2) of the labeling kernels: the
// monitor's next-state and violation tables staged in shared memory, and per
// edge the letter formed from the label's relevant bits.
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

// Programmatic dependent launch.  The kernels of one frame (plane packing,
// frame transform, pyramid, labels) each depend on the one before; launched
// with pdl_launch, a kernel's CTAs are placed on the SMs while the kernel
// before it finishes (that kernel lets them in with pdl_trigger at its start),
// so the launch gap between the two shrinks.  A kernel launched this way calls
// pdl_wait first: it returns once the kernel before has completed and its
// writes are visible, so nothing is read or written early.  Launched the usual
// way, pdl_wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// One roadmap's share of a batched labeling launch (device table entry).
struct BatchItem {
  const int64_t *rowptr;
  const int32_t *colidx;
  const int64_t *part;  // warps + 1 entries
  const void *O;  // gather base: words of the table's word_bytes (O itself, or the item's pyramid)
  uint64_t *L, *next;
  uint16_t *viol;
  const uint64_t *T;  // monitor tables, NULL without a monitor
  const uint16_t *V;
  uint64_t mask;
  int64_t warp0, warps;  // work units [warp0, warp0 + warps) of the batch
  const int32_t *perm;   // output index of row e (NULL: e)
  int32_t m;
  uint8_t rel[8];
};

// One frame's share of a batched frame-transform launch (device table entry).
struct FrameItem {
  int64_t A00, A01, B0, A10, A11, B1;  // Q32.32 map
  int64_t At, Bt;                      // Q32.32 time map
  const uint8_t *planes;
  uint64_t *O;
  int64_t plane_cells;  // ww * wh * wd
  int64_t cell0;        // first global cell of this frame
  int32_t ww, wh, wd, aw, ah, ad, P, order;
  const void *words;  // packed world words (bit p = plane p), or NULL: read the planes
  uint64_t wmask;     // 2^P - 1, applied to packed words
  int32_t word_bytes; // width of a packed word: 1, 2, 4 or 8
};

// Packing world planes into one word per world cell (bit p = plane p != 0).
struct PackItem {
  const uint8_t *planes;
  void *words;         // cells words of word_bytes each
  int64_t cells;       // world cells (w * h * d)
  int32_t P;
  int32_t word_bytes;  // 1, 2, 4 or 8, at least P bits
};

// Width of a packed world word: the narrowest of 1, 2, 4 and 8 bytes that holds P bits.
inline int packed_word_bytes(int32_t P) { return P <= 8 ? 1 : P <= 16 ? 2 : P <= 32 ? 4 : 8; }
// Sessions pack the planes when they hold at least kPackedMinPlaneBytes (below
// that, a second small launch costs more than the byte gathers it saves) and
// the world has at most kPackedWorldRatio times the agent's cells.
constexpr int64_t kPackedMinPlaneBytes = 8ll << 20;
constexpr int64_t kPackedWorldRatio = 4;

// Batched launches take their whole item table as one kernel parameter.
constexpr int kMaxBatch = 128;
struct BatchTable {
  BatchItem items[kMaxBatch];
  int32_t n;
  int32_t wide;   // some item has 2^31 - 4096 or more nonzeros or edges (64-bit words only)
  int32_t depth;  // groups in flight per warp: 12 when every item streams quadtree rows, else 8
  int32_t word_bytes;  // width of every item's gathered words: 1, 2, 4 or 8 (0 = 8)
  int64_t total;  // work units
};
struct FrameTable {
  FrameItem items[kMaxBatch];
  int32_t n;
  int64_t total;  // cells
};

// Batched packing: item i packs lanes [lane0[i], lane0[i+1]) of the launch, a
// lane per four world cells, into 64-bit words.
struct PackTable {
  PackItem items[kMaxBatch];
  int32_t vec[kMaxBatch];  // the item's planes and words allow vector loads and stores
  int64_t lane0[kMaxBatch + 1];
  int32_t n;
};

// Levels of the quadtree form: blocks of up to 4^4 = 256 cells.
constexpr int kQuadLevels = 4;
// Default register pipeline depth of the quadtree stream (groups of 32 entries
// in flight per warp).  With the rows in locality order a third of the
// gathers hit L1, and four CTAs per SM at depth 8 beat three at depth 12
// (and five or six at depths 6 or 4) on every single-frame workload.
constexpr int kQuadDepth = 8;
// The locality order sorts the quadtree rows inside each of this many equal
// ranges of the caller's edges, not across the whole roadmap (with the moving
// front: 0.2528 vs 0.2618 ms on the 1M-edge call, rows pre-sorted).
constexpr int kOrderRanges = 4;
// Host-buffer sessions label roadmaps of at least this many edges on their own
// stream, pyramid and partition.
constexpr int64_t kSessionChunkMinEdges = 1 << 16;
struct QuadOffsets {
  int64_t at[kQuadLevels + 1];  // first pyramid word of each level
};

// Cell (x, y) of a row-major grid tiled_w cells wide that tiled index
// 256 * tile + t stands for: tiles of 16 x 16 cells in row-major order, t the
// z-order index inside the tile (x in the odd bits, y in the even bits).
__device__ __forceinline__ void tiled_cell(int32_t tiled_w, int64_t tile, uint32_t t, uint32_t &x, uint32_t &y) {
  const int64_t tw = tiled_w >> 4;
  uint32_t lx = 0, ly = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    lx |= ((t >> (2 * i + 1)) & 1u) << i;
    ly |= ((t >> (2 * i)) & 1u) << i;
  }
  x = static_cast<uint32_t>((tile % tw) * 16) + lx;
  y = static_cast<uint32_t>((tile / tw) * 16) + ly;
}

// Quadtree pyramid of O (compressed A): level k holds, for every block of 4^k
// consecutive cells in the grid's cell order that lies wholly inside the
// grid, the OR of their words; level 0 is O itself.  Word of block b at level
// k: pyr[off.at[k] + b].  One CTA of kThreads covers the 256 consecutive
// cells of top-level block `blk`, thread t holding v = the word of cell
// blk * 256 + t (0 past the grid): levels 1-2 (4 and 16 cells) by butterfly
// shuffles inside each warp, levels 3-4 (64 and 256 cells) from the eight
// 32-cell warp words in `wsum`.  Used by the pyramid kernels (which read v
// from O) and by the frame transform that builds the pyramid of the words it
// computes.
template <typename T>
__device__ __forceinline__ void quad_pyramid_of(uint64_t v, int64_t cells, const QuadOffsets &off,
                                                T *__restrict__ pyr, int64_t blk, uint64_t *wsum) {
  static_assert(kThreads == 256 && kQuadLevels == 4, "one CTA = one block of the top level");
  constexpr unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i = blk * kThreads + threadIdx.x;
  if (i < cells) pyr[i] = static_cast<T>(v);
  v |= __shfl_xor_sync(full, v, 1);
  v |= __shfl_xor_sync(full, v, 2);  // every lane: OR of its aligned 4-cell block
  if ((lane & 3) == 0 && (i >> 2) < (cells >> 2)) pyr[off.at[1] + (i >> 2)] = static_cast<T>(v);
  v |= __shfl_xor_sync(full, v, 4);
  v |= __shfl_xor_sync(full, v, 8);  // 16-cell block
  if ((lane & 15) == 0 && (i >> 4) < (cells >> 4)) pyr[off.at[2] + (i >> 4)] = static_cast<T>(v);
  v |= __shfl_xor_sync(full, v, 16);  // the warp's 32 cells
  if (lane == 0) wsum[wid] = v;
  __syncthreads();
  if (threadIdx.x < 4) {  // 64-cell blocks: warps (2t, 2t+1)
    const int t = threadIdx.x;
    const int64_t b = blk * 4 + t;
    if (b < (cells >> 6)) pyr[off.at[3] + b] = static_cast<T>(wsum[2 * t] | wsum[2 * t + 1]);
  } else if (threadIdx.x == 4) {  // the 256-cell block
    uint64_t a = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) a |= wsum[w];
    if (blk < (cells >> 8)) pyr[off.at[4] + blk] = static_cast<T>(a);
  }
}

// One item of a batched pyramid launch: O of a frame -> that frame's pyramid.
struct PyrItem {
  const uint64_t *O;
  void *pyr;       // words of word_bytes each
  int64_t cells;
  int64_t block0;  // first 256-cell block of this item in the launch
  QuadOffsets off;
  int32_t word_bytes;  // 1, 2, 4 or 8
  int32_t tiled_w;     // > 0: the pyramid is in the tiled order of a row-major grid this wide
};
// Batched label launches group their items by gathered word width.
constexpr int kWordClasses = 4;  // 1, 2, 4, 8 bytes
inline int word_class(int word_bytes) { return word_bytes == 1 ? 0 : word_bytes == 2 ? 1 : word_bytes == 4 ? 2 : 3; }
struct PyrTable {
  PyrItem items[128];
  int32_t n;
  int64_t total;  // 256-cell blocks over all items
};

// One streamed row set: CSR rows over some gather base (cells, sectors or
// pyramid words) with its warp partition.
struct StreamRows {
  const int64_t *rowptr;
  const int32_t *idx;
  const int64_t *part;
  int part_ctas;
  int64_t E, entries;
  const int32_t *perm;  // output index of row e (NULL: e); with perm the outputs are not offset
  int front_chunk = -1;  // moving front over chunks of this many edges; 0 = per-warp stream, -1 = by range size
};

// Memory owned by the library's objects (roadmaps, monitors, sessions,
// batches, servers) comes from the stream-ordered allocator.  Each object logs
// the last piece of work it enqueued on every stream it used (an event per
// stream); its *_free makes a library stream wait for those events and frees
// the memory there with cudaFreeAsync, so releasing one object neither waits
// for nor stalls work of others on the device.  Work a CUDA graph replays is
// not logged: the caller frees an object only after the replays that use it.
struct UseLog {
  std::mutex mu;
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> ev;
  void note(cudaStream_t s);  // record the object's latest work on s (skipped while s is capturing)
  // free `ptrs` in stream order after every logged use (the device must be the object's)
  void release(int device, const std::vector<void *> &ptrs);
};

struct Roadmap {
  std::shared_ptr<UseLog> uses = std::make_shared<UseLog>();
  int device = 0;
  int num_sms = 0;
  lbl_grid agent{};
  int64_t E = 0, nnz = 0, cells = 0;
  int64_t *rowptr = nullptr;
  int32_t *colidx = nullptr;
  // block form (optional)
  bool has_bt = false;
  int64_t n_bt = 0;        // entries
  int64_t n_blocks = 0;    // ceil(cells / 64)
  int64_t *bt_rowptr = nullptr;
  uint32_t *bt_block = nullptr;
  uint64_t *bt_mask = nullptr;
  uint64_t *planes = nullptr;  // n_blocks * 64 words of working memory
  // sector form (optional): per edge the entries (sector << 4) | 4-cell mask
  bool has_sec = false;
  int64_t n_sec = 0;
  int64_t *sec_rowptr = nullptr;
  int32_t *sec = nullptr;      // n_sec entries, padded like colidx
  int64_t *sec_part = nullptr;  // partition of the sector kernel's grid
  int sec_part_ctas = 0;
  // quadtree form (optional): per edge the pyramid indices of its maximal blocks
  bool has_qd = false;
  int64_t n_qd = 0;
  int64_t *qd_rowptr = nullptr;
  int32_t *qd_idx = nullptr;    // n_qd entries, padded like colidx
  // Quadtree row i is the caller's edge qd_perm[i]: inside each of the
  // kOrderRanges edge ranges the rows of a 2-D grid are sorted by the z-order
  // of their middle cell's (x, y), so a CTA's edges lie close together and
  // share pyramid lines in L1; NULL keeps the caller's order (time-augmented
  // grids, LBL_UPLOAD_KEEP_ORDER, roadmaps of 2^31 edges or more)
  int32_t *qd_perm = nullptr;
  int64_t *qd_part = nullptr;   // partition of the quadtree stream's grid
  int qd_part_ctas = 0;
  QuadOffsets qd_off{};
  int64_t pyr_words = 0;
  // > 0: the quadtree rows and the pyramid use the tiled order of this
  // row-major 2-D grid (its width; sides multiples of 16), 0: the cell order
  int32_t qd_tiled_w = 0;
  uint64_t *pyr = nullptr;      // per-frame pyramid (working memory)
  int pyr_built_bytes = 0;      // word width of the pyramid last enqueued into `pyr` (0: none yet)
  // dense tensor-core form (optional): edges in locality order in tiles of 128,
  // per tile the K-blocks of 128 cells its rows touch, as 128 x 128 bit
  // matrices (16 bytes per row); per-frame B operand as working memory
  bool has_mma = false;
  int64_t mma_T = 0;             // tiles
  int64_t n_mma = 0;             // (tile, K-block) pairs
  int32_t mma_nkb = 0;           // K-blocks of the grid
  int32_t *mma_perm = nullptr;   // sorted position -> the caller's edge
  int64_t *mma_tptr = nullptr;   // tile t's K-blocks: [mma_tptr[t], mma_tptr[t+1])
  int32_t *mma_tblk = nullptr;   // K-block ids, ascending per tile
  uint32_t *mma_bits = nullptr;  // n_mma x 128 rows x 4 words
  uint8_t *mma_b = nullptr;      // mma_nkb x 64 x 128 e4m3 bytes
  // edge partition of the streaming CSR kernel: warp w owns [part[w], part[w+1])
  int64_t *part = nullptr;
  int64_t part_cap = 0;  // entries allocated
  int part_ctas = 0;     // CTAs per SM the partition was made for
  int *err = nullptr;    // device flag: a bounded wait in a kernel ran out
  int64_t wait_ns = 2000000000;  // limit of those waits (lbl_roadmap_set_wait_limit)
  // AUTO choice per proposition count, set by lbl_roadmap_autotune
  bool tuned_valid[65] = {false};
  lbl_config tuned[65] = {};
  int64_t bytes = 0;
};

struct Monitor {
  std::shared_ptr<UseLog> uses = std::make_shared<UseLog>();
  int device = 0;
  int32_t n_states = 0, m = 0, reject = -1;
  uint8_t rel[8] = {0};
  uint64_t hT[256] = {0};
  uint16_t hV[256] = {0};
  uint64_t *T = nullptr;
  uint16_t *V = nullptr;
};

// Even-position bits of v packed into the low half: the inverse of the 2-D
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

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// --------------------------------------------------------------- kernels
struct FrameMap {
  int64_t A00, A01, B0, A10, A11, B1;  // Q32.32 (x, y)
  int64_t At, Bt;                      // Q32.32 time slab map (time-augmented worlds)
};

// Cells of a grid (d <= 1 counts as one slab).
inline int64_t grid_cells(const lbl_grid &g) {
  return static_cast<int64_t>(g.w) * g.h * (g.d > 1 ? g.d : 1);
}
inline int32_t grid_depth(const lbl_grid &g) { return g.d > 1 ? g.d : 1; }

// Fixed-point map of the equivariant frame transform (world grid W, agent
// grid A, pose p); false (with the error set) if it could overflow.
bool frame_map(const lbl_grid &W, const lbl_grid &A, const lbl_pose &p, FrameMap *out);
struct FrameItem;
FrameItem frame_item(const FrameMap &m, const lbl_grid &W, const lbl_grid &A, const uint8_t *planes, int32_t P,
                     uint64_t *O, int64_t cell0);

cudaError_t launch_frame_transform(const FrameItem &f, cudaStream_t s);
// z-order agent grids, or row-major 2-D grids in the quadtree form's tiled
// order (tiled_w > 0), packed world words: the transform (O written unless
// f.O is NULL) and the quadtree pyramid of its words (pyr_bytes-wide words at
// `off`) in one kernel
cudaError_t launch_frame_transform_pyramid(const FrameItem &f, const QuadOffsets &off, int pyr_bytes, void *pyr,
                                           int32_t tiled_w, cudaStream_t s);
cudaError_t launch_pack_planes(const PackItem &it, cudaStream_t s);
cudaError_t launch_pack_batch(const PackTable &tab, cudaStream_t s);
bool pack_vec_ok(const PackItem &it);

cudaError_t launch_label_csr(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L, const MonitorTables *mon,
                             int lanes_per_edge, bool early_exit, int ctas_per_sm, cudaStream_t s);

// streaming CSR form: CTAs per SM it runs with, its partition, its launch
int stream_ctas_per_sm(int depth);
int tma_ctas_per_sm();
int async_ctas_per_sm();
cudaError_t launch_label_async(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                               const MonitorTables *mon, cudaStream_t s);
cudaError_t launch_label_tma(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L, const MonitorTables *mon,
                             cudaStream_t s);
cudaError_t launch_partition(const Roadmap &rm, int ctas_per_sm, cudaStream_t s);
cudaError_t launch_label_stream(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                                const MonitorTables *mon, int depth, cudaStream_t s);
// base: words of word_bytes (1, 2, 4 or 8) each; rows of 2^31 entries or more need 8
cudaError_t launch_label_rows(const StreamRows &r, const void *base, int word_bytes, int32_t P, uint64_t *L,
                              const MonitorTables *mon, int depth, int num_sms, cudaStream_t s);

// quadtree form: pyramid of O, then the stream over the quadtree rows
// pyramid word width for n_props propositions: 1, 2, 4 or 8 bytes
int quad_word_bytes(const Roadmap &rm, int32_t P);
int mma_n_of(int32_t P);
cudaError_t launch_mma_count(const int64_t *rowptr, const int32_t *colidx, const int32_t *perm, int64_t E,
                             int32_t nkb, int64_t *count, cudaStream_t s);
cudaError_t launch_mma_fill(const int64_t *rowptr, const int32_t *colidx, const int32_t *perm, int64_t E,
                            int32_t nkb, const int64_t *tptr, int32_t *tblk, uint32_t *bits, cudaStream_t s);
cudaError_t launch_label_mma(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L, const MonitorTables *mon,
                             cudaStream_t s);
int front_chunk_for(int64_t E, int num_sms);
// pyramid of O into `pyr` (rm.pyr, or a buffer of rm.pyr_words 64-bit words owned elsewhere)
cudaError_t launch_quad_pyramid(const Roadmap &rm, const uint64_t *O, int word_bytes, void *pyr, cudaStream_t s);
// O NULL: label from rm.pyr as it stands (built by the frame transform)
cudaError_t launch_label_quad(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                                const MonitorTables *mon, int depth, cudaStream_t s, int front_chunk = -1);
cudaError_t launch_quad_pyramid_batch(const PyrTable &tab, cudaStream_t s);
// quadtree row e from CSR row rowmap[e] (rowmap NULL: row e); key[e] = z-order
// of the (x, y) of row e's middle cell (2-D grids of w columns in `order`)
cudaError_t launch_row_keys(const int64_t *rowptr, const int32_t *colidx, int64_t E, int32_t order, int32_t w,
                            uint32_t *key, cudaStream_t s);
// tiled_w > 0: rows in the tiled order of a row-major grid tiled_w cells wide
// (16 x 16 tiles in row-major order, z-order inside a tile), else in the cell order
cudaError_t launch_quad_count(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int32_t *rowmap,
                                int32_t tiled_w, int32_t *count, cudaStream_t s);
cudaError_t launch_quad_fill(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int32_t *rowmap,
                               int32_t tiled_w, QuadOffsets off, const int64_t *drow, int32_t *idx, cudaStream_t s);

cudaError_t launch_label_bittile(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                                 const MonitorTables *mon, bool early_exit, int ctas_per_sm, cudaStream_t s);

cudaError_t launch_monitor_step(const MonitorTables &mon, const uint64_t *L, int64_t n, int num_sms, cudaStream_t s);

// batched launches over device tables of items
int sector_ctas_per_sm(int depth);
cudaError_t launch_label_sector(const Roadmap &rm, const uint64_t *O, int32_t P, uint64_t *L,
                                const MonitorTables *mon, int depth, cudaStream_t s);
cudaError_t launch_sector_count(const int64_t *rowptr, const int32_t *colidx, int64_t E, int32_t *count,
                                cudaStream_t s);
cudaError_t launch_sector_fill(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int64_t *srow,
                               int32_t *sec, cudaStream_t s);
int batch_ctas_per_sm(int depth);
cudaError_t launch_label_batch(const BatchTable &tab, unsigned long long *counter, int num_sms, int ctas_per_sm,
                               cudaStream_t s);
cudaError_t launch_partition_into(const int64_t *rowptr, int64_t E, int64_t W, int64_t *part, cudaStream_t s);
cudaError_t launch_frame_batch(const FrameTable &tab, int num_sms, cudaStream_t s);

// roadmap preparation: row checks, block counts, block fill
cudaError_t launch_scan_rows(const int64_t *rowptr, const int32_t *colidx, int64_t E, int64_t nnz, int64_t cells,
                             unsigned long long *n_bad, int32_t *bt_count, cudaStream_t s);
cudaError_t launch_bt_fill(const int64_t *rowptr, const int32_t *colidx, int64_t E, const int64_t *bt_rowptr,
                           uint32_t *bt_block, uint64_t *bt_mask, cudaStream_t s);

}  // namespace lbl

// The opaque handles of the C ABI are the internal objects.
struct lbl_roadmap_s : lbl::Roadmap {};
struct lbl_monitor_s : lbl::Monitor {};

// Host helpers shared by the entry points (defined in lbl_api.cu).
namespace lbl {
int roadmap_new(const lbl_grid &agent, int64_t n_edges, int64_t nnz, lbl_roadmap_s **out);
int roadmap_finish(lbl_roadmap_s *rm, uint32_t flags, cudaStream_t st);
void free_roadmap(Roadmap *rm);
// a grid the entry points accept: 1..32768 cells a side, < 2^31 cells, finite
// geometry; need_order also checks the cell order (z-order: a power-of-two square or cube)
bool valid_grid(const lbl_grid *g, const char *name, bool need_order);
int device_sms(int dev);    // SM count (cached per device)
bool same_device(int dev);  // the current device is `dev` (else sets the error)
// lbl_frame_transform_pyramid into an explicit pyramid buffer (a roadmap's or
// a session's, pyr_words of rm): status code; O may be NULL on z-order grids
int transform_pyramid(const lbl_grid *world, const void *d_words, int32_t n_props, lbl_pose pose, const Roadmap &rm,
                      uint64_t *d_O, void *pyr, cudaStream_t st);
void clear_error();         // empty lbl_last_error at the start of an entry point
MonitorTables tables_of(const Monitor &mon, uint64_t *next, uint16_t *viol);
// the quadtree form's labeling (d_O NULL: from the pyramid already built)
int quad_label(lbl_roadmap_s *rm, const uint64_t *d_O, int32_t n_props, uint64_t *d_L, const MonitorTables *mt,
               const lbl_config *cfg, cudaStream_t st);
// lbl_label's body: argument checks, form resolution, re-partitioning, launch
int label_impl(lbl_roadmap rm, const uint64_t *d_O, int32_t n_props, uint64_t *d_L, lbl_monitor mon,
               uint64_t *d_next, uint16_t *d_viol, const lbl_config *cfg, cudaStream_t st);

// cudaMalloc of `count` elements (at least 16 bytes), adding the bytes to *bytes if given
// Object-owned memory (see UseLog): stream-ordered allocation on the legacy
// stream, which is then synchronised so any stream may use it at once.
template <typename T>
cudaError_t obj_alloc(T **p, size_t count, int64_t *bytes) {
  const size_t b = count * sizeof(T);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(p), b ? b : 16, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
  if (e == cudaSuccess && bytes) *bytes += static_cast<int64_t>(b);
  return e;
}

// Free object memory whose uses the host has already waited for.
inline void obj_free_now(void *p) {
  if (p) cudaFreeAsync(p, nullptr);
}

// Temporary device memory of one call, freed with cudaFree before it returns.
template <typename T>
cudaError_t dev_alloc(T **p, size_t count, int64_t *bytes) {
  const size_t b = count * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), b ? b : 16);
  if (e == cudaSuccess && bytes) *bytes += static_cast<int64_t>(b);
  return e;
}
}  // namespace lbl
