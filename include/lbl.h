/*
 * lbl.h — C ABI of liblbl: GPU labeling of a fixed discrete abstraction with
 * atomic propositions (arXiv 1810.02612, Paden, Liu & Cullen, "Accelerated
 * Labeling of Discrete Abstractions for Planning Under LTL Specifications").
 *
 * The method (Sec. 4): every edge e of a precomputed roadmap is stored as the
 * set of workspace cells its swept footprint covers (a row of the Boolean
 * trajectory matrix M, eq. 10, stored in CSR form as in eq. 11).  The perceived
 * scene is a Boolean matrix P with one column per atomic proposition.  The edge
 * labels are the Boolean product  L(e, p) = OR_k M(e, k) AND P(k, p)  (eq. 10),
 * i.e. proposition p labels edge e iff its region meets the swept cells
 * (eq. 7).  Because the dynamics are equivariant to planar motions (Sec. 5,
 * eq. 13), one roadmap built in the agent frame is re-used at every planning
 * pose by resampling the world-frame proposition grids into the agent frame.
 * A safety monitor (Sec. 3.2) then reads each label.
 *
 * Conventions for every entry point:
 *   - The return value is a status code (LBL_OK or a negative LBL_E*).  On
 *     failure lbl_last_error() returns a message for the calling thread.
 *   - "d_" pointers are CUDA device pointers owned by the caller; "h_" pointers
 *     are host pointers owned by the caller.  The library owns only the objects
 *     behind its opaque handles and frees them in the matching *_free call.
 *   - Work is enqueued asynchronously on the caller's stream (NULL = the legacy
 *     default stream); outputs are valid once that stream has completed.
 *     Calls on different streams that write the same outputs race.
 *   - Proposition words are uint64: bit p is proposition p, bits >= n_props are
 *     zero.  At most 64 propositions.
 *   - No C++ exception crosses this interface; nothing here calls exit().
 *   - The library computes on the CUDA device current on the calling thread
 *     when the handle was created; it never falls back to the CPU.
 */
#ifndef LBL_H_
#define LBL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *lbl_stream;

/* ----------------------------------------------------------- status codes */
#define LBL_OK 0
#define LBL_EINVAL (-1)      /* bad argument, limit exceeded, malformed CSR */
#define LBL_ENOMEM (-2)      /* device or host allocation failed */
#define LBL_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define LBL_ETIMEOUT (-4)    /* a bounded wait ran out */
#define LBL_EUNSUPPORTED (-5)/* valid request the library does not implement */

/* ------------------------------------------------------------ cell order */
#define LBL_ORDER_ROWMAJOR 0 /* index = iy * w + ix */
#define LBL_ORDER_MORTON 1   /* z-order (Sec. 4.1, Alg. 1): bit i of ix -> bit 2i+1,
                                bit i of iy -> bit 2i; needs w == h, a power of two */

/*
 * Occupancy grid (Sec. 4.1): w x h square cells of side res metres.  Cell
 * (ix, iy) covers [x0 + ix*res, x0 + (ix+1)*res) x [y0 + iy*res, y0 + (iy+1)*res)
 * in the grid's own frame (world frame for perception grids, agent frame for
 * the roadmap grid).  `order` numbers the cells (LBL_ORDER_*).
 * Time-augmented workspace (Sec. 5, (x, y, tau) with dynamic objects as static
 * volumes): d > 1 time slabs, slab it covering [t0 + it*tres, t0 + (it+1)*tres)
 * seconds (relative to the query time in the agent frame).  d <= 1 is a plain
 * 2-D grid (tres and t0 ignored); cell index = (it*h + iy)*w + ix row-major, or
 * the 3-D z-order (bit i of ix -> 3i+2, of iy -> 3i+1, of it -> 3i; needs
 * w == h == d, a power of two).
 * Limits: 1 <= w, h, d <= 32768; w*h*d <= 2^31 - 1; res > 0; tres > 0 if d > 1.
 */
typedef struct {
  int32_t w, h;
  double res, x0, y0;
  int32_t order;
  int32_t d;        /* time slabs, <= 1 = 2-D */
  double tres, t0;  /* slab length and start, seconds */
} lbl_grid;

/* Agent pose in the world frame: position (x, y) in metres, heading theta in
   radians (the agent frame's +x axis points along theta), and the query time t
   in seconds (used by time-augmented grids, eq. 13's shift in t). */
typedef struct {
  double x, y, theta, t;
} lbl_pose;

/* Labeling algorithm (Sec. 4.3: both compute eq. 10 exactly). */
#define LBL_ALGO_AUTO 0    /* pick from the roadmap's shape and n_props */
#define LBL_ALGO_CSR 1     /* gather-OR over the CSR cell lists */
#define LBL_ALGO_BITTILE 2 /* AND over per-edge 64-cell block masks */
#define LBL_ALGO_SECTOR 3  /* gather-OR over per-edge 4-cell sectors (compressed A):
                              one u32 (sector << 4 | cell mask) per touched 32-byte
                              sector of O; needs O 32-byte aligned */
#define LBL_ALGO_QUAD 4    /* gather-OR over each row's maximal quadtree blocks
                              (compressed A): a row is the union of blocks of 4^k
                              consecutive cells of the cell order (k <= 4) that
                              start at a multiple of 4^k (in z-order: the
                              2^k x 2^k squares of the quadtree).  On a 2-D
                              row-major grid whose sides are multiples of 16
                              the blocks follow a tiled order (16 x 16 tiles in
                              row-major order, z-order inside each tile), so
                              they are squares too; other row-major grids use
                              aligned runs of a grid row.  Per frame the library ORs O
                              over every such block (a pyramid of ~4/3 words per
                              cell) and each edge ORs one word per block.  Exact:
                              OR is associative and idempotent */
#define LBL_ALGO_MMA 5     /* the dense product of eq. 8-10 on the tensor cores:
                              tiles of 128 edges (in locality order) times
                              K-blocks of 128 cells, each touched tile-block a
                              0/1 matrix multiplied with O's 0/1 bits as e4m3
                              (tcgen05.mma kind::f8f6f4, fp32 counts in tensor
                              memory, exact); label bit p = count > 0 */

typedef struct {
  int32_t algo;           /* LBL_ALGO_* */
  int32_t lanes_per_edge; /* CSR: 0 = streaming form (each warp streams a contiguous,
                             nonzero-balanced range of edges); 4/8/16/32 = lane
                             groups of that size, one edge each */
  int32_t early_exit;     /* 1 = stop a row once every proposition is set (Sec. 5,
                             early termination; lane-group CSR and block forms);
                             0 or -1 = off */
  int32_t ctas_per_sm;    /* persistent grid size per SM, 0 = auto */
  int32_t pipeline;       /* streaming CSR: index stream (LBL_PIPE_REGISTERS/BULK/ASYNC);
                             quadtree: LBL_PIPE_FRONT or LBL_PIPE_REGISTERS (below);
                             0 = the form's default */
  int32_t depth;          /* register pipelines: groups of 32 entries in flight per
                             warp, 0 = the form's default: CSR 8 (default), 12 or 16;
                             quadtree 8 (default), 12 or 16; sector form 4 (default)
                             or 8.  Deeper variants run fewer CTAs per SM */
} lbl_config;

/* How the streaming CSR form moves each warp's column indices from HBM. */
#define LBL_PIPE_REGISTERS 1 /* loads into registers, 8 groups of 32 ahead */
#define LBL_PIPE_BULK 2      /* cp.async.bulk (TMA engine) into a shared-memory ring */
#define LBL_PIPE_ASYNC 3     /* per-lane cp.async into a shared-memory ring */
/* How the quadtree form spreads edges over warps.  LBL_PIPE_REGISTERS: every
   warp streams a fixed contiguous range of edges.  LBL_PIPE_FRONT (depth 8):
   one CTA per SM takes the SM's range and its warps take chunks of
   neighbouring edges in order, so the rows labeled at the same time on an SM
   share pyramid words in its L1.  0 (default): the front on ranges of about
   3,000 edges per SM or more, else the fixed ranges. */
#define LBL_PIPE_FRONT 4

typedef struct lbl_roadmap_s *lbl_roadmap;
typedef struct lbl_monitor_s *lbl_monitor;
typedef struct lbl_session_s *lbl_session;
typedef struct lbl_batch_s *lbl_batch;
typedef struct lbl_server_s *lbl_server;

/* Message describing the last failure on the calling thread ("" if none).
   The pointer stays valid until the thread's next lbl_* call. */
const char *lbl_last_error(void);

/* ABI version of this header (major * 10000 + minor * 100 + patch): 1.1.0
   (1.0.0 plus lbl_frame_transform_pyramid and lbl_label_pyramid). */
int lbl_version(void);

/* --------------------------------------------------------------- roadmap */

#define LBL_UPLOAD_DEVICE_PTRS 1u /* rowptr/colidx are device pointers (default: host) */
#define LBL_UPLOAD_BITTILE 2u     /* also derive the 64-cell block form used by
                                     LBL_ALGO_BITTILE (costs ~12 B per touched block) */
#define LBL_UPLOAD_SECTOR 4u      /* also derive the 4-cell sector form used by
                                     LBL_ALGO_SECTOR (4 B per touched sector; grids of
                                     at most 2^30 cells) */
#define LBL_UPLOAD_QUAD 8u        /* also derive the quadtree form used by LBL_ALGO_QUAD
                                     (4 B per maximal block of a row, plus a pyramid of
                                     ~11 B per cell; grids of fewer than 2^30 cells).
                                     On 2-D grids its rows are stored in locality order:
                                     inside each quarter of the edges (E*c/4 .. E*(c+1)/4),
                                     sorted by the z-order of the (x, y) of the row's
                                     middle cell, 4 B per edge; outputs still land at the
                                     caller's edge positions */
#define LBL_UPLOAD_KEEP_ORDER 16u /* with LBL_UPLOAD_QUAD: keep the caller's edge order
                                     for the quadtree rows (for roadmaps already ordered
                                     for locality) */
#define LBL_UPLOAD_MMA 32u        /* also derive the tensor-core form used by LBL_ALGO_MMA
                                     (grids of at most 2^22 cells): the edges sorted by
                                     the z-order of their middle cell, in tiles of 128;
                                     per tile the 128-cell blocks its rows touch, 2 KiB
                                     each; 8 KiB of working memory per 128 cells */

/*
 * lbl_roadmap_upload — make a roadmap resident on the device.
 * The trajectory matrix M of eq. 10 in the CSR layout of eq. 11: row e (edge e)
 * holds the cells swept by X(e) (eq. 7 discretised on `agent`, Sec. 4.1).
 *   agent   grid of the roadmap, agent frame (its `order` numbers colidx)
 *   rowptr  int64[n_edges + 1], rowptr[0] = 0, non-decreasing, rowptr[n_edges] = nnz
 *   colidx  int32[nnz], each row strictly increasing, 0 <= colidx < w*h
 *   flags   LBL_UPLOAD_*; host arrays may be pageable or pinned
 *   s       stream for the copies and derivation kernels
 * The call copies both arrays into library-owned device memory, checks them on
 * the device (LBL_EINVAL if malformed), derives the structures the kernels use
 * and synchronises `s` before returning.  The caller's arrays may be freed
 * afterwards.  n_edges = 0 is allowed.
 */
int lbl_roadmap_upload(const lbl_grid *agent, const int64_t *rowptr, const int32_t *colidx, int64_t n_edges,
                       int64_t nnz, uint32_t flags, lbl_stream s, lbl_roadmap *out);

/*
 * lbl_roadmap_rasterize — build a roadmap's rows on the device: row e holds the
 * cells of `agent` whose centre lies within `radius` of arc e (eq. 7 with the
 * closed disc footprint of eq. 5, discretised by cell centres as in Sec. 4.1),
 * sorted in agent.order.  h_arcs = double[n_edges][5] on the host: start x, y
 * (agent frame, metres), heading (rad), curvature (1/m; |c| < 1e-9 is a
 * straight segment), length (m, >= 0).  Each membership decision equals the
 * fp64 evaluation of that distance test: the arc geometry is computed on the
 * host, cells within 1 mm of the radius are decided in fp64 with correctly
 * rounded operations, the rest by an fp32 screen.  2-D grids only
 * (LBL_EUNSUPPORTED for time-augmented ones); flags: LBL_UPLOAD_BITTILE /
 * LBL_UPLOAD_SECTOR as for lbl_roadmap_upload.  Synchronises `s`.
 */
int lbl_roadmap_rasterize(const lbl_grid *agent, const double *h_arcs, int64_t n_edges, double radius,
                          uint32_t flags, lbl_stream s, lbl_roadmap *out);

/* Copy a roadmap's rows (CSR of eq. 11, in the caller's edge order) into
   caller device buffers d_rowptr int64[E+1], d_colidx int32[nnz], on `s`. */
int lbl_roadmap_rows(lbl_roadmap rm, int64_t *d_rowptr, int32_t *d_colidx, lbl_stream s);

/*
 * Release a roadmap.  NULL is accepted.  Its device memory is freed in stream
 * order after the work the library enqueued with it (lbl_label and the calls
 * built on it, lbl_roadmap_rows, sessions, batch launches) has run; the call
 * itself waits for nothing on the device and stalls no other stream.  Work a
 * caller captured into a CUDA graph is not tracked: free a roadmap only after
 * the replays that use it have completed, and free the sessions, batches and
 * servers that hold it first.  The same holds for lbl_monitor_free,
 * lbl_session_free and lbl_batch_free; lbl_server_free waits for the server's
 * own lanes only.
 */
int lbl_roadmap_free(lbl_roadmap rm);

/*
 * lbl_roadmap_status — synchronise `s`, then report whether any labeling kernel
 * on this roadmap gave up a bounded wait (the bulk-copy index stream of
 * LBL_PIPE_BULK or the tensor-core form's MMA completion did not arrive within
 * the roadmap's wait limit): LBL_ETIMEOUT if so (the labels of that call are
 * incomplete; the flag is cleared), LBL_OK otherwise.  Kernels never spin
 * without a bound; after giving up, a kernel still waits (at most 2 s) for
 * the copies and MMAs it has in flight before it returns.
 */
int lbl_roadmap_status(lbl_roadmap rm, lbl_stream s);

/*
 * lbl_roadmap_set_wait_limit — the limit of those waits for later launches on
 * this roadmap, in nanoseconds (default 2,000,000,000; 0..60e9).  0 tests the
 * awaited phase once without waiting, which makes a launch give up at its
 * first wait whose data has not arrived: a way to exercise the failure path.
 */
int lbl_roadmap_set_wait_limit(lbl_roadmap rm, int64_t limit_ns);

/* Shape of a roadmap: edges, nonzeros, (block, mask) entries of the block form
   (0 without LBL_UPLOAD_BITTILE), entries of the sector form (0 without
   LBL_UPLOAD_SECTOR), entries of the quadtree form (0 without LBL_UPLOAD_QUAD)
   and device bytes held.  Any out pointer may be NULL. */
int lbl_roadmap_info(lbl_roadmap rm, int64_t *n_edges, int64_t *nnz, int64_t *n_block_entries,
                     int64_t *n_sector_entries, int64_t *n_qdadic_entries, int64_t *device_bytes);

/* Size of one labeling form of a roadmap: *entries = what its kernels stream
   per frame (LBL_ALGO_CSR: nonzeros; LBL_ALGO_BITTILE: (block, mask) entries;
   LBL_ALGO_SECTOR: sector entries; LBL_ALGO_QUAD: quadtree entries;
   LBL_ALGO_MMA: (tile of 128 edges, 128-cell block) pairs, 2 KiB each), 0 when
   the roadmap lacks the form; *tiles (LBL_ALGO_MMA: tiles of 128 edges, else
   0).  Either pointer may be NULL.  LBL_EINVAL for an unknown algo. */
int lbl_roadmap_form_info(lbl_roadmap rm, int32_t algo, int64_t *entries, int64_t *tiles);

/* ------------------------------------------------------- frame transform */

/*
 * lbl_frame_transform — equivariant re-use of the roadmap (Sec. 5, eq. 13).
 * For every cell (ix, iy) of `agent`, take its centre c in the agent frame,
 * move it to the world point q = (pose.x, pose.y) + R(pose.theta) c, and set
 * bit p of d_O[index(ix, iy)] iff d_planes[p] is non-zero at the world cell
 * containing q; world points outside `world` read as 0.  Time-augmented
 * grids: agent slab it (centre t0 + (it+.5)tres) reads the world slab holding
 * pose.t + that centre; a 2-D world under a time-augmented agent grid is a
 * static world (every slab reads its single plane); a time-augmented world
 * needs a time-augmented agent grid.
 * Exactness: the map (ix, iy) -> world cell coordinates is affine; its six
 * coefficients are computed once in double on the host and rounded (half to
 * even) to Q32.32 fixed point; the map is then evaluated exactly in 64-bit
 * integers and floored, so every device and every run give the same cells.
 *   world     grid of the planes (row-major planes, its `order` is ignored)
 *   d_planes  uint8[n_props][world.d][world.h][world.w], non-zero = occupied
 *   n_props   0..64
 *   agent     roadmap grid; d_O is written in agent.order
 *   d_O       uint64[agent.w * agent.h * agent.d]
 * Errors: LBL_EINVAL for bad grids, n_props > 64, or a pose whose fixed-point
 * map could overflow 64 bits.
 */
int lbl_frame_transform(const lbl_grid *world, const uint8_t *d_planes, int32_t n_props, lbl_pose pose,
                        const lbl_grid *agent, uint64_t *d_O, lbl_stream s);

/*
 * lbl_pack_planes — the world planes as one word per world cell: bit p of
 * word c is set iff d_planes[p][c] != 0 (c in the world grid's row-major cell
 * order, time slabs outermost; the same cells lbl_frame_transform reads).
 *   d_planes  uint8[n_props][cells of world]              (device)
 *   d_words   cells of world words, each LBL_PACKED_WORD_BYTES(n_props)
 *             bytes: uint8 for n_props <= 8, uint16 <= 16, uint32 <= 32,
 *             else uint64 (device, caller-owned; bits >= n_props zero)
 * One coalesced pass over the planes (whole 128-byte lines of a plane per
 * warp load, with 4-byte aligned planes and a cell count divisible by 4; byte
 * loads otherwise).  With lbl_frame_transform_words it gives exactly
 * lbl_frame_transform's O.  LBL_EINVAL on a bad grid, n_props outside 0..64,
 * a NULL buffer or words not aligned to their width.  Asynchronous on `s`.
 */
#define LBL_PACKED_WORD_BYTES(n_props) ((n_props) <= 8 ? 1 : (n_props) <= 16 ? 2 : (n_props) <= 32 ? 4 : 8)
int lbl_pack_planes(const lbl_grid *world, const uint8_t *d_planes, int32_t n_props, void *d_words,
                    lbl_stream s);

/*
 * lbl_frame_transform_words — lbl_frame_transform (Sec. 5, eq. 13) reading the
 * packed words of lbl_pack_planes (LBL_PACKED_WORD_BYTES(n_props) bytes each)
 * instead of the planes: one gather per agent cell instead of n_props byte
 * gathers.  Word bits >= n_props are ignored.  Same arguments, layouts and
 * errors as lbl_frame_transform, and LBL_EINVAL for words or d_O not aligned
 * to their width.
 */
int lbl_frame_transform_words(const lbl_grid *world, const void *d_words, int32_t n_props, lbl_pose pose,
                              const lbl_grid *agent, uint64_t *d_O, lbl_stream s);

/* --------------------------------------------------------------- monitor */

/*
 * lbl_monitor_create — deterministic safety monitor (Sec. 3.2: the automaton
 * whose rejected words are the bad prefixes of an LTL safety formula), given as
 * a table.  A label word is read as the letter
 *   letter = sum_j bit(L, relbits[j]) << j,  j < m
 * and state q moves to delta[q * 2^m + letter].
 *   n_states  1..16       m  0..8       relbits  uint8[m], each < 64
 *   delta     uint8[n_states << m], each < n_states      reject  state id or -1
 * The table is copied; the host arrays may be freed afterwards.
 */
int lbl_monitor_create(int32_t n_states, int32_t m, const uint8_t *relbits, const uint8_t *delta, int32_t reject,
                       lbl_monitor *out);
int lbl_monitor_free(lbl_monitor mon);

/*
 * lbl_monitor_step — for each of n labels and every state q < n_states:
 *   d_next[i] bits [4q, 4q+4) = delta(q, letter(d_L[i])),
 *   d_viol[i] bit q           = (that state == reject).
 * Fields of states >= n_states are zero.  d_next/d_viol: uint64[n] / uint16[n].
 */
int lbl_monitor_step(lbl_monitor mon, const uint64_t *d_L, int64_t n, uint64_t *d_next, uint16_t *d_viol,
                     lbl_stream s);

/* ---------------------------------------------------------------- labels */

/*
 * lbl_label — the labeling operation (eq. 7) as the Boolean product of eq. 10:
 *   d_L[e] = (OR over cells k of row e of d_O[k]) & (2^n_props - 1)
 * in the caller's edge order.  With `mon` non-NULL the monitor step above is
 * fused into the same kernel and d_next/d_viol (uint64[E] / uint16[E]) are
 * written too; with `mon` NULL they are ignored.
 *   d_O      uint64[agent cells] in the roadmap grid's order (lbl_frame_transform)
 *   n_props  0..64
 *   d_L      uint64[n_edges]
 *   cfg      NULL = defaults (LBL_ALGO_AUTO)
 * LBL_ALGO_BITTILE / LBL_ALGO_SECTOR / LBL_ALGO_QUAD / LBL_ALGO_MMA need a
 * roadmap uploaded with LBL_UPLOAD_BITTILE / LBL_UPLOAD_SECTOR /
 * LBL_UPLOAD_QUAD / LBL_UPLOAD_MMA
 * (LBL_EUNSUPPORTED otherwise).  LBL_ALGO_AUTO takes the form
 * lbl_roadmap_autotune chose for n_props, else the quadtree form when the roadmap
 * has it, else the block form for n_props <= 8 when present, else CSR.  The
 * roadmap holds per-launch working memory (block planes, quadtree pyramid), so
 * two lbl_label calls on the same roadmap must not overlap on the device.
 */
int lbl_label(lbl_roadmap rm, const uint64_t *d_O, int32_t n_props, uint64_t *d_L, lbl_monitor mon, uint64_t *d_next,
              uint16_t *d_viol, const lbl_config *cfg, lbl_stream s);

/*
 * lbl_frame_transform_pyramid — lbl_frame_transform_words (Sec. 5, eq. 13)
 * for the roadmap's agent grid that also builds, from the words it computes,
 * the roadmap's per-frame quadtree pyramid: for every aligned block of 4^k
 * consecutive cells (k <= 4) the OR of their words, i.e. eq. 10 over that
 * block, which the quadtree rows gather (LBL_ALGO_QUAD).  On a z-order agent
 * grid, and on a 2-D row-major grid whose sides are multiples of 16 (the
 * quadtree form's tiled order), the pyramid is built inside the transform
 * kernel (one launch, O not read back); on other row-major grids the
 * transform and the pyramid are two launches.  lbl_label_pyramid then labels
 * the frame from it.
 *   rm       uploaded with LBL_UPLOAD_QUAD (LBL_EUNSUPPORTED otherwise, unless
 *            the roadmap has no edges: then only O is written)
 *   d_words  packed world words of lbl_pack_planes (LBL_PACKED_WORD_BYTES(n_props) each)
 *   d_O      uint64[agent cells], written as by lbl_frame_transform_words;
 *            may be NULL where the pyramid is built in one launch (the words
 *            then exist only as the pyramid's level 0)
 * Same errors as lbl_frame_transform_words.  The pyramid is the roadmap's
 * working memory: a quadtree lbl_label or another lbl_frame_transform_pyramid
 * on this roadmap overwrites it, and calls on one roadmap must not overlap on
 * the device.  Asynchronous on `s`.
 */
int lbl_frame_transform_pyramid(lbl_roadmap rm, const lbl_grid *world, const void *d_words, int32_t n_props,
                                lbl_pose pose, uint64_t *d_O, lbl_stream s);

/*
 * lbl_label_pyramid — lbl_label's quadtree form (eq. 10 over each row's
 * maximal quadtree blocks) gathering from the pyramid the last
 * lbl_frame_transform_pyramid (or quadtree lbl_label) enqueued on this roadmap,
 * so a frame is labeled without a pyramid launch.  Outputs, the fused monitor
 * and `cfg` as in lbl_label; cfg->algo must be LBL_ALGO_AUTO or LBL_ALGO_QUAD
 * (AUTO takes the quadtree configuration lbl_roadmap_autotune measured, if it
 * chose the quadtree form).  LBL_EINVAL when no pyramid for n_props'
 * word width (1, 2, 4 or 8 bytes) was enqueued on this roadmap.  The pyramid
 * is read as the stream finds it: order this call after the transform that
 * built it, on the same stream or behind an event.
 */
int lbl_label_pyramid(lbl_roadmap rm, int32_t n_props, uint64_t *d_L, lbl_monitor mon, uint64_t *d_next,
                      uint16_t *d_viol, const lbl_config *cfg, lbl_stream s);

/*
 * lbl_label_blocks_noalloc — the block-form labeling of lbl_label
 * (LBL_ALGO_BITTILE) for callers that cannot allocate device memory: planning
 * loops under real-time or safety rules that forbid allocation once the system
 * runs, and host frameworks that own every device allocation.  The paper has no
 * counterpart: it is lbl_label's block form on the same kernels, with its
 * working memory moved into the library.
 *
 * The kernels' one piece of working memory, the bit-plane copy of d_O (one word
 * per 64-cell block and proposition), is a fixed device array of
 * LBL_NOALLOC_MAX_PLANE_WORDS words (4 MiB) inside the library; every GPU that
 * loads the library holds it until the process exits.  The call allocates and
 * frees nothing.
 *   d_block_rowptr  int64[n_edges + 1]: edge e owns entries
 *                   [d_block_rowptr[e], d_block_rowptr[e+1]), non-decreasing
 *   d_block_id      uint32[entries]: block b = cells [64b, 64b+64) of d_O's
 *                   order, each < ceil(n_cells / 64)
 *   d_block_mask    uint64[entries]: bit i set iff cell 64b+i is in the edge
 *   d_O             uint64[n_cells]  proposition words (lbl_frame_transform)
 *   d_L             uint64[n_edges]  labels, as lbl_label writes them
 * The block form is not checked (malformed entries are undefined behaviour);
 * it equals what lbl_roadmap_upload derives with LBL_UPLOAD_BITTILE.
 * Returns LBL_EINVAL when ceil(n_cells / 64) * n_props exceeds
 * LBL_NOALLOC_MAX_PLANE_WORDS.  A call looks up the array's device address
 * (under a lock) unless its stream is being captured; a call on a capturing
 * stream reuses the last address looked up on that device.  So make the first
 * call on a device, and the first after a cudaDeviceReset (which can move the
 * array), before any stream capture.  Every call uses the same array: calls that can
 * overlap on the GPU (on different streams, or from several threads) race and
 * must be serialised by the caller.  Nothing in the array needs clearing: each
 * call writes every word it reads.
 */
#define LBL_NOALLOC_MAX_PLANE_WORDS 524288
int lbl_label_blocks_noalloc(const int64_t *d_block_rowptr, const uint32_t *d_block_id, const uint64_t *d_block_mask,
                             int64_t n_edges, const uint64_t *d_O, int64_t n_cells, int32_t n_props, uint64_t *d_L,
                             lbl_stream s);

/*
 * lbl_mma_probe — the tensor-core rate behind LBL_ALGO_MMA, measured on the
 * current device.  Every CTA (ctas_per_sm per SM, 1..4) keeps one 128 x K
 * 0/1 tile of A and one n x K tile of B in shared memory and accumulates
 * their product `reps` times with tcgen05.mma into fp32 tensor memory:
 * kind 0 = kind::f8f6f4 with e4m3 operands (K = 128; n 16, 64 or 128), the
 * form LBL_ALGO_MMA uses; kind 1 = kind::f16 with bf16 operands (K = 64; n
 * 16 or 64), for comparison.  *tflops = 2 x 128 x n x K x reps x CTAs / time
 * (CUDA events around one launch); *exact = 1 iff every accumulated count of
 * one CTA equals reps x (A.B^T) computed on the host.  The paper has no
 * counterpart: it bounds what the dense form of eq. 8-10 can reach.
 * Runs on the legacy default stream and synchronises it; allocates and frees
 * its own small buffers.
 */
int lbl_mma_probe(int32_t kind, int32_t n, int32_t reps, int32_t ctas_per_sm, double *tflops, int32_t *exact);

/*
 * lbl_roadmap_autotune — pick the labeling form of this roadmap by measurement
 * (the two forms of Sec. 4.3 and their variants compute the same eq. 10; which
 * is fastest depends on the roadmap, the grid order and n_props).  Every
 * applicable variant (streaming CSR with each LBL_PIPE_*, lane groups of 8, 16
 * and 32, and the block and sector forms if the roadmap has them) labels d_O
 * once untimed and
 * `reps` times timed with CUDA events on `s`; the fastest becomes what
 * LBL_ALGO_AUTO runs for this n_props on this roadmap.  d_L (and d_next/d_viol
 * with a monitor) receive labels as lbl_label writes them.  *chosen (may be
 * NULL) gets the winner.  Synchronises `s`.  1 <= reps <= 1000.
 */
int lbl_roadmap_autotune(lbl_roadmap rm, const uint64_t *d_O, int32_t n_props, lbl_monitor mon, uint64_t *d_L,
                         uint64_t *d_next, uint16_t *d_viol, int32_t reps, lbl_config *chosen, lbl_stream s);

/* ----------------------------------------------------------------- batch */

/*
 * Batched frames: many roadmaps (agents, or uneven abstractions), one frame each,
 * transformed and labeled by two kernel launches in total instead of two per
 * frame.  Sec. 5 runs one labeling query at a time; the batch runs many.  Every
 * item's labels equal what lbl_frame_transform + lbl_label produce for it.
 *
 * lbl_batch_create    plan for n (1..128) roadmaps with their proposition counts
 *                     and optional monitors (mons may be NULL): every roadmap is
 *                     cut into edge ranges ("work units") of about equal cost
 *                     (nonzeros + 32 per edge), about 8 per warp of one
 *                     persistent grid; warps take units in roadmap order from a
 *                     counter, so the load balances and few frames are live in
 *                     L2 at once.  ctas_per_sm 0 = as many as fit.
 *                     Synchronises the legacy default stream.
 * lbl_batch_set_frames  frames[i] is item i's world planes, pose and output
 *                     buffers (see lbl_frame).  Checked here.  Host-side, except
 *                     that it allocates a larger packed-word buffer (cudaMalloc)
 *                     when the packed worlds outgrow the batch's; the buffer it
 *                     replaces stays allocated until lbl_batch_free, so graphs
 *                     captured earlier remain valid.
 * lbl_batch_launch    enqueues on `s`, for the frames last set, the stages asked
 *                     for: LBL_STAGE_TRANSFORM (all frame transforms: one launch
 *                     packs the planes of every frame whose world has at most
 *                     4x its agent's cells into 64-bit words, one launch
 *                     transforms all frames, from those words or from the
 *                     planes) and/or LBL_STAGE_LABEL (all labels with the fused
 *                     monitors, one launch after a 8-byte memset of the unit
 *                     counter; reads each frame's d_O).  It only enqueues
 *                     kernels and that memset, so it can be captured in a CUDA
 *                     graph and replayed; replays use the buffers and poses of
 *                     the frames set before capture.  Launches of one batch
 *                     must not overlap on the device (they share the counter).
 */
typedef struct {
  lbl_grid world;          /* world grid of d_planes (its order is ignored) */
  const uint8_t *d_planes; /* uint8[n_props][world.d][world.h][world.w] */
  lbl_pose pose;           /* agent pose in the world */
  uint64_t *d_O;           /* uint64[agent cells]: transformed words (written) */
  uint64_t *d_L;           /* uint64[E]: labels */
  uint64_t *d_next;        /* uint64[E], uint16[E]: monitor outputs when the item */
  uint16_t *d_viol;        /*   has a monitor, else ignored */
} lbl_frame;

int lbl_batch_create(int32_t n, const lbl_roadmap *rms, const int32_t *n_props, const lbl_monitor *mons,
                     int32_t ctas_per_sm, lbl_batch *out);
int lbl_batch_set_frames(lbl_batch b, const lbl_frame *frames);
#define LBL_STAGE_TRANSFORM 1u
#define LBL_STAGE_LABEL 2u
int lbl_batch_launch(lbl_batch b, uint32_t stages, lbl_stream s);
int lbl_batch_free(lbl_batch b);

/*
 * lbl_batch_autotune — choose the batched labeling launch by measurement, as
 * lbl_roadmap_autotune does for one roadmap (Sec. 4.3: every variant computes
 * the same eq. 10; which is fastest depends on the rows, the grids and the
 * proposition counts).  The batch's items are labeled in one launch per class
 * of gathered word width (1, 2, 4, 8 bytes: the bins of the batch); for each
 * class with items the call times, on the frames last set, the stream depth
 * (8 or 12 groups of 32 entries in flight per warp), CTAs per SM (the most
 * that fit and up to two fewer) and the work-unit size (2, 4, 8, 16 or 32
 * units per warp, the items cut into units of equal cost), `reps` launches
 * each (CUDA events on `s`, after one untimed launch), and keeps the fastest
 * plan for later lbl_batch_launch calls.  Labels written meanwhile are the
 * frames' labels.  A CUDA graph captured before keeps the plan it captured
 * (its memory stays allocated until lbl_batch_free); capture after tuning to
 * replay the tuned plan.  out[LBL_BATCH_CLASSES] (may be NULL) receives, per
 * class (index 0..3 = 1, 2, 4, 8-byte words), the choice and its time next to
 * the time of the plan lbl_batch_create made.  Synchronises `s`;
 * 1 <= reps <= 1000.
 */
#define LBL_BATCH_CLASSES 4
typedef struct {
  int32_t word_bytes;     /* 1, 2, 4 or 8; 0 = the class has no items */
  int32_t items;          /* items labeled by the class's launch */
  int32_t depth;          /* groups of 32 entries in flight per warp */
  int32_t ctas_per_sm;    /* CTAs per SM of the launch */
  int32_t units_per_warp; /* work units per warp */
  float ms;               /* measured label-launch time of the chosen plan, ms */
  float ms_default;       /* the same for the plan lbl_batch_create made, ms */
} lbl_batch_tuning;
int lbl_batch_autotune(lbl_batch b, int32_t reps, lbl_stream s, lbl_batch_tuning *out);

/* ---------------------------------------------------------------- server */

/*
 * A serving loop with continuous batching.  The roadmaps stay resident; each
 * request is one planning query (Sec. 5): a pose and world proposition planes
 * in host memory, answered with the labels (and monitor outputs) of one
 * roadmap, copied back to host memory.  A scheduler thread inside the library
 *   - admits requests first come first served into a device arena of
 *     `mem_budget` bytes (planes, agent words and outputs of each request), so
 *     a request waits until memory frees up;
 *   - whenever one of `lanes` execution lanes (CUDA streams) is free, launches
 *     everything admitted so far (up to 128 requests) as one batch: copies in,
 *     one batched frame-transform launch, one batched labeling launch over
 *     work units precomputed per roadmap, copies out.  Requests that arrive
 *     while batches run join the next batch, and batches on different lanes
 *     overlap on the device.  max_batch = 1 gives the plain form: one request
 *     per launch pair.
 * Every request's outputs equal what lbl_session_run returns for it alone.
 *
 * lbl_server_create  n resident roadmaps (1..), their proposition counts and
 *                    optional monitors (mons may be NULL), 1..16 lanes, the
 *                    largest batch (1..128), arena bytes.  Allocates everything
 *                    the loop needs up front.
 * lbl_server_submit  queue a request against roadmap `roadmap`: h_planes
 *                    uint8[n_props][world.h][world.w]; outputs h_L uint64[E],
 *                    h_next/h_viol (monitor only, may be NULL).  All host
 *                    buffers must stay valid until the request completes; use
 *                    pinned memory for asynchronous copies (planes are
 *                    uint8[n_props][world.d][world.h][world.w]).  arrival_ns: the
 *                    request's arrival on CLOCK_MONOTONIC (0 = now), the start
 *                    of its latency.  LBL_ENOMEM if it can never fit the arena.
 * lbl_server_wait    block up to timeout_ms for a ticket (LBL_ETIMEOUT
 *                    otherwise); on return the outputs are in host memory and
 *                    *latency_ns = completion - arrival.  Each ticket is waited
 *                    for once.
 * lbl_server_stats   batches launched, requests completed, largest batch,
 *                    arena bytes in use (any pointer may be NULL).
 * lbl_server_free    stop the loop after the batches in flight, release all.
 */
int lbl_server_create(int32_t n, const lbl_roadmap *rms, const int32_t *n_props, const lbl_monitor *mons,
                      int32_t lanes, int32_t max_batch, int64_t mem_budget, lbl_server *out);
int lbl_server_submit(lbl_server srv, int32_t roadmap, const lbl_grid *world, const uint8_t *h_planes, lbl_pose pose,
                      uint64_t *h_L, uint64_t *h_next, uint16_t *h_viol, int64_t arrival_ns, int64_t *ticket);
int lbl_server_wait(lbl_server srv, int64_t ticket, int64_t timeout_ms, int64_t *latency_ns);
int lbl_server_stats(lbl_server srv, int64_t *batches, int64_t *completed, int64_t *max_batch, int64_t *arena_used);
int lbl_server_free(lbl_server srv);

/* --------------------------------------------------------------- session */

/*
 * A session bundles one roadmap, one world grid shape and the device buffers of
 * a whole planning query, so a frame can be run from host memory in one call:
 * copy the world planes in, transform them to the agent frame, label (with the
 * monitor, if any) and copy the results out.
 *   lbl_session_create  allocates the device buffers (planes, O, labels,
 *                       monitor outputs) for `world` and n_props; when the
 *                       planes take 8 MiB or more and the world has at most
 *                       4x the agent's cells, also a packed word per world
 *                       cell, and each frame's transform is then
 *                       lbl_pack_planes + lbl_frame_transform_words.
 *   lbl_session_run     enqueues H2D(h_planes) -> transform -> label -> D2H;
 *                       everything is ordered before the end of `s`.  h_planes:
 *                       uint8[n_props][world.d][world.h][world.w]; h_L: uint64[E];
 *                       h_next/h_viol: uint64[E]/uint16[E] or NULL.  Host buffers
 *                       should be pinned for asynchronous copies and stay
 *                       untouched until `s` completes; results are valid then.
 * Frames run back to back overlap their copies with the neighbouring frames'
 * kernels: the planes go in on the session's own copy stream into one of two
 * device buffers (frame i+1's copy runs while frame i is labeled), and on
 * roadmaps of 2^16 edges or more labeled by a streamed form (quadtree, or CSR
 * without lane groups) the labels leave on a second copy stream once the
 * frame's single labeling launch (the moving front on quadtree roadmaps of
 * about 3,000 edges per SM or more, else the per-warp stream) has ended.  Such a session keeps its own
 * pyramid and output buffers (two sets), runs its kernels on its own stream
 * and only makes `s` wait for each frame's end, so frame i+1 is computed while
 * frame i is still being copied out; it reads nothing on the device that the
 * caller writes.  Other sessions run their kernels on `s` and use the
 * roadmap's working memory like lbl_label: sessions of that kind sharing a
 * roadmap must not run at the same time.  Calls on one session must not be
 * made from several threads at once.
 */
int lbl_session_create(lbl_roadmap rm, const lbl_grid *world, int32_t n_props, lbl_monitor mon,
                       const lbl_config *cfg, lbl_session *out);
int lbl_session_run(lbl_session ss, const uint8_t *h_planes, lbl_pose pose, uint64_t *h_L, uint64_t *h_next,
                    uint16_t *h_viol, lbl_stream s);
int lbl_session_free(lbl_session ss);

#ifdef __cplusplus
}
#endif

#endif /* LBL_H_ */
