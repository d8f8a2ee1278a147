/*
 * Seeded synthetic workload generator (test and benchmark input only).
 *
 * Builds the two inputs of the labeling problem of arXiv 1810.02612:
 *   - the trajectory matrix M of eq. 10 as CSR rows (Sec. 4.3, eq. 11): for
 *     every edge, the sorted list of agent-grid cells swept by a disc
 *     footprint (eq. 5) moving along a constant-curvature arc;
 *   - world-frame proposition occupancy planes S_pi (eq. 6) made of discs,
 *     lane bands and convex polygons.
 *
 * Random numbers are drawn by the caller and passed in as shape parameters;
 * nothing here is part of the labeling arithmetic (no frame transform, no
 * Boolean product, no monitor).  A cell belongs to a set iff its centre lies in
 * the set (closed), the reading used for "intersects region i" (Sec. 4.1).
 *
 * Cell order of the emitted column indices: 0 = row-major (iy*w+ix), 1 = z-order
 * (x bit i at position 2i+1, y bit i at position 2i; square power-of-two grid).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SYN_ORDER_ROWMAJOR 0
#define SYN_ORDER_MORTON 1

/* ---------------------------------------------------------------- geometry */

typedef struct {
  int straight, full, wide;
  double ax, ay, bx, by; /* start and end points */
  double dx, dy, len;    /* unit heading and length (straight) */
  double cx, cy, R, sgn; /* circle centre, radius, sign of curvature */
  double u0x, u0y, u1x, u1y;
} arcgeom_t;

static void arc_setup(arcgeom_t *g, double px, double py, double th, double kappa, double len) {
  memset(g, 0, sizeof(*g));
  g->ax = px;
  g->ay = py;
  g->len = len;
  if (fabs(kappa) < 1e-9 || !(len > 0.0)) { /* a segment, or a zero-length arc: its start point */
    g->straight = 1;
    g->dx = cos(th);
    g->dy = sin(th);
    g->bx = px + len * g->dx;
    g->by = py + len * g->dy;
    return;
  }
  double inv = 1.0 / kappa;
  g->sgn = kappa > 0 ? 1.0 : -1.0;
  g->R = fabs(inv);
  g->cx = px - inv * sin(th);
  g->cy = py + inv * cos(th);
  double th1 = th + kappa * len;
  g->bx = g->cx + inv * sin(th1);
  g->by = g->cy - inv * cos(th1);
  g->u0x = g->sgn * sin(th);
  g->u0y = -g->sgn * cos(th);
  g->u1x = g->sgn * sin(th1);
  g->u1y = -g->sgn * cos(th1);
  double sweep = fabs(kappa * len);
  g->full = sweep >= 2.0 * M_PI;
  g->wide = sweep > M_PI;
}

/* Euclidean distance from (x,y) to the arc (closed form). */
static double arc_dist(const arcgeom_t *g, double x, double y) {
  if (g->straight) {
    double t = (x - g->ax) * g->dx + (y - g->ay) * g->dy;
    if (t < 0) t = 0;
    if (t > g->len) t = g->len;
    double ex = x - g->ax - t * g->dx, ey = y - g->ay - t * g->dy;
    return sqrt(ex * ex + ey * ey);
  }
  double wx = x - g->cx, wy = y - g->cy;
  double rho = sqrt(wx * wx + wy * wy);
  int in = 1;
  if (!g->full && rho > 0) {
    if (!g->wide) {
      double c0 = g->sgn * (g->u0x * wy - g->u0y * wx);
      double c1 = g->sgn * (wx * g->u1y - wy * g->u1x);
      in = (c0 >= 0) && (c1 >= 0);
    } else {
      double c0 = g->sgn * (g->u1x * wy - g->u1y * wx);
      double c1 = g->sgn * (wx * g->u0y - wy * g->u0x);
      in = !((c0 > 0) && (c1 > 0));
    }
  }
  if (in) return fabs(rho - g->R);
  double ex = x - g->ax, ey = y - g->ay, fx = x - g->bx, fy = y - g->by;
  double d0 = sqrt(ex * ex + ey * ey), d1 = sqrt(fx * fx + fy * fy);
  return d0 < d1 ? d0 : d1;
}

/* Conservative bounding box of the arc (samples plus chord sagitta). */
static void arc_bbox(const arcgeom_t *g, double *xlo, double *xhi, double *ylo, double *yhi) {
  double lo_x = g->ax < g->bx ? g->ax : g->bx, hi_x = g->ax < g->bx ? g->bx : g->ax;
  double lo_y = g->ay < g->by ? g->ay : g->by, hi_y = g->ay < g->by ? g->by : g->ay;
  if (!g->straight) {
    double phi0 = atan2(g->u0y, g->u0x);
    double sweep = g->full ? 2.0 * M_PI : fabs(g->len / g->R);
    int n = (int)ceil(sweep / 0.05) + 1;
    double step = sweep / n;
    for (int i = 0; i <= n; i++) {
      double a = phi0 + g->sgn * step * i;
      double x = g->cx + g->R * cos(a), y = g->cy + g->R * sin(a);
      if (x < lo_x) lo_x = x;
      if (x > hi_x) hi_x = x;
      if (y < lo_y) lo_y = y;
      if (y > hi_y) hi_y = y;
    }
    double sag = g->R * (1.0 - cos(step * 0.5)) + 1e-9;
    lo_x -= sag;
    hi_x += sag;
    lo_y -= sag;
    hi_y += sag;
  }
  *xlo = lo_x;
  *xhi = hi_x;
  *ylo = lo_y;
  *yhi = hi_y;
}

/* --------------------------------------------------------------- cell order */

static uint64_t spread_bits(uint64_t v) {
  v &= 0xFFFFFFFFull;
  v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
  v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
  v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

static inline uint32_t cell_key(int order, int w, int ix, int iy) {
  if (order == SYN_ORDER_MORTON) return (uint32_t)((spread_bits((uint64_t)ix) << 1) | spread_bits((uint64_t)iy));
  return (uint32_t)iy * (uint32_t)w + (uint32_t)ix;
}

/* ------------------------------------------------------- per-thread scratch */

typedef struct {
  uint32_t *stamp;
  size_t stamp_cap;
  uint32_t gen;
  int32_t *queue;
  size_t queue_cap;
  uint32_t *keys, *tmp;
  size_t keys_cap, tmp_cap;
} scratch_t;

static int grow(void **p, size_t *cap, size_t need, size_t elem) {
  if (need <= *cap) return 0;
  size_t nc = *cap ? *cap : 1024;
  while (nc < need) nc *= 2;
  void *q = realloc(*p, nc * elem);
  if (!q) return -1;
  *p = q;
  *cap = nc;
  return 0;
}

static void radix_sort_u32(uint32_t *a, uint32_t *tmp, size_t n) {
  size_t cnt[256];
  for (int shift = 0; shift < 32; shift += 8) {
    memset(cnt, 0, sizeof(cnt));
    int any = 0;
    for (size_t i = 0; i < n; i++) {
      uint32_t d = (a[i] >> shift) & 255u;
      cnt[d]++;
      any |= (d != 0);
    }
    if (!any) continue;
    size_t s = 0;
    for (int d = 0; d < 256; d++) {
      size_t c = cnt[d];
      cnt[d] = s;
      s += c;
    }
    for (size_t i = 0; i < n; i++) tmp[cnt[(a[i] >> shift) & 255u]++] = a[i];
    memcpy(a, tmp, n * sizeof(uint32_t));
  }
}

/*
 * Swept cells of one arc: all in-grid cells whose centre is within `radius` of
 * the arc.  Flood fill over the unclipped lattice from the cell holding the
 * start point (the lattice set of a closed disc of radius > res/sqrt(2) moved
 * along a curve is 4-connected); a plain bounding-box scan otherwise.
 * Returns the number of keys written to s->keys (sorted, unique), or -1.
 */
static long sweep_one(scratch_t *s, const arcgeom_t *g, double radius, int w, int h, double res, double x0, double y0,
                      int order) {
  double bx0, bx1, by0, by1;
  arc_bbox(g, &bx0, &bx1, &by0, &by1);
  long i_lo = (long)floor((bx0 - radius - x0) / res) - 2, i_hi = (long)floor((bx1 + radius - x0) / res) + 2;
  long j_lo = (long)floor((by0 - radius - y0) / res) - 2, j_hi = (long)floor((by1 + radius - y0) / res) + 2;
  long bw = i_hi - i_lo + 1, bh = j_hi - j_lo + 1;
  size_t area = (size_t)bw * (size_t)bh;
  long n = 0;
  int flood = radius > res * 0.70711;
  long si = (long)floor((g->ax - x0) / res), sj = (long)floor((g->ay - y0) / res);
  if (flood) {
    double cxs = x0 + (si + 0.5) * res, cys = y0 + (sj + 0.5) * res;
    if (!(arc_dist(g, cxs, cys) <= radius)) flood = 0;
  }
  if (!flood) {
    /* bounding-box scan clipped to the grid */
    long a0 = i_lo < 0 ? 0 : i_lo, a1 = i_hi >= w ? w - 1 : i_hi;
    long b0 = j_lo < 0 ? 0 : j_lo, b1 = j_hi >= h ? h - 1 : j_hi;
    if (a0 > a1 || b0 > b1) return 0;
    size_t need = (size_t)(a1 - a0 + 1) * (size_t)(b1 - b0 + 1);
    if (grow((void **)&s->keys, &s->keys_cap, need, sizeof(uint32_t))) return -1;
    if (grow((void **)&s->tmp, &s->tmp_cap, need, sizeof(uint32_t))) return -1;
    for (long j = b0; j <= b1; j++)
      for (long i = a0; i <= a1; i++)
        if (arc_dist(g, x0 + (i + 0.5) * res, y0 + (j + 0.5) * res) <= radius)
          s->keys[n++] = cell_key(order, w, (int)i, (int)j);
  } else {
    if (area > s->stamp_cap) {
      size_t cap = s->stamp_cap ? s->stamp_cap : 4096;
      while (cap < area) cap *= 2;
      free(s->stamp);
      s->stamp = (uint32_t *)calloc(cap, sizeof(uint32_t));
      if (!s->stamp) return -1;
      s->stamp_cap = cap;
      s->gen = 0;
    }
    if (s->gen == 0xFFFFFFFFu) {
      memset(s->stamp, 0, s->stamp_cap * sizeof(uint32_t));
      s->gen = 0;
    }
    /* one generation per edge: stamps left by earlier edges never match */
    uint32_t gen = ++s->gen;
    if (grow((void **)&s->queue, &s->queue_cap, 2 * area, sizeof(int32_t))) return -1;
    size_t head = 0, tail = 0;
    s->queue[tail++] = (int32_t)(si - i_lo);
    s->queue[tail++] = (int32_t)(sj - j_lo);
    s->stamp[(size_t)(sj - j_lo) * bw + (si - i_lo)] = gen;
    while (head < tail) {
      long li = s->queue[head++], lj = s->queue[head++];
      long i = li + i_lo, j = lj + j_lo;
      if (!(arc_dist(g, x0 + (i + 0.5) * res, y0 + (j + 0.5) * res) <= radius)) continue;
      if (i >= 0 && i < w && j >= 0 && j < h) {
        if (grow((void **)&s->keys, &s->keys_cap, (size_t)n + 1, sizeof(uint32_t))) return -1;
        s->keys[n++] = cell_key(order, w, (int)i, (int)j);
      }
      static const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
      for (int k = 0; k < 4; k++) {
        long ni = li + di[k], nj = lj + dj[k];
        if (ni < 0 || nj < 0 || ni >= bw || nj >= bh) continue;
        uint32_t *st = &s->stamp[(size_t)nj * bw + ni];
        if (*st == gen) continue;
        *st = gen;
        s->queue[tail++] = (int32_t)ni;
        s->queue[tail++] = (int32_t)nj;
      }
    }
    if (grow((void **)&s->tmp, &s->tmp_cap, (size_t)n + 1, sizeof(uint32_t))) return -1;
  }
  radix_sort_u32(s->keys, s->tmp, (size_t)n);
  return n;
}

/* --------------------------------------------------------------- roadmaps */

typedef struct {
  int64_t n_edges, n_chunks, chunk;
  int64_t *counts;    /* per edge */
  uint32_t **bufs;    /* per chunk */
  int64_t *chunk_nnz; /* per chunk */
  int64_t nnz;
} build_t;

void synth_free_build(void *hb) {
  build_t *b = (build_t *)hb;
  if (!b) return;
  if (b->bufs)
    for (int64_t c = 0; c < b->n_chunks; c++) free(b->bufs[c]);
  free(b->bufs);
  free(b->counts);
  free(b->chunk_nnz);
  free(b);
}

/*
 * Rasterise n_edges arcs; arcs = float64[n_edges][5] (x, y, heading, curvature,
 * length) in the grid's frame.  Returns an opaque build holding the rows, or
 * NULL on allocation failure; *nnz_out receives the total swept-cell count.
 */
void *synth_sweep_build(int64_t n_edges, const double *arcs, double radius, int32_t w, int32_t h, double res,
                        double x0, double y0, int32_t order, int32_t n_threads, int64_t *nnz_out) {
  build_t *b = (build_t *)calloc(1, sizeof(build_t));
  if (!b) return NULL;
  b->n_edges = n_edges;
  b->chunk = 1024;
  b->n_chunks = (n_edges + b->chunk - 1) / b->chunk;
  b->counts = (int64_t *)calloc((size_t)(n_edges > 0 ? n_edges : 1), sizeof(int64_t));
  b->bufs = (uint32_t **)calloc((size_t)(b->n_chunks > 0 ? b->n_chunks : 1), sizeof(uint32_t *));
  b->chunk_nnz = (int64_t *)calloc((size_t)(b->n_chunks > 0 ? b->n_chunks : 1), sizeof(int64_t));
  if (!b->counts || !b->bufs || !b->chunk_nnz) {
    synth_free_build(b);
    return NULL;
  }
  int failed = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel reduction(| : failed)
  {
    scratch_t s;
    memset(&s, 0, sizeof(s));
#pragma omp for schedule(dynamic, 1)
    for (int64_t c = 0; c < b->n_chunks; c++) {
      int64_t e0 = c * b->chunk, e1 = e0 + b->chunk < n_edges ? e0 + b->chunk : n_edges;
      size_t cap = 0, used = 0;
      uint32_t *buf = NULL;
      for (int64_t e = e0; e < e1 && !failed; e++) {
        arcgeom_t g;
        const double *a = arcs + 5 * e;
        arc_setup(&g, a[0], a[1], a[2], a[3], a[4]);
        long n = sweep_one(&s, &g, radius, w, h, res, x0, y0, order);
        if (n < 0 || grow((void **)&buf, &cap, used + (size_t)n + 1, sizeof(uint32_t))) {
          failed = 1;
          break;
        }
        memcpy(buf + used, s.keys, (size_t)n * sizeof(uint32_t));
        used += (size_t)n;
        b->counts[e] = n;
      }
      b->bufs[c] = buf;
      b->chunk_nnz[c] = (int64_t)used;
    }
    free(s.stamp);
    free(s.queue);
    free(s.keys);
    free(s.tmp);
  }
  if (failed) {
    synth_free_build(b);
    return NULL;
  }
  int64_t nnz = 0;
  for (int64_t c = 0; c < b->n_chunks; c++) nnz += b->chunk_nnz[c];
  b->nnz = nnz;
  *nnz_out = nnz;
  return b;
}

/* Copy a build into caller arrays rowptr[n_edges+1], colidx[nnz]; frees it. */
int synth_sweep_take(void *hb, int64_t *rowptr, int32_t *colidx) {
  build_t *b = (build_t *)hb;
  if (!b) return -1;
  rowptr[0] = 0;
  for (int64_t e = 0; e < b->n_edges; e++) rowptr[e + 1] = rowptr[e] + b->counts[e];
  int64_t *off = (int64_t *)malloc((size_t)(b->n_chunks + 1) * sizeof(int64_t));
  if (!off) return -1;
  off[0] = 0;
  for (int64_t c = 0; c < b->n_chunks; c++) off[c + 1] = off[c] + b->chunk_nnz[c];
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t c = 0; c < b->n_chunks; c++)
    if (b->chunk_nnz[c]) memcpy(colidx + off[c], b->bufs[c], (size_t)b->chunk_nnz[c] * sizeof(int32_t));
  free(off);
  synth_free_build(b);
  return 0;
}

/* Distance from points to one arc (for tests that need the generator's own
   geometry, e.g. lane bands). */
void synth_arc_dist(const double *arc5, int64_t n, const double *xy, double *out) {
  arcgeom_t g;
  arc_setup(&g, arc5[0], arc5[1], arc5[2], arc5[3], arc5[4]);
  for (int64_t i = 0; i < n; i++) out[i] = arc_dist(&g, xy[2 * i], xy[2 * i + 1]);
}

/* --------------------------------------------------- world occupancy planes */

/* All plane writers: plane = uint8[h][w] over a grid with corner (x0,y0) and
   resolution res; a cell is set iff its centre lies in the shape.  Each returns
   the number of cells that changed from 0 to 1. */

int64_t synth_plane_disc(uint8_t *plane, int32_t w, int32_t h, double res, double x0, double y0, double cx, double cy,
                         double rad) {
  long i0 = (long)floor((cx - rad - x0) / res) - 1, i1 = (long)floor((cx + rad - x0) / res) + 1;
  long j0 = (long)floor((cy - rad - y0) / res) - 1, j1 = (long)floor((cy + rad - y0) / res) + 1;
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i1 >= w) i1 = w - 1;
  if (j1 >= h) j1 = h - 1;
  int64_t added = 0;
  double r2 = rad * rad;
  for (long j = j0; j <= j1; j++)
    for (long i = i0; i <= i1; i++) {
      double dx = x0 + (i + 0.5) * res - cx, dy = y0 + (j + 0.5) * res - cy;
      if (dx * dx + dy * dy <= r2) {
        uint8_t *p = &plane[(size_t)j * w + i];
        added += (*p == 0);
        *p = 1;
      }
    }
  return added;
}

int64_t synth_plane_band(uint8_t *plane, int32_t w, int32_t h, double res, double x0, double y0, const double *arc5,
                         double half_width) {
  arcgeom_t g;
  arc_setup(&g, arc5[0], arc5[1], arc5[2], arc5[3], arc5[4]);
  double bx0, bx1, by0, by1;
  arc_bbox(&g, &bx0, &bx1, &by0, &by1);
  long i0 = (long)floor((bx0 - half_width - x0) / res) - 1, i1 = (long)floor((bx1 + half_width - x0) / res) + 1;
  long j0 = (long)floor((by0 - half_width - y0) / res) - 1, j1 = (long)floor((by1 + half_width - y0) / res) + 1;
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i1 >= w) i1 = w - 1;
  if (j1 >= h) j1 = h - 1;
  int64_t added = 0;
  for (long j = j0; j <= j1; j++)
    for (long i = i0; i <= i1; i++)
      if (arc_dist(&g, x0 + (i + 0.5) * res, y0 + (j + 0.5) * res) <= half_width) {
        uint8_t *p = &plane[(size_t)j * w + i];
        added += (*p == 0);
        *p = 1;
      }
  return added;
}

/* Convex polygon with n counter-clockwise vertices xs[i], ys[i]. */
int64_t synth_plane_polygon(uint8_t *plane, int32_t w, int32_t h, double res, double x0, double y0, const double *xs,
                            const double *ys, int32_t n) {
  double lx = xs[0], hx = xs[0], ly = ys[0], hy = ys[0];
  for (int k = 1; k < n; k++) {
    if (xs[k] < lx) lx = xs[k];
    if (xs[k] > hx) hx = xs[k];
    if (ys[k] < ly) ly = ys[k];
    if (ys[k] > hy) hy = ys[k];
  }
  long i0 = (long)floor((lx - x0) / res) - 1, i1 = (long)floor((hx - x0) / res) + 1;
  long j0 = (long)floor((ly - y0) / res) - 1, j1 = (long)floor((hy - y0) / res) + 1;
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i1 >= w) i1 = w - 1;
  if (j1 >= h) j1 = h - 1;
  int64_t added = 0;
  for (long j = j0; j <= j1; j++)
    for (long i = i0; i <= i1; i++) {
      double px = x0 + (i + 0.5) * res, py = y0 + (j + 0.5) * res;
      int inside = 1;
      for (int k = 0; k < n && inside; k++) {
        int k1 = (k + 1) % n;
        double ex = xs[k1] - xs[k], ey = ys[k1] - ys[k];
        if (ex * (py - ys[k]) - ey * (px - xs[k]) < 0) inside = 0;
      }
      if (inside) {
        uint8_t *p = &plane[(size_t)j * w + i];
        added += (*p == 0);
        *p = 1;
      }
    }
  return added;
}

/* ------------------------------------------- time-augmented (x, y, tau) grids */

static uint64_t spread3_bits(uint64_t v) {
  uint64_t r = 0;
  for (int i = 0; i < 21; i++) r |= ((v >> i) & 1ull) << (3 * i);
  return r;
}

static inline uint32_t cell_key3(int order, int w, int h, int ix, int iy, int it) {
  if (order == SYN_ORDER_MORTON)
    return (uint32_t)((spread3_bits((uint64_t)ix) << 2) | (spread3_bits((uint64_t)iy) << 1) |
                      spread3_bits((uint64_t)it));
  return ((uint32_t)it * (uint32_t)h + (uint32_t)iy) * (uint32_t)w + (uint32_t)ix;
}

/*
 * Swept cells of arcs travelled at constant speed from time 0: arcs =
 * float64[n][6] (x, y, heading, curvature, length, speed).  Cell (ix, iy, it)
 * belongs to the row iff some point of the arc reached during time slab it
 * (closed interval [t0 + it*tres, t0 + (it+1)*tres]) lies within `radius` of
 * the cell's (x, y) centre.  Same build/take protocol as synth_sweep_build.
 */
void *synth_sweep3_build(int64_t n_edges, const double *arcs, double radius, int32_t w, int32_t h, int32_t d,
                         double res, double x0, double y0, double tres, double t0, int32_t order, int32_t n_threads,
                         int64_t *nnz_out) {
  build_t *b = (build_t *)calloc(1, sizeof(build_t));
  if (!b) return NULL;
  b->n_edges = n_edges;
  b->chunk = 256;
  b->n_chunks = (n_edges + b->chunk - 1) / b->chunk;
  b->counts = (int64_t *)calloc((size_t)(n_edges > 0 ? n_edges : 1), sizeof(int64_t));
  b->bufs = (uint32_t **)calloc((size_t)(b->n_chunks > 0 ? b->n_chunks : 1), sizeof(uint32_t *));
  b->chunk_nnz = (int64_t *)calloc((size_t)(b->n_chunks > 0 ? b->n_chunks : 1), sizeof(int64_t));
  if (!b->counts || !b->bufs || !b->chunk_nnz) {
    synth_free_build(b);
    return NULL;
  }
  int failed = 0;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel reduction(| : failed)
  {
    scratch_t s;
    memset(&s, 0, sizeof(s));
    uint32_t *row = NULL, *tmp = NULL;
    size_t row_cap = 0, tmp_cap = 0;
#pragma omp for schedule(dynamic, 1)
    for (int64_t c = 0; c < b->n_chunks; c++) {
      int64_t e0 = c * b->chunk, e1 = e0 + b->chunk < n_edges ? e0 + b->chunk : n_edges;
      size_t cap = 0, used = 0;
      uint32_t *buf = NULL;
      for (int64_t e = e0; e < e1 && !failed; e++) {
        const double *a = arcs + 6 * e;
        const double len = a[4], v = a[5];
        size_t n_row = 0;
        for (int32_t it = 0; it < d && !failed; it++) {
          double sa = v * (t0 + it * tres), sb = v * (t0 + (it + 1) * tres);
          if (sa < 0) sa = 0;
          if (sb > len) sb = len;
          if (sa > sb) continue;
          /* the sub-arc travelled during the slab, as an arc of its own */
          const double k = a[3], th = a[2];
          double px, py;
          if (fabs(k) < 1e-9) {
            px = a[0] + sa * cos(th);
            py = a[1] + sa * sin(th);
          } else {
            px = a[0] + (sin(th + k * sa) - sin(th)) / k;
            py = a[1] - (cos(th + k * sa) - cos(th)) / k;
          }
          arcgeom_t g;
          arc_setup(&g, px, py, th + k * sa, k, sb - sa);
          long n = sweep_one(&s, &g, radius, w, h, res, x0, y0, SYN_ORDER_ROWMAJOR);
          if (n < 0 || grow((void **)&row, &row_cap, n_row + (size_t)n + 1, sizeof(uint32_t))) {
            failed = 1;
            break;
          }
          for (long i = 0; i < n; i++) {
            const int ix = (int)(s.keys[i] % (uint32_t)w), iy = (int)(s.keys[i] / (uint32_t)w);
            row[n_row++] = cell_key3(order, w, h, ix, iy, it);
          }
        }
        if (failed || grow((void **)&tmp, &tmp_cap, n_row + 1, sizeof(uint32_t)) ||
            grow((void **)&buf, &cap, used + n_row + 1, sizeof(uint32_t))) {
          failed = 1;
          break;
        }
        radix_sort_u32(row, tmp, n_row);
        memcpy(buf + used, row, n_row * sizeof(uint32_t));
        used += n_row;
        b->counts[e] = (int64_t)n_row;
      }
      b->bufs[c] = buf;
      b->chunk_nnz[c] = (int64_t)used;
    }
    free(s.stamp);
    free(s.queue);
    free(s.keys);
    free(s.tmp);
    free(row);
    free(tmp);
  }
  if (failed) {
    synth_free_build(b);
    return NULL;
  }
  int64_t nnz = 0;
  for (int64_t c = 0; c < b->n_chunks; c++) nnz += b->chunk_nnz[c];
  b->nnz = nnz;
  *nnz_out = nnz;
  return b;
}

/* A disc of radius rad whose centre moves as (cx + vx t, cy + vy t): in every
   time slab of the volume (uint8[d][h][w]) the cells whose centre lies in the
   disc at the slab's mid time.  Returns the cells that changed from 0 to 1. */
int64_t synth_volume_moving_disc(uint8_t *vol, int32_t w, int32_t h, int32_t d, double res, double x0, double y0,
                                 double tres, double t0, double cx, double cy, double vx, double vy, double rad) {
  int64_t added = 0;
  for (int32_t it = 0; it < d; it++) {
    const double t = t0 + (it + 0.5) * tres;
    added += synth_plane_disc(vol + (size_t)it * w * h, w, h, res, x0, y0, cx + vx * t, cy + vy * t, rad);
  }
  return added;
}
