/*
 * ORACLE — test infrastructure only.  Plain, slow, obviously correct CPU
 * definition of the labeling path of arXiv 1810.02612 (Paden, Liu, Cullen,
 * "Accelerated Labeling of Discrete Abstractions for Planning Under LTL
 * Specifications").  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library; the product path never does.
 *
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Functions and the passage each follows:
 *   orc_morton / orc_cell_index  z-order cell index, Sec. 4.1 (Algorithm 1 and
 *                                the bit-interleaving equivalence stated with it)
 *   orc_frame_coeffs             fixed-point affine map of the equivariance step,
 *   orc_frame_transform          Sec. 5 (eq. 13): the roadmap lives in the agent
 *                                frame; the perceived world grids are re-expressed
 *                                there at the planning pose
 *   orc_label / orc_label_rows   Boolean matrix product L = M.P over the CSR
 *                                rows of M (eq. 10, rows stored as in eq. 11)
 *   orc_monitor                  safety-monitor transition delta(q, L(e)) for every
 *                                monitor state, Sec. 3.2
 *   orc_arc_geometry / orc_arc_dist / orc_sweep
 *                                swept-cell rows of a roadmap: eq. 7 with the closed
 *                                disc footprint of eq. 5, discretised by cell centres
 *                                (Sec. 4.1)
 *   orc_morton3 / orc_cell_index3 / orc_time_coeffs / orc_frame_transform3
 *                                the time-augmented (x, y, tau) workspace of Sec. 5:
 *                                3-D z-order and the frame transform with the
 *                                time shift of eq. 13
 *
 * Readings of the paper used here (the paper is silent or garbled at these
 * points):
 *   - CSR: row pointer r and column indices c as in eq. 11 and Algorithm 2.
 *   - z-order: x bit i goes to index bit 2i+1, y bit i to bit 2i (axis 0 split
 *     first, at the most significant level).
 *   - Agent grid cell (ix,iy) has its centre at (x0+(ix+.5)res, y0+(iy+.5)res)
 *     in the agent frame; the world point under it is (X,Y)+R(theta)*centre.
 *     The world cell is the floor of ((p - corner)/res_w), evaluated as a Q32.32
 *     fixed-point affine map of (ix,iy) whose six coefficients are rounded once
 *     (half to even) from double; outside the world grid reads as false.
 *   - Label bits at positions >= P are zero.
 *   - Monitor: deterministic table delta[q][letter] with an explicit reject
 *     state; the letter is formed from m <= 8 selected proposition bits.
 *   - Time axis: agent time cell it has its centre at t0 + (it+.5)tres relative
 *     to the query time T; the world time cell is the floor of
 *     ((T + centre) - t0_w)/tres_w, again a Q32.32 affine map rounded once.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off (no contraction, so the
 * double arithmetic of orc_frame_coeffs is evaluated exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ROWMAJOR 0
#define ORC_MORTON 1

/* ------------------------------------------------------------ cell index */

/* z-order index: interleave the bits of ix and iy one at a time. */
uint64_t orc_morton(uint32_t ix, uint32_t iy) {
  uint64_t n = 0;
  for (int i = 0; i < 32; i++) {
    uint64_t xb = (ix >> i) & 1u;
    uint64_t yb = (iy >> i) & 1u;
    n |= xb << (2 * i + 1);
    n |= yb << (2 * i);
  }
  return n;
}

int64_t orc_cell_index(int32_t order, int32_t w, int32_t ix, int32_t iy) {
  if (order == ORC_MORTON) return (int64_t)orc_morton((uint32_t)ix, (uint32_t)iy);
  return (int64_t)iy * w + ix;
}

/* --------------------------------------------------------- frame transform */

/* floor(v / 2^32) for any signed v, written without relying on shifts of
   negative numbers. */
static int64_t floor_q32(int64_t v) {
  const int64_t one = (int64_t)1 << 32;
  int64_t q = v / one;
  if (v % one != 0 && v < 0) q -= 1;
  return q;
}

static int64_t to_q32(double a) {
  /* a * 2^32 is exact in double; nearbyint rounds half to even */
  return (int64_t)nearbyint(a * 4294967296.0);
}

/*
 * Coefficients of the map (ix,iy) -> continuous world-cell coordinates (u,v):
 *   u = a00*ix + a01*iy + b0,   v = a10*ix + a11*iy + b1
 * out = {A00, A01, B0, A10, A11, B1} in Q32.32.
 */
void orc_frame_coeffs(double wres, double wx0, double wy0, double ares, double ax0, double ay0, double X, double Y,
                      double theta, int64_t *out) {
  double c = cos(theta);
  double s = sin(theta);
  double k = ares / wres;
  double a00 = c * k;
  double a01 = -(s * k);
  double a10 = s * k;
  double a11 = c * k;
  double xa = ax0 + 0.5 * ares; /* centre of agent cell (0,0), agent frame */
  double ya = ay0 + 0.5 * ares;
  double b0 = ((X + ((c * xa) - (s * ya))) - wx0) / wres;
  double b1 = ((Y + ((s * xa) + (c * ya))) - wy0) / wres;
  out[0] = to_q32(a00);
  out[1] = to_q32(a01);
  out[2] = to_q32(b0);
  out[3] = to_q32(a10);
  out[4] = to_q32(a11);
  out[5] = to_q32(b1);
}

/*
 * O[cell_index(ix,iy)] bit p = planes[p][wy][wx] != 0 at the world cell under
 * the agent cell's centre; 0 when that world cell is outside the world grid.
 * planes: uint8[P][wh][ww] row-major.  O: uint64[aw*ah].
 */
int orc_frame_transform(int32_t ww, int32_t wh, double wres, double wx0, double wy0, const uint8_t *planes, int32_t P,
                        double X, double Y, double theta, int32_t aw, int32_t ah, double ares, double ax0, double ay0,
                        int32_t aorder, uint64_t *O) {
  if (P < 0 || P > 64) return -1;
  int64_t q[6];
  orc_frame_coeffs(wres, wx0, wy0, ares, ax0, ay0, X, Y, theta, q);
  for (int32_t iy = 0; iy < ah; iy++) {
    for (int32_t ix = 0; ix < aw; ix++) {
      int64_t u = q[0] * ix + q[1] * iy + q[2];
      int64_t v = q[3] * ix + q[4] * iy + q[5];
      int64_t wxc = floor_q32(u);
      int64_t wyc = floor_q32(v);
      uint64_t word = 0;
      if (wxc >= 0 && wxc < ww && wyc >= 0 && wyc < wh) {
        for (int32_t p = 0; p < P; p++) {
          uint8_t occ = planes[(size_t)p * ww * wh + (size_t)wyc * ww + (size_t)wxc];
          if (occ != 0) word |= (uint64_t)1 << p;
        }
      }
      O[orc_cell_index(aorder, aw, ix, iy)] = word;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ labels */

/*
 * L(e, p) = OR over the nonzeros k of row e of P(colidx[k], p)  (eq. 10).
 * Bit p of an OR of words is the OR of their bits p, so each row ORs the whole
 * words of its cells and then clears the bits at positions >= P.  No early
 * exit.  Rows are independent, so the row loop may be split across n_threads
 * OpenMP threads without changing any result.
 */
void orc_label(int64_t n_edges, const int64_t *rowptr, const int32_t *colidx, const uint64_t *O, int32_t P,
               uint64_t *L, int32_t n_threads) {
  const uint64_t keep = P <= 0 ? 0 : (P >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << P) - 1));
#pragma omp parallel for schedule(dynamic, 1024) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t e = 0; e < n_edges; e++) {
    uint64_t word = 0;
    for (int64_t k = rowptr[e]; k < rowptr[e + 1]; k++) word |= O[colidx[k]];
    L[e] = word & keep;
  }
}

/* The same product for a list of rows, one element (edge, proposition) at a
   time: bit p of L[i] is set iff some nonzero k of row rows[i] has bit p of
   O[colidx[k]] set. */
void orc_label_rows(int64_t n_rows, const int64_t *rows, const int64_t *rowptr, const int32_t *colidx,
                    const uint64_t *O, int32_t P, uint64_t *L) {
  for (int64_t i = 0; i < n_rows; i++) {
    int64_t e = rows[i];
    uint64_t word = 0;
    for (int32_t p = 0; p < P; p++) {
      uint64_t hit = 0;
      for (int64_t k = rowptr[e]; k < rowptr[e + 1]; k++) hit |= (O[colidx[k]] >> p) & 1u;
      word |= hit << p;
    }
    L[i] = word;
  }
}

/* ----------------------------------------------------------------- monitor */

/*
 * For every edge e and monitor state q < n_states:
 *   letter = sum_j bit(L[e], relbits[j]) << j,   q' = delta[q][letter]
 * next[e] holds q' in bits [4q, 4q+4); viol[e] bit q is set iff q' == reject.
 * delta: uint8[n_states][2^m].
 */
int orc_monitor(int32_t n_states, int32_t m, const uint8_t *relbits, const uint8_t *delta, int32_t reject,
                const uint64_t *L, int64_t n, uint64_t *next, uint16_t *viol) {
  if (n_states < 1 || n_states > 16 || m < 0 || m > 8) return -1;
  for (int64_t e = 0; e < n; e++) {
    uint32_t letter = 0;
    for (int32_t j = 0; j < m; j++) letter |= (uint32_t)((L[e] >> relbits[j]) & 1u) << j;
    uint64_t word = 0;
    uint16_t v = 0;
    for (int32_t q = 0; q < n_states; q++) {
      uint32_t qn = delta[(size_t)q * ((size_t)1 << m) + letter];
      word |= (uint64_t)(qn & 15u) << (4 * q);
      if ((int32_t)qn == reject) v |= (uint16_t)(1u << q);
    }
    next[e] = word;
    viol[e] = v;
  }
  return 0;
}

/* ------------------------------------------------ time-augmented workspace */

/*
 * Sec. 5: the workspace is (x, y, tau); dynamic objects become static volumes.
 * 3-D z-order (Algorithm 1 with k = 3, axis 0 = x split first): bit i of ix
 * goes to index bit 3i+2, of iy to 3i+1, of it (time) to 3i.
 */
uint64_t orc_morton3(uint32_t ix, uint32_t iy, uint32_t it) {
  uint64_t n = 0;
  for (int i = 0; i < 21; i++) {
    n |= (uint64_t)((ix >> i) & 1u) << (3 * i + 2);
    n |= (uint64_t)((iy >> i) & 1u) << (3 * i + 1);
    n |= (uint64_t)((it >> i) & 1u) << (3 * i);
  }
  return n;
}

int64_t orc_cell_index3(int32_t order, int32_t w, int32_t h, int32_t ix, int32_t iy, int32_t it) {
  if (order == ORC_MORTON) return (int64_t)orc_morton3((uint32_t)ix, (uint32_t)iy, (uint32_t)it);
  return ((int64_t)it * h + iy) * w + ix;
}

/* Q32.32 time map it -> continuous world time-cell coordinate:
   v_t = at * it + bt, the agent time-cell centre shifted by the query time T
   (the equivariance of eq. 13 in t).  out = {At, Bt}. */
void orc_time_coeffs(double wtres, double wt0, double atres, double at0, double T, int64_t *out) {
  double a = atres / wtres;
  double ta = at0 + 0.5 * atres; /* centre of agent time cell 0 */
  double b = ((T + ta) - wt0) / wtres;
  out[0] = to_q32(a);
  out[1] = to_q32(b);
}

/*
 * 3-D frame transform: agent cell (ix, iy, it) reads the world volume cell
 * (wx, wy, wt) with (wx, wy) as in orc_frame_transform and wt the floor of the
 * time map; volumes: uint8[P][wd][wh][ww]; outside the world volume reads 0.
 * O: uint64[aw * ah * ad] in the agent order.
 */
int orc_frame_transform3(int32_t ww, int32_t wh, int32_t wd, double wres, double wx0, double wy0, double wtres,
                         double wt0, const uint8_t *vols, int32_t P, double X, double Y, double theta, double T,
                         int32_t aw, int32_t ah, int32_t ad, double ares, double ax0, double ay0, double atres,
                         double at0, int32_t aorder, uint64_t *O) {
  if (P < 0 || P > 64) return -1;
  int64_t q[6], qt[2];
  orc_frame_coeffs(wres, wx0, wy0, ares, ax0, ay0, X, Y, theta, q);
  orc_time_coeffs(wtres, wt0, atres, at0, T, qt);
  for (int32_t it = 0; it < ad; it++) {
    int64_t wtc = floor_q32(qt[0] * it + qt[1]);
    for (int32_t iy = 0; iy < ah; iy++) {
      for (int32_t ix = 0; ix < aw; ix++) {
        int64_t wxc = floor_q32(q[0] * ix + q[1] * iy + q[2]);
        int64_t wyc = floor_q32(q[3] * ix + q[4] * iy + q[5]);
        uint64_t word = 0;
        if (wxc >= 0 && wxc < ww && wyc >= 0 && wyc < wh && wtc >= 0 && wtc < wd) {
          for (int32_t p = 0; p < P; p++) {
            size_t off = (((size_t)p * wd + (size_t)wtc) * wh + (size_t)wyc) * ww + (size_t)wxc;
            if (vols[off] != 0) word |= (uint64_t)1 << p;
          }
        }
        O[orc_cell_index3(aorder, aw, ah, ix, iy, it)] = word;
      }
    }
  }
  return 0;
}

/* -------------------------------------------- swept cells (roadmap rows) */

/*
 * The swept set of eq. 7 discretised as in Sec. 4.1: cell c belongs to row e
 * iff the distance from c's centre to the arc X(e) is at most the footprint
 * radius (closed disc footprint, F of eq. 5).  Arc = (x, y, heading,
 * curvature, length): a straight segment if |curvature| < 1e-9, else a circle
 * arc of radius 1/|curvature| turning by curvature * length.
 *
 * Geometry (12 doubles): straight: {1, x, y, cos, sin, len, ...}; circle:
 * {0, cx, cy, R, sgn, u0x, u0y, u1x, u1y, px1, py1, sweep class} where u0/u1 are
 * the unit vectors from the centre to the start/end, (px1, py1) the end point
 * and the class is 2 (full turn), 1 (more than half a turn) or 0.
 */
void orc_arc_geometry(const double *a, double *g) {
  const double x = a[0], y = a[1], th = a[2], k = a[3], len = a[4];
  for (int i = 0; i < 12; i++) g[i] = 0.0;
  if (fabs(k) < 1e-9 || !(len > 0.0)) { /* a segment, or a zero-length arc: its start point */
    g[0] = 1.0;
    g[1] = x;
    g[2] = y;
    g[3] = cos(th);
    g[4] = sin(th);
    g[5] = len;
    return;
  }
  const double inv = 1.0 / k;
  const double sg = k > 0 ? 1.0 : -1.0;
  const double cx = x - inv * sin(th);
  const double cy = y + inv * cos(th);
  const double th1 = th + k * len;
  const double sweep = fabs(k * len);
  g[0] = 0.0;
  g[1] = cx;
  g[2] = cy;
  g[3] = fabs(inv);
  g[4] = sg;
  g[5] = sg * sin(th);
  g[6] = -sg * cos(th);
  g[7] = sg * sin(th1);
  g[8] = -sg * cos(th1);
  g[9] = cx + inv * sin(th1);
  g[10] = cy - inv * cos(th1);
  g[11] = sweep >= 2.0 * M_PI ? 2.0 : (sweep > M_PI ? 1.0 : 0.0);
}

/* Distance from (px, py) to the arc: the nearest circle point if its angle is
   inside the arc's sweep (tested with cross products against the end
   directions), else the nearer end point; for segments, the clamped
   projection. */
double orc_arc_dist(const double *g, const double *a, double px, double py) {
  if (g[0] == 1.0) {
    double t = (px - g[1]) * g[3] + (py - g[2]) * g[4];
    if (t < 0.0) t = 0.0;
    if (t > g[5]) t = g[5];
    const double ex = (px - g[1]) - t * g[3];
    const double ey = (py - g[2]) - t * g[4];
    return sqrt(ex * ex + ey * ey);
  }
  const double wx = px - g[1], wy = py - g[2];
  const double rho = sqrt(wx * wx + wy * wy);
  int inside = 1;
  if (g[11] != 2.0 && rho > 0.0) {
    if (g[11] == 0.0) {
      const double c0 = g[4] * (g[5] * wy - g[6] * wx);
      const double c1 = g[4] * (wx * g[8] - wy * g[7]);
      inside = (c0 >= 0.0) && (c1 >= 0.0);
    } else {
      const double c0 = g[4] * (g[7] * wy - g[8] * wx);
      const double c1 = g[4] * (wx * g[6] - wy * g[5]);
      inside = !((c0 > 0.0) && (c1 > 0.0));
    }
  }
  if (inside) return fabs(rho - g[3]);
  const double ax = px - a[0], ay = py - a[1], bx = px - g[9], by = py - g[10];
  const double d0 = sqrt(ax * ax + ay * ay), d1 = sqrt(bx * bx + by * by);
  return d0 < d1 ? d0 : d1;
}

/* Rows of the listed arcs over every cell of a 2-D grid (plain scan in cell
   index order, so each row comes out sorted).  counts[i] receives row i's
   length; keys (may be NULL) receives the rows one after another. */
int64_t orc_sweep(int64_t n, const double *arcs, double radius, int32_t w, int32_t h, double res, double x0,
                  double y0, int32_t order, int64_t *counts, int32_t *keys) {
  int64_t total = 0;
  const int64_t cells = (int64_t)w * h;
  for (int64_t i = 0; i < n; i++) {
    double g[12];
    orc_arc_geometry(arcs + 5 * i, g);
    int64_t cnt = 0;
    for (int64_t idx = 0; idx < cells; idx++) {
      int32_t ix, iy;
      if (order == ORC_MORTON) {
        uint32_t xs = 0, ys = 0;
        for (int b = 0; b < 16; b++) {
          xs |= (uint32_t)((idx >> (2 * b + 1)) & 1) << b;
          ys |= (uint32_t)((idx >> (2 * b)) & 1) << b;
        }
        ix = (int32_t)xs;
        iy = (int32_t)ys;
      } else {
        iy = (int32_t)(idx / w);
        ix = (int32_t)(idx - (int64_t)iy * w);
      }
      const double cx = x0 + (ix + 0.5) * res, cy = y0 + (iy + 0.5) * res;
      if (orc_arc_dist(g, arcs + 5 * i, cx, cy) <= radius) {
        if (keys) keys[total] = (int32_t)idx;
        total++;
        cnt++;
      }
    }
    counts[i] = cnt;
  }
  return total;
}
