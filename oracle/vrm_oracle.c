/*
 * CPU oracle for the splitting-free vorticity redistribution method (VRM)
 * diffusion operator of Kirchhart & Obi, "A Splitting-free Vorticity
 * Redistribution Method" (arXiv 1508.06379).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 restatement of
 * the method, written to be checked against the paper by eye.  Only the test
 * suite, the smoke check and the timed CPU baseline of bench.py load it.  It
 * shares no code, header, table or helper with the CUDA library, and the
 * CUDA library never calls it.
 *
 * Built with -O2 -ffp-contract=off so that every a*b+c below is two roundings,
 * except where fma() is called explicitly.
 *
 * Parity pins (what ties each function to something other than itself) are in
 * tests/test_oracle_*.py.  Every function here has at least one pin.
 *
 * Conventions
 *   - r_ij = x_j - x_i (Sec. 2, definition of r_ij); xi_ij = r_ij * (1/h).
 *   - f~ = h^2 f is the h-scaled weight (Sec. 2, last paragraph), so that the
 *     moment conditions read V(xi) f~ = b with the b of Eq. (cond_two).
 *   - Indices are 0-based.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define ORC_PIVOT_CAP 64
#define ORC_TOL_PRICE 1e-9    /* entering: reduced cost < -tol */
#define ORC_TOL_PIVOT 1e-9    /* ratio test: pivot element > tol */
#define ORC_TOL_TIE 1e-12     /* ratio ties: within tol * max(1, min ratio) */
#define ORC_TOL_PHASE1 1e-10  /* feasible iff phase-I objective <= tol */
#define ORC_TOL_SNAP 1e-11    /* basic values <= tol are degenerate zeros */
#define ORC_TOL_RESID 1e-12   /* accepted iff max |V f - b| <= tol */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* Growth control: the reduced operator (Sec. 3.5, Eq. reduced_bound).       */
/* ------------------------------------------------------------------------ */

/* floor(t) for 0 <= t < 2^127 as an unsigned 128-bit integer: hi/lo split. */
static u128 dbl_floor_to_u128(double t) {
  const double two64 = 18446744073709551616.0;
  uint64_t hi = (uint64_t)(t / two64);
  double rem = t - (double)hi * two64;
  uint64_t lo = (uint64_t)rem;
  return ((u128)hi << 64) | (u128)lo;
}

/* Nearest-ish double of an unsigned 128-bit integer by a fixed sequence:
   RN(RN(hi) * 2^64 + RN(lo)). */
static double u128_to_dbl(u128 s) {
  const double two64 = 18446744073709551616.0;
  uint64_t hi = (uint64_t)(s >> 64), lo = (uint64_t)s;
  return (double)hi * two64 + (double)lo;
}

typedef struct {
  uint64_t key;
  int64_t idx;
} orc_key;

static int cmp_key(const void* a, const void* b) {
  const orc_key* p = (const orc_key*)a;
  const orc_key* q = (const orc_key*)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
  return 0;
}

/*
 * Sec. 3.5: particles are left out of diffusion, smallest |Gamma_i| first, as
 * long as the l1 norm of the left-out set I stays within
 *     ||Gamma_I||_1 <= C_diff h^{n+2} ||Gamma||_1          (Eq. reduced_bound)
 * Reading: I is the longest prefix of the particles sorted by (|Gamma_i|, i)
 * whose sum stays within the bound; D is the rest.
 *
 * Sums are exact so that the choice of D does not depend on summation order:
 * |Gamma_i| is scaled by the power of two 2^(96-E) (max|Gamma| < 2^E) and
 * truncated to an integer q_i; sum S and the bound tau = floor(c * dbl(S))
 * are 128-bit integers.  c_bound = C_diff * h^{n+2} is given by the caller.
 *
 * Writes diffused[i] in {0,1}; returns |D|.
 */
long orc_reduce(const double* gamma, long n, double c_bound, unsigned char* diffused) {
  if (n <= 0) return 0;
  double amax = 0.0;
  for (long i = 0; i < n; ++i) {
    double a = fabs(gamma[i]);
    if (a > amax) amax = a;
  }
  if (amax == 0.0 || !(c_bound < 1.0)) {
    /* no circulation, or a bound of at least ||Gamma||_1: nothing diffuses */
    memset(diffused, 0, (size_t)n);
    return 0;
  }
  int E;
  frexp(amax, &E); /* amax = m 2^E, m in [0.5, 1): amax < 2^E */
  u128* q = (u128*)malloc(sizeof(u128) * (size_t)n);
  orc_key* keys = (orc_key*)malloc(sizeof(orc_key) * (size_t)n);
  u128 S = 0;
  for (long i = 0; i < n; ++i) {
    double a = fabs(gamma[i]);
    q[i] = dbl_floor_to_u128(ldexp(a, 96 - E));
    S += q[i];
    uint64_t bits;
    memcpy(&bits, &a, sizeof bits);
    keys[i].key = bits; /* non-negative doubles order like their bit patterns */
    keys[i].idx = i;
  }
  u128 tau = dbl_floor_to_u128(c_bound * u128_to_dbl(S));
  qsort(keys, (size_t)n, sizeof(orc_key), cmp_key);
  for (long i = 0; i < n; ++i) diffused[i] = 1;
  u128 cum = 0;
  long left_out = 0;
  for (long k = 0; k < n; ++k) {
    long i = (long)keys[k].idx;
    if (cum + q[i] > tau) break;
    cum += q[i];
    diffused[i] = 0;
    ++left_out;
  }
  free(q);
  free(keys);
  return n - left_out;
}

/* ------------------------------------------------------------------------ */
/* Neighbourhoods (Sec. 2, Eq. neighbourhood) and 45-degree segments        */
/* (Sec. 4.2).                                                               */
/* ------------------------------------------------------------------------ */

/*
 * Segment k covers the half-open angle [k pi/4, (k+1) pi/4) counter-clockwise
 * from +x.  Written with comparisons only, so that seg(-r) = seg(r) + 4 mod 8
 * holds exactly.  (dx, dy) = (0, 0) never reaches here (r > 0).
 */
int orc_segment(double dx, double dy) {
  if (dx > 0 && dy >= 0) return dy < dx ? 0 : 1;
  if (dx <= 0 && dy > 0) return dy > -dx ? 2 : 3;
  if (dx < 0 && dy <= 0) return dy > dx ? 4 : 5;
  /* dx >= 0 && dy < 0 */
  return -dy > dx ? 6 : 7;
}

static int segment_f(float dx, float dy) {
  if (dx > 0 && dy >= 0) return dy < dx ? 0 : 1;
  if (dx <= 0 && dy > 0) return dy > -dx ? 2 : 3;
  if (dx < 0 && dy <= 0) return dy > dx ? 4 : 5;
  return -dy > dx ? 6 : 7;
}

/*
 * Annulus test r h <= |x_j - x_i| <= R h (Eq. neighbourhood), on squared
 * distances lo2 = (r h)^2, hi2 = (R h)^2, inclusive at both ends.
 * d2 = dx*dx + dy*dy: two products and one sum, no fused multiply-add.
 * fp32 != 0 evaluates the same sequence in binary32 on positions rounded to
 * binary32 (the mixed-precision search of the library).
 * Returns 1 if j is in the annulus, with d2 and the segment of r_ij.
 */
static int annulus(const double* x, const double* y, long i, long j, double lo2, double hi2, int fp32,
                   double* d2_out, int* seg_out) {
  if (fp32) {
    float dx = (float)x[j] - (float)x[i];
    float dy = (float)y[j] - (float)y[i];
    float d2 = dx * dx + dy * dy;
    if (d2 < (float)lo2 || d2 > (float)hi2) return 0;
    *d2_out = (double)d2;
    *seg_out = segment_f(dx, dy);
    return 1;
  }
  double dx = x[j] - x[i];
  double dy = y[j] - y[i];
  double d2 = dx * dx + dy * dy;
  if (d2 < lo2 || d2 > hi2) return 0;
  *d2_out = d2;
  *seg_out = orc_segment(dx, dy);
  return 1;
}

/* Uniform bucket grid over the particles (the paper's neighbourhood search is
   hash based, Sec. 5.2); bucket side slightly above R h so that the 3 x 3
   buckets around a particle hold its whole annulus. */
typedef struct {
  double x0, y0, cs;
  long nx, ny;
  long* start; /* nx*ny + 1 */
  long* items; /* particle indices grouped by bucket, ascending within one */
} orc_grid;

static void grid_build(orc_grid* g, const double* x, const double* y, long n, double Rh) {
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  for (long i = 0; i < n; ++i) {
    if (x[i] < xmin) xmin = x[i];
    if (x[i] > xmax) xmax = x[i];
    if (y[i] < ymin) ymin = y[i];
    if (y[i] > ymax) ymax = y[i];
  }
  if (n == 0) xmin = xmax = ymin = ymax = 0.0;
  g->cs = Rh * (1.0 + 1e-6);
  /* keep the bucket count near n for very sparse clouds */
  double w = xmax - xmin, hgt = ymax - ymin;
  while ((w / g->cs + 1.0) * (hgt / g->cs + 1.0) > 4.0 * (double)n + 64.0) g->cs *= 2.0;
  g->x0 = xmin;
  g->y0 = ymin;
  g->nx = (long)floor(w / g->cs) + 1;
  g->ny = (long)floor(hgt / g->cs) + 1;
  long nb = g->nx * g->ny;
  g->start = (long*)calloc((size_t)nb + 1, sizeof(long));
  g->items = (long*)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
  long* cell = (long*)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
  for (long i = 0; i < n; ++i) {
    long cx = (long)floor((x[i] - g->x0) / g->cs);
    long cy = (long)floor((y[i] - g->y0) / g->cs);
    if (cx < 0) cx = 0;
    if (cx >= g->nx) cx = g->nx - 1;
    if (cy < 0) cy = 0;
    if (cy >= g->ny) cy = g->ny - 1;
    cell[i] = cy * g->nx + cx;
    g->start[cell[i] + 1]++;
  }
  for (long b = 0; b < nb; ++b) g->start[b + 1] += g->start[b];
  long* fill = (long*)malloc(sizeof(long) * (size_t)nb);
  memcpy(fill, g->start, sizeof(long) * (size_t)nb);
  for (long i = 0; i < n; ++i) g->items[fill[cell[i]]++] = i;
  free(fill);
  free(cell);
}

static void grid_free(orc_grid* g) {
  free(g->start);
  free(g->items);
}

/* Bucket coordinates of a point, clamped to the grid. */
static void grid_cell(const orc_grid* g, double px, double py, long* cx, long* cy) {
  long a = (long)floor((px - g->x0) / g->cs);
  long b = (long)floor((py - g->y0) / g->cs);
  /* points outside the grid by more than one bucket have no neighbours in it;
     clamping to one bucket outside keeps the 3x3 loop correct */
  if (a < -1) a = -1;
  if (a > g->nx) a = g->nx;
  if (b < -1) b = -1;
  if (b > g->ny) b = g->ny;
  *cx = a;
  *cy = b;
}

static int cmp_long(const void* a, const void* b) {
  long p = *(const long*)a, q = *(const long*)b;
  return (p > q) - (p < q);
}

/*
 * Neighbourhood N_i minus {i} of every particle (Eq. neighbourhood), the mask
 * of occupied 45-degree segments (Sec. 4.2), and the small neighbourhood: the
 * closest particle of every segment, ties to the smaller index (Sec. 4.3).
 *
 * count[i]        = |N_i \ {i}| (true size, even above k_cap)
 * idx[i*k_cap+t]  = the min(count, k_cap) smallest member indices, ascending
 * mask[i]         = bit s set iff segment s holds a member
 * small[i*8+s]    = closest member of segment s, -1 if empty
 * Returns the largest count.
 */
long orc_neighbours(const double* x, const double* y, long n, double lo2, double hi2, double Rh, int fp32,
                    int* count, int* idx, int k_cap, unsigned char* mask, int* small) {
  orc_grid g;
  grid_build(&g, x, y, n, Rh);
  long maxc = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(max : maxc)
  for (long i = 0; i < n; ++i) {
    long cx, cy;
    grid_cell(&g, x[i], y[i], &cx, &cy);
    long cap = 64, cnt = 0;
    long* list = (long*)malloc(sizeof(long) * (size_t)cap);
    double best_d2[8];
    long best_j[8];
    for (int s = 0; s < 8; ++s) {
      best_d2[s] = INFINITY;
      best_j[s] = -1;
    }
    unsigned char m = 0;
    for (long by = cy - 1; by <= cy + 1; ++by) {
      if (by < 0 || by >= g.ny) continue;
      for (long bx = cx - 1; bx <= cx + 1; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        long b = by * g.nx + bx;
        for (long t = g.start[b]; t < g.start[b + 1]; ++t) {
          long j = g.items[t];
          if (j == i) continue;
          double d2;
          int s;
          if (!annulus(x, y, i, j, lo2, hi2, fp32, &d2, &s)) continue;
          if (cnt == cap) {
            cap *= 2;
            list = (long*)realloc(list, sizeof(long) * (size_t)cap);
          }
          list[cnt++] = j;
          m |= (unsigned char)(1u << s);
          if (d2 < best_d2[s] || (d2 == best_d2[s] && j < best_j[s])) {
            best_d2[s] = d2;
            best_j[s] = j;
          }
        }
      }
    }
    qsort(list, (size_t)cnt, sizeof(long), cmp_long);
    count[i] = (int)cnt;
    for (long t = 0; t < cnt && t < k_cap; ++t) idx[(size_t)i * k_cap + t] = (int)list[t];
    for (long t = cnt; t < k_cap; ++t) idx[(size_t)i * k_cap + t] = -1;
    mask[i] = m;
    for (int s = 0; s < 8; ++s) small[(size_t)i * 8 + s] = (int)best_j[s];
    if (cnt > maxc) maxc = cnt;
    free(list);
  }
  grid_free(&g);
  return maxc;
}

/* ------------------------------------------------------------------------ */
/* Insertion of zero-strength particles (Sec. 2 and Sec. 4.2).              */
/* ------------------------------------------------------------------------ */

/*
 * Offsets of the insertion points: radius 1.5 h on the centre line of segment
 * s, at angle (s + 1/2) pi/4.  cos and sin of 22.5 degrees are taken from the
 * half-angle identities so that every platform gets the same bits:
 * cos = sqrt(2 + sqrt 2)/2, sin = sqrt(2 - sqrt 2)/2.
 */
void orc_insertion_offsets(double h, double* ox, double* oy) {
  double c = 0.5 * sqrt(2.0 + sqrt(2.0));
  double s = 0.5 * sqrt(2.0 - sqrt(2.0));
  double ux[8] = {c, s, -s, -c, -c, -s, s, c};
  double uy[8] = {s, c, c, s, -s, -c, -c, -s};
  double a = 1.5 * h;
  for (int k = 0; k < 8; ++k) {
    ox[k] = a * ux[k];
    oy[k] = a * uy[k];
  }
}

/*
 * Insertion rounds.  Reading of Sec. 4.2 for simultaneous insertions:
 *   one round = for every diffused i (ascending) the segments of its annulus
 *   that hold no particle of the current cloud give candidates with key (i, s)
 *   at p = x_i + offset_s; a candidate is dropped if a candidate with a
 *   smaller key lies closer than r h (d2 < lo2); the rest are appended in key
 *   order with Gamma = 0.  Rounds repeat until no candidate is left, at most
 *   max_rounds times.  Only diffused particles ask for insertion (Sec. 2:
 *   neighbours are needed for circulation-carrying particles).
 *
 * x, y have room for `capacity` entries; [0, n) are given.  Returns n' (the
 * new count), or -(needed) if capacity is too small.  *rounds = insertion
 * rounds that appended something; *open_out = empty segments of diffused
 * particles left after the last round (0 unless max_rounds was hit).
 */
long orc_insert(double* x, double* y, long n, long capacity, const unsigned char* diffused, double h, double lo2,
                double hi2, double Rh, int max_rounds, int* rounds, long* open_out) {
  double ox[8], oy[8];
  orc_insertion_offsets(h, ox, oy);
  long n_cur = n;
  *rounds = 0;
  *open_out = 0;
  unsigned char* mask = (unsigned char*)malloc((size_t)(n > 0 ? n : 1));
  for (int round = 0; round <= max_rounds; ++round) {
    /* occupancy of the annulus segments of every diffused particle */
    orc_grid g;
    grid_build(&g, x, y, n_cur, Rh);
#pragma omp parallel for schedule(dynamic, 256)
    for (long i = 0; i < n; ++i) {
      mask[i] = 0xFF;
      if (!diffused[i]) continue;
      unsigned char m = 0;
      long cx, cy;
      grid_cell(&g, x[i], y[i], &cx, &cy);
      for (long by = cy - 1; by <= cy + 1; ++by) {
        if (by < 0 || by >= g.ny) continue;
        for (long bx = cx - 1; bx <= cx + 1; ++bx) {
          if (bx < 0 || bx >= g.nx) continue;
          long b = by * g.nx + bx;
          for (long t = g.start[b]; t < g.start[b + 1]; ++t) {
            long j = g.items[t];
            double d2;
            int s;
            if (j == i) continue;
            if (annulus(x, y, i, j, lo2, hi2, 0, &d2, &s)) m |= (unsigned char)(1u << s);
          }
        }
      }
      mask[i] = m;
    }
    grid_free(&g);
    long ncand = 0;
    for (long i = 0; i < n; ++i)
      for (int s = 0; s < 8; ++s)
        if (!((mask[i] >> s) & 1)) ++ncand;
    if (ncand == 0) break;
    if (round == max_rounds) {
      *open_out = ncand;
      break;
    }
    double* px = (double*)malloc(sizeof(double) * (size_t)ncand);
    double* py = (double*)malloc(sizeof(double) * (size_t)ncand);
    long c = 0;
    for (long i = 0; i < n; ++i)
      for (int s = 0; s < 8; ++s)
        if (!((mask[i] >> s) & 1)) {
          px[c] = x[i] + ox[s];
          py[c] = y[i] + oy[s];
          ++c;
        }
    unsigned char* keep = (unsigned char*)malloc((size_t)ncand);
#pragma omp parallel for schedule(dynamic, 64)
    for (long a = 0; a < ncand; ++a) {
      keep[a] = 1;
      for (long b = 0; b < a; ++b) {
        double dx = px[a] - px[b];
        double dy = py[a] - py[b];
        if (dx * dx + dy * dy < lo2) {
          keep[a] = 0;
          break;
        }
      }
    }
    long nacc = 0;
    for (long a = 0; a < ncand; ++a) nacc += keep[a];
    if (n_cur + nacc > capacity) {
      free(px);
      free(py);
      free(keep);
      free(mask);
      return -(n_cur + nacc);
    }
    for (long a = 0; a < ncand; ++a)
      if (keep[a]) {
        x[n_cur] = px[a];
        y[n_cur] = py[a];
        ++n_cur;
      }
    *rounds = round + 1;
    free(px);
    free(py);
    free(keep);
  }
  free(mask);
  return n_cur;
}

/* ------------------------------------------------------------------------ */
/* Moment conditions and the phase-I simplex (Sec. 2, Eqs. cond_two,        */
/* cond_alpha, momcondmv; Sec. 4.1).                                         */
/* ------------------------------------------------------------------------ */

/* Number of moment rows: multi-indices 1 <= |alpha| <= n+1 (Eq. momcondmv). */
int orc_rows(int order) { return order == 2 ? 9 : 5; }

/* Stencil slots kept per particle: a basic solution of the m-row LP has at
   most m nonzero weights, so 8 slots hold every n = 1 stencil (m = 5) and
   12 every n = 2 stencil (m = 9). */
int orc_stencil_width(int order) { return order == 2 ? 12 : 8; }

/*
 * Column of the Vandermonde matrix for one neighbour (Eq. momcondmv), rows in
 * the order (1,0) (0,1) (2,0) (1,1) (0,2) [(3,0) (2,1) (1,2) (0,3)], in the
 * scaled offsets xi = r_ij / h.  Right-hand side b: 2 at (2,0) and (0,2),
 * 0 elsewhere (Eqs. cond_two, cond_alpha).
 */
void orc_vandermonde_column(int order, double xi, double eta, double* col) {
  double xx = xi * xi, yy = eta * eta;
  col[0] = xi;
  col[1] = eta;
  col[2] = xx;
  col[3] = xi * eta;
  col[4] = yy;
  if (order == 2) {
    col[5] = xx * xi;
    col[6] = xx * eta;
    col[7] = xi * yy;
    col[8] = yy * eta;
  }
}

void orc_rhs(int order, double* b) {
  int m = orc_rows(order);
  for (int a = 0; a < m; ++a) b[a] = 0.0;
  b[2] = 2.0;
  b[4] = 2.0;
}

/* LU factorisation with partial pivoting of the m x m matrix A (row-major),
   in place; piv[k] = row swapped with k (first row of largest |A[r][k]|),
   rcp[k] = 1 / U[k][k].  The multipliers are A[r][k] * rcp[k].
   Returns 0 if singular. */
static int lu_factor(int m, double* A, int* piv, double* rcp) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = fabs(A[k * m + k]);
    for (int r = k + 1; r < m; ++r)
      if (fabs(A[r * m + k]) > best) {
        best = fabs(A[r * m + k]);
        p = r;
      }
    piv[k] = p;
    if (best == 0.0) return 0;
    if (p != k)
      for (int c = 0; c < m; ++c) {
        double t = A[k * m + c];
        A[k * m + c] = A[p * m + c];
        A[p * m + c] = t;
      }
    rcp[k] = 1.0 / A[k * m + k];
    for (int r = k + 1; r < m; ++r) {
      double l = A[r * m + k] * rcp[k];
      A[r * m + k] = l;
      for (int c = k + 1; c < m; ++c) A[r * m + c] = A[r * m + c] - l * A[k * m + c];
    }
  }
  return 1;
}

/* Solve A z = rhs with the factors of lu_factor (z overwrites rhs). */
static void lu_solve(int m, const double* LU, const int* piv, const double* rcp, double* z) {
  for (int k = 0; k < m; ++k)
    if (piv[k] != k) {
      double t = z[k];
      z[k] = z[piv[k]];
      z[piv[k]] = t;
    }
  for (int r = 1; r < m; ++r)
    for (int c = 0; c < r; ++c) z[r] = z[r] - LU[r * m + c] * z[c];
  for (int r = m - 1; r >= 0; --r) {
    for (int c = r + 1; c < m; ++c) z[r] = z[r] - LU[r * m + c] * z[c];
    z[r] = z[r] * rcp[r];
  }
}

/* Solve A^T z = rhs with the factors of lu_factor (P A = L U, so
   A^T = U^T L^T P). */
static void lu_solve_transposed(int m, const double* LU, const int* piv, const double* rcp, double* z) {
  for (int r = 0; r < m; ++r) {
    for (int c = 0; c < r; ++c) z[r] = z[r] - LU[c * m + r] * z[c];
    z[r] = z[r] * rcp[r];
  }
  for (int r = m - 1; r >= 0; --r)
    for (int c = r + 1; c < m; ++c) z[r] = z[r] - LU[c * m + r] * z[c];
  for (int k = m - 1; k >= 0; --k)
    if (piv[k] != k) {
      double t = z[k];
      z[k] = z[piv[k]];
      z[piv[k]] = t;
    }
}

/*
 * Phase I of the simplex method for V f = b, f >= 0 (Eq. momcondmv, Sec. 4.1):
 *   minimise sum(a)  s.t.  V f + a = b,  f >= 0,  a >= 0     (b >= 0).
 * Revised form: every iteration solves the m x m systems of the current
 * basis from scratch by LU (Sec. 4.1), as the paper does.
 * Variables: artificial a_k has index k (0..m-1), structural f_j has index
 * m + j.  Start basis: the artificials.  Entering: the structural column of
 * lowest index with reduced cost < -1e-9 (Bland); artificials that left are
 * never re-entered.  Leaving: minimum ratio over pivot elements > 1e-9, the
 * basic values at or below 1e-11 taken as the zeros they are; ratios within
 * 1e-12 max(1, min) are tied and the tie goes to the basic variable of lowest
 * index (Bland).  At most 64 pivots.
 *
 * V: m x K row-major.  f: K outputs: basic values above 1e-11, others 0
 * (degenerate basics come out at rounding level, of either sign; they are
 * zeros of the vertex and are snapped to 0 so that f >= 0 holds exactly).
 * Returns 0 feasible (phase-I objective <= 1e-10 and max |V f - b| <= 1e-12,
 * 1 infeasible, 2 pivot cap or singular basis.  *npiv = pivots taken,
 * *resid = max |V f - b|.
 */
int orc_phase1(int m, int K, const double* V, const double* b, double* f, int* npiv, double* resid) {
  int basis[9];
  double B[81], xB[9], y[9], d[9], rcp[9];
  int piv[9];
  for (int k = 0; k < m; ++k) basis[k] = k;
  int it = 0, status = 0;
  for (;;) {
    /* basis matrix: column k is the column of variable basis[k] */
    for (int r = 0; r < m; ++r)
      for (int k = 0; k < m; ++k) {
        int v = basis[k];
        B[r * m + k] = v < m ? (r == v ? 1.0 : 0.0) : V[r * K + (v - m)];
      }
    if (!lu_factor(m, B, piv, rcp)) {
      status = 2;
      break;
    }
    for (int r = 0; r < m; ++r) xB[r] = b[r];
    lu_solve(m, B, piv, rcp, xB);
    for (int k = 0; k < m; ++k) y[k] = basis[k] < m ? 1.0 : 0.0;
    lu_solve_transposed(m, B, piv, rcp, y);
    /* pricing (Bland): lowest structural index with reduced cost < -tol */
    int q = -1;
    for (int j = 0; j < K && q < 0; ++j) {
      int in_basis = 0;
      for (int k = 0; k < m; ++k)
        if (basis[k] == m + j) in_basis = 1;
      if (in_basis) continue;
      double s = 0.0;
      for (int r = 0; r < m; ++r) s += y[r] * V[r * K + j];
      double dj = 0.0 - s;
      if (dj < -ORC_TOL_PRICE) q = j;
    }
    if (q < 0) break; /* optimal for phase I */
    if (it == ORC_PIVOT_CAP) {
      status = 2;
      break;
    }
    for (int r = 0; r < m; ++r) d[r] = V[r * K + q];
    lu_solve(m, B, piv, rcp, d);
    /* ratio test */
    /* basic values at or below the snap tolerance are degenerate zeros */
    double xr[9];
    for (int k = 0; k < m; ++k) xr[k] = xB[k] > ORC_TOL_SNAP ? xB[k] : 0.0;
    double theta = INFINITY;
    for (int k = 0; k < m; ++k)
      if (d[k] > ORC_TOL_PIVOT) {
        double ratio = xr[k] / d[k];
        if (ratio < theta) theta = ratio;
      }
    if (theta == INFINITY) {
      status = 2;
      break;
    }
    double lim = theta + ORC_TOL_TIE * (theta > 1.0 ? theta : 1.0);
    int leave = -1;
    for (int k = 0; k < m; ++k)
      if (d[k] > ORC_TOL_PIVOT && xr[k] / d[k] <= lim)
        if (leave < 0 || basis[k] < basis[leave]) leave = k;
    basis[leave] = m + q;
    ++it;
  }
  *npiv = it;
  for (int j = 0; j < K; ++j) f[j] = 0.0;
  *resid = INFINITY;
  if (status != 0) return status;
  /* final basic solution */
  for (int r = 0; r < m; ++r)
    for (int k = 0; k < m; ++k) {
      int v = basis[k];
      B[r * m + k] = v < m ? (r == v ? 1.0 : 0.0) : V[r * K + (v - m)];
    }
  if (!lu_factor(m, B, piv, rcp)) return 2;
  for (int r = 0; r < m; ++r) xB[r] = b[r];
  lu_solve(m, B, piv, rcp, xB);
  double w = 0.0;
  for (int k = 0; k < m; ++k)
    if (basis[k] < m) w += xB[k];
    else f[basis[k] - m] = xB[k] > ORC_TOL_SNAP ? xB[k] : 0.0;
  double rmax = 0.0;
  for (int r = 0; r < m; ++r) {
    double s = 0.0;
    for (int j = 0; j < K; ++j) s += V[r * K + j] * f[j];
    double e = fabs(s - b[r]);
    if (e > rmax) rmax = e;
  }
  *resid = rmax;
  if (w > ORC_TOL_PHASE1 || rmax > ORC_TOL_RESID) {
    for (int j = 0; j < K; ++j) f[j] = 0.0;
    return 1;
  }
  return 0;
}

typedef struct {
  double d2;
  long j;
  double dx, dy;
} orc_col;

static int cmp_col(const void* a, const void* b) {
  const orc_col* p = (const orc_col*)a;
  const orc_col* q = (const orc_col*)b;
  if (p->d2 != q->d2) return p->d2 < q->d2 ? -1 : 1;
  return (p->j > q->j) - (p->j < q->j);
}

/* Solve one particle's LP on the given column set (ordered by (d2, j)). */
static int solve_columns(int order, double inv_h, orc_col* cols, int K, double* f, int* npiv, double* resid) {
  int m = orc_rows(order);
  double* V = (double*)malloc(sizeof(double) * (size_t)m * (size_t)(K > 0 ? K : 1));
  double colv[9], b[9];
  orc_rhs(order, b);
  for (int j = 0; j < K; ++j) {
    orc_vandermonde_column(order, cols[j].dx * inv_h, cols[j].dy * inv_h, colv);
    for (int r = 0; r < m; ++r) V[r * K + j] = colv[r];
  }
  int st = orc_phase1(m, K, V, b, f, npiv, resid);
  free(V);
  return st;
}

/*
 * Redistribution weights of every diffused particle (Sec. 4.1, 4.3):
 * LP on the small neighbourhood (columns ordered by (d2, j)); if that is
 * infeasible and fallback != 0, LP on the whole N_i \ {i} (at most k_cap
 * columns, ordered by (d2, j)); if that fails too the stencil is zero and the
 * particle does not diffuse (a reading: the paper is silent).
 * f~_ii = -sum_j f~_ij in column order (Eq. fii).
 *
 * Outputs per particle i (W slots): cols[i*W+t], f[i*W+t] = the nonzero
 * weights in column order, padded with -1 / 0; fii[i]; status[i] =
 *   0 not diffused, 1 small neighbourhood, 2 full neighbourhood, 3 no stencil.
 * npiv[i] = pivots of the last LP solved for i.
 */
void orc_solve_weights(const double* x, const double* y, long n, const unsigned char* diffused, const int* count,
                       const int* idx, int k_cap, const int* small, double h, int order, int fallback, int W,
                       int* cols, double* f, double* fii, unsigned char* status, int* npiv) {
  double inv_h = 1.0 / h;
#pragma omp parallel for schedule(dynamic, 256)
  for (long i = 0; i < n; ++i) {
    for (int t = 0; t < W; ++t) {
      cols[(size_t)i * W + t] = -1;
      f[(size_t)i * W + t] = 0.0;
    }
    fii[i] = 0.0;
    status[i] = 0;
    npiv[i] = 0;
    if (!diffused[i]) continue;
    int kfull = count[i] < k_cap ? count[i] : k_cap;
    int kmax = kfull > 8 ? kfull : 8;
    orc_col* cl = (orc_col*)malloc(sizeof(orc_col) * (size_t)kmax);
    double* fv = (double*)malloc(sizeof(double) * (size_t)kmax);
    int K = 0;
    for (int s = 0; s < 8; ++s) {
      long j = small[(size_t)i * 8 + s];
      if (j < 0) continue;
      cl[K].j = j;
      cl[K].dx = x[j] - x[i];
      cl[K].dy = y[j] - y[i];
      cl[K].d2 = cl[K].dx * cl[K].dx + cl[K].dy * cl[K].dy;
      ++K;
    }
    qsort(cl, (size_t)K, sizeof(orc_col), cmp_col);
    double resid;
    int np;
    int st = solve_columns(order, inv_h, cl, K, fv, &np, &resid);
    unsigned char code = 1;
    if (st != 0 && fallback) {
      /* full neighbourhood: k_cap smallest (d2, j) of N_i \ {i} */
      int Kf = 0;
      for (int t = 0; t < kfull; ++t) {
        long j = idx[(size_t)i * k_cap + t];
        cl[Kf].j = j;
        cl[Kf].dx = x[j] - x[i];
        cl[Kf].dy = y[j] - y[i];
        cl[Kf].d2 = cl[Kf].dx * cl[Kf].dx + cl[Kf].dy * cl[Kf].dy;
        ++Kf;
      }
      qsort(cl, (size_t)Kf, sizeof(orc_col), cmp_col);
      K = Kf;
      st = solve_columns(order, inv_h, cl, K, fv, &np, &resid);
      code = 2;
    }
    npiv[i] = np;
    if (st != 0) {
      status[i] = 3;
    } else {
      status[i] = code;
      int t = 0;
      double s = 0.0;
      for (int c = 0; c < K; ++c) {
        if (fv[c] == 0.0) continue;
        if (t < W) {
          cols[(size_t)i * W + t] = (int)cl[c].j;
          f[(size_t)i * W + t] = fv[c];
        }
        ++t;
        s += fv[c];
      }
      fii[i] = -s;
    }
    free(cl);
    free(fv);
  }
}

/* ------------------------------------------------------------------------ */
/* Operator application and Euler step (Sec. 3.3 and Eq. nsode).            */
/* ------------------------------------------------------------------------ */

/*
 * dGamma_j/dt = nu sum_i f_ij Gamma_i = (nu/h^2) sum_i f~_ij Gamma_i
 * (Eq. nsode, second line), over diffused i (Eq. reducedop), terms summed in
 * ascending i with the self term f~_jj Gamma_j at i = j; products and sums
 * rounded separately.  Particles j >= n_gamma carry Gamma = 0 (inserted).
 * nu_over_h2 = nu / (h*h) is given by the caller.
 */
void orc_apply(long n_total, long n_gamma, const double* gamma, const unsigned char* diffused, const int* cols,
               const double* f, const double* fii, int W, double nu_over_h2, double* dgamma) {
  double* acc = (double*)calloc((size_t)(n_total > 0 ? n_total : 1), sizeof(double));
  for (long i = 0; i < n_gamma && i < n_total; ++i) {
    if (!diffused[i]) continue;
    double g = gamma[i];
    /* each column j appears at most once per i, and at most once as i itself */
    for (int t = 0; t < W; ++t) {
      int j = cols[(size_t)i * W + t];
      if (j < 0) continue;
      acc[j] = acc[j] + f[(size_t)i * W + t] * g;
    }
    acc[i] = acc[i] + fii[i] * g;
  }
  for (long j = 0; j < n_total; ++j) dgamma[j] = nu_over_h2 * acc[j];
  free(acc);
}

/* Forward Euler on the semi-discrete system (Sec. 3.3):
   Gamma^{n+1}_j = fma(dt, dGamma_j, Gamma^n_j); Gamma^n_j = 0 for j >= n_gamma. */
void orc_euler(long n_total, long n_gamma, const double* gamma, const double* dgamma, double dt, double* gamma_out) {
  for (long j = 0; j < n_total; ++j) gamma_out[j] = fma(dt, dgamma[j], j < n_gamma ? gamma[j] : 0.0);
}

/* Counters of one oracle step. */
typedef struct {
  long n_in, n_out, n_diffused, n_inserted, open_segments;
  long small_ok, full_ok, no_stencil, max_pivots;
  int rounds;
  double max_dt_ratio; /* max over diffused i of nu dt (-f~_ii) / h^2 (Thm. stability) */
} orc_stats;

/*
 * One VRM step (Sec. 3.3 with the reduced operator of Sec. 3.5 and the
 * algorithms of Sec. 4): reduce, insert, neighbourhoods, weights, apply,
 * Euler.  x, y: capacity entries, [0, n) given; inserted particles are
 * appended.  gamma_in: n values; gamma_out: capacity entries.
 * Derived constants are computed here exactly as documented:
 *   lo2 = (r h)^2, hi2 = (R h)^2, c_bound = C_diff * h^{n+2} (repeated
 *   products), nu_over_h2 = nu / (h h).
 * Returns n' >= n, or -(needed capacity).
 */
long orc_step(double* x, double* y, long n, long capacity, const double* gamma_in, double* gamma_out, double h,
              double r, double R, double nu, double c_diff, int order, double dt, int k_cap, int max_rounds,
              int fallback, int fp32_search, orc_stats* st) {
  double rh = r * h, Rh = R * h;
  double lo2 = rh * rh, hi2 = Rh * Rh;
  double hp = h * h * h;
  if (order == 2) hp = hp * h;
  double c_bound = c_diff * hp;
  double nu_over_h2 = nu / (h * h);
  memset(st, 0, sizeof(*st));
  st->n_in = n;
  unsigned char* diffused = (unsigned char*)calloc((size_t)(capacity > 0 ? capacity : 1), 1);
  st->n_diffused = orc_reduce(gamma_in, n, c_bound, diffused);
  long open = 0;
  long n2 = orc_insert(x, y, n, capacity, diffused, h, lo2, hi2, Rh, max_rounds, &st->rounds, &open);
  if (n2 < 0) {
    free(diffused);
    return n2;
  }
  st->open_segments = open;
  st->n_inserted = n2 - n;
  st->n_out = n2;
  int W = orc_stencil_width(order);
  int* count = (int*)malloc(sizeof(int) * (size_t)n2);
  int* idx = (int*)malloc(sizeof(int) * (size_t)n2 * (size_t)k_cap);
  unsigned char* mask = (unsigned char*)malloc((size_t)n2);
  int* small = (int*)malloc(sizeof(int) * (size_t)n2 * 8);
  orc_neighbours(x, y, n2, lo2, hi2, Rh, fp32_search, count, idx, k_cap, mask, small);
  int* cols = (int*)malloc(sizeof(int) * (size_t)n2 * W);
  double* f = (double*)malloc(sizeof(double) * (size_t)n2 * W);
  double* fii = (double*)malloc(sizeof(double) * (size_t)n2);
  unsigned char* status = (unsigned char*)malloc((size_t)n2);
  int* npiv = (int*)malloc(sizeof(int) * (size_t)n2);
  orc_solve_weights(x, y, n2, diffused, count, idx, k_cap, small, h, order, fallback, W, cols, f, fii, status, npiv);
  for (long i = 0; i < n2; ++i) {
    if (status[i] == 1) st->small_ok++;
    if (status[i] == 2) st->full_ok++;
    if (status[i] == 3) st->no_stencil++;
    if (npiv[i] > st->max_pivots) st->max_pivots = npiv[i];
    if (status[i] == 1 || status[i] == 2) {
      double q = nu * dt * (-fii[i]) / (h * h);
      if (q > st->max_dt_ratio) st->max_dt_ratio = q;
    }
  }
  double* dg = (double*)malloc(sizeof(double) * (size_t)n2);
  orc_apply(n2, n, gamma_in, diffused, cols, f, fii, W, nu_over_h2, dg);
  orc_euler(n2, n, gamma_in, dg, dt, gamma_out);
  free(dg);
  free(diffused);
  free(count);
  free(idx);
  free(mask);
  free(small);
  free(cols);
  free(f);
  free(fii);
  free(status);
  free(npiv);
  return n2;
}

/* ------------------------------------------------------------------------ */
/* Particle removal (the outlook of Sec. 6.2): a particle that has come too    */
/* close to another is redistributed to its neighbours by an approximation  */
/* of the identity operator, then removed.                                   */
/* ------------------------------------------------------------------------ */

/* Key of the removal order: (|Gamma|, index); of two particles closer than
   r h the one with the smaller key goes. */
static int removal_key_less(const double* gamma, long a, long b) {
  double ga = fabs(gamma[a]), gb = fabs(gamma[b]);
  if (ga != gb) return ga < gb;
  return a < b;
}

/*
 * close[i] = 1 iff a particle j != i lies strictly closer than r h
 * (dx*dx + dy*dy < lo2, the inner bound of Eq. neighbourhood) and has the
 * larger key.  Returns the number of such candidates.
 */
long orc_close(const double* x, const double* y, const double* gamma, long n, double lo2, double Rh,
               unsigned char* close) {
  orc_grid g;
  grid_build(&g, x, y, n, Rh);
  long cnt = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : cnt)
  for (long i = 0; i < n; ++i) {
    long cx, cy;
    grid_cell(&g, x[i], y[i], &cx, &cy);
    unsigned char c = 0;
    for (long by = cy - 1; by <= cy + 1 && !c; ++by) {
      if (by < 0 || by >= g.ny) continue;
      for (long bx = cx - 1; bx <= cx + 1 && !c; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        long b = by * g.nx + bx;
        for (long t = g.start[b]; t < g.start[b + 1]; ++t) {
          long j = g.items[t];
          if (j == i) continue;
          double dx = x[j] - x[i], dy = y[j] - y[i];
          double d2 = dx * dx + dy * dy;
          if (d2 < lo2 && removal_key_less(gamma, i, j)) {
            c = 1;
            break;
          }
        }
      }
    }
    close[i] = c;
    cnt += c;
  }
  grid_free(&g);
  return cnt;
}

/*
 * Identity stencils of the candidates.  Columns: the closest kept particle
 * (close[j] == 0) of every 45-degree segment of the annulus of i (ties to
 * the smaller index), ordered by (d2, j).  Rows (0,0) (1,0) (0,1) in
 * xi = r_ij / h with b = (1, 0, 0): sum_j g_ij = 1 and sum_j g_ij r_ij = 0,
 * g >= 0 (the moment conditions of the identity that non-negative weights
 * can meet: the second moments of g are positive).  The phase-I simplex of
 * orc_phase1.  removed[i] = 1 with the nonzero weights in column order
 * (at most 3, slots of 4, padded -1 / 0) where it is feasible; otherwise the
 * candidate stays.
 */
void orc_remove_weights(const double* x, const double* y, long n, const unsigned char* close, double h, double lo2,
                        double hi2, double Rh, unsigned char* removed, int* cols, double* w) {
  orc_grid g;
  grid_build(&g, x, y, n, Rh);
  double inv_h = 1.0 / h;
#pragma omp parallel for schedule(dynamic, 256)
  for (long i = 0; i < n; ++i) {
    removed[i] = 0;
    for (int t = 0; t < 4; ++t) {
      cols[(size_t)i * 4 + t] = -1;
      w[(size_t)i * 4 + t] = 0.0;
    }
    if (!close[i]) continue;
    long cx, cy;
    grid_cell(&g, x[i], y[i], &cx, &cy);
    double best_d2[8];
    long best_j[8];
    for (int s = 0; s < 8; ++s) {
      best_d2[s] = INFINITY;
      best_j[s] = -1;
    }
    for (long by = cy - 1; by <= cy + 1; ++by) {
      if (by < 0 || by >= g.ny) continue;
      for (long bx = cx - 1; bx <= cx + 1; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        long b = by * g.nx + bx;
        for (long t = g.start[b]; t < g.start[b + 1]; ++t) {
          long j = g.items[t];
          if (j == i || close[j]) continue;
          double d2;
          int s;
          if (!annulus(x, y, i, j, lo2, hi2, 0, &d2, &s)) continue;
          if (d2 < best_d2[s] || (d2 == best_d2[s] && j < best_j[s])) {
            best_d2[s] = d2;
            best_j[s] = j;
          }
        }
      }
    }
    orc_col cl[8];
    int K = 0;
    for (int s = 0; s < 8; ++s) {
      if (best_j[s] < 0) continue;
      long j = best_j[s];
      cl[K].j = j;
      cl[K].dx = x[j] - x[i];
      cl[K].dy = y[j] - y[i];
      cl[K].d2 = cl[K].dx * cl[K].dx + cl[K].dy * cl[K].dy;
      ++K;
    }
    qsort(cl, (size_t)K, sizeof(orc_col), cmp_col);
    double V[3 * 8], b3[3] = {1.0, 0.0, 0.0}, f[8];
    for (int k = 0; k < K; ++k) {
      V[0 * K + k] = 1.0;
      V[1 * K + k] = cl[k].dx * inv_h;
      V[2 * K + k] = cl[k].dy * inv_h;
    }
    int np;
    double res;
    if (orc_phase1(3, K, V, b3, f, &np, &res) != 0) continue;
    removed[i] = 1;
    int t = 0;
    for (int k = 0; k < K; ++k) {
      if (f[k] == 0.0) continue;
      if (t < 4) {
        cols[(size_t)i * 4 + t] = (int)cl[k].j;
        w[(size_t)i * 4 + t] = f[k];
      }
      ++t;
    }
  }
  grid_free(&g);
}

/*
 * One removal pass: candidates (orc_close), their identity stencils, then
 * Gamma_j + sum_i g_ij Gamma_i for every kept j, the removed i taken in
 * ascending order (products and sums rounded separately), and the kept
 * particles compacted in index order into x_out, y_out, gamma_out.
 * removed: n flags out.  Returns the number kept.
 */
long orc_remove(const double* x, const double* y, const double* gamma, long n, double h, double r, double R,
                double* x_out, double* y_out, double* gamma_out, unsigned char* removed, long* candidates) {
  double rh = r * h, Rh = R * h;
  double lo2 = rh * rh, hi2 = Rh * Rh;
  unsigned char* close = (unsigned char*)malloc((size_t)(n > 0 ? n : 1));
  int* cols = (int*)malloc(sizeof(int) * 4 * (size_t)(n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
  double* acc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  *candidates = orc_close(x, y, gamma, n, lo2, Rh, close);
  orc_remove_weights(x, y, n, close, h, lo2, hi2, Rh, removed, cols, w);
  for (long j = 0; j < n; ++j) acc[j] = gamma[j];
  for (long i = 0; i < n; ++i) {
    if (!removed[i]) continue;
    for (int t = 0; t < 4; ++t) {
      int j = cols[(size_t)i * 4 + t];
      if (j < 0) continue;
      double p = w[(size_t)i * 4 + t] * gamma[i];
      acc[j] = acc[j] + p;
    }
  }
  long k = 0;
  for (long i = 0; i < n; ++i) {
    if (removed[i]) continue;
    x_out[k] = x[i];
    y_out[k] = y[i];
    gamma_out[k] = acc[i];
    ++k;
  }
  free(close);
  free(cols);
  free(w);
  free(acc);
  return k;
}
