// Redistribution weights: phase-I simplex per diffused particle (Sec. 2 Eq.
// momcondmv, Sec. 4.1, small neighbourhoods Sec. 4.3).
//
// The LP  V f = b, f >= 0  has m = 5 rows (1,0) (0,1) (2,0) (1,1) (0,2) in
// xi = r_ij / h for n = 1, and m = 9 with (3,0) (2,1) (1,2) (0,3) added for
// n = 2 (Eqs. cond_two, cond_alpha); b = 2 on (2,0) and (0,2), 0 elsewhere.
// Phase I minimises the sum of m artificials; they start the basis and, once
// they leave, never re-enter.  Both kernels are templates on m and on the
// stencil width W (8 for n = 1, 12 for n = 2: a basic solution has at most m
// nonzero weights).
// Rules (identical to the FP64 oracle, which solves the basis systems by LU
// every iteration while this code updates a tableau):
//   entering: lowest column with reduced cost < -1e-9 (Bland);
//   leaving:  minimum ratio over pivot elements > 1e-9, basic values at or
//             below 1e-11 taken as zero; ratios within 1e-12 max(1, min)
//             tie, the tie goes to the basic variable of lowest index
//             (artificials 0..m-1 before structurals m..);
//   at most 64 pivots; feasible iff the phase-I objective <= 1e-10 and
//   max |V f - b| <= 1e-12 (the moment conditions met to 1e-12 per
//   particle); basic values <= 1e-11 are zeros.
//
// GB300 has about 1/60 of its FP32 rate in FP64, and every FP64 instruction
// of a warp costs the same whether its lanes are busy or not.  The small
// neighbourhood LP therefore runs one particle per thread with the m x 8
// tableau in registers: every FP64 lane-operation does useful work, and
// pivot row/column selections are register selects on the integer pipes.
// The rare full-neighbourhood retry runs one particle per warp, one tableau
// column per lane (K <= 32), with the pivot column broadcast by shuffles.
// For n = 1 the default kernel, k_lp_small32, pivots in binary32 with
// certified decisions and keeps FP64 for the column offsets and the final
// basis solve (see the section before it); k_lp_small re-runs the particles
// it hands back, and serves n = 2 and the FP64-pivot schedule.
#include <climits>

#include "vrm_internal.cuh"

namespace vrm {

constexpr double kTolPrice = 1e-9;
constexpr double kTolPivot = 1e-9;
constexpr double kTolTie = 1e-12;
constexpr double kTolPhase1 = 1e-10;
constexpr double kTolSnap = 1e-11;
constexpr double kTolResid = 1e-12;
constexpr int kPivotCap = 64;

// FP64 comparisons on the integer pipes: for non-NaN doubles the signed
// 64-bit pattern orders the non-negative values, so these tests spend no
// FP64 instruction (GB300's FP64 pipe is the bottleneck of this kernel).
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// x > t, for t > 0
__device__ __forceinline__ bool gt_pos(double x, double t) { return dbits(x) > dbits(t); }
// x < -t, for t > 0
__device__ __forceinline__ bool lt_neg(double x, double t) {
  const long long b = dbits(x);
  return b < 0 && (b & 0x7FFFFFFFFFFFFFFFLL) > dbits(t);
}
// a < b, for a, b in [+0, inf]
__device__ __forceinline__ bool lt_nonneg(double a, double b) {
  return (unsigned long long)dbits(a) < (unsigned long long)dbits(b);
}
// |a| > |b|
__device__ __forceinline__ bool abs_gt(double a, double b) {
  return (dbits(a) & 0x7FFFFFFFFFFFFFFFLL) > (dbits(b) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double dneg(double x) { return __longlong_as_double(dbits(x) ^ (long long)0x8000000000000000ULL); }

// Reciprocal of a > 0 (a in the binary32 normal range) for the tableau: a
// binary32 seed made from the bit pattern (rounded mantissa, integer ops),
// a binary32 reciprocal, widened by integer ops, then Newton steps
// r <- r + r (1 - a r) in FP64; one step gives about 2^-45 relative error,
// two give full FP64 accuracy.  Only the pivot decisions use these values;
// the weights come from the exact basis solve below.
template <int STEPS>
__device__ __forceinline__ double rcp_newton(double a) {
  const unsigned long long b = (unsigned long long)dbits(a);
  const unsigned long long mr = (b + 0x10000000ULL) >> 29;  // round the mantissa to 23 bits
  const int e32 = (int)((mr >> 23) & 0x7FF) - 1023 + 127;
  const float af = __int_as_float((e32 << 23) | (int)(mr & 0x7FFFFF));
  const unsigned rb = __float_as_uint(__frcp_rn(af));
  const unsigned long long db =
      ((unsigned long long)((int)((rb >> 23) & 0xFF) - 127 + 1023) << 52) | ((unsigned long long)(rb & 0x7FFFFF) << 29);
  double r = __longlong_as_double((long long)db);
#pragma unroll
  for (int k = 0; k < STEPS; ++k) r = __fma_rn(r, __fma_rn(-a, r, 1.0), r);
  return r;
}

// Binary32 value of a double in the binary32 normal range, from the bit
// pattern (mantissa rounded to 23 bits, exponent rebiased; integer ops only).
__device__ __forceinline__ float f32_of(double a) {
  const unsigned long long b = (unsigned long long)dbits(a);
  const unsigned long long mr = ((b & 0x7FFFFFFFFFFFFFFFULL) + 0x10000000ULL) >> 29;
  const int e32 = (int)((mr >> 23) & 0x7FF) - 1023 + 127;
  return __int_as_float((int)((b >> 32) & 0x80000000u) | (e32 << 23) | (int)(mr & 0x7FFFFF));
}

template <typename P>
__device__ __forceinline__ void cswap(double* d2, int* j, P* a, P* b, int p, int q) {
  const unsigned long long bq = (unsigned long long)dbits(d2[q]), bp = (unsigned long long)dbits(d2[p]);
  bool sw = (bq < bp) || (bq == bp && j[q] < j[p]);
  double t0 = sw ? d2[q] : d2[p], t1 = sw ? d2[p] : d2[q];
  d2[p] = t0;
  d2[q] = t1;
  int u0 = sw ? j[q] : j[p], u1 = sw ? j[p] : j[q];
  j[p] = u0;
  j[q] = u1;
  P v0 = sw ? a[q] : a[p], v1 = sw ? a[p] : a[q];
  a[p] = v0;
  a[q] = v1;
  P w0 = sw ? b[q] : b[p], w1 = sw ? b[p] : b[q];
  b[p] = w0;
  b[q] = w1;
}

// Batcher odd-even merge sort of 8 (d2, j) keys with two payloads.
template <typename P>
__device__ __forceinline__ void sort8(double* d2, int* j, P* a, P* b) {
  cswap(d2, j, a, b, 0, 1); cswap(d2, j, a, b, 2, 3); cswap(d2, j, a, b, 4, 5); cswap(d2, j, a, b, 6, 7);
  cswap(d2, j, a, b, 0, 2); cswap(d2, j, a, b, 1, 3); cswap(d2, j, a, b, 4, 6); cswap(d2, j, a, b, 5, 7);
  cswap(d2, j, a, b, 1, 2); cswap(d2, j, a, b, 5, 6);
  cswap(d2, j, a, b, 0, 4); cswap(d2, j, a, b, 1, 5); cswap(d2, j, a, b, 2, 6); cswap(d2, j, a, b, 3, 7);
  cswap(d2, j, a, b, 2, 4); cswap(d2, j, a, b, 3, 5);
  cswap(d2, j, a, b, 1, 2); cswap(d2, j, a, b, 3, 4); cswap(d2, j, a, b, 5, 6);
}

// Vandermonde column r^alpha of one neighbour, xi = r_ij / h (Eq. momcondmv),
// each product rounded once: the cubic rows are (xi xi) xi, (xi xi) eta,
// xi (eta eta), (eta eta) eta.
template <int M>
__device__ __forceinline__ void vcol(double xi, double eta, double* v) {
  v[0] = xi;
  v[1] = eta;
  v[2] = __dmul_rn(xi, xi);
  v[3] = __dmul_rn(xi, eta);
  v[4] = __dmul_rn(eta, eta);
  if constexpr (M == 9) {
    v[5] = __dmul_rn(v[2], xi);
    v[6] = __dmul_rn(v[2], eta);
    v[7] = __dmul_rn(xi, v[4]);
    v[8] = __dmul_rn(v[4], eta);
  }
}

__device__ __forceinline__ double b_of(int r) { return (r == 2 || r == 4) ? 2.0 : 0.0; }

// The identity's rows of the removal LP: (0,0) (1,0) (0,1), b = (1, 0, 0).
__device__ __forceinline__ void vcol_id(double xi, double eta, double* v) {
  v[0] = 1.0;
  v[1] = xi;
  v[2] = eta;
}
__device__ __forceinline__ double b_id(int r) { return r == 0 ? 1.0 : 0.0; }


// Upper bound in binary32 of |a| for a double a with |a| < 2^127, from the
// high word of its bit pattern (three integer ops: the sign cleared, the
// exponent rebiased with the 20 high mantissa bits moved into place, and one
// unit of the 20th mantissa bit added, which covers the bits dropped);
// values below the smallest normal binary32 number (zeros included) give
// about that number.
__device__ __forceinline__ float f32_up_abs(double a) {
  unsigned hi = (unsigned)__double2hiint(a) & 0x7FFFFFFFu;
  hi = hi > 0x38100000u ? hi : 0x38100000u;
  return __uint_as_float((hi << 3) + 0x40000008u);
}

// Residual certificate of a basis solve.  The computed x of the LU solve
// below satisfies (B + dB) x = b with |dB| <= 2 gamma_3m |L||U| (Higham,
// Accuracy and Stability of Numerical Algorithms, Thm. 9.4; the factor 2
// covers the multipliers and quotients taken through reciprocals, two
// roundings each), so |B x - b| <= 2 gamma_3m s with s = max_r (|L||U||x|)_r.
// Any FP64 evaluation of the residual sum over at most 8 columns (the
// oracle's) adds at most gamma_8 (|B||x|)_r <= gamma_8 s (1 + 2 gamma_3m) and
// one rounding.  s <= cert_s<M>() keeps the sum of these under 1e-12 / 1.2.
// Partial pivoting gives |L| <= 1 + 4u, so s <= (1 + 4u) sum_c (|U||x|)_c,
// the quantity basis_solve evaluates (the factor 1.2 covers 1 + 4u and the
// binary32 rounding of the evaluation).
__host__ __device__ constexpr double gamma_n(int n) { return n * 0x1p-53 / (1.0 - n * 0x1p-53); }
template <int M>
__host__ __device__ constexpr float cert_s() {
  return (float)(1e-12 / (1.2 * (2.0 * gamma_n(3 * M) + gamma_n(8) * (1.0 + 2.0 * gamma_n(3 * M)))));
}

// Basic solution of the final basis, by the same LU sequence as the oracle's
// basis solves (partial pivoting on the first largest |pivot|, full row
// swaps, multipliers A[r][k] * (1/A[k][k]), products and differences rounded
// separately), so that equal bases give bit-identical weights.  Column k of
// B is the unit vector e_v for an artificial v = basis[k] < m, else the
// Vandermonde column of (bxi[k], beta[k]).  Returns false if B is singular.
// With cert non-null, *cert = sum over the rows of |U||z| in binary32 from
// upper bounds of |U| and |z| (an upper bound of max_r (|L||U||z|)_r up to
// the factor 1 + 4u and binary32 rounding); +inf if some |z| >= 256, where
// the bounds of the conversion no longer hold and no stencil is that large.
template <int M, bool ID = false>
__device__ __forceinline__ bool basis_solve(const int* basis, const double* bxi, const double* beta, double* z,
                                            float* cert = nullptr) {
  double A[M][M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    double v[M];
    if constexpr (ID)
      vcol_id(bxi[k], beta[k], v);
    else
      vcol<M>(bxi[k], beta[k], v);
#pragma unroll
    for (int r = 0; r < M; ++r) A[r][k] = basis[k] < M ? (basis[k] == r ? 1.0 : 0.0) : v[r];
  }
  int piv[M];
  double rcp[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    int p = k;
    double best = A[k][k];
#pragma unroll
    for (int r = k + 1; r < M; ++r)
      if (abs_gt(A[r][k], best)) {
        best = A[r][k];
        p = r;
      }
    piv[k] = p;
    if ((dbits(best) & 0x7FFFFFFFFFFFFFFFLL) == 0) return false;
#pragma unroll
    for (int r = k + 1; r < M; ++r)
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const double a = A[k][c], b = A[r][c];
        A[k][c] = (p == r) ? b : a;
        A[r][c] = (p == r) ? a : b;
      }
    rcp[k] = __drcp_rn(A[k][k]);
#pragma unroll
    for (int r = k + 1; r < M; ++r) {
      const double l = __dmul_rn(A[r][k], rcp[k]);
      A[r][k] = l;
#pragma unroll
      for (int c = k + 1; c < M; ++c) A[r][c] = __dsub_rn(A[r][c], __dmul_rn(l, A[k][c]));
    }
  }
#pragma unroll
  for (int r = 0; r < M; ++r) z[r] = ID ? b_id(r) : b_of(r);
#pragma unroll
  for (int k = 0; k < M; ++k)
#pragma unroll
    for (int r = k + 1; r < M; ++r) {
      const double a = z[k], b = z[r];
      z[k] = (piv[k] == r) ? b : a;
      z[r] = (piv[k] == r) ? a : b;
    }
#pragma unroll
  for (int r = 1; r < M; ++r)
#pragma unroll
    for (int c = 0; c < r; ++c) z[r] = __dsub_rn(z[r], __dmul_rn(A[r][c], z[c]));
#pragma unroll
  for (int r = M - 1; r >= 0; --r) {
#pragma unroll
    for (int c = r + 1; c < M; ++c) z[r] = __dsub_rn(z[r], __dmul_rn(A[r][c], z[c]));
    z[r] = __dmul_rn(z[r], rcp[r]);
  }
  if (cert) {
    // sum_r (|U||z|)_r = sum_c |z_c| (sum_{r <= c} |U_rc|)
    unsigned zhi = 0;
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const unsigned h = (unsigned)__double2hiint(z[c]) & 0x7FFFFFFFu;
      zhi = h > zhi ? h : zhi;
      float col = 0.0f;
#pragma unroll
      for (int r = 0; r <= c; ++r) col += f32_up_abs(A[r][c]);
      acc = __fmaf_rn(col, f32_up_abs(z[c]), acc);
    }
    *cert = zhi < 0x40700000u ? acc : INFINITY;
  }
  return true;
}

// Sorts M (key, payload) entries by ascending key: odd-even transposition
// (M rounds of neighbour compare-exchanges), selects only.
template <int M, int NP>
__device__ __forceinline__ void sort_by_key(int (&key)[M], double (&pay)[NP][M]) {
#pragma unroll
  for (int t = 0; t < M; ++t)
#pragma unroll
    for (int a = t & 1; a + 1 < M; a += 2) {
      const bool sw = key[a + 1] < key[a];
      const int k0 = sw ? key[a + 1] : key[a], k1 = sw ? key[a] : key[a + 1];
      key[a] = k0;
      key[a + 1] = k1;
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const double p0 = sw ? pay[q][a + 1] : pay[q][a], p1 = sw ? pay[q][a] : pay[q][a + 1];
        pay[q][a] = p0;
        pay[q][a + 1] = p1;
      }
    }
}

// max_r |sum_j V_rj f_j - b_r| evaluated as the oracle evaluates it: the
// terms in ascending column order, each product and sum rounded separately,
// then the difference with b_r.  Columns outside the basis carry f = 0 and
// leave the sum unchanged, so only the basic columns are summed: entry r is
// basis variable basis[r] (structural column basis[r] - M, offsets bxi[r],
// beta[r], snapped value v[r]; artificials carry v = 0).
template <int M, bool ID = false>
__device__ __forceinline__ double resid_in_column_order(const int (&basis)[M], const double (&bxi)[M],
                                                        const double (&beta)[M], const double (&v)[M]) {
  int key[M];
  double pay[3][M];
#pragma unroll
  for (int r = 0; r < M; ++r) {
    key[r] = basis[r];
    pay[0][r] = bxi[r];
    pay[1][r] = beta[r];
    pay[2][r] = v[r];
  }
  sort_by_key<M, 3>(key, pay);
  double acc[M];
#pragma unroll
  for (int q = 0; q < M; ++q) acc[q] = 0.0;
#pragma unroll
  for (int r = 0; r < M; ++r) {
    double col[M];
    if constexpr (ID)
      vcol_id(pay[0][r], pay[1][r], col);
    else
      vcol<M>(pay[0][r], pay[1][r], col);
#pragma unroll
    for (int q = 0; q < M; ++q) acc[q] = __dadd_rn(acc[q], __dmul_rn(col[q], pay[2][r]));
  }
  double rmax = 0.0;
#pragma unroll
  for (int q = 0; q < M; ++q) {
    const double e = __dsub_rn(acc[q], ID ? b_id(q) : b_of(q));
    rmax = abs_gt(e, rmax) ? fabs(e) : rmax;
  }
  return rmax;
}

struct WarpStats {
  int ok, none, maxpiv;
  double maxratio;
};

__device__ __forceinline__ void flush_stats(DevStats* ds, int ok, int none, int maxpiv, double maxratio, bool full,
                                            int solved, int pivots) {
  solved = __reduce_add_sync(0xffffffffu, solved);
  pivots = __reduce_add_sync(0xffffffffu, pivots);
  ok = __reduce_add_sync(0xffffffffu, ok);
  none = __reduce_add_sync(0xffffffffu, none);
  maxpiv = __reduce_max_sync(0xffffffffu, maxpiv);
  unsigned long long rb = (unsigned long long)__double_as_longlong(maxratio);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, rb, o);
    rb = t > rb ? t : rb;
  }
  if ((threadIdx.x & 31) == 0) {
    if (ok) atomicAdd(full ? &ds->full_ok : &ds->small_ok, ok);
    if (none) atomicAdd(&ds->no_stencil, none);
    if (maxpiv) atomicMax(&ds->max_pivots, maxpiv);
    if (rb) atomicMax(&ds->max_dt_ratio_bits, rb);
    if (solved) atomicAdd(full ? &ds->lp_full_solved : &ds->lp_small_solved, solved);
    if (pivots) atomicAdd(full ? &ds->lp_full_pivots : &ds->lp_small_pivots, (unsigned long long)pivots);
  }
}

// Columns of one small-neighbourhood LP: the occupied slots of particle i's
// small neighbourhood ordered by (d2, index) (Sec. 4.3), offsets in units of
// h; empty slots get index INT_MAX and zero offsets (a zero column).
__device__ __forceinline__ void lp_columns(const Consts& c, const double* __restrict__ x,
                                           const double* __restrict__ y, const int* __restrict__ small, int i,
                                           int (&cj)[8], double (&cxi)[8], double (&ceta)[8]) {
  const double xi0 = x[i], yi0 = y[i];
  const int4 s0 = reinterpret_cast<const int4*>(small + (size_t)i * 8)[0];
  const int4 s1 = reinterpret_cast<const int4*>(small + (size_t)i * 8)[1];
  cj[0] = s0.x; cj[1] = s0.y; cj[2] = s0.z; cj[3] = s0.w;
  cj[4] = s1.x; cj[5] = s1.y; cj[6] = s1.z; cj[7] = s1.w;
  double cd2[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (cj[k] >= 0) {
      const double dx = __dsub_rn(x[cj[k]], xi0), dy = __dsub_rn(y[cj[k]], yi0);
      cd2[k] = dist2(dx, dy);
      cxi[k] = dx;
      ceta[k] = dy;
    } else {
      cd2[k] = 1e300;
      cj[k] = INT_MAX;
      cxi[k] = 0.0;
      ceta[k] = 0.0;
    }
  }
  sort8(cd2, cj, cxi, ceta);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    cxi[k] = __dmul_rn(cxi[k], c.inv_h);
    ceta[k] = __dmul_rn(ceta[k], c.inv_h);
  }
}

struct LpTally {
  int ok = 0, none = 0, maxpiv = 0, solved = 0, pivots = 0;
  double ratio = 0.0;
};

// Basic solution of the final basis (fresh LU solve, bit-identical to the
// oracle's), snapped; feasibility from the phase-I objective and the
// residual over the basic columns; the stencil (or the fallback queue, or a
// zero stencil) written out.
// Offsets of the basic columns (zero for artificials) selected from the
// columns' offsets.
template <int M>
__device__ __forceinline__ void basic_offsets(const int (&basis)[M], const double (&cxi)[8],
                                              const double (&ceta)[8], double (&bxi)[M], double (&beta)[M]) {
#pragma unroll
  for (int r = 0; r < M; ++r) {
    double a = 0.0, e = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a = (basis[r] == M + k) ? cxi[k] : a;
      e = (basis[r] == M + k) ? ceta[k] : e;
    }
    bxi[r] = a;
    beta[r] = e;
  }
}

template <int M, int W>
__device__ __forceinline__ void lp_finish(const Consts& c, int i, int code, const int (&basis)[M], int it,
                                          const int (&cj)[8], const double (&bxi)[M], const double (&beta)[M],
                                          int* __restrict__ cols, double* __restrict__ f, double* __restrict__ fii,
                                          uint8_t* __restrict__ status, int* __restrict__ fail_list,
                                          DevStats* __restrict__ ds, double nu_dt, double inv_h2, LpTally& tl) {
  double fv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) fv[k] = 0.0;
  double wsum = 0.0, rmax = 0.0;
  if (code == 0) {
    double xB[M];
    float cert = INFINITY;
    if (!basis_solve<M>(basis, bxi, beta, xB, &cert)) code = 2;
    // Residual certificate: when every basic variable is structural (the
    // phase-I sum is then exactly 0) and none is snapped, the residual
    // V f - b is that of the basis solve, and cert <= cert_s<M>() proves it
    // (and the oracle's FP64 evaluation of it) below 1e-12 without
    // computing it.  Otherwise the residual is evaluated as the oracle does.
    bool all_struct = true, snapped = false;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      all_struct = all_struct && basis[r] >= M;
      snapped = snapped || !gt_pos(xB[r], kTolSnap);
    }
    const bool certified = all_struct && !snapped && cert <= cert_s<M>();
    double v[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
      v[r] = (basis[r] >= M && gt_pos(xB[r], kTolSnap)) ? xB[r] : 0.0;
      if (basis[r] < M) wsum = __dadd_rn(wsum, xB[r]);
#pragma unroll
      for (int k = 0; k < 8; ++k) fv[k] = (basis[r] == M + k) ? v[r] : fv[k];
    }
    if (code == 0 && !certified) rmax = resid_in_column_order<M>(basis, bxi, beta, v);
  }
  const bool feasible = code == 0 && !gt_pos(wsum, kTolPhase1) && !gt_pos(rmax, kTolResid);
  tl.maxpiv = it > tl.maxpiv ? it : tl.maxpiv;
  ++tl.solved;
  tl.pivots += it;
  int* crow = cols + (size_t)i * W;
  double* frow = f + (size_t)i * W;
  if (feasible) {
    int slot = 0;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (dbits(fv[k]) != 0) {
        crow[slot] = cj[k];
        frow[slot] = fv[k];
        ++slot;
        s = __dadd_rn(s, fv[k]);
      }
    for (int k = slot; k < W; ++k) {
      crow[k] = -1;
      frow[k] = 0.0;
    }
    fii[i] = -s;
    status[i] = VRM_LP_SMALL;
    ++tl.ok;
    const double q = __dmul_rn(__dmul_rn(nu_dt, s), inv_h2);
    tl.ratio = q > tl.ratio ? q : tl.ratio;
  } else if (c.fallback) {
    fail_list[atomicAdd(&ds->n_fail, 1)] = i;
  } else {
    for (int k = 0; k < W; ++k) {
      crow[k] = -1;
      frow[k] = 0.0;
    }
    fii[i] = 0.0;
    status[i] = VRM_LP_NONE;
    ++tl.none;
  }
}

// Leaving row of an FP64 pivot whose entering column is a (the ratio test;
// one function for the FP64 kernels, so that they decide alike): basic
// values <= kTolSnap are zeros.  The ratios are screened in binary32
// (operands rounded from their bit patterns: relative error < 1e-6, no FP64
// instruction); the rows within 1e-5 of the smallest binary32 ratio are the
// only ones that can lie in the FP64 tie window (1e-12), so the leaving row
// is decided without FP64 unless two of them differ and are not exact zeros,
// and then in FP64 (Newton reciprocal, relative error ~2^-45) on those rows.
// Returns false when no row is eligible; else the leaving row and its basic
// variable.
template <int M>
__device__ __forceinline__ bool lp_leave(const double (&a)[M], const double (&rhs)[M], const int (&basis)[M],
                                         int& leave, int& lbas) {
  bool elig[M], any = false;
  float r32[M], m32 = 3.0e38f;
#pragma unroll
  for (int r = 0; r < M; ++r) {
    elig[r] = gt_pos(a[r], kTolPivot);
    const bool nz = gt_pos(rhs[r], kTolSnap);
    r32[r] = !elig[r] ? 3.0e38f : nz ? __fmul_rn(f32_of(rhs[r]), __frcp_rn(f32_of(a[r]))) : 0.0f;
    any = any || elig[r];
    m32 = fminf(m32, r32[r]);
  }
  leave = -1;
  lbas = INT_MAX;
  if (!any) return false;
  const float marg = __fmaf_rn(1e-5f, fmaxf(m32, 1.0f), m32);
  unsigned cont = 0;
  bool allzero = true;
#pragma unroll
  for (int r = 0; r < M; ++r)
    if (elig[r] && r32[r] <= marg) {
      cont |= 1u << r;
      allzero = allzero && r32[r] == 0.0f;
    }
  if (__popc(cont) > 1 && !allzero) {
    double ratio[M], theta = 1e308;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      const double num = gt_pos(rhs[r], kTolSnap) ? rhs[r] : 0.0;
      ratio[r] = ((cont >> r) & 1u) ? __dmul_rn(num, rcp_newton<1>(a[r])) : 1e308;
      theta = lt_nonneg(ratio[r], theta) ? ratio[r] : theta;
    }
    const double lim = __fma_rn(kTolTie, gt_pos(theta, 1.0) ? theta : 1.0, theta);
#pragma unroll
    for (int r = 0; r < M; ++r)
      if (((cont >> r) & 1u) && lt_nonneg(lim, ratio[r])) cont &= ~(1u << r);
  }
  // the tied rows: the one with the lowest basic variable leaves
#pragma unroll
  for (int r = 0; r < M; ++r)
    if (((cont >> r) & 1u) && basis[r] < lbas) {
      leave = r;
      lbas = basis[r];
    }
  return true;
}

template <int M, int W>
__global__ void __launch_bounds__(128) k_lp_small(Consts c, const double* __restrict__ x,
                                                  const double* __restrict__ y, const int* __restrict__ list,
                                                  const int* __restrict__ list_count, const int* __restrict__ small,
                                                  int* __restrict__ cols, double* __restrict__ f,
                                                  double* __restrict__ fii, uint8_t* __restrict__ status,
                                                  int* __restrict__ fail_list, DevStats* __restrict__ ds,
                                                  double nu_dt, const double* __restrict__ dt_dev, double nu) {
  if (dt_dev) nu_dt = nu * *dt_dev;
  const int m = *list_count;
  const double inv_h2 = 1.0 / (c.h * c.h);
  LpTally tl;
  // grid-stride over whole warps so that the warp-level statistics below run converged
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x; base < m; base += stride) {
    const long t = base + threadIdx.x;
    if (t < m) {
      const int i = list[t];
      int cj[8];
      double cxi[8], ceta[8];
      lp_columns(c, x, y, small, i, cj, cxi, ceta);
      // tableau: T[r][k] = (B^-1 V)_rk, rhs = B^-1 b, d = phase-I reduced costs
      double T[M][8], rhs[M], d[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        double v[M];
        vcol<M>(cxi[k], ceta[k], v);
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < M; ++r) {
          T[r][k] = v[r];
          s = __dadd_rn(s, v[r]);
        }
        d[k] = dneg(s);
      }
#pragma unroll
      for (int r = 0; r < M; ++r) rhs[r] = b_of(r);
      int basis[M];
#pragma unroll
    for (int r = 0; r < M; ++r) basis[r] = r;
      unsigned basic = 0;
      int it = 0, code = 0;
      int n_art = M;  // artificials in the basis
      for (;;) {
        // with no artificial left the phase-I costs of the basis are zero, so
        // every reduced cost is exactly zero: phase I is over (the updated
        // cost row only holds rounding noise then)
        if (n_art == 0) break;
        int q = -1;
#pragma unroll
        for (int k = 7; k >= 0; --k)
          if (!((basic >> k) & 1u) && lt_neg(d[k], kTolPrice)) q = k;
        if (q < 0) break;
        if (it == kPivotCap) {
          code = 2;
          break;
        }
        double a[M];
#pragma unroll
        for (int r = 0; r < M; ++r) {
          double v = T[r][0];
#pragma unroll
          for (int k = 1; k < 8; ++k) v = (q == k) ? T[r][k] : v;
          a[r] = v;
        }
        int leave, lbas;
        if (!lp_leave<M>(a, rhs, basis, leave, lbas)) {
          code = 2;
          break;
        }
        double piv = a[0], prhs_raw = rhs[0];
#pragma unroll
        for (int r = 1; r < M; ++r) {
          piv = (leave == r) ? a[r] : piv;
          prhs_raw = (leave == r) ? rhs[r] : prhs_raw;
        }
        const double rcp = rcp_newton<2>(piv);
        double prow[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          double v = T[0][k];
#pragma unroll
          for (int r = 1; r < M; ++r) v = (leave == r) ? T[r][k] : v;
          prow[k] = (k == q) ? 1.0 : __dmul_rn(v, rcp);
        }
        const double prhs = __dmul_rn(prhs_raw, rcp);
        // row r <- row r - a_r prow; the leaving row becomes prow itself
        // (zeroed, multiplier -1), and column q becomes exactly e_leave
        // because prow[q] = 1 and T[r][q] = a_r
#pragma unroll
        for (int r = 0; r < M; ++r) {
          const bool lr = (leave == r);
          const double ar = lr ? -1.0 : a[r];
#pragma unroll
          for (int k = 0; k < 8; ++k) T[r][k] = __fma_rn(-ar, prow[k], lr ? 0.0 : T[r][k]);
          rhs[r] = __fma_rn(-ar, prhs, lr ? 0.0 : rhs[r]);
        }
        double dq = d[0];
#pragma unroll
        for (int k = 1; k < 8; ++k) dq = (q == k) ? d[k] : dq;
#pragma unroll
        for (int k = 0; k < 8; ++k) d[k] = __fma_rn(-dq, prow[k], d[k]);
        if (lbas >= M) basic &= ~(1u << (lbas - M));
        else --n_art;
        basic |= 1u << q;
#pragma unroll
        for (int r = 0; r < M; ++r) basis[r] = (leave == r) ? M + q : basis[r];
        ++it;
      }
      double bxi[M], beta[M];
      basic_offsets<M>(basis, cxi, ceta, bxi, beta);
      lp_finish<M, W>(c, i, code, basis, it, cj, bxi, beta, cols, f, fii, status, fail_list, ds, nu_dt, inv_h2, tl);
    }
  }
  flush_stats(ds, tl.ok, tl.none, tl.maxpiv, tl.ratio, false, tl.solved, tl.pivots);
}

// ---------------------------------------------------------------------------
// Certified binary32 pivoting.  Every pivot decision of the phase-I simplex
// (entering column, eligible pivot rows, zero basic values, the minimum
// ratio and its ties) is a comparison of a tableau quantity with a
// threshold.  k_lp_small32 runs the tableau in binary32 and carries, for
// every entry, a rigorous bound on its distance from the exact rational
// tableau of the same pivot sequence started from the FP64 Vandermonde
// matrix (running error analysis: each update adds the propagated operand
// bounds and the rounding of its own result, u = 2^-24).  A decision whose
// binary32 value lies farther from the threshold than its bound is the
// decision of exact arithmetic, and therefore the decision of the FP64
// tableau, whose own distance from exact is smaller by 2^-29 (the safety
// factor 1.25 covers it and the rounding of the bound arithmetic).  So a
// run whose decisions are all certified ends on the FP64 run's basis with
// its pivot count, and the weights come from the same FP64 LU solve of that
// basis (lp_finish): bit-identical output.  A particle with one uncertain
// decision (near-degenerate ratios, entries near the tolerances, growth of
// the bounds under small pivots) goes to a retry list that k_lp_small
// solves in FP64.  This moves the m x 8 tableau updates (about 60% of the
// FP64 instructions of an LP) to the binary32 pipes, which GB300 runs at
// about 64 times the FP64 rate.
// ---------------------------------------------------------------------------
constexpr float kU32 = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of binary32
constexpr float kCertSafety = 1.25f;
// a product by an approximate reciprocal (at most 1 ulp = 2u) and its rounding
constexpr float kRcpMul = 3.01f * kU32;
// FP64 tolerances bracketed by binary32 values (below, above)
constexpr float kTolPriceLo = 0.99999994e-9f, kTolPriceHi = 1.0000001e-9f;
constexpr float kTolPivotLo = 0.99999994e-9f, kTolPivotHi = 1.0000001e-9f;
constexpr float kTolSnapLo = 0.99999994e-11f, kTolSnapHi = 1.0000001e-11f;
constexpr float kTolTieLo = 0.9999999e-12f, kTolTieHi = 1.0000001e-12f;

// Approximate binary32 reciprocal (PTX rcp.approx: at most 1 ulp from 1/a
// for normal a); the error bounds below account for it.
__device__ __forceinline__ float rcp_approx(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// Binary32 value of an FP64 offset (f32_of), zero kept; magnitudes outside
// [2^-100, 2^100] set `bad` (the bounds assume normal binary32 operands).
__device__ __forceinline__ float f32_checked(double a, bool& bad) {
  const long long b = dbits(a) & 0x7FFFFFFFFFFFFFFFLL;
  if (b == 0) return 0.0f;
  const int e = (int)(b >> 52) - 1023;
  bad = bad || e < -100 || e > 100;
  return f32_of(a);
}

// Columns of one LP as in lp_columns, carrying binary32 offsets
// xi32 = f32(dx) * f32(1/h) (within 3.01 u of the FP64 offset) instead of
// the FP64 ones.
__device__ __forceinline__ void lp_columns32(const double* __restrict__ x, const double* __restrict__ y,
                                             const int* __restrict__ small, int i, double xi0, double yi0,
                                             float inv_h32, int (&cj)[8], float (&xs)[8], float (&es)[8],
                                             bool& bad) {
  const int4 s0 = reinterpret_cast<const int4*>(small + (size_t)i * 8)[0];
  const int4 s1 = reinterpret_cast<const int4*>(small + (size_t)i * 8)[1];
  cj[0] = s0.x; cj[1] = s0.y; cj[2] = s0.z; cj[3] = s0.w;
  cj[4] = s1.x; cj[5] = s1.y; cj[6] = s1.z; cj[7] = s1.w;
  double cd2[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (cj[k] >= 0) {
      const double dx = __dsub_rn(x[cj[k]], xi0), dy = __dsub_rn(y[cj[k]], yi0);
      cd2[k] = dist2(dx, dy);
      xs[k] = __fmul_rn(f32_checked(dx, bad), inv_h32);
      es[k] = __fmul_rn(f32_checked(dy, bad), inv_h32);
    } else {
      cd2[k] = 1e300;
      cj[k] = INT_MAX;
      xs[k] = 0.0f;
      es[k] = 0.0f;
    }
  }
  sort8(cd2, cj, xs, es);
}

// The certified binary32 phase-I pivots of one LP whose columns have the
// binary32 offsets xs, es: the final basis, the pivot count and the code
// (2: pivot cap or no eligible row), or `unc` when a decision could not be
// certified (the LP then goes to the FP64 re-run).
template <int M>
__device__ __forceinline__ void lp_pivots32(const float (&xs)[8], const float (&es)[8], int (&basis)[M], int& it,
                                            int& code, bool& unc) {
  // T, rhs: tableau; E, Eb: bounds on their distance from exact; d, Ed:
  // phase-I reduced costs and bounds
  float T[M][8], E[M][8], d[8], Ed[8], rhs[M], Eb[M];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float v[M] = {xs[k], es[k], __fmul_rn(xs[k], xs[k]), __fmul_rn(xs[k], es[k]), __fmul_rn(es[k], es[k])};
    float sum = 0.0f, sa = 0.0f, se = 0.0f;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      T[r][k] = v[r];
      // offsets within 3.01 u of the FP64 ones; their products within 7.01 u
      E[r][k] = (r < 2 ? 3.01f : 7.01f) * kU32 * fabsf(v[r]);
      sum = __fadd_rn(sum, v[r]);
      sa += fabsf(v[r]);
      se += E[r][k];
    }
    d[k] = -sum;
    Ed[k] = __fmaf_rn(4.01f * kU32, sa, se);
  }
#pragma unroll
  for (int r = 0; r < M; ++r) {
    rhs[r] = (r == 2 || r == 4) ? 2.0f : 0.0f;
    Eb[r] = 0.0f;
  }
  unsigned basic = 0;
  int n_art = M;
  for (;;) {
    if (unc || n_art == 0) break;
    // entering column: the lowest k certainly below -tol; a lower column
    // that is not certainly above it makes the choice uncertain
    unsigned yes = 0, un = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float mg = kCertSafety * Ed[k];
      const bool nb = !((basic >> k) & 1u);
      yes |= (nb && d[k] < -kTolPriceHi - mg) ? 1u << k : 0u;
      un |= (nb && !(d[k] < -kTolPriceHi - mg) && !(d[k] > -kTolPriceLo + mg)) ? 1u << k : 0u;
    }
    if (yes == 0) {
      unc = un != 0;
      break;
    }
    const int q = __ffs(yes) - 1;
    unc = (un & ((1u << q) - 1u)) != 0;
    if (it == kPivotCap) {
      code = 2;
      break;
    }
    float a[M], ea[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
      float v = T[r][0], e = E[r][0];
#pragma unroll
      for (int k = 1; k < 8; ++k) {
        v = (q == k) ? T[r][k] : v;
        e = (q == k) ? E[r][k] : e;
      }
      a[r] = v;
      ea[r] = e;
    }
    // eligible rows, zero basic values, ratios with bounds.  A row whose
    // eligibility is uncertain (pivot element within its bound of the
    // tolerance, mostly exact zeros) but whose basic value is certainly
    // positive would, if eligible, have a ratio of at least
    // (rhs - Eb) / (a + Ea): when that is above every possible tie limit,
    // the row can neither be the minimum nor tie with it, and the leaving
    // row is the same either way
    unsigned elig = 0, amb = 0;
    float lo[M], hi[M], thlo = 3.0e38f, thhi = 3.0e38f;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      const float mg = kCertSafety * ea[r];
      const bool el = a[r] > kTolPivotHi + mg;
      const bool am = !el && !(a[r] < kTolPivotLo - mg);
      const float mb = kCertSafety * Eb[r];
      const bool nzr = rhs[r] > kTolSnapHi + mb;
      unc = unc || (am && !nzr);
      unc = unc || (el && !nzr && !(rhs[r] < kTolSnapLo - mb));
      amb |= am ? 1u << r : 0u;
      const float inv = rcp_approx(a[r]);
      const float ratio = nzr ? rhs[r] * inv : 0.0f;
      // relative bound of the pivot element; for g <= 1/2,
      // |1/a - 1/a*| <= (g / a) / (1 - g) <= (g / a) (1 + 2 g)
      const float g = ea[r] * inv;
      const float gg = __fmaf_rn(2.0f * g, g, g);
      const float er = nzr ? kCertSafety * __fmaf_rn(kRcpMul, ratio, __fmaf_rn(gg, rhs[r] + Eb[r], Eb[r]) * inv)
                           : 0.0f;
      unc = unc || (el && nzr && (!(g <= 0.5f) || !(er < 1.0e30f)));
      elig |= el ? 1u << r : 0u;
      lo[r] = el ? fmaxf(ratio - er, 0.0f) : 3.0e38f;  // exact ratios of eligible rows are >= 0
      hi[r] = el ? ratio + er : 3.0e38f;
      thlo = fminf(thlo, lo[r]);
      thhi = fminf(thhi, hi[r]);
    }
    if (elig == 0) {
      // an uncertain row decides between no eligible row and a pivot
      unc = unc || amb != 0;
      code = 2;
      break;
    }
    // a row can tie with the minimum only if its interval reaches the
    // largest possible tie limit theta + 1e-12 max(theta, 1)
    const float l0 = __fmaf_rn(kTolTieLo, fmaxf(thlo, 1.0f), thlo);
    const float l1 = __fmaf_rn(kTolTieHi, fmaxf(thhi, 1.0f), thhi);
    const float limlo = __fmaf_rn(-4.0f * kU32, fabsf(l0), l0);
    const float limhi = __fmaf_rn(4.0f * kU32, fabsf(l1), l1);
    unsigned poss = 0, tied = 0;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      poss |= (((elig >> r) & 1u) && lo[r] <= limhi) ? 1u << r : 0u;
      tied |= (hi[r] <= limlo) ? 1u << r : 0u;
    }
    if (amb != 0) {
      // (rhs - mb) / (a + mg) > limhi without a division: a + mg is at least
      // the pivot tolerance for these rows, and the factor covers the
      // roundings of the difference, the sum and the product (< 4 u)
#pragma unroll
      for (int r = 0; r < M; ++r) {
        const float num = __fsub_rn(rhs[r], kCertSafety * Eb[r]);
        const float lim = __fmul_rn(limhi, __fadd_rn(a[r], kCertSafety * ea[r]));
        unc = unc || (((amb >> r) & 1u) && !(__fmul_rn(num, 1.0f - 8.0f * kU32) > lim));
      }
    }
    if (__popc(poss) == 1)
      tied = poss;
    else
      unc = unc || (poss & ~tied) != 0;
    tied &= poss;
    int leave = 0, lbas = INT_MAX;
#pragma unroll
    for (int r = 0; r < M; ++r)
      if (((tied >> r) & 1u) && basis[r] < lbas) {
        leave = r;
        lbas = basis[r];
      }
    float piv = a[0], pe = ea[0], prhs_raw = rhs[0], pebr = Eb[0];
#pragma unroll
    for (int r = 1; r < M; ++r) {
      piv = (leave == r) ? a[r] : piv;
      pe = (leave == r) ? ea[r] : pe;
      prhs_raw = (leave == r) ? rhs[r] : prhs_raw;
      pebr = (leave == r) ? Eb[r] : pebr;
    }
    const float P = rcp_approx(piv);
    const float rho = pe * P;  // relative bound of the pivot; the bounds below take rho <= 1/2
    unc = unc || !(rho <= 0.5f);
    const float rr = __fmaf_rn(2.0f * rho, rho, rho);  // rho / (1 - rho) <= rho (1 + 2 rho)
    if (unc) break;
    // pivot on (leave, q)
    float prow[8], Ep[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float v = T[0][k], e = E[0][k];
#pragma unroll
      for (int r = 1; r < M; ++r) {
        v = (leave == r) ? T[r][k] : v;
        e = (leave == r) ? E[r][k] : e;
      }
      const float pr = v * P, eP = e * P;
      prow[k] = (k == q) ? 1.0f : pr;
      Ep[k] = (k == q) ? 0.0f : __fmaf_rn(kRcpMul, fabsf(pr), __fmaf_rn(rr, fabsf(pr) + eP, eP));
    }
    const float prhs = prhs_raw * P, ebP = pebr * P;
    const float Ebp = __fmaf_rn(kRcpMul, fabsf(prhs), __fmaf_rn(rr, fabsf(prhs) + ebP, ebP));
#pragma unroll
    for (int r = 0; r < M; ++r) {
      const bool lr = (leave == r);
      const float ar = lr ? -1.0f : a[r];
      const float ear = lr ? 0.0f : ea[r];
      const float aar = fabsf(ar) + ear;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        // column q of the other rows becomes an exact 0 (its bound stays, conservatively)
        const float tn = __fmaf_rn(-ar, prow[k], lr ? 0.0f : T[r][k]);
        const float en = __fmaf_rn(kU32, fabsf(tn), __fmaf_rn(aar, Ep[k], __fmaf_rn(ear, fabsf(prow[k]), E[r][k])));
        T[r][k] = tn;
        E[r][k] = lr ? Ep[k] : en;
      }
      const float rn = __fmaf_rn(-ar, prhs, lr ? 0.0f : rhs[r]);
      const float ebn = __fmaf_rn(kU32, fabsf(rn), __fmaf_rn(aar, Ebp, __fmaf_rn(ear, fabsf(prhs), Eb[r])));
      rhs[r] = rn;
      Eb[r] = lr ? Ebp : ebn;
    }
    float dq = d[0], edq = Ed[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      dq = (q == k) ? d[k] : dq;
      edq = (q == k) ? Ed[k] : edq;
    }
    const float adq = fabsf(dq) + edq;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      d[k] = __fmaf_rn(-dq, prow[k], d[k]);
      Ed[k] = __fmaf_rn(kU32, fabsf(d[k]), __fmaf_rn(adq, Ep[k], __fmaf_rn(edq, fabsf(prow[k]), Ed[k])));
    }
    if (lbas >= M)
      basic &= ~(1u << (lbas - M));
    else
      --n_art;
    basic |= 1u << q;
#pragma unroll
    for (int r = 0; r < M; ++r) basis[r] = (leave == r) ? M + q : basis[r];
    ++it;
  }
}

template <int M, int W>
__global__ void __launch_bounds__(128, 3) k_lp_small32(Consts c, const double* __restrict__ x,
                                                    const double* __restrict__ y, const int* __restrict__ list,
                                                    const int* __restrict__ list_count, const int* __restrict__ small,
                                                    int* __restrict__ cols, double* __restrict__ f,
                                                    double* __restrict__ fii, uint8_t* __restrict__ status,
                                                    int* __restrict__ fail_list, int* __restrict__ retry_list,
                                                    DevStats* __restrict__ ds, double nu_dt,
                                                    const double* __restrict__ dt_dev, double nu) {
  static_assert(M == 5, "certified binary32 pivoting is written for the n = 1 rows");
  if (dt_dev) nu_dt = nu * *dt_dev;
  const int m = *list_count;
  const double inv_h2 = 1.0 / (c.h * c.h);
  const float inv_h32 = f32_of(c.inv_h);
  LpTally tl;
  int n_retry = 0;
  const unsigned lane = threadIdx.x & 31;
  // the sorted column indices wait in shared memory while the tableau holds the registers
  __shared__ int s_cj[8][128];
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x; base < m; base += stride) {
    const long t = base + threadIdx.x;
    const bool active = t < m;
    int i = 0, it = 0, code = 0;
    int basis[M];
    bool unc = false;
#pragma unroll
    for (int r = 0; r < M; ++r) basis[r] = r;
    if (active) {
      i = list[t];
      float xs[8], es[8];
      {
        int cj[8];
        lp_columns32(x, y, small, i, x[i], y[i], inv_h32, cj, xs, es, unc);
#pragma unroll
        for (int k = 0; k < 8; ++k) s_cj[k][threadIdx.x] = cj[k];
      }
      lp_pivots32<M>(xs, es, basis, it, code, unc);
    }
    // the lanes leave the pivot loop at different counts: join them so that
    // the FP64 solve below runs once per warp
    __syncwarp();
    const bool retry = active && unc;
    if (active && !unc) {
      // FP64 offsets of the basic columns, computed as lp_columns computes them
      int cj[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) cj[k] = s_cj[k][threadIdx.x];
      const double xi0 = x[i], yi0 = y[i];
      double bxi[M], beta[M];
#pragma unroll
      for (int r = 0; r < M; ++r) {
        int j = INT_MAX;
#pragma unroll
        for (int k = 0; k < 8; ++k) j = (basis[r] == M + k) ? cj[k] : j;
        bxi[r] = 0.0;
        beta[r] = 0.0;
        if (j != INT_MAX) {
          bxi[r] = __dmul_rn(__dsub_rn(x[j], xi0), c.inv_h);
          beta[r] = __dmul_rn(__dsub_rn(y[j], yi0), c.inv_h);
        }
      }
      lp_finish<M, W>(c, i, code, basis, it, cj, bxi, beta, cols, f, fii, status, fail_list, ds, nu_dt, inv_h2, tl);
    }
    // warp-aggregated append to the FP64 retry list
    const unsigned rb = __ballot_sync(0xffffffffu, retry);
    if (rb) {
      const int lead = __ffs(rb) - 1;
      int slot0 = 0;
      if ((int)lane == lead) slot0 = atomicAdd(&ds->n_retry, __popc(rb));
      slot0 = __shfl_sync(0xffffffffu, slot0, lead);
      if (retry) retry_list[slot0 + __popc(rb & ((1u << lane) - 1u))] = i;
      n_retry += (lane == 0) ? __popc(rb) : 0;
    }
  }
  flush_stats(ds, tl.ok, tl.none, tl.maxpiv, tl.ratio, false, tl.solved, tl.pivots);
  if (lane == 0 && n_retry) atomicAdd(&ds->lp_small_retries, (unsigned long long)n_retry);
}

// ---------------------------------------------------------------------------
// The same LPs with the work split by warps: per block, PW warps take the
// columns and the certified binary32 pivots of 32 LPs each, and FW warps
// take the FP64 part (basis offsets, LU solve, certificate, stencil) of the
// LPs the pivot warps finished before, handed over in shared memory (three
// buffers, a full and an empty named barrier each).  The FP64 pipe then
// works on one batch while the binary32 and integer pipes work on the next,
// instead of every warp alternating between the two phases.  Results are
// those of k_lp_small32 bit for bit (the same device functions in the same
// order).  Two shapes: 4 + 2 warps with two blocks per SM, and 8 + 4 warps
// with one block per SM (the same 12 warps per SM at 168 registers; the
// wider block is 6% faster on the 1M-particle workload).
// ---------------------------------------------------------------------------
constexpr int kLpWsThreads = 32 * (4 + 2);
constexpr int kLpWsThreadsWide = 32 * (8 + 4);

// Hand-over of the warp-specialised LP: kWsSlots buffers, and per buffer two
// named barriers over every thread of the block.  FULL (1 + slot): the pivot
// warps arrive once they have written the batch, the FP64 warps wait there
// before reading it; EMPTY (1 + kWsSlots + slot): the FP64 warps arrive once
// they have read it, the pivot warps wait there before writing the slot
// again.  With three buffers the pivot warps may run two batches ahead, so
// that neither role waits for the other's slowest batch.  Both roles count
// the same rounds, and the last arrival on each EMPTY barrier that no later
// round waits for is left out, so every barrier generation completes.
constexpr int kWsSlots = 3;
// (immediate barrier numbers, so that the block reserves barriers 1 to 6
// only; the switch is uniform over the warp)
#define VRM_WS_BAR(op, id) asm volatile("bar." op " " #id ", %0;" ::"n"(NT) : "memory")
template <int NT>
__device__ __forceinline__ void ws_arrive(int id) {
  switch (id) {
    case 1: VRM_WS_BAR("arrive", 1); break;
    case 2: VRM_WS_BAR("arrive", 2); break;
    case 3: VRM_WS_BAR("arrive", 3); break;
    case 4: VRM_WS_BAR("arrive", 4); break;
    case 5: VRM_WS_BAR("arrive", 5); break;
    default: VRM_WS_BAR("arrive", 6); break;
  }
}
template <int NT>
__device__ __forceinline__ void ws_sync(int id) {
  switch (id) {
    case 1: VRM_WS_BAR("sync", 1); break;
    case 2: VRM_WS_BAR("sync", 2); break;
    case 3: VRM_WS_BAR("sync", 3); break;
    case 4: VRM_WS_BAR("sync", 4); break;
    case 5: VRM_WS_BAR("sync", 5); break;
    default: VRM_WS_BAR("sync", 6); break;
  }
}
#undef VRM_WS_BAR

template <int M, int W, int PW, int FW, int MINB>
__global__ void __launch_bounds__(32 * (PW + FW), MINB) k_lp_small32_ws(
    Consts c, const double* __restrict__ x, const double* __restrict__ y, const int* __restrict__ list,
    const int* __restrict__ list_count, const int* __restrict__ small, int* __restrict__ cols,
    double* __restrict__ f, double* __restrict__ fii, uint8_t* __restrict__ status, int* __restrict__ fail_list,
    int* __restrict__ retry_list, DevStats* __restrict__ ds, double nu_dt, const double* __restrict__ dt_dev,
    double nu) {
  static_assert(M == 5, "certified binary32 pivoting is written for the n = 1 rows");
  constexpr int kLpPivotWarps = PW, kLpFinishWarps = FW, kLpBatch = 32 * PW, kThreads = 32 * (PW + FW);
  if (dt_dev) nu_dt = nu * *dt_dev;
  const int m = *list_count;
  const double inv_h2 = 1.0 / (c.h * c.h);
  const float inv_h32 = f32_of(c.inv_h);
  LpTally tl;
  int n_retry = 0;
  const unsigned lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const bool pivot_warp = warp < kLpPivotWarps;
  // hand-over of a batch: particle, basis (4 bits per row) | pivots << 20 |
  // code << 27 | 1 << 30 (valid), and the sorted column indices
  __shared__ int s_i[kWsSlots][kLpBatch];
  __shared__ int s_meta[kWsSlots][kLpBatch];
  __shared__ int s_cj[kWsSlots][8][kLpBatch];
  const long nchunks = ((long)m + kLpBatch - 1) / kLpBatch;
  // the block's batches: chunks blockIdx.x + r gridDim.x, r < rounds; the
  // pivot warps take batch r into slot r mod kWsSlots, the FP64 warps finish
  // it from there
  const long rounds = (long)blockIdx.x < nchunks ? (nchunks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  if (pivot_warp) {
    int buf = 0;
    for (long r = 0; r < rounds; ++r) {
      const long chunk = (long)blockIdx.x + r * gridDim.x;
      if (r >= kWsSlots) ws_sync<kThreads>(1 + kWsSlots + buf);  // batch r - kWsSlots read
      {
        const int slot = warp * 32 + (int)lane;
        const long t = chunk * kLpBatch + slot;
        const bool active = t < m;
        int i = 0, it = 0, code = 0;
        int basis[M];
        bool unc = false;
#pragma unroll
        for (int q = 0; q < M; ++q) basis[q] = q;
        if (active) {
          i = list[t];
          float xs[8], es[8];
          int cj[8];
          lp_columns32(x, y, small, i, x[i], y[i], inv_h32, cj, xs, es, unc);
#pragma unroll
          for (int k = 0; k < 8; ++k) s_cj[buf][k][slot] = cj[k];
          lp_pivots32<M>(xs, es, basis, it, code, unc);
        }
        int meta = 0;
        if (active && !unc) {
          meta = (1 << 30) | (code << 27) | (it << 20);
#pragma unroll
          for (int q = 0; q < M; ++q) meta |= basis[q] << (4 * q);
        }
        s_i[buf][slot] = i;
        s_meta[buf][slot] = meta;
        // warp-aggregated append to the FP64 retry list
        const bool retry = active && unc;
        const unsigned rb = __ballot_sync(0xffffffffu, retry);
        if (rb) {
          const int lead = __ffs(rb) - 1;
          int slot0 = 0;
          if ((int)lane == lead) slot0 = atomicAdd(&ds->n_retry, __popc(rb));
          slot0 = __shfl_sync(0xffffffffu, slot0, lead);
          if (retry) retry_list[slot0 + __popc(rb & ((1u << lane) - 1u))] = i;
          n_retry += (lane == 0) ? __popc(rb) : 0;
        }
      }
      ws_arrive<kThreads>(1 + buf);  // batch r written
      buf = buf + 1 == kWsSlots ? 0 : buf + 1;
    }
  } else {
    int pb = 0;
    for (long d = 0; d < rounds; ++d) {
      ws_sync<kThreads>(1 + pb);  // batch d written
      {
#pragma unroll 1
        for (int slot = (warp - kLpPivotWarps) * 32 + (int)lane; slot < kLpBatch; slot += 32 * kLpFinishWarps) {
          const int meta = s_meta[pb][slot];
          if (meta & (1 << 30)) {
            const int i = s_i[pb][slot];
            int basis[M];
#pragma unroll
            for (int q = 0; q < M; ++q) basis[q] = (meta >> (4 * q)) & 15;
            const int it = (meta >> 20) & 127, code = (meta >> 27) & 3;
            int cj[8];
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) cj[kk] = s_cj[pb][kk][slot];
            // FP64 offsets of the basic columns, computed as lp_columns computes them
            const double xi0 = x[i], yi0 = y[i];
            double bxi[M], beta[M];
#pragma unroll
            for (int q = 0; q < M; ++q) {
              int j = INT_MAX;
#pragma unroll
              for (int kk = 0; kk < 8; ++kk) j = (basis[q] == M + kk) ? cj[kk] : j;
              bxi[q] = 0.0;
              beta[q] = 0.0;
              if (j != INT_MAX) {
                bxi[q] = __dmul_rn(__dsub_rn(x[j], xi0), c.inv_h);
                beta[q] = __dmul_rn(__dsub_rn(y[j], yi0), c.inv_h);
              }
            }
            lp_finish<M, W>(c, i, code, basis, it, cj, bxi, beta, cols, f, fii, status, fail_list, ds, nu_dt,
                            inv_h2, tl);
          }
        }
      }
      if (d + kWsSlots < rounds) ws_arrive<kThreads>(1 + kWsSlots + pb);  // batch d read
      pb = pb + 1 == kWsSlots ? 0 : pb + 1;
    }
  }
  flush_stats(ds, tl.ok, tl.none, tl.maxpiv, tl.ratio, false, tl.solved, tl.pivots);
  if (lane == 0 && n_retry) atomicAdd(&ds->lp_small_retries, (unsigned long long)n_retry);
}

// Monomial of Vandermonde row r at (xi, eta), rounded exactly as vcol<M>
// rounds it: rows 0, 1 are xi, eta; 2, 3, 4 are xi xi, xi eta, eta eta; 5 to
// 8 are (xi xi) xi, (xi xi) eta, xi (eta eta), (eta eta) eta.
__device__ __forceinline__ double vrow(int r, double xi, double eta) {
  const double u = (r == 4 || r == 7 || r == 8) ? eta : xi;
  const double v = (r == 2 || r == 5 || r == 6) ? xi : eta;
  const double quad = __dmul_rn(u, v);
  const double cub = __dmul_rn(quad, (r == 5 || r == 7) ? xi : eta);
  return r == 0 ? xi : r == 1 ? eta : r < 5 ? quad : cub;
}

// One column K of the lane-parallel LU of an M x M matrix (row r on lane
// r): the first largest |A[r][K]| at or below the diagonal is the pivot, its
// row and the right-hand side swap with row K, rcpd[K] = 1 / pivot, and the
// rows below store the multiplier A[r][K] rcpd[K] and subtract it times the
// pivot row, products and differences rounded separately.  Recursion over K
// keeps every index static (the matrix stays in registers).
template <int K, int M>
__device__ __forceinline__ void lu_rows(double (&A)[M], double& z, double (&rcpd)[M], bool& sing, int lane) {
  if constexpr (K < M) {
    constexpr unsigned kAll = 0xffffffffu;
    const bool rowk = lane >= K && lane < M;
    const unsigned long long key = rowk ? (unsigned long long)(dbits(A[K]) & 0x7FFFFFFFFFFFFFFFLL) : 0ull;
    unsigned long long best = key;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(kAll, best, o);
      best = ob > best ? ob : best;
    }
    sing = sing || best == 0ull;
    const int p = __ffs(__ballot_sync(kAll, rowk && key == best)) - 1;
    const int partner = lane == K ? p : (lane == p ? K : lane);
#pragma unroll
    for (int q = 0; q < M; ++q) A[q] = __shfl_sync(kAll, A[q], partner);
    z = __shfl_sync(kAll, z, partner);
    rcpd[K] = __drcp_rn(__shfl_sync(kAll, A[K], K));
    const bool below = lane > K && lane < M;
    const double l = __dmul_rn(A[K], rcpd[K]);
    if (below) A[K] = l;
#pragma unroll
    for (int q = K + 1; q < M; ++q) {
      const double pq = __shfl_sync(kAll, A[q], K);
      if (below) A[q] = __dsub_rn(A[q], __dmul_rn(l, pq));
    }
    lu_rows<K + 1, M>(A, z, rcpd, sing, lane);
  }
}

// Full-neighbourhood retry: one warp per particle.  Lane l holds tableau
// column l (K <= 32 columns, the FP64 work of the pivots); the per-row
// quantities (right-hand side, basic variable, ratio) live on lane r for row
// r, so that the ratio test costs one reciprocal per lane and a warp minimum
// instead of m divisions on every lane.  The final basis is factored with
// row r on lane r (the oracle's LU sequence: first largest pivot, full row
// swaps, multipliers times the pivot's reciprocal, separately rounded
// updates), forward substitution in column order, back substitution row by
// row; the result is bit-identical to the oracle's basis solve.
template <int M, int W>
__global__ void __launch_bounds__(128) k_lp_full(Consts c, const double* __restrict__ x,
                                                 const double* __restrict__ y, const int* __restrict__ fail_list,
                                                 const int* __restrict__ fail_count,
                                                 const int* __restrict__ nbr_count, const int* __restrict__ nbr_idx,
                                                 int* __restrict__ cols, double* __restrict__ f,
                                                 double* __restrict__ fii, uint8_t* __restrict__ status,
                                                 DevStats* __restrict__ ds, double nu_dt,
                                                 const double* __restrict__ dt_dev, double nu) {
  constexpr unsigned kAll = 0xffffffffu;
  if (dt_dev) nu_dt = nu * *dt_dev;
  const int lane = threadIdx.x & 31;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
  const int m = *fail_count;
  const double inv_h2 = 1.0 / (c.h * c.h);
  int st_ok = 0, st_none = 0, st_maxpiv = 0, st_solved = 0, st_pivots = 0;
  unsigned st_cols = 0;
  unsigned long long st_colpiv = 0;
  double st_ratio = 0.0;
  for (long t = warp; t < m; t += nwarps) {
    const int i = fail_list[t];
    const int cnt = nbr_count[i];
    const int K = cnt < c.row_cap ? cnt : c.row_cap;
    const double xi0 = x[i], yi0 = y[i];
    double d2 = 1e300, dx = 0.0, dy = 0.0;
    int j = INT_MAX;
    if (lane < K) {
      j = nbr_idx[(size_t)i * c.k_cap + lane];
      dx = __dsub_rn(x[j], xi0);
      dy = __dsub_rn(y[j], yi0);
      d2 = dist2(dx, dy);
    }
    // bitonic sort of (d2, j) across the warp, ascending
    for (int size = 2; size <= 32; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const double od2 = __shfl_xor_sync(kAll, d2, stride);
        const int oj = __shfl_xor_sync(kAll, j, stride);
        const double odx = __shfl_xor_sync(kAll, dx, stride);
        const double ody = __shfl_xor_sync(kAll, dy, stride);
        const bool up = ((lane & size) == 0);
        const bool lower = ((lane & stride) == 0);
        const bool eq = dbits(od2) == dbits(d2);  // d2 >= +0: bit order is value order
        const bool other_less = lt_nonneg(od2, d2) || (eq && oj < j);
        const bool take = (lower == up) ? other_less : !other_less && !(eq && oj == j);
        if (take) {
          d2 = od2;
          j = oj;
          dx = odx;
          dy = ody;
        }
      }
    }
    const double cxi = __dmul_rn(dx, c.inv_h), ceta = __dmul_rn(dy, c.inv_h);
    double T[M], v[M];
    vcol<M>(cxi, ceta, v);
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      T[r] = v[r];
      s = __dadd_rn(s, v[r]);
    }
    double d = 0.0 - s;
    // row r on lane r: right-hand side and basic variable (artificials first)
    double rhs = lane < M ? b_of(lane) : 0.0;
    int bas = lane < M ? lane : INT_MAX;
    bool isb = false;
    int it = 0, code = 0;
    int n_art = M;
    for (;;) {
      if (n_art == 0) break;  // phase I over: every reduced cost is zero
      const unsigned cand = __ballot_sync(kAll, lane < K && !isb && lt_neg(d, kTolPrice));
      if (!cand) break;
      if (it == kPivotCap) {
        code = 2;
        break;
      }
      const int q = __ffs(cand) - 1;
      double a[M], amine = 0.0;
#pragma unroll
      for (int r = 0; r < M; ++r) {
        a[r] = __shfl_sync(kAll, T[r], q);
        amine = (lane == r) ? a[r] : amine;
      }
      // ratio test, row r on lane r: basic values <= kTolSnap are zeros.
      // As in k_lp_small, the ratios are screened in binary32 (operands
      // rounded from their bit patterns, relative error < 1e-6): the rows
      // within 1e-5 of the smallest binary32 ratio are the only ones that
      // can lie in the FP64 tie window, so FP64 ratios (Newton reciprocal,
      // relative error ~2^-45) are taken only when two of them differ and
      // are not exact zeros, and only on those rows
      const bool elig = lane < M && gt_pos(amine, kTolPivot);
      const bool nzr = gt_pos(rhs, kTolSnap);
      const float r32 = !elig ? 3.0e38f : nzr ? __fmul_rn(f32_of(rhs), __frcp_rn(f32_of(amine))) : 0.0f;
      const unsigned eligm = __ballot_sync(kAll, elig);
      if (!eligm) {
        code = 2;
        break;
      }
      const float m32 = __uint_as_float(__reduce_min_sync(kAll, __float_as_uint(r32)));
      const float marg = __fmaf_rn(1e-5f, fmaxf(m32, 1.0f), m32);
      const bool contr = elig && r32 <= marg;
      unsigned cont = __ballot_sync(kAll, contr);
      const bool allzero = __ballot_sync(kAll, contr && r32 != 0.0f) == 0u;
      if (__popc(cont) > 1 && !allzero) {
        const double num = nzr ? rhs : 0.0;
        const double ratio = contr ? __dmul_rn(num, rcp_newton<1>(amine)) : 1e308;
        unsigned long long rb = contr ? (unsigned long long)dbits(ratio) : ~0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long ob = __shfl_xor_sync(kAll, rb, o);
          rb = ob < rb ? ob : rb;
        }
        const double theta = __longlong_as_double((long long)rb);
        const double lim = __fma_rn(kTolTie, gt_pos(theta, 1.0) ? theta : 1.0, theta);
        cont = __ballot_sync(kAll, contr && !lt_nonneg(lim, ratio));
      }
      // leaving row: the lowest basic variable among the tied rows
      const int key = ((cont >> lane) & 1u) ? bas : INT_MAX;
      const int lbas = __reduce_min_sync(kAll, key);
      const int leave = __ffs(__ballot_sync(kAll, key == lbas)) - 1;
      const double piv = __shfl_sync(kAll, amine, leave);
      const double prhs_raw = __shfl_sync(kAll, rhs, leave);
      double prow_raw = T[0];
#pragma unroll
      for (int r = 1; r < M; ++r) prow_raw = (leave == r) ? T[r] : prow_raw;
      const double rcp = rcp_newton<2>(piv);
      const double prow = (lane == q) ? 1.0 : __dmul_rn(prow_raw, rcp);
      const double prhs = __dmul_rn(prhs_raw, rcp);
#pragma unroll
      for (int r = 0; r < M; ++r) {
        const bool lr = (leave == r);
        const double ar = lr ? 0.0 : a[r];
        const double u = __fma_rn(-ar, prow, T[r]);
        T[r] = lr ? prow : ((lane == q) ? 0.0 : u);
      }
      rhs = (lane == leave) ? prhs : __fma_rn(-amine, prhs, rhs);
      const double dq = __shfl_sync(kAll, d, q);
      d = (lane == q) ? 0.0 : __fma_rn(-dq, prow, d);
      if (lbas >= M && lane == lbas - M) isb = false;
      if (lbas < M) --n_art;
      if (lane == q) isb = true;
      if (lane == leave) bas = M + q;
      ++it;
    }
    // basic solution of the final basis by the oracle's LU sequence, row r of
    // B on lane r: column k is e_v for an artificial v = basis[k] < m, else
    // the Vandermonde column of the basic structural
    double fv = 0.0, wsum = 0.0, rmax = 0.0;
    if (code == 0) {
      double A[M], B0[M];
      int bk[M];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        bk[k] = __shfl_sync(kAll, bas, k);
        const int src = bk[k] >= M ? bk[k] - M : 0;
        const double bx = __shfl_sync(kAll, cxi, src), be = __shfl_sync(kAll, ceta, src);
        A[k] = bk[k] < M ? (bk[k] == lane ? 1.0 : 0.0) : vrow(lane, bx, be);
        B0[k] = A[k];
      }
      double z = lane < M ? b_of(lane) : 0.0;
      double rcpd[M];
      bool sing = false;
      lu_rows<0, M>(A, z, rcpd, sing, lane);
      // forward substitution: row r takes its terms in ascending column order
#pragma unroll
      for (int q = 0; q < M - 1; ++q) {
        const double zq = __shfl_sync(kAll, z, q);
        if (lane > q && lane < M) z = __dsub_rn(z, __dmul_rn(A[q], zq));
      }
      // back substitution row by row (ascending columns within a row)
      double xB[M];
#pragma unroll
      for (int r = M - 1; r >= 0; --r) {
        double acc = z;
#pragma unroll
        for (int q = r + 1; q < M; ++q) acc = __dsub_rn(acc, __dmul_rn(A[q], xB[q]));
        xB[r] = __shfl_sync(kAll, __dmul_rn(acc, rcpd[r]), r);
      }
      if (sing) code = 2;
      // residual V f - b of the snapped structural weights, row r on lane r,
      // evaluated as the oracle does: the terms B[r][k] f_k (the basis matrix
      // kept before its LU) in ascending column order, products and sums
      // rounded separately, then the difference with b_r; the largest |row|
      // over the row lanes
      int key[M];
      double pay[2][M];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        double vk = 0.0;
        if (bk[k] < M) {
          wsum = __dadd_rn(wsum, xB[k]);
        } else {
          vk = gt_pos(xB[k], kTolSnap) ? xB[k] : 0.0;
          if (bk[k] == M + lane) fv = vk;
        }
        key[k] = bk[k];
        pay[0][k] = B0[k];
        pay[1][k] = vk;
      }
      sort_by_key<M, 2>(key, pay);
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < M; ++k) acc = __dadd_rn(acc, __dmul_rn(pay[0][k], pay[1][k]));
      acc = __dsub_rn(acc, lane < M ? b_of(lane) : 0.0);
      unsigned long long eb = lane < M ? ((unsigned long long)dbits(acc) & 0x7FFFFFFFFFFFFFFFull) : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(kAll, eb, o);
        eb = ob > eb ? ob : eb;
      }
      rmax = __longlong_as_double((long long)eb);
    }
    const bool feasible = code == 0 && !gt_pos(wsum, kTolPhase1) && !gt_pos(rmax, kTolResid);
    int* crow = cols + (size_t)i * W;
    double* frow = f + (size_t)i * W;
    const unsigned nz = __ballot_sync(kAll, feasible && dbits(fv) != 0);
    if (feasible) {
      const int slot = __popc(nz & ((1u << lane) - 1u));
      if (dbits(fv) != 0 && slot < W) {
        crow[slot] = j;
        frow[slot] = fv;
      }
      const int used = __popc(nz);
      if (lane >= used && lane < W) {
        crow[lane] = -1;
        frow[lane] = 0.0;
      }
      // f~_ii = -sum of the nonzero weights in column order
      double sacc = 0.0;
      unsigned rest = nz;
      while (rest) {
        const int l = __ffs(rest) - 1;
        rest &= rest - 1;
        sacc = __dadd_rn(sacc, __shfl_sync(kAll, fv, l));
      }
      if (lane == 0) {
        fii[i] = -sacc;
        status[i] = VRM_LP_FULL;
        ++st_ok;
        const double qr = __dmul_rn(__dmul_rn(nu_dt, sacc), inv_h2);
        st_ratio = qr > st_ratio ? qr : st_ratio;
      }
    } else {
      if (lane < W) {
        crow[lane] = -1;
        frow[lane] = 0.0;
      }
      if (lane == 0) {
        fii[i] = 0.0;
        status[i] = VRM_LP_NONE;
        ++st_none;
      }
    }
    st_maxpiv = it > st_maxpiv ? it : st_maxpiv;
    if (lane == 0) {
      ++st_solved;
      st_pivots += it;
      st_cols += K;
      st_colpiv += (unsigned long long)K * it;
    }
  }
  flush_stats(ds, st_ok, st_none, st_maxpiv, st_ratio, true, st_solved, st_pivots);
  st_cols = __reduce_add_sync(kAll, (unsigned)st_cols);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) st_colpiv += __shfl_xor_sync(kAll, st_colpiv, o);
  if (lane == 0 && st_cols) {
    atomicAdd(&ds->lp_full_columns, (unsigned long long)st_cols);
    atomicAdd(&ds->lp_full_column_pivots, st_colpiv);
  }
}

// Identity weights of the removal candidates (particle removal, the outlook
// of Sec. 6.2): the phase-I simplex of k_lp_small with rows (0,0) (1,0) (0,1)
// of r_ij / h and b = (1, 0, 0), i.e. sum g = 1 and sum g r = 0 with g >= 0,
// on the closest kept particle (close[j] == 0) of every 45-degree segment of
// the candidate's annulus row (ties to the smaller index), columns ordered by
// (d2, j).  The same entering, leaving, snapping and feasibility rules; the
// final basis solved by the oracle's LU sequence.  One candidate per thread.
// removed[i] = 1 and the nonzero weights (at most 3 of the 4 slots, column
// order, padded -1 / 0) where feasible; otherwise the candidate stays.
__global__ void __launch_bounds__(128) k_lp_identity(Consts c, const double* __restrict__ x,
                                                     const double* __restrict__ y, const int* __restrict__ list,
                                                     const int* __restrict__ list_count,
                                                     const int* __restrict__ nbr_count,
                                                     const int* __restrict__ nbr_idx,
                                                     const uint8_t* __restrict__ close, uint8_t* __restrict__ removed,
                                                     int* __restrict__ cols4, double* __restrict__ w4) {
  constexpr int M = 3;
  const int m = *list_count;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) {
    const int i = list[t];
    const double xi0 = x[i], yi0 = y[i];
    const int cnt0 = nbr_count[i];
    const int K = cnt0 < c.row_cap ? cnt0 : c.row_cap;
    const int* row = nbr_idx + (size_t)i * c.k_cap;
    // closest kept member of every segment
    double cd2[8], cxi[8], ceta[8];
    int cj[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      cd2[s] = 1e300;
      cj[s] = INT_MAX;
      cxi[s] = ceta[s] = 0.0;
    }
    for (int e = 0; e < K; ++e) {
      const int j = row[e];
      if (close[j]) continue;
      const double dx = __dsub_rn(x[j], xi0), dy = __dsub_rn(y[j], yi0);
      const double d2 = dist2(dx, dy);
      const int sg = segment_of(dx, dy);
      double cb = cd2[0];
      int cjb = cj[0];
#pragma unroll
      for (int s = 1; s < 8; ++s) {
        cb = (sg == s) ? cd2[s] : cb;
        cjb = (sg == s) ? cj[s] : cjb;
      }
      const bool take = lt_nonneg(d2, cb) || (dbits(d2) == dbits(cb) && j < cjb);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const bool here = take && sg == s;
        cd2[s] = here ? d2 : cd2[s];
        cj[s] = here ? j : cj[s];
        cxi[s] = here ? dx : cxi[s];
        ceta[s] = here ? dy : ceta[s];
      }
    }
    sort8(cd2, cj, cxi, ceta);
    unsigned basic = 0;  // empty columns never enter
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (cj[k] == INT_MAX) basic |= 1u << k;
      cxi[k] = __dmul_rn(cxi[k], c.inv_h);
      ceta[k] = __dmul_rn(ceta[k], c.inv_h);
    }
    double T[M][8], rhs[M], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double v[M];
      vcol_id(cxi[k], ceta[k], v);
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < M; ++r) {
        T[r][k] = v[r];
        s = __dadd_rn(s, v[r]);
      }
      d[k] = dneg(s);
    }
#pragma unroll
    for (int r = 0; r < M; ++r) rhs[r] = b_id(r);
    int basis[M];
#pragma unroll
    for (int r = 0; r < M; ++r) basis[r] = r;
    int it = 0, code = 0, n_art = M;
    for (;;) {
      if (n_art == 0) break;  // phase I over
      int q = -1;
#pragma unroll
      for (int k = 7; k >= 0; --k)
        if (!((basic >> k) & 1u) && lt_neg(d[k], kTolPrice)) q = k;
      if (q < 0) break;
      if (it == kPivotCap) {
        code = 2;
        break;
      }
      double a[M];
#pragma unroll
      for (int r = 0; r < M; ++r) {
        double v = T[r][0];
#pragma unroll
        for (int k = 1; k < 8; ++k) v = (q == k) ? T[r][k] : v;
        a[r] = v;
      }
      double ratio[M], theta = 1e308;
      bool elig[M], any = false;
#pragma unroll
      for (int r = 0; r < M; ++r) {
        elig[r] = gt_pos(a[r], kTolPivot);
        const double num = gt_pos(rhs[r], kTolSnap) ? rhs[r] : 0.0;
        ratio[r] = elig[r] ? __dmul_rn(num, rcp_newton<1>(a[r])) : 1e308;
        if (elig[r]) {
          any = true;
          theta = lt_nonneg(ratio[r], theta) ? ratio[r] : theta;
        }
      }
      if (!any) {
        code = 2;
        break;
      }
      const double lim = __fma_rn(kTolTie, gt_pos(theta, 1.0) ? theta : 1.0, theta);
      int leave = -1, lbas = INT_MAX;
#pragma unroll
      for (int r = 0; r < M; ++r)
        if (elig[r] && !lt_nonneg(lim, ratio[r]) && basis[r] < lbas) {
          leave = r;
          lbas = basis[r];
        }
      double piv = a[0], prhs_raw = rhs[0];
#pragma unroll
      for (int r = 1; r < M; ++r) {
        piv = (leave == r) ? a[r] : piv;
        prhs_raw = (leave == r) ? rhs[r] : prhs_raw;
      }
      const double rcp = rcp_newton<2>(piv);
      double prow[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        double v = T[0][k];
#pragma unroll
        for (int r = 1; r < M; ++r) v = (leave == r) ? T[r][k] : v;
        prow[k] = (k == q) ? 1.0 : __dmul_rn(v, rcp);
      }
      const double prhs = __dmul_rn(prhs_raw, rcp);
#pragma unroll
      for (int r = 0; r < M; ++r) {
        const bool lr = (leave == r);
        const double ar = lr ? -1.0 : a[r];
#pragma unroll
        for (int k = 0; k < 8; ++k) T[r][k] = __fma_rn(-ar, prow[k], lr ? 0.0 : T[r][k]);
        rhs[r] = __fma_rn(-ar, prhs, lr ? 0.0 : rhs[r]);
      }
      double dq = d[0];
#pragma unroll
      for (int k = 1; k < 8; ++k) dq = (q == k) ? d[k] : dq;
#pragma unroll
      for (int k = 0; k < 8; ++k) d[k] = __fma_rn(-dq, prow[k], d[k]);
      if (lbas >= M) basic &= ~(1u << (lbas - M));
      else --n_art;
      basic |= 1u << q;
#pragma unroll
      for (int r = 0; r < M; ++r) basis[r] = (leave == r) ? M + q : basis[r];
      ++it;
    }
    double fv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fv[k] = 0.0;
    double wsum = 0.0, rmax = 0.0;
    if (code == 0) {
      double bxi[M], beta[M], xB[M];
#pragma unroll
      for (int r = 0; r < M; ++r) {
        double av = 0.0, ev = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          av = (basis[r] == M + k) ? cxi[k] : av;
          ev = (basis[r] == M + k) ? ceta[k] : ev;
        }
        bxi[r] = av;
        beta[r] = ev;
      }
      if (!basis_solve<M, true>(basis, bxi, beta, xB)) code = 2;
      double v[M];
#pragma unroll
      for (int r = 0; r < M; ++r) {
        v[r] = (basis[r] >= M && gt_pos(xB[r], kTolSnap)) ? xB[r] : 0.0;
        if (basis[r] < M) wsum = __dadd_rn(wsum, xB[r]);
#pragma unroll
        for (int k = 0; k < 8; ++k) fv[k] = (basis[r] == M + k) ? v[r] : fv[k];
      }
      if (code == 0) rmax = resid_in_column_order<M, true>(basis, bxi, beta, v);
    }
    const bool feasible = code == 0 && !gt_pos(wsum, kTolPhase1) && !gt_pos(rmax, kTolResid);
    int* crow = cols4 + (size_t)i * 4;
    double* wrow = w4 + (size_t)i * 4;
    int slot = 0;
    if (feasible) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (dbits(fv[k]) != 0 && slot < 4) {
          crow[slot] = cj[k];
          wrow[slot] = fv[k];
          ++slot;
        }
    }
    for (; slot < 4; ++slot) {
      crow[slot] = -1;
      wrow[slot] = 0.0;
    }
    removed[i] = feasible ? 1 : 0;
  }
}

__global__ void k_lp_clear(int n, int w, const uint8_t* __restrict__ diffused, int* __restrict__ cols,
                           double* __restrict__ f, double* __restrict__ fii, uint8_t* __restrict__ status) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    if (diffused[i]) continue;
    for (int k = 0; k < w; ++k) {
      cols[i * w + k] = -1;
      f[i * w + k] = 0.0;
    }
    fii[i] = 0.0;
    status[i] = VRM_LP_NOT_DIFFUSED;
  }
}

cudaError_t lp_small(const Consts& c, const double* x, const double* y, const int* list, const int* list_count,
                     int cap, const int* small, int* cols, double* f, double* fii, uint8_t* status, int* fail_list,
                     int* retry_list, DevStats* ds, double nu_dt, cudaStream_t s, const double* dt_dev, double nu) {
  if (cap <= 0) return cudaSuccess;
  // lp_block = kLpWsThreads or kLpWsThreadsWide selects the warp-specialised
  // binary32 LP; the other LP kernels then run with 128 threads per block
  const bool ws = c.lp_block == kLpWsThreads || c.lp_block == kLpWsThreadsWide;
  const int tb = ws ? 128 : c.lp_block;
  int blocks = (int)(((long)cap + tb - 1) / tb);
  if (blocks > c.lp_blocks_per_sm * sm_count()) blocks = c.lp_blocks_per_sm * sm_count();
  if (c.order == 2) {
    k_lp_small<9, 12><<<blocks, tb, 0, s>>>(c, x, y, list, list_count, small, cols, f, fii, status, fail_list, ds,
                                            nu_dt, dt_dev, nu);
    note_launch();
  } else if (c.lp_fp64_pivots || !(c.inv_h > 1e-20 && c.inv_h < 1e20)) {
    k_lp_small<5, 8><<<blocks, tb, 0, s>>>(c, x, y, list, list_count, small, cols, f, fii, status, fail_list, ds,
                                           nu_dt, dt_dev, nu);
    note_launch();
  } else {
    // certified binary32 pivots, then the uncertain particles in FP64
    cudaError_t e = cudaMemsetAsync(&ds->n_retry, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (c.lp_block == kLpWsThreads) {
      // warp-specialised form, 4 + 2 warps: two resident blocks per SM
      k_lp_small32_ws<5, 8, 4, 2, 2><<<2 * sm_count(), kLpWsThreads, 0, s>>>(
          c, x, y, list, list_count, small, cols, f, fii, status, fail_list, retry_list, ds, nu_dt, dt_dev, nu);
    } else if (c.lp_block == kLpWsThreadsWide) {
      // 8 + 4 warps: one resident block per SM
      k_lp_small32_ws<5, 8, 8, 4, 1><<<sm_count(), kLpWsThreadsWide, 0, s>>>(
          c, x, y, list, list_count, small, cols, f, fii, status, fail_list, retry_list, ds, nu_dt, dt_dev, nu);
    } else {
      k_lp_small32<5, 8><<<blocks, tb, 0, s>>>(c, x, y, list, list_count, small, cols, f, fii, status, fail_list,
                                               retry_list, ds, nu_dt, dt_dev, nu);
    }
    note_launch();
    // the re-run list is a few percent of the LPs: one-warp blocks spread it
    // over every SM instead of over the first few hundred blocks
    int rblocks = (int)(((long)cap + 31) / 32);
    if (rblocks > 32 * sm_count()) rblocks = 32 * sm_count();
    k_lp_small<5, 8><<<rblocks, 32, 0, s>>>(c, x, y, retry_list, &ds->n_retry, small, cols, f, fii, status,
                                           fail_list, ds, nu_dt, dt_dev, nu);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t lp_full(const Consts& c, const double* x, const double* y, const int* fail_list, const int* fail_count,
                    int cap, const int* nbr_count, const int* nbr_idx, int* cols, double* f, double* fii,
                    uint8_t* status, DevStats* ds, double nu_dt, cudaStream_t s, const double* dt_dev, double nu) {
  if (cap <= 0) return cudaSuccess;
  long warps = cap;
  long blocks = (warps * 32 + 127) / 128;
  if (blocks > 4 * sm_count()) blocks = 4 * sm_count();
  if (c.order == 2)
    k_lp_full<9, 12><<<(int)blocks, 128, 0, s>>>(c, x, y, fail_list, fail_count, nbr_count, nbr_idx, cols, f, fii,
                                                 status, ds, nu_dt, dt_dev, nu);
  else
    k_lp_full<5, 8><<<(int)blocks, 128, 0, s>>>(c, x, y, fail_list, fail_count, nbr_count, nbr_idx, cols, f, fii,
                                                status, ds, nu_dt, dt_dev, nu);
  note_launch();
  return cudaGetLastError();
}

cudaError_t lp_clear(int n, int w, const uint8_t* diffused, int* cols, double* f, double* fii, uint8_t* status,
                     cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (n + kBlock - 1) / kBlock;
  if (blocks > 8 * sm_count()) blocks = 8 * sm_count();
  k_lp_clear<<<blocks, kBlock, 0, s>>>(n, w, diffused, cols, f, fii, status); note_launch();
  return cudaGetLastError();
}

cudaError_t lp_identity(const Consts& c, const double* x, const double* y, const int* list, const int* list_count,
                        int cap, const int* nbr_count, const int* nbr_idx, const uint8_t* close, uint8_t* removed,
                        int* cols4, double* w4, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  int blocks = (cap + 127) / 128;
  if (blocks > 16 * sm_count()) blocks = 16 * sm_count();
  k_lp_identity<<<blocks, 128, 0, s>>>(c, x, y, list, list_count, nbr_count, nbr_idx, close, removed, cols4, w4);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
