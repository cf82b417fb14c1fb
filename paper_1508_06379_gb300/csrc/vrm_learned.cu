// The learned weight proposal around the network (vrm_mlp.cu): input rows
// from the neighbourhoods, and the exact correction of the proposals onto the
// moment conditions with the acceptance test.  Rejected particles go to the
// LP of Sec. 4.1 (vrm_lp.cu), which stays the arbiter of validity.
//
// Slots: the annulus neighbours of particle i (Eq. neighbourhood) ordered by
// (45-degree segment of Sec. 4.2, squared distance, index), at most 32.
// Input row: xi_x of the slots, xi_y, mask, 32 zeros (bf16), xi = (x_j -
// x_i) / h (Eq. momcondmv scaling) in fp32 from fp32 positions, then bf16.
//
// Candidates are the slots holding the small neighbourhood of Sec. 4.3 (the
// closest particle of every segment, the LP's own columns), ranked by the
// network's proposal (larger first, ties to the lower slot).  The proposal
// chooses the stencil's support: five candidates at a time, in a fixed
// order (increasing sum of ranks, ties lexicographic: the network's top five
// first), the moment conditions V_S f = b (rows (1,0) (0,1) (2,0) (1,1)
// (0,2) of Eq. momcondmv, b = (0, 0, 2, 0, 2) from Eqs. cond_two and
// cond_alpha) are solved on the support S, and the first support whose
// solution is non-negative (Sec. 3.1) with |V_S f - b|_inf <= 1e-12 gives
// the stencil: the projection of the proposal onto the moment conditions
// within its support, an exact vertex of the set the LP searches.  Every
// support is first screened in binary32 (GB300 runs fp32 at about 60 times
// its FP64 rate): Gaussian elimination with every operation rounded to
// float32, passed on when all weights are >= -1e-6; only then the FP64
// solve (FP64 weights in [-1e-13, 0) are zeros of the vertex and dropped),
// at most four FP64 solves per particle.  A particle with no passing support
// goes to the LP.
#include <cuda_bf16.h>

#include "vrm_mlp.cuh"

namespace vrm {

namespace {

constexpr int kSlots = 32;
constexpr int kRow = 128;  // input row stride
constexpr int kSup = 8;    // support cap (= stencil width)
constexpr double kAcceptResid = 1e-12;
constexpr double kSnap = 1e-13;        // FP64 weights in [-kSnap, 0) are zeros
constexpr float kScreenTol = 1e-6f;    // binary32 screen: weights >= -kScreenTol pass
constexpr float kScreenPivot = 1e-6f;  // binary32 screen: relative pivot threshold
constexpr int kSubsets = 56;           // 5-subsets of 8 candidate ranks
constexpr int kMaxSolves = 4;          // FP64 solves per particle at most

}  // namespace

// fp32 copy of the positions (the network's input precision).
__global__ void k_mirror(const double* __restrict__ x, const double* __restrict__ y, int n_bound,
                         const int* __restrict__ n_dev, float2* __restrict__ xyf) {
  const int n = n_dev ? *n_dev : n_bound;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    xyf[i] = make_float2(__double2float_rn(x[i]), __double2float_rn(y[i]));
}

// One warp per listed particle: lane l takes neighbour l of the row, the
// warp sorts the keys (segment, squared distance, index) and lane l writes
// slot l.  Everything is fp32 (the network's input precision): the offset
// is fp32(x_j) - fp32(x_i), then the segment, the squared distance
// (products and sum rounded separately) and xi = dx * fp32(1/h).  The sort
// key is one 32-bit word, segment << 28 | bits(d2) >> 3 (d2 >= 0, so its bit
// pattern orders like the value; the 3 lowest mantissa bits are dropped),
// with the index breaking ties: the sort runs on the integer pipes, on one
// 64-bit value per lane, and does not depend on the row's order.
__global__ void k_features(Consts c, const float2* __restrict__ xyf,
                           const int* __restrict__ list, const int* __restrict__ list_count, int m_bound,
                           const int* __restrict__ nbr_count, const int* __restrict__ nbr_idx,
                           __nv_bfloat16* __restrict__ X, int* __restrict__ slots) {
  const int lane = threadIdx.x & 31;
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
  const int m = list_count ? *list_count : m_bound;
  const float inv_hf = __double2float_rn(c.inv_h);
  for (long t = warp; t < m; t += nwarps) {
    const int i = list ? list[t] : (int)t;
    const int cnt = nbr_count[i];
    const int K = cnt < c.row_cap ? cnt : c.row_cap;
    unsigned key = 0xFFFFFFFFu;  // empty slots last
    int j = INT_MAX;
    float fdx = 0.0f, fdy = 0.0f;
    if (lane < K) {
      j = nbr_idx[(size_t)i * c.k_cap + lane];
      const float2 pj = xyf[j], pi = xyf[i];
      fdx = __fsub_rn(pj.x, pi.x);
      fdy = __fsub_rn(pj.y, pi.y);
      const float d2 = dist2f(fdx, fdy);
      key = ((unsigned)segment_of(fdx, fdy) << 28) | (__float_as_uint(d2) >> 3);
    }
    // ties are broken by the index (rows may be in any order): one distinct
    // 64-bit value per lane, (key << 32) | j
    unsigned long long v = ((unsigned long long)key << 32) | (unsigned)j;
    // a row of K <= 8 (16) entries sits in lanes 0..7 (0..15): a bitonic
    // network of that width sorts it (lanes past it keep their empties)
    const int width = K <= 8 ? 8 : K <= 16 ? 16 : 32;
    for (int size = 2; size <= width; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, v, stride);
        const bool up = ((lane & size) == 0);
        const bool lower = ((lane & stride) == 0);
        // ascending runs keep the smaller value in the lower lane
        const bool take = (lower == up) ? ov < v : ov > v;
        v = take ? ov : v;
      }
    }
    const bool valid = lane < K;
    j = (int)(unsigned)(v & 0xFFFFFFFFull);
    float sdx = 0.0f, sdy = 0.0f;
    if (valid) {  // the sorted entry's offset, recomputed as above
      const float2 pj = xyf[j], pi = xyf[i];
      sdx = __fsub_rn(pj.x, pi.x);
      sdy = __fsub_rn(pj.y, pi.y);
    }
    __nv_bfloat16* row = X + (size_t)t * kRow;
    row[lane] = __float2bfloat16_rn(valid ? __fmul_rn(sdx, inv_hf) : 0.0f);
    row[kSlots + lane] = __float2bfloat16_rn(valid ? __fmul_rn(sdy, inv_hf) : 0.0f);
    row[2 * kSlots + lane] = __float2bfloat16_rn(valid ? 1.0f : 0.0f);
    row[3 * kSlots + lane] = __float2bfloat16_rn(0.0f);
    slots[(size_t)t * kSlots + lane] = valid ? j : -1;
  }
}

// |d| through the bit pattern (integer compares: GB300's FP64 pipe is narrow).
__device__ __forceinline__ unsigned long long abs_bits(double d) {
  return (unsigned long long)__double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFull;
}
// d >= 0 (and not NaN) through the bit pattern.
__device__ __forceinline__ bool nonneg_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return b <= 0x7FF0000000000000ull || b == 0x8000000000000000ull;
}

// binary32 seed of |a| from the bit pattern (mantissa rounded to 23 bits,
// exponent rebiased; |a| must lie in the binary32 normal range), by integer ops.
__device__ __forceinline__ float seed32(double a) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long mr = (b + 0x10000000ull) >> 29;
  const int e32 = (int)((mr >> 23) & 0x7FF) - 1023 + 127;
  return __int_as_float((e32 << 23) | (int)(mr & 0x7FFFFF));
}
// binary32 value widened to binary64 by integer ops (normal range).
__device__ __forceinline__ double widen32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long d = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)((int)((u >> 23) & 0xFF) - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7FFFFF) << 29);
  return __longlong_as_double((long long)d);
}
// 1/a for |a| in the binary32 normal range: binary32 seed, two Newton steps
// r <- r + r (1 - a r) in FP64 (full FP64 accuracy; no FP64 division).
__device__ __forceinline__ double rcp64(double a) {
  float r32 = __frcp_rn(seed32(a));
  if (__double_as_longlong(a) < 0) r32 = -r32;
  double r = widen32(r32);
  r = fma(r, fma(-a, r, 1.0), r);
  r = fma(r, fma(-a, r, 1.0), r);
  return r;
}
// The square system V f = b on five neighbours (columns xi, eta) by Gaussian
// elimination with partial pivoting (first largest |pivot|), FP64.  Returns
// false when a pivot is at most 1e-12 of the largest |entry| or the result
// (weights in [-kSnap, 0) set to zero) is not a non-negative solution with
// residual <= kAcceptResid.
__device__ __forceinline__ bool square_stencil(const double* xi, const double* eta, double* fo) {
  double A[5][6];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    A[0][s] = xi[s];
    A[1][s] = eta[s];
    A[2][s] = xi[s] * xi[s];
    A[3][s] = xi[s] * eta[s];
    A[4][s] = eta[s] * eta[s];
  }
  unsigned long long vmax = 0;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const unsigned long long ab = abs_bits(A[r][s]);
      vmax = ab > vmax ? ab : vmax;
    }
    A[r][5] = (r == 2 || r == 4) ? 2.0 : 0.0;
  }
  const unsigned long long tiny = abs_bits(1e-12 * __longlong_as_double((long long)vmax));
  double inv[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    int p = k;
    unsigned long long best = abs_bits(A[k][k]);
#pragma unroll
    for (int r = k + 1; r < 5; ++r) {
      const unsigned long long ab = abs_bits(A[r][k]);
      if (ab > best) {
        best = ab;
        p = r;
      }
    }
    if (best <= tiny) return false;
#pragma unroll
    for (int r = k + 1; r < 5; ++r) {
      const bool sw = r == p;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const double a = A[k][q], b = A[r][q];
        A[k][q] = sw ? b : a;
        A[r][q] = sw ? a : b;
      }
    }
    inv[k] = rcp64(A[k][k]);
#pragma unroll
    for (int r = k + 1; r < 5; ++r) {
      const double mlt = A[r][k] * inv[k];
#pragma unroll
      for (int q = k + 1; q < 6; ++q) A[r][q] = fma(-mlt, A[k][q], A[r][q]);
    }
  }
  double f[5];
#pragma unroll
  for (int k = 4; k >= 0; --k) {
    double acc = A[k][5];
#pragma unroll
    for (int q = k + 1; q < 5; ++q) acc = fma(-A[k][q], f[q], acc);
    f[k] = acc * inv[k];
  }
  // weights in [-kSnap, 0) are rounding zeros of the vertex
  const unsigned long long snap = abs_bits(kSnap);
  bool ok = true;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    if (!nonneg_bits(f[s]) && abs_bits(f[s]) <= snap) f[s] = 0.0;
    ok = ok && nonneg_bits(f[s]);
  }
  const unsigned long long lim = abs_bits(kAcceptResid);
  // residual with the Vandermonde entries formed again (fewer live registers)
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    double acc = (r == 2 || r == 4) ? -2.0 : 0.0;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      const double vr = r == 0 ? xi[s] : r == 1 ? eta[s] : r == 2 ? xi[s] * xi[s] : r == 3 ? xi[s] * eta[s]
                                                                                           : eta[s] * eta[s];
      acc = fma(vr, f[s], acc);
    }
    ok = ok && abs_bits(acc) <= lim;
  }
#pragma unroll
  for (int s = 0; s < 5; ++s) fo[s] = f[s];
  return ok;
}

// 5-subsets of the candidate ranks 0..7 in the order they are tried
// (increasing sum of ranks, ties in lexicographic order of the sorted rank
// tuple), as bit masks over ranks, with the highest rank each one uses.
struct SubsetOrder {
  unsigned char mask[kSubsets];
  unsigned char top[kSubsets];
};

// Of two 5-subsets with equal rank sums, the one holding the lowest rank at
// which they differ comes first (lexicographic order of the sorted tuples).
constexpr bool tuple_less(int a, int b) {
  for (int bit = 0; bit < 8; ++bit) {
    const int x = (a >> bit) & 1, y = (b >> bit) & 1;
    if (x != y) return x > y;
  }
  return false;
}

constexpr SubsetOrder make_subset_order() {
  SubsetOrder o{};
  int sums[kSubsets] = {};
  int k = 0;
  for (int m = 0; m < 256; ++m) {
    int cnt = 0, sm = 0, top = 0;
    for (int b = 0; b < 8; ++b)
      if ((m >> b) & 1) {
        ++cnt;
        sm += b;
        top = b;
      }
    if (cnt != 5) continue;
    o.mask[k] = (unsigned char)m;
    o.top[k] = (unsigned char)top;
    sums[k] = sm;
    ++k;
  }
  // insertion sort by (sum of ranks, lexicographic rank tuple)
  for (int a = 1; a < kSubsets; ++a)
    for (int b = a; b > 0; --b) {
      const bool less = sums[b] < sums[b - 1] || (sums[b] == sums[b - 1] && tuple_less(o.mask[b], o.mask[b - 1]));
      if (!less) break;
      const unsigned char tm = o.mask[b], tt = o.top[b];
      const int ts = sums[b];
      o.mask[b] = o.mask[b - 1];
      o.top[b] = o.top[b - 1];
      sums[b] = sums[b - 1];
      o.mask[b - 1] = tm;
      o.top[b - 1] = tt;
      sums[b - 1] = ts;
    }
  return o;
}

// read by broadcast: the support loop is warp-uniform
__constant__ SubsetOrder kOrder = make_subset_order();

// One column of the binary32 elimination: pivot = first largest |entry| at
// or below the diagonal (one row swap), then the rows below get
// A[q][c] - (A[q][K] / A[K][K]) A[K][c].  A template per column so that the
// matrix stays in registers.
template <int K>
__device__ __forceinline__ void screen_column(float (&A)[5][6], float (&rcp)[5], float tiny, bool& ok) {
  int p = K;
  float best = fabsf(A[K][K]);
#pragma unroll
  for (int q = K + 1; q < 5; ++q) {
    const float v = fabsf(A[q][K]);
    p = v > best ? q : p;
    best = v > best ? v : best;
  }
  ok = ok && best > tiny;
#pragma unroll
  for (int q = K + 1; q < 5; ++q) {
    const bool sw = q == p;
#pragma unroll
    for (int c = K; c < 6; ++c) {
      const float a = A[K][c], b = A[q][c];
      A[K][c] = sw ? b : a;
      A[q][c] = sw ? a : b;
    }
  }
  rcp[K] = __frcp_rn(A[K][K]);
#pragma unroll
  for (int q = K + 1; q < 5; ++q) {
    const float m = __fmul_rn(A[q][K], rcp[K]);
#pragma unroll
    for (int c = K + 1; c < 6; ++c) A[q][c] = __fsub_rn(A[q][c], __fmul_rn(m, A[K][c]));
  }
}

// Binary32 screen of a support (columns xs, es = float32 xi, eta): Gaussian
// elimination of V_S f = b with every product, reciprocal and difference
// rounded to float32 in a fixed order (back substitution multiplies by the
// pivots' reciprocals) (the oracle repeats it operation by
// operation).  True iff no pivot is at most kScreenPivot times the largest
// |entry| of V_S and every weight is >= -kScreenTol.  (After a failed pivot
// the remaining arithmetic runs on but its result is not used.)
__device__ __forceinline__ bool screen32(const float* xs, const float* es) {
  float A[5][6];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const float a = xs[c], e = es[c];
    A[0][c] = a;
    A[1][c] = e;
    A[2][c] = __fmul_rn(a, a);
    A[3][c] = __fmul_rn(a, e);
    A[4][c] = __fmul_rn(e, e);
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) A[r][5] = (r == 2 || r == 4) ? 2.0f : 0.0f;
  float vmax = 0.0f;
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) vmax = fmaxf(vmax, fabsf(A[r][c]));
  const float tiny = __fmul_rn(kScreenPivot, vmax);
  bool ok = true;
  float rcp[5];
  screen_column<0>(A, rcp, tiny, ok);
  screen_column<1>(A, rcp, tiny, ok);
  screen_column<2>(A, rcp, tiny, ok);
  screen_column<3>(A, rcp, tiny, ok);
  screen_column<4>(A, rcp, tiny, ok);
  float f[5];
#pragma unroll
  for (int k = 4; k >= 0; --k) {
    float acc = A[k][5];
#pragma unroll
    for (int q = k + 1; q < 5; ++q) acc = __fsub_rn(acc, __fmul_rn(A[k][q], f[q]));
    f[k] = __fmul_rn(acc, rcp[k]);
    ok = ok && f[k] >= -kScreenTol;
  }
  return ok;
}

// Per listed particle, what the screen chose: the five particles of the
// support in slot order, the next support index, and whether it was the
// first support tried (stats).
struct ProjSel {
  int j[5];
  int next;    // the next support to screen
  int first;   // the support is the first one tried (stats)
  int solves;  // FP64 solves made so far
};

// Appends v to list (warp-aggregated; the whole warp calls it converged).
__device__ __forceinline__ void warp_append(bool take, int v, int* list, int* count) {
  const unsigned bal = __ballot_sync(0xffffffffu, take);
  int basepos = 0;
  if ((threadIdx.x & 31) == 0 && bal) basepos = atomicAdd(count, __popc(bal));
  basepos = __shfl_sync(0xffffffffu, basepos, 0);
  if (take) list[basepos + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = v;
}

// A rejected particle: to the LP's list (reject_list) or a zero stencil
// with status VRM_LP_NONE.  Called converged by the whole warp.
__device__ __forceinline__ void reject_particle(bool rej, int i, int* cols, double* f, double* fii, uint8_t* status,
                                                int* reject_list, int* reject_count) {
  if (reject_list) {
    warp_append(rej, i, reject_list, reject_count);
  } else if (rej) {
    int* crow = cols + (size_t)i * VRM_STENCIL_W;
    double* frow = f + (size_t)i * VRM_STENCIL_W;
#pragma unroll
    for (int s = 0; s < VRM_STENCIL_W; ++s) {
      crow[s] = -1;
      frow[s] = 0.0;
    }
    fii[i] = 0.0;
    status[i] = VRM_LP_NONE;
  }
}

// Screening: one thread per entry (round 0: every listed particle from the
// first support; later rounds: the particles whose FP64 solve failed, from
// their next support).  The support loop runs warp-uniformly (all lanes step
// through the subset order together until each has a support passing the
// binary32 screen or none is left), so that the subset table in constant
// memory is read by broadcast.  A particle with a passing support goes to
// solve_list, one without any to the rejects.
__global__ void __launch_bounds__(128) k_screen(Consts c, const double* __restrict__ x, const double* __restrict__ y,
                                                const int* __restrict__ list, const int* __restrict__ list_count,
                                                int m_bound, const int* __restrict__ in_list,
                                                const int* __restrict__ in_count, const int* __restrict__ slots,
                                                const float* __restrict__ f0, const int* __restrict__ small,
                                                ProjSel* __restrict__ sel, int budget,
                                                int* __restrict__ solve_list, int* __restrict__ solve_count,
                                                int* __restrict__ pend_list, int* __restrict__ pend_count,
                                                int* __restrict__ cols,
                                                double* __restrict__ f, double* __restrict__ fii,
                                                uint8_t* __restrict__ status, int* __restrict__ reject_list,
                                                int* __restrict__ reject_count, DevStats* __restrict__ ds) {
  const int m = in_list ? *in_count : (list_count ? *list_count : m_bound);
  unsigned long long n_trials = 0;
  int n_rej = 0;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x; base < m; base += stride) {
    const long e = base + threadIdx.x;
    const bool active = e < m;
    int t = 0, i = -1, nc = 0, start = 0, solves = 0;
    int js[kSup], rank[kSup];
    float xf[kSup], ef[kSup];
#pragma unroll
    for (int s = 0; s < kSup; ++s) {
      js[s] = -1;
      rank[s] = kSup;
      xf[s] = ef[s] = 0.0f;
    }
    if (active) {
      t = in_list ? in_list[e] : (int)e;
      start = in_list ? sel[t].next : 0;
      solves = in_list ? sel[t].solves : 0;
      i = list ? list[t] : t;
      const int* slr = slots + (size_t)t * kSlots;
      const float* pr = f0 + (size_t)t * kSlots;
      // candidates: the slots holding a small-neighbourhood particle (at
      // most 8, one per segment), in slot order; the slot row read in
      // 16-byte loads (the scalar reads below then hit the same lines)
      const int4 s0 = reinterpret_cast<const int4*>(small + (size_t)i * 8)[0];
      const int4 s1 = reinterpret_cast<const int4*>(small + (size_t)i * 8)[1];
      unsigned cand = 0;
#pragma unroll
      for (int k4 = 0; k4 < kSlots / 4; ++k4) {
        const int4 a4 = reinterpret_cast<const int4*>(slr)[k4];
        const int jv[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = jv[u];
          const bool in_small = j >= 0 && (j == s0.x || j == s0.y || j == s0.z || j == s0.w || j == s1.x ||
                                           j == s1.y || j == s1.z || j == s1.w);
          if (in_small) cand |= 1u << (4 * k4 + u);
        }
      }
      nc = __popc(cand) < kSup ? __popc(cand) : kSup;
      float cv[kSup];
#pragma unroll
      for (int s = 0; s < kSup; ++s) {
        const int kk = s < nc ? (int)__fns(cand, 0, s + 1) : 0;
        js[s] = s < nc ? slr[kk] : -1;
        cv[s] = s < nc ? pr[kk] : 0.0f;
      }
      const double xi0 = x[i], yi0 = y[i];
#pragma unroll
      for (int s = 0; s < kSup; ++s) {
        const double xi = s < nc ? __dmul_rn(__dsub_rn(x[js[s]], xi0), c.inv_h) : 0.0;
        const double eta = s < nc ? __dmul_rn(__dsub_rn(y[js[s]], yi0), c.inv_h) : 0.0;
        xf[s] = __double2float_rn(xi);
        ef[s] = __double2float_rn(eta);
      }
      // rank of every candidate (larger proposal first, ties to the lower slot)
#pragma unroll
      for (int s = 0; s < kSup; ++s) {
        int r = 0;
#pragma unroll
        for (int q = 0; q < kSup; ++q) r += (q < nc && q != s) && (cv[q] > cv[s] || (cv[q] == cv[s] && q < s));
        rank[s] = s < nc ? r : kSup;
      }
    }
    bool done = !active || nc < 5, have = false, pend = false;
    unsigned pm = 0;
    int trials = 0, u_pass = 0;
    for (int u = 0; u < kSubsets; ++u) {
      if (__all_sync(0xffffffffu, done)) break;
      if (done || u < start || kOrder.top[u] >= nc) continue;
      if (trials == budget) {  // this round's screens are spent: go on next round from u
        done = pend = true;
        u_pass = u - 1;
        continue;
      }
      ++trials;
      const unsigned rm = kOrder.mask[u];
      unsigned um = 0;  // the support as positions (slot order)
#pragma unroll
      for (int s = 0; s < kSup; ++s) um |= ((rm >> (rank[s] & 7)) & (rank[s] < kSup ? 1u : 0u)) << s;
      float xs[5], es[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int pos = (int)__fns(um, 0, q + 1);
        float a = xf[0], b = ef[0];
#pragma unroll
        for (int s = 1; s < kSup; ++s) {
          a = pos == s ? xf[s] : a;
          b = pos == s ? ef[s] : b;
        }
        xs[q] = a;
        es[q] = b;
      }
      if (screen32(xs, es)) {
        have = done = true;
        pm = um;
        u_pass = u;
      }
    }
    if (have || pend) {
      ProjSel o;
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int pos = (int)__fns(pm, 0, q + 1);
        int jj = js[0];
#pragma unroll
        for (int s = 1; s < kSup; ++s) jj = pos == s ? js[s] : jj;
        o.j[q] = jj;
      }
      o.next = u_pass + 1;
      o.first = have && !in_list && trials == 1;
      o.solves = solves;
      sel[t] = o;
    }
    n_trials += trials;
    const bool rej = active && !have && !pend;
    n_rej += rej;
    warp_append(have, t, solve_list, solve_count);
    warp_append(pend, t, pend_list, pend_count);
    reject_particle(rej, i, cols, f, fii, status, reject_list, reject_count);
  }
  n_rej = __reduce_add_sync(0xffffffffu, n_rej);
  n_trials = __reduce_add_sync(0xffffffffu, (unsigned)n_trials);
  if ((threadIdx.x & 31) == 0) {
    if (n_rej) atomicAdd(&ds->learned_rejected, n_rej);
    if (n_trials) atomicAdd(&ds->learned_screens, n_trials);
  }
}

// FP64 solve of the screened supports: one thread per entry of solve_list,
// all lanes on the same work (the FP64 pipe runs full warps).  Accepted
// stencils are written like the LP's (nonzero weights in slot order,
// f~_ii = -sum in that order, status VRM_LP_LEARNED); a failed solve sends
// the particle to retry_list (the next round screens on from its next
// support), after its kMaxSolves-th solve or in the last round to the
// rejects.
__global__ void __launch_bounds__(128) k_solve(Consts c, const double* __restrict__ x, const double* __restrict__ y,
                                               const int* __restrict__ list, const int* __restrict__ solve_list,
                                               const int* __restrict__ solve_count, ProjSel* __restrict__ sel,
                                               int* __restrict__ retry_list, int* __restrict__ retry_count,
                                               bool last_round, int* __restrict__ cols, double* __restrict__ f,
                                               double* __restrict__ fii, uint8_t* __restrict__ status,
                                               int* __restrict__ reject_list, int* __restrict__ reject_count,
                                               DevStats* __restrict__ ds, const double* __restrict__ dt_dev, double nu) {
  const int m = *solve_count;
  const double nu_dt = dt_dev ? nu * *dt_dev : 0.0;
  const double inv_h2 = 1.0 / (c.h * c.h);
  int n_ok = 0, n_rej = 0, n_square = 0;
  double st_ratio = 0.0;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x; base < m; base += stride) {
    const long e = base + threadIdx.x;
    const bool active = e < m;
    bool ok = false;
    int t = 0, i = -1;
    ProjSel o{};
    if (active) {
      t = solve_list[e];
      i = list ? list[t] : t;
      o = sel[t];
      const double xi0 = x[i], yi0 = y[i];
      double x5[5], e5[5], f5[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        x5[q] = __dmul_rn(__dsub_rn(x[o.j[q]], xi0), c.inv_h);
        e5[q] = __dmul_rn(__dsub_rn(y[o.j[q]], yi0), c.inv_h);
      }
      ok = square_stencil(x5, e5, f5);
      if (!ok) sel[t].solves = o.solves + 1;
      if (ok) {
        int* crow = cols + (size_t)i * VRM_STENCIL_W;
        double* frow = f + (size_t)i * VRM_STENCIL_W;
        double sum = 0.0;
        int w = 0;
#pragma unroll
        for (int q = 0; q < 5; ++q)
          if (abs_bits(f5[q]) != 0) {
            crow[w] = o.j[q];
            frow[w] = f5[q];
            sum = __dadd_rn(sum, f5[q]);
            ++w;
          }
        for (; w < VRM_STENCIL_W; ++w) {
          crow[w] = -1;
          frow[w] = 0.0;
        }
        fii[i] = -sum;
        status[i] = VRM_LP_LEARNED;
        const double qr = __dmul_rn(__dmul_rn(nu_dt, sum), inv_h2);
        st_ratio = qr > st_ratio ? qr : st_ratio;
        ++n_ok;
        n_square += o.first;
      }
    }
    const bool failed = active && !ok;
    const bool rej = failed && (last_round || o.solves + 1 >= kMaxSolves);
    n_rej += rej;
    warp_append(failed && !rej, t, retry_list, retry_count);
    reject_particle(rej, i, cols, f, fii, status, reject_list, reject_count);
  }
  n_ok = __reduce_add_sync(0xffffffffu, n_ok);
  n_rej = __reduce_add_sync(0xffffffffu, n_rej);
  n_square = __reduce_add_sync(0xffffffffu, n_square);
  unsigned long long rb = (unsigned long long)__double_as_longlong(st_ratio);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t2 = __shfl_xor_sync(0xffffffffu, rb, o);
    rb = t2 > rb ? t2 : rb;
  }
  if ((threadIdx.x & 31) == 0) {
    if (n_ok) atomicAdd(&ds->learned_ok, n_ok);
    if (n_rej) atomicAdd(&ds->learned_rejected, n_rej);
    if (n_square) atomicAdd(&ds->learned_square, n_square);
    if (rb) atomicMax(&ds->max_dt_ratio_bits, rb);
  }
}

// Training targets: T[t][k] = f~ of the LP stencil of particle list[t] at
// the particle in slot k (0 where the stencil has no weight).
__global__ void k_targets(const int* __restrict__ list, int m, const int* __restrict__ slots,
                          const int* __restrict__ cols, const double* __restrict__ f, float* __restrict__ T) {
  const long total = (long)m * kSlots;
  for (long u = (long)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += (long)gridDim.x * blockDim.x) {
    const long t = u / kSlots;
    const int i = list[t];
    const int j = slots[u];
    float v = 0.0f;
    if (j >= 0) {
#pragma unroll
      for (int s = 0; s < VRM_STENCIL_W; ++s)
        if (cols[(size_t)i * VRM_STENCIL_W + s] == j) v = (float)f[(size_t)i * VRM_STENCIL_W + s];
    }
    T[u] = v;
  }
}

cudaError_t learned_features(const Consts& c, const double* x, const double* y, int n_bound, const int* n_dev,
                             float2* xyf, const int* list, const int* list_count, int m_bound, const int* nbr_count,
                             const int* nbr_idx, __nv_bfloat16* X, int* slots, cudaStream_t s) {
  if (m_bound <= 0 || n_bound <= 0) return cudaSuccess;
  long mb = ((long)n_bound + 255) / 256;
  if (mb > 8L * sm_count()) mb = 8L * sm_count();
  k_mirror<<<(int)mb, 256, 0, s>>>(x, y, n_bound, n_dev, xyf);
  note_launch();
  long blocks = ((long)m_bound * 32 + 255) / 256;
  if (blocks > 16L * sm_count()) blocks = 16L * sm_count();
  k_features<<<(int)blocks, 256, 0, s>>>(c, xyf, list, list_count, m_bound, nbr_count, nbr_idx, X, slots);
  note_launch();
  return cudaGetLastError();
}

cudaError_t proj_alloc(ProjScratch* p, int cap) {
  proj_free(p);
  cudaError_t e = cudaMalloc(&p->sel, sizeof(ProjSel) * (size_t)cap);
  if (e == cudaSuccess) e = cudaMalloc(&p->list_s, sizeof(int) * (size_t)cap);
  if (e == cudaSuccess) e = cudaMalloc(&p->list_r, sizeof(int) * (size_t)cap);
  if (e == cudaSuccess) e = cudaMalloc(&p->list_p, sizeof(int) * (size_t)cap);
  if (e == cudaSuccess) e = cudaMalloc(&p->counts, sizeof(int) * 2 * kProjRounds);
  if (e != cudaSuccess) {
    proj_free(p);
    return e;
  }
  p->cap = cap;
  return cudaSuccess;
}

void proj_free(ProjScratch* p) {
  cudaFree(p->sel);
  cudaFree(p->list_s);
  cudaFree(p->list_r);
  cudaFree(p->list_p);
  cudaFree(p->counts);
  *p = ProjScratch{};
}

// Rounds of (screen, FP64 solve).  Round r screens at most kBudget[r]
// supports per particle: the particles still searching when their budget is
// spent, and those whose FP64 solve failed, form the next round's list
// (compacted, so later rounds run full warps on the few that need many
// screens), each from its next support.  The budgets grow to the whole
// subset order and a particle makes at most kMaxSolves FP64 solves, so
// kProjRounds rounds cover every particle's full search.  Fixed launches
// (graph-capturable), the lists and their sizes on the device.
cudaError_t learned_project(const Consts& c, const double* x, const double* y, const int* list, const int* list_count,
                            int m_bound, const int* slots, const float* f0, const int* small, int* cols, double* f,
                            double* fii, uint8_t* status, int* reject_list, int* reject_count, DevStats* ds,
                            const double* dt_dev, double nu, ProjScratch* ps, cudaStream_t s) {
  static const int kBudget[kProjRounds] = {2, 4, 8, kSubsets, kSubsets, kSubsets, kSubsets};
  if (m_bound <= 0) return cudaSuccess;
  if (!ps || ps->cap < m_bound) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(ps->counts, 0, sizeof(int) * 2 * kProjRounds, s);
  if (e != cudaSuccess) return e;
  int blocks = (m_bound + 127) / 128;
  if (blocks > 16 * sm_count()) blocks = 16 * sm_count();
  int* lists[2] = {ps->list_r, ps->list_p};
  for (int r = 0; r < kProjRounds; ++r) {
    int* solve_count = ps->counts + 2 * r;
    int* next_count = ps->counts + 2 * r + 1;
    const int* in_list = r == 0 ? nullptr : lists[(r - 1) & 1];
    const int* in_count = r == 0 ? nullptr : ps->counts + 2 * r - 1;
    int* next_list = lists[r & 1];
    k_screen<<<blocks, 128, 0, s>>>(c, x, y, list, list_count, m_bound, in_list, in_count, slots, f0, small,
                                    reinterpret_cast<ProjSel*>(ps->sel), kBudget[r], ps->list_s, solve_count,
                                    next_list, next_count, cols, f, fii, status, reject_list, reject_count, ds);
    note_launch();
    k_solve<<<blocks, 128, 0, s>>>(c, x, y, list, ps->list_s, solve_count, reinterpret_cast<ProjSel*>(ps->sel),
                                   next_list, next_count, r == kProjRounds - 1, cols, f, fii, status, reject_list,
                                   reject_count, ds, dt_dev, nu);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t learned_targets(const int* list, int m, const int* slots, const int* cols, const double* f, float* T,
                            cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  long blocks = ((long)m * kSlots + 255) / 256;
  if (blocks > 16L * sm_count()) blocks = 16L * sm_count();
  k_targets<<<(int)blocks, 256, 0, s>>>(list, m, slots, cols, f, T);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
