// The learned weight proposal around the network (vrm_mlp.cu): input rows
// from the neighbourhoods, and the exact correction of the proposals onto the
// moment conditions with the acceptance test.  Rejected particles go to the
// LP of Sec. 4.1 (vrm_lp.cu), which stays the arbiter of validity.
//
// Slots: the annulus neighbours of particle i (Eq. neighbourhood) ordered by
// (45-degree segment of Sec. 4.2, squared distance, index), at most 32.
// Input row: xi_x of the slots, xi_y, mask, 32 zeros (bf16), xi = (x_j -
// x_i) / h (Eq. momcondmv scaling) rounded to fp32 and then bf16.
//
// First the square system V_5 f = b on the five slots with the largest
// proposals (the network's choice of basis; Gaussian elimination with partial
// pivoting, FP64): its solution is accepted under the test below.  Otherwise,
// correction (FP64): S = the up to 8 slots with the largest positive
// proposal (ties to the lower slot), in slot order; with V_S the rows (1,0)
// (0,1) (2,0) (1,1) (0,2) of Eq. momcondmv at S and b = (0, 0, 2, 0, 2)
// (Eqs. cond_two, cond_alpha),
//   f_S = f0_S + V_S^T (V_S V_S^T)^{-1} (b - V_S f0_S),
// the least change of f0_S that meets V_S f = b (Cholesky of the 5 x 5
// Gram matrix).  Accepted iff |S| >= 5, the Gram matrix is well conditioned,
// every f_j >= 0 (Sec. 3.1's non-negativity) and |V_S f_S - b|_inf <= 1e-12.
// While a corrected weight is negative and |S| > 5, the position with the
// smallest corrected weight (ties: the later one) leaves S and the original
// proposal is corrected again on the rest (at most three times).
#include <cuda_bf16.h>

#include "vrm_internal.cuh"

namespace vrm {

namespace {

constexpr int kSlots = 32;
constexpr int kRow = 128;  // input row stride
constexpr int kSup = 8;    // support cap (= stencil width)
constexpr double kAcceptResid = 1e-12;
constexpr double kGramPivot = 1e-10;  // relative to the largest diagonal entry
constexpr int kMaxDrops = 3;          // support refinements (8 -> 5 slots)

}  // namespace

// One warp per listed particle: lane l takes neighbour l of the row, the
// warp sorts the keys (segment, squared distance, index) and lane l writes
// slot l.  Only x_j - x_i is FP64; it is rounded to fp32, and the segment,
// the squared distance (products and sum rounded separately) and xi =
// dx * fp32(1/h) are fp32 (the network's input precision).  d2 >= 0 is
// compared through its bit pattern, so the sort runs on the integer pipes.
__global__ void k_features(Consts c, const double* __restrict__ x, const double* __restrict__ y,
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
    unsigned long long key = ~0ull;  // segment (8 = empty) << 32 | d2 bits
    int j = INT_MAX;
    float fdx = 0.0f, fdy = 0.0f;
    if (lane < K) {
      j = nbr_idx[(size_t)i * c.k_cap + lane];
      fdx = __double2float_rn(__dsub_rn(x[j], x[i]));
      fdy = __double2float_rn(__dsub_rn(y[j], y[i]));
      const float d2 = dist2f(fdx, fdy);
      key = ((unsigned long long)segment_of(fdx, fdy) << 32) | __float_as_uint(d2);
    }
    int src = lane;
    for (int size = 2; size <= 32; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, stride);
        const int oj = __shfl_xor_sync(0xffffffffu, j, stride);
        const int os = __shfl_xor_sync(0xffffffffu, src, stride);
        const bool up = ((lane & size) == 0);
        const bool lower = ((lane & stride) == 0);
        const bool other_less = ok < key || (ok == key && oj < j);
        const bool same = ok == key && oj == j;
        const bool take = (lower == up) ? other_less : (!other_less && !same);
        if (take) {
          key = ok;
          j = oj;
          src = os;
        }
      }
    }
    const bool valid = lane < K;
    const float sdx = __shfl_sync(0xffffffffu, fdx, src);
    const float sdy = __shfl_sync(0xffffffffu, fdy, src);
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

// The square system V f = b on five neighbours (columns xi, eta) by Gaussian
// elimination with partial pivoting (first largest |pivot|), FP64.  Returns
// false when a pivot is at most 1e-12 of the largest |entry| or the result
// is not a non-negative solution with residual <= kAcceptResid.
__device__ __forceinline__ bool square_stencil(const double* xi, const double* eta, double* fo) {
  double A[5][6], V[5][5];
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    V[0][s] = xi[s];
    V[1][s] = eta[s];
    V[2][s] = xi[s] * xi[s];
    V[3][s] = xi[s] * eta[s];
    V[4][s] = eta[s] * eta[s];
  }
  unsigned long long vmax = 0;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      A[r][s] = V[r][s];
      const unsigned long long ab = abs_bits(V[r][s]);
      vmax = ab > vmax ? ab : vmax;
    }
    A[r][5] = (r == 2 || r == 4) ? 2.0 : 0.0;
  }
  const unsigned long long tiny = abs_bits(1e-12 * __longlong_as_double((long long)vmax));
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
      if (r == p) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const double tmp = A[k][q];
          A[k][q] = A[r][q];
          A[r][q] = tmp;
        }
      }
    }
    const double inv = 1.0 / A[k][k];
#pragma unroll
    for (int r = k + 1; r < 5; ++r) {
      const double mlt = A[r][k] * inv;
#pragma unroll
      for (int q = k; q < 6; ++q) A[r][q] = fma(-mlt, A[k][q], A[r][q]);
    }
  }
  double f[5];
#pragma unroll
  for (int k = 4; k >= 0; --k) {
    double acc = A[k][5];
#pragma unroll
    for (int q = k + 1; q < 5; ++q) acc = fma(-A[k][q], f[q], acc);
    f[k] = acc / A[k][k];
  }
  bool ok = true;
#pragma unroll
  for (int s = 0; s < 5; ++s) ok = ok && nonneg_bits(f[s]);
  const unsigned long long lim = abs_bits(kAcceptResid);
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    double acc = (r == 2 || r == 4) ? -2.0 : 0.0;
#pragma unroll
    for (int s = 0; s < 5; ++s) acc = fma(V[r][s], f[s], acc);
    ok = ok && abs_bits(acc) <= lim;
  }
#pragma unroll
  for (int s = 0; s < 5; ++s) fo[s] = f[s];
  return ok;
}

// One thread per listed particle.  Accepted stencils are written like the
// LP's (columns in slot order, f~, f~_ii = -sum in that order, status
// VRM_LP_LEARNED); rejected particles are appended to reject_list (if given)
// or marked VRM_LP_NONE.
__global__ void __launch_bounds__(128) k_project(Consts c, const double* __restrict__ x, const double* __restrict__ y,
                                                 const int* __restrict__ list, const int* __restrict__ list_count,
                                                 int m_bound, const int* __restrict__ slots, const float* __restrict__ f0,
                                                 int* __restrict__ cols, double* __restrict__ f,
                                                 double* __restrict__ fii, uint8_t* __restrict__ status,
                                                 int* __restrict__ reject_list, int* __restrict__ reject_count,
                                                 DevStats* __restrict__ ds, const double* __restrict__ dt_dev,
                                                 double nu) {
  const int m = list_count ? *list_count : m_bound;
  const double nu_dt = dt_dev ? nu * *dt_dev : 0.0;
  const double inv_h2 = 1.0 / (c.h * c.h);
  int n_ok = 0, n_rej = 0, n_square = 0;
  double st_ratio = 0.0;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x; base < m; base += stride) {
    const long t = base + threadIdx.x;
    bool accepted = false, active = t < m;
    int i = -1;
    if (active) {
      i = list ? list[t] : (int)t;
      const float* p = f0 + (size_t)t * kSlots;
      const int* sl = slots + (size_t)t * kSlots;
      // support: rank each positive valid slot among the positive valid ones
      float v[kSlots];
      unsigned ok_mask = 0;
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        v[k] = p[k];
        if (sl[k] >= 0 && v[k] > 0.0f) ok_mask |= 1u << k;
      }
      unsigned sup = 0, sup5 = 0;
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        if (!((ok_mask >> k) & 1u)) continue;
        int rank = 0;
#pragma unroll
        for (int q = 0; q < kSlots; ++q)
          rank += ((ok_mask >> q) & 1u) && (v[q] > v[k] || (v[q] == v[k] && q < k));
        if (rank < kSup) sup |= 1u << k;
        if (rank < 5) sup5 |= 1u << k;
      }
      const int ns = __popc(sup);
      // the network's basis alone: the square system on the top five slots
      if (__popc(sup5) == 5) {
        int j5[5];
        double xi5[5], eta5[5], f5[5];
        int q5 = 0;
        const double xi0 = x[i], yi0 = y[i];
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
          if (((sup5 >> k) & 1u) && q5 < 5) {
            j5[q5] = sl[k];
            ++q5;
          }
        }
#pragma unroll
        for (int s2 = 0; s2 < 5; ++s2) {
          xi5[s2] = __dmul_rn(__dsub_rn(x[j5[s2]], xi0), c.inv_h);
          eta5[s2] = __dmul_rn(__dsub_rn(y[j5[s2]], yi0), c.inv_h);
        }
        if (square_stencil(xi5, eta5, f5)) {
          accepted = true;
          int* crow = cols + (size_t)i * VRM_STENCIL_W;
          double* frow = f + (size_t)i * VRM_STENCIL_W;
          double sum = 0.0;
#pragma unroll
          for (int s2 = 0; s2 < VRM_STENCIL_W; ++s2) {
            crow[s2] = s2 < 5 ? j5[s2] : -1;
            frow[s2] = s2 < 5 ? f5[s2] : 0.0;
            if (s2 < 5) sum = __dadd_rn(sum, f5[s2]);
          }
          fii[i] = -sum;
          status[i] = VRM_LP_LEARNED;
          const double qr = __dmul_rn(__dmul_rn(nu_dt, sum), inv_h2);
          st_ratio = qr > st_ratio ? qr : st_ratio;
          ++n_square;
        }
      }
      if (!accepted && ns >= 5) {

        int js[kSup];
        double xi[kSup], eta[kSup], f0s[kSup], fs[kSup];
        int q = 0;
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
          if (((sup >> k) & 1u) && q < kSup) {
            js[q] = sl[k];
            f0s[q] = (double)v[k];
            ++q;
          }
        }
        const double xi0 = x[i], yi0 = y[i];
#pragma unroll
        for (int s2 = 0; s2 < kSup; ++s2) {
          if (s2 < ns) {
            xi[s2] = __dmul_rn(__dsub_rn(x[js[s2]], xi0), c.inv_h);
            eta[s2] = __dmul_rn(__dsub_rn(y[js[s2]], yi0), c.inv_h);
          } else {
            js[s2] = -1;
            xi[s2] = eta[s2] = f0s[s2] = 0.0;
          }
        }
        const double b[5] = {0.0, 0.0, 2.0, 0.0, 2.0};
        unsigned act = (1u << ns) - 1u;  // support positions still in S
        for (int attempt = 0; attempt <= kMaxDrops; ++attempt) {
          const int na = __popc(act);
          if (na < 5) break;
          double V[5][kSup];
#pragma unroll
          for (int s2 = 0; s2 < kSup; ++s2) {
            const bool on = (act >> s2) & 1u;
            V[0][s2] = on ? xi[s2] : 0.0;
            V[1][s2] = on ? eta[s2] : 0.0;
            V[2][s2] = on ? xi[s2] * xi[s2] : 0.0;
            V[3][s2] = on ? xi[s2] * eta[s2] : 0.0;
            V[4][s2] = on ? eta[s2] * eta[s2] : 0.0;
            fs[s2] = on ? f0s[s2] : 0.0;
          }
          // Gram matrix G = V V^T (lower triangle) and r = b - V f0
          double G[5][5], r[5];
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            double acc = 0.0;
#pragma unroll
            for (int s2 = 0; s2 < kSup; ++s2) acc = fma(V[a][s2], fs[s2], acc);
            r[a] = b[a] - acc;
#pragma unroll
            for (int e = 0; e <= a; ++e) {
              double g = 0.0;
#pragma unroll
              for (int s2 = 0; s2 < kSup; ++s2) g = fma(V[a][s2], V[e][s2], g);
              G[a][e] = g;
            }
          }
          // Cholesky G = L L^T in place (lower triangle), pivots checked
          double gmax = 0.0;
#pragma unroll
          for (int a = 0; a < 5; ++a) gmax = G[a][a] > gmax ? G[a][a] : gmax;
          bool spd = true;
          double dinv[5];
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            double d = G[a][a];
#pragma unroll
            for (int e = 0; e < a; ++e) d = fma(-G[a][e], G[a][e], d);
            spd = spd && d > kGramPivot * gmax;
            const double l = sqrt(d > 0.0 ? d : 1.0);
            G[a][a] = l;
            dinv[a] = 1.0 / l;
#pragma unroll
            for (int q2 = a + 1; q2 < 5; ++q2) {
              double s3 = G[q2][a];
#pragma unroll
              for (int e = 0; e < a; ++e) s3 = fma(-G[q2][e], G[a][e], s3);
              G[q2][a] = s3 * dinv[a];
            }
          }
          if (!spd) break;  // nearly dependent rows: reject
          // solve L z = r, L^T w = z
          double w[5];
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            double s3 = r[a];
#pragma unroll
            for (int e = 0; e < a; ++e) s3 = fma(-G[a][e], w[e], s3);
            w[a] = s3 * dinv[a];
          }
#pragma unroll
          for (int a = 4; a >= 0; --a) {
            double s3 = w[a];
#pragma unroll
            for (int e = a + 1; e < 5; ++e) s3 = fma(-G[e][a], w[e], s3);
            w[a] = s3 * dinv[a];
          }
          // f = f0 + V^T w on S, then the sign test and the residual in FP64
          bool nonneg = true;
#pragma unroll
          for (int s2 = 0; s2 < kSup; ++s2) {
            double acc = fs[s2];
#pragma unroll
            for (int a = 0; a < 5; ++a) acc = fma(V[a][s2], w[a], acc);
            const bool on = (act >> s2) & 1u;
            fs[s2] = on ? acc : 0.0;
            nonneg = nonneg && fs[s2] >= 0.0;
          }
          double rmax = 0.0;
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            double acc = 0.0;
#pragma unroll
            for (int s2 = 0; s2 < kSup; ++s2) acc = fma(V[a][s2], fs[s2], acc);
            const double e2 = fabs(acc - b[a]);
            rmax = e2 > rmax ? e2 : rmax;
          }
          if (nonneg && rmax <= kAcceptResid) {
            accepted = true;
            int* crow = cols + (size_t)i * VRM_STENCIL_W;
            double* frow = f + (size_t)i * VRM_STENCIL_W;
            double sum = 0.0;
            int o = 0;
#pragma unroll
            for (int s2 = 0; s2 < kSup; ++s2) {
              if ((act >> s2) & 1u) {
                crow[o] = js[s2];
                frow[o] = fs[s2];
                sum = __dadd_rn(sum, fs[s2]);
                ++o;
              }
            }
            for (; o < VRM_STENCIL_W; ++o) {
              crow[o] = -1;
              frow[o] = 0.0;
            }
            fii[i] = -sum;
            status[i] = VRM_LP_LEARNED;
            const double qr = __dmul_rn(__dmul_rn(nu_dt, sum), inv_h2);
            st_ratio = qr > st_ratio ? qr : st_ratio;
            break;
          }
          if (na == 5) break;
          // drop the smallest corrected weight (ties: the later position)
          int worst = 0;
          double wv = 1e308;
#pragma unroll
          for (int s2 = 0; s2 < kSup; ++s2)
            if (((act >> s2) & 1u) && fs[s2] <= wv) {
              wv = fs[s2];
              worst = s2;
            }
          act &= ~(1u << worst);
        }
      }
      if (accepted) {
        ++n_ok;
      } else {
        ++n_rej;
        if (!reject_list) {
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
    }
    // warp-aggregated append of the rejected particles (the warp is converged here)
    if (reject_list) {
      const bool rej = active && !accepted;
      const unsigned bal = __ballot_sync(0xffffffffu, rej);
      int basepos = 0;
      if ((threadIdx.x & 31) == 0 && bal) basepos = atomicAdd(reject_count, __popc(bal));
      basepos = __shfl_sync(0xffffffffu, basepos, 0);
      if (rej) reject_list[basepos + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u))] = i;
    }
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

cudaError_t learned_features(const Consts& c, const double* x, const double* y, const int* list, const int* list_count,
                             int m_bound, const int* nbr_count, const int* nbr_idx, __nv_bfloat16* X, int* slots,
                             cudaStream_t s) {
  if (m_bound <= 0) return cudaSuccess;
  long blocks = ((long)m_bound * 32 + 255) / 256;
  if (blocks > 16L * sm_count()) blocks = 16L * sm_count();
  k_features<<<(int)blocks, 256, 0, s>>>(c, x, y, list, list_count, m_bound, nbr_count, nbr_idx, X, slots);
  note_launch();
  return cudaGetLastError();
}

cudaError_t learned_project(const Consts& c, const double* x, const double* y, const int* list, const int* list_count,
                            int m_bound, const int* slots, const float* f0, int* cols, double* f, double* fii,
                            uint8_t* status, int* reject_list, int* reject_count, DevStats* ds, const double* dt_dev,
                            double nu, cudaStream_t s) {
  if (m_bound <= 0) return cudaSuccess;
  int blocks = (m_bound + 127) / 128;
  if (blocks > 16 * sm_count()) blocks = 16 * sm_count();
  k_project<<<blocks, 128, 0, s>>>(c, x, y, list, list_count, m_bound, slots, f0, cols, f, fii, status, reject_list,
                                   reject_count, ds, dt_dev, nu);
  note_launch();
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
