// Growth control (Sec. 3.5, Eq. reduced_bound) as an exact radix select.
//
// Particles are left out of diffusion, smallest |Gamma_i| first (ties by
// index), while the left-out l1 norm stays within C_diff h^{n+2} ||Gamma||_1.
// The choice must not depend on summation order, so the sums are exact
// integers: q_i = floor(|Gamma_i| 2^(96-E)) with max|Gamma| < 2^E, summed as
// three 32-bit limbs in 64-bit counters (no carries lost for n < 2^31).
//
// Instead of sorting, eight passes select the threshold key T (the bit
// pattern of |Gamma|, which orders like the value for non-negative doubles)
// one byte at a time: each pass histograms the exact q-sums of the particles
// whose key matches the bytes chosen so far, and one thread picks the first
// byte at which the running sum crosses the remaining budget.  Particles with
// key == T are tied; the first k_tie of them by index stay out, found with a
// scan of the tie flags.
#include "vrm_internal.cuh"

namespace vrm {

__device__ __forceinline__ u128 dbl_floor_to_u128(double t) {
  const double two64 = 18446744073709551616.0;
  unsigned long long hi = __double2ull_rz(__dmul_rn(t, 5.421010862427522170e-20));  // t * 2^-64, exact
  double rem = __dsub_rn(t, __dmul_rn(__ull2double_rn(hi), two64));
  unsigned long long lo = __double2ull_rz(rem);
  return ((u128)hi << 64) | (u128)lo;
}

__device__ __forceinline__ double u128_to_dbl(u128 s) {
  const double two64 = 18446744073709551616.0;
  unsigned long long hi = (unsigned long long)(s >> 64), lo = (unsigned long long)s;
  return __dadd_rn(__dmul_rn(__ull2double_rn(hi), two64), __ull2double_rn(lo));
}

__device__ __forceinline__ u128 limbs_value(const unsigned long long* h) {
  return (u128)h[0] + ((u128)h[1] << 32) + ((u128)h[2] << 64);
}

__global__ void k_reduce_init(ReduceState* st) {
  int t = threadIdx.x;
  for (int b = t; b < 256; b += blockDim.x) st->hist[b][0] = st->hist[b][1] = st->hist[b][2] = st->hist[b][3] = 0;
  if (t == 0) {
    st->amax_bits = 0;
    st->E = 0;
    st->done = 0;
    st->prefix = 0;
    st->tau_lo = st->tau_hi = 0;
    st->T = 0;
    st->k_tie = 0;
    st->all_out = 0;
  }
}

__global__ void k_absmax(const double* __restrict__ g, int n, ReduceState* __restrict__ st, DevStats* ds) {
  unsigned long long m = 0;
  int bad = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double v = g[i];
    if (!isfinite(v)) {
      bad = 1;
      continue;
    }
    unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicMax(&st->amax_bits, m);
    if (bad) atomicOr(&ds->nonfinite, 1);
  }
}

__global__ void k_reduce_prepare(ReduceState* st, double c_bound) {
  if (st->amax_bits == 0 || !(c_bound < 1.0)) {
    // no circulation, or a bound of at least ||Gamma||_1: nothing diffuses
    st->all_out = 1;
    st->done = 1;
    return;
  }
  int E;
  frexp(__longlong_as_double((long long)st->amax_bits), &E);
  st->E = E;
}

__global__ void k_reduce_hist(const double* __restrict__ g, int n, ReduceState* __restrict__ st, int pass) {
  __shared__ unsigned long long h[256][4];
  for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b][0] = h[b][1] = h[b][2] = h[b][3] = 0;
  __syncthreads();
  const int done = st->done;
  const int E = st->E;
  const unsigned long long prefix = st->prefix;
  if (!done) {
    const int shift = 56 - 8 * pass;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
      double a = fabs(g[i]);
      unsigned long long key = (unsigned long long)__double_as_longlong(a);
      if (pass > 0 && (key >> (shift + 8)) != prefix) continue;
      int d = (int)((key >> shift) & 0xFF);
      u128 q = dbl_floor_to_u128(ldexp(a, 96 - E));
      unsigned long long l0 = (unsigned long long)(q & 0xFFFFFFFFull);
      unsigned long long l1 = (unsigned long long)((q >> 32) & 0xFFFFFFFFull);
      unsigned long long l2 = (unsigned long long)(q >> 64);
      if (l0) atomicAdd(&h[d][0], l0);
      if (l1) atomicAdd(&h[d][1], l1);
      if (l2) atomicAdd(&h[d][2], l2);
      atomicAdd(&h[d][3], 1ull);
    }
  }
  __syncthreads();
  if (!done)
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
      if (h[b][3]) {
        atomicAdd(&st->hist[b][0], h[b][0]);
        atomicAdd(&st->hist[b][1], h[b][1]);
        atomicAdd(&st->hist[b][2], h[b][2]);
        atomicAdd(&st->hist[b][3], h[b][3]);
      }
}

__global__ void k_reduce_choose(ReduceState* st, double c_bound, int pass) {
  if (threadIdx.x != 0) return;
  if (st->done) return;
  u128 tau;
  if (pass == 0) {
    u128 S = 0;
    for (int b = 0; b < 256; ++b) S += limbs_value(st->hist[b]);
    tau = dbl_floor_to_u128(__dmul_rn(c_bound, u128_to_dbl(S)));
    if (S <= tau) {
      st->all_out = 1;
      st->done = 1;
      return;
    }
  } else {
    tau = ((u128)st->tau_hi << 64) | (u128)st->tau_lo;
  }
  u128 cum = 0;
  int bsel = 255;
  for (int b = 0; b < 256; ++b) {
    u128 sb = limbs_value(st->hist[b]);
    if (cum + sb > tau) {
      bsel = b;
      break;
    }
    cum += sb;
  }
  tau -= cum;
  unsigned long long count_sel = st->hist[bsel][3];
  st->prefix = (st->prefix << 8) | (unsigned long long)bsel;
  st->tau_lo = (unsigned long long)tau;
  st->tau_hi = (unsigned long long)(tau >> 64);
  for (int b = 0; b < 256; ++b) st->hist[b][0] = st->hist[b][1] = st->hist[b][2] = st->hist[b][3] = 0;
  if (pass == 7) {
    // all particles with key == T have the same q_T > 0; the first k_tie by
    // index fit: k_tie = max k <= count with k q_T <= tau (binary search)
    unsigned long long T = st->prefix;
    u128 qT = dbl_floor_to_u128(ldexp(__longlong_as_double((long long)T), 96 - st->E));
    unsigned long long lo = 0, hi = count_sel;
    while (lo < hi) {
      unsigned long long mid = (lo + hi + 1) / 2;
      if ((u128)mid * qT <= tau) lo = mid;
      else hi = mid - 1;
    }
    st->T = T;
    st->k_tie = (int)lo;
    st->done = 1;
  }
}

__global__ void k_reduce_mark(const double* __restrict__ g, int n, const ReduceState* __restrict__ st,
                              uint8_t* __restrict__ diffused, uint8_t* __restrict__ tie_flag) {
  const int all_out = st->all_out;
  const unsigned long long T = st->T;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    unsigned long long key = (unsigned long long)__double_as_longlong(fabs(g[i]));
    uint8_t d = 0, t = 0;
    if (!all_out) {
      d = key > T;
      t = key == T;
    }
    diffused[i] = d;
    tie_flag[i] = t;
  }
}

__global__ void k_reduce_ties(int n, const ReduceState* __restrict__ st, const uint8_t* __restrict__ tie_flag,
                              const int* __restrict__ tie_rank, uint8_t* __restrict__ diffused) {
  const int k_tie = st->k_tie;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (tie_flag[i] && tie_rank[i] >= k_tie) diffused[i] = 1;
}

cudaError_t reduce_select(const double* gamma, int n, double c_bound, uint8_t* diffused, ReduceState* st,
                          uint8_t* tie_flag, int* tie_rank, int* scan_tmp, DevStats* ds, cudaStream_t s) {
  int blocks = n > 0 ? (n + kBlock - 1) / kBlock : 1;
  int pblocks = blocks < 4 * sm_count() ? blocks : 4 * sm_count();
  k_reduce_init<<<1, 256, 0, s>>>(st); note_launch();
  k_absmax<<<pblocks, kBlock, 0, s>>>(gamma, n, st, ds); note_launch();
  k_reduce_prepare<<<1, 1, 0, s>>>(st, c_bound); note_launch();
  for (int pass = 0; pass < 8; ++pass) {
    k_reduce_hist<<<pblocks, kBlock, 0, s>>>(gamma, n, st, pass); note_launch();
    k_reduce_choose<<<1, 32, 0, s>>>(st, c_bound, pass); note_launch();
  }
  k_reduce_mark<<<pblocks, kBlock, 0, s>>>(gamma, n, st, diffused, tie_flag); note_launch();
  cudaError_t e = scan_exclusive_u8(tie_flag, tie_rank, n, scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_reduce_ties<<<pblocks, kBlock, 0, s>>>(n, st, tie_flag, tie_rank, diffused); note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
