// Growth control (Sec. 3.5, Eq. reduced_bound) as an exact radix select.
//
// Particles are left out of diffusion, smallest |Gamma_i| first (ties by
// index), while the left-out l1 norm stays within C_diff h^{n+2} ||Gamma||_1.
// The choice must not depend on summation order, so the sums are exact
// integers: q_i = floor(|Gamma_i| 2^(96-E)) with max|Gamma| < 2^E, summed as
// three 32-bit limbs in 64-bit counters (no carries lost for n < 2^31).
// q_i is formed from the bit pattern with integer shifts (the same value as
// floor(ldexp(|Gamma_i|, 96-E)), computed without FP64 instructions).
//
// Instead of sorting, eight passes select the threshold key T (the bit
// pattern of |Gamma|, which orders like the value for non-negative doubles)
// one byte at a time: each pass histograms the exact q-sums of the particles
// whose key matches the bytes chosen so far; the last block of the pass to
// finish scans the 256 buckets in parallel and picks the first byte at which
// the running sum crosses the remaining budget.  Passes 3 to 7 run in one
// single-block launch over the list of pass 2's matches.  Particles with key == T are
// tied; the first k_tie of them by index stay out, found with a scan of the
// tie flags.
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

// floor(|a| 2^(96-E)) from the bit pattern key of |a| (a finite, |a| < 2^E):
// |a| = M 2^(e-1075) for a normal (M with the hidden bit), M 2^-1074 for a
// subnormal; the product by 2^(96-E) is a shift, floor a right shift.
__device__ __forceinline__ u128 q_of_key(unsigned long long key, int E) {
  const int ebits = (int)(key >> 52);
  const unsigned long long frac = key & 0xFFFFFFFFFFFFFull;
  const unsigned long long M = ebits ? (frac | 0x10000000000000ull) : frac;
  const int sh = (ebits ? ebits - 1075 : -1074) + 96 - E;
  if (sh >= 0) return (u128)M << sh;  // sh <= 43 because |a| < 2^E
  if (sh <= -64) return 0;
  return (u128)(M >> (-sh));
}

// E with max|Gamma| < 2^E (frexp exponent) from the bit pattern, no FP64.
__device__ __forceinline__ int exponent_of_key(unsigned long long key) {
  const int ebits = (int)(key >> 52);
  if (ebits) return ebits - 1022;
  const unsigned long long frac = key & 0xFFFFFFFFFFFFFull;
  return (64 - __clzll((long long)frac)) - 1074;  // bit length of frac - 1074
}

// Bucket value from its limbs; read past L1 (other blocks wrote them by atomics).
__device__ __forceinline__ u128 limbs_value(const unsigned long long* h) {
  return (u128)__ldcg(h) + ((u128)__ldcg(h + 1) << 32) + ((u128)__ldcg(h + 2) << 64);
}


// max |Gamma| (Inf/NaN flagged in ds->nonfinite) and the selection state
// set up for pass 0: each block leaves its maximum in the histogram memory,
// and the last block to finish takes the maximum, clears the histograms and
// the state, and marks the selection done when nothing can diffuse (no
// circulation, or a bound of at least ||Gamma||_1).  st->blocks_done is 0
// on entry (after allocation and after every pass).
__global__ void k_absmax(const double* __restrict__ g, int n, const int* __restrict__ n_dev, ReduceState* __restrict__ st,
                         DevStats* ds, double c_bound, const double* __restrict__ x, const double* __restrict__ y,
                         unsigned long long* __restrict__ bb) {
  if (n_dev) n = *n_dev;
  unsigned long long m = 0;
  int bad = 0;
  // with bb: the bounding box of the same particles, as k_bbox takes it
  // (ordered bit patterns; a NaN or Inf position flagged)
  unsigned long long mnx = ~0ull, mxx = 0, mny = ~0ull, mxy = 0;
  int badxy = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(g[i]) & 0x7FFFFFFFFFFFFFFFull;
    if (bb) {
      const double a = x[i], c = y[i];
      if (!isfinite(a) || !isfinite(c)) {
        badxy = 1;
      } else {
        const unsigned long long oa = ordered_bits(a), oc = ordered_bits(c);
        mnx = oa < mnx ? oa : mnx;
        mxx = oa > mxx ? oa : mxx;
        mny = oc < mny ? oc : mny;
        mxy = oc > mxy ? oc : mxy;
      }
    }
    if (b >= 0x7FF0000000000000ull) {  // Inf or NaN
      bad = 1;
      continue;
    }
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  bad = __any_sync(0xffffffffu, bad);
  if (bb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t;
      t = __shfl_xor_sync(0xffffffffu, mnx, o);
      mnx = t < mnx ? t : mnx;
      t = __shfl_xor_sync(0xffffffffu, mxx, o);
      mxx = t > mxx ? t : mxx;
      t = __shfl_xor_sync(0xffffffffu, mny, o);
      mny = t < mny ? t : mny;
      t = __shfl_xor_sync(0xffffffffu, mxy, o);
      mxy = t > mxy ? t : mxy;
    }
    badxy = __any_sync(0xffffffffu, badxy);
    // one atomic per block and quantity
    __shared__ unsigned long long w_bb[4][32];
    __shared__ int w_badxy[32];
    const int wb = threadIdx.x >> 5, nwb = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
      w_bb[0][wb] = mnx;
      w_bb[1][wb] = mxx;
      w_bb[2][wb] = mny;
      w_bb[3][wb] = mxy;
      w_badxy[wb] = badxy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < nwb; ++w) {
        mnx = w_bb[0][w] < mnx ? w_bb[0][w] : mnx;
        mxx = w_bb[1][w] > mxx ? w_bb[1][w] : mxx;
        mny = w_bb[2][w] < mny ? w_bb[2][w] : mny;
        mxy = w_bb[3][w] > mxy ? w_bb[3][w] : mxy;
        badxy |= w_badxy[w];
      }
      if (mnx != ~0ull) atomicMin(&bb[0], mnx);
      if (mxx) atomicMax(&bb[1], mxx);
      if (mny != ~0ull) atomicMin(&bb[2], mny);
      if (mxy) atomicMax(&bb[3], mxy);
      if (badxy) atomicOr(&bb[4], 1ull);
    }
  }
  __shared__ unsigned long long w_m[32];
  __shared__ int w_bad[32];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    w_m[warp] = m;
    w_bad[warp] = bad;
  }
  __syncthreads();
  unsigned long long* const part = &st->hist[0][0];  // 1024 slots >= gridDim.x
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      m = w_m[w] > m ? w_m[w] : m;
      bad |= w_bad[w];
    }
    part[blockIdx.x] = m;
    if (bad) atomicOr(&ds->nonfinite, 1);
    __threadfence();
    last = atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  unsigned long long amax = 0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const unsigned long long v = ((volatile unsigned long long*)part)[b];
    amax = v > amax ? v : amax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, amax, o);
    amax = t > amax ? t : amax;
  }
  if ((threadIdx.x & 31) == 0) w_m[warp] = amax;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w) amax = w_m[w] > amax ? w_m[w] : amax;
  __syncthreads();  // every part[] read before it is cleared
  for (int b = threadIdx.x; b < 256 * 4; b += blockDim.x) part[b] = 0;
  if (threadIdx.x == 0) {
    st->amax_bits = amax;
    st->E = 0;
    st->prefix = 0;
    st->tau_lo = st->tau_hi = 0;
    st->T = 0;
    st->k_tie = 0;
    st->n_sub = 0;
    const int none = amax == 0 || !(c_bound < 1.0);
    st->all_out = none;
    st->done = none;
    st->blocks_done = 0;
  }
}

// Choice of the byte of pass `pass` from the 256 bucket sums, by all 256
// threads of the last block: inclusive scan of the 128-bit bucket sums, then
// the first bucket whose running sum exceeds the budget.
__device__ void choose_digit(ReduceState* st, double c_bound, int pass) {
  __shared__ unsigned long long s_lo[8], s_hi[8];
  __shared__ int s_sel;
  const int b = threadIdx.x;  // 256 threads, one per bucket
  const u128 v = limbs_value(st->hist[b]);
  const unsigned long long cnt = __ldcg(&st->hist[b][3]);
  // inclusive scan: shuffles within each warp, then the warps' totals
  u128 acc = v;
  const int lane = b & 31, w = b >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long lo = __shfl_up_sync(0xffffffffu, (unsigned long long)acc, o);
    const unsigned long long hi = __shfl_up_sync(0xffffffffu, (unsigned long long)(acc >> 64), o);
    if (lane >= o) acc += ((u128)hi << 64) | (u128)lo;
  }
  if (lane == 31) {
    s_lo[w] = (unsigned long long)acc;
    s_hi[w] = (unsigned long long)(acc >> 64);
  }
  __syncthreads();
  u128 total = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const u128 wk = ((u128)s_hi[k] << 64) | (u128)s_lo[k];
    if (k < w) acc += wk;
    total += wk;
  }
  u128 tau;
  if (pass == 0) {
    tau = dbl_floor_to_u128(__dmul_rn(c_bound, u128_to_dbl(total)));
  } else {
    tau = ((u128)st->tau_hi << 64) | (u128)st->tau_lo;
  }
  if (b == 0) s_sel = 255;
  __syncthreads();
  if (pass == 0 && total <= tau) {
    if (b == 0) {
      st->all_out = 1;
      st->done = 1;
    }
    return;
  }
  // first bucket with inclusive sum > tau (exists: the total exceeds tau)
  const u128 excl = acc - v;
  if (acc > tau && excl <= tau) atomicMin(&s_sel, b);
  __syncthreads();
  const int sel = s_sel;
  if (b == sel) {
    const u128 rem = tau - excl;
    st->prefix = (st->prefix << 8) | (unsigned long long)sel;
    st->tau_lo = (unsigned long long)rem;
    st->tau_hi = (unsigned long long)(rem >> 64);
    if (pass == 7) {
      // all particles with key == T have the same q_T > 0; the first k_tie
      // by index fit: k_tie = max k <= count with k q_T <= rem (bisection)
      const unsigned long long T = st->prefix;
      const u128 qT = q_of_key(T, st->E);
      unsigned long long lo = 0, hi = cnt;
      while (lo < hi) {
        const unsigned long long mid = (lo + hi + 1) / 2;
        if ((u128)mid * qT <= rem) lo = mid;
        else hi = mid - 1;
      }
      st->T = T;
      st->k_tie = (int)lo;
      st->done = 1;
    }
  }
  __syncthreads();
  st->hist[b][0] = st->hist[b][1] = st->hist[b][2] = st->hist[b][3] = 0;
}

// One pass: block histograms of the exact q-sums per byte of the key, merged
// into st->hist; the last block to finish chooses the byte.  Passes 0 to 2
// read every particle; pass 2 also lists the particles that match the two
// chosen bytes (sign, exponent and the top mantissa bits: a sixteenth of a
// binade of |Gamma|, a small fraction), and passes 3 to 7 read that list
// only.  The sums are exact integers, so the list's order (atomic appends)
// does not matter.
constexpr int kReduceUnroll = 4;  // particles per lane whose loads one pass issues together

__global__ void __launch_bounds__(256) k_reduce_pass(const double* __restrict__ g, int n, const int* __restrict__ n_dev,
                                                     ReduceState* __restrict__ st, double c_bound, int pass,
                                                     int* __restrict__ sub) {
  if (n_dev) n = *n_dev;
  if (pass >= 3) n = st->n_sub;
  __shared__ unsigned long long h[256][4];
  __shared__ bool last;
  for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b][0] = h[b][1] = h[b][2] = h[b][3] = 0;
  if (pass == 0 && blockIdx.x == 0 && threadIdx.x == 0 && st->amax_bits != 0) st->E = exponent_of_key(st->amax_bits);
  __syncthreads();
  const int done = st->done;
  if (!done) {
    const unsigned long long amax = st->amax_bits;
    const int E = exponent_of_key(amax);
    const unsigned long long prefix = st->prefix;
    const int shift = 56 - 8 * pass;
    const int lane = threadIdx.x & 31;
    // whole warps step through the particles so that lanes holding the same
    // byte merge their exact limb sums before one shared atomic per byte (the
    // leading bytes are shared by nearly all particles); each warp takes
    // kReduceUnroll x 32 particles at a time, their loads issued together
    const long stride = (long)gridDim.x * blockDim.x * kReduceUnroll;
    for (long base = ((long)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * kReduceUnroll; base < n;
         base += stride) {
      int idxs[kReduceUnroll];
      unsigned long long keys[kReduceUnroll];
#pragma unroll
      for (int u = 0; u < kReduceUnroll; ++u) {
        const long i = base + u * 32 + lane;
        idxs[u] = -1;
        keys[u] = 0;
        if (i < n) {
          idxs[u] = pass >= 3 ? sub[i] : (int)i;
          keys[u] = (unsigned long long)__double_as_longlong(g[idxs[u]]) & 0x7FFFFFFFFFFFFFFFull;
        }
      }
#pragma unroll
      for (int u = 0; u < kReduceUnroll; ++u) {
        bool pending = false;
        int d = 0;
        const int idx = idxs[u];
        unsigned long long l0 = 0, l1 = 0, l2 = 0;
        if (idx >= 0) {
          const unsigned long long key = keys[u];
          if (pass == 0 || (key >> (shift + 8)) == prefix) {
            pending = true;
            d = (int)((key >> shift) & 0xFF);
            const u128 q = q_of_key(key, E);
            l0 = (unsigned long long)(q & 0xFFFFFFFFull);
            l1 = (unsigned long long)((q >> 32) & 0xFFFFFFFFull);
            l2 = (unsigned long long)(q >> 64);
          }
        }
        unsigned todo = __ballot_sync(0xffffffffu, pending);
        if (pass == 2 && todo) {
          // list the matches for the later passes (warp-aggregated append)
          const int lead = __ffs(todo) - 1;
          int slot0 = 0;
          if (lane == lead) slot0 = atomicAdd(&st->n_sub, __popc(todo));
          slot0 = __shfl_sync(0xffffffffu, slot0, lead);
          if (pending) sub[slot0 + __popc(todo & ((1u << lane) - 1u))] = idx;
        }
        if (pass > 0) {
          // bytes after the first are spread over many values: one shared
          // atomic per lane and limb (equal bytes in a warp serialise, rarely)
          if (pending) {
            if (l0) atomicAdd(&h[d][0], l0);
            if (l1) atomicAdd(&h[d][1], l1);
            if (l2) atomicAdd(&h[d][2], l2);
            atomicAdd(&h[d][3], 1ull);
          }
          todo = 0;
        }
        while (todo) {
          const int leader = __ffs(todo) - 1;
          const int dl = __shfl_sync(0xffffffffu, d, leader);
          const bool mine = pending && d == dl;
          const unsigned peers = __ballot_sync(0xffffffffu, mine);
          // 16-bit halves of the 32-bit limbs: sums of 32 lanes stay below 2^21
          unsigned long long sum[3];
          const unsigned long long lim[3] = {l0, l1, l2};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const unsigned lo = mine ? (unsigned)(lim[k] & 0xFFFFu) : 0u;
            const unsigned hi = mine ? (unsigned)(lim[k] >> 16) : 0u;
            sum[k] = (unsigned long long)__reduce_add_sync(0xffffffffu, lo) +
                     ((unsigned long long)__reduce_add_sync(0xffffffffu, hi) << 16);
          }
          if (lane == leader) {
            if (sum[0]) atomicAdd(&h[dl][0], sum[0]);
            if (sum[1]) atomicAdd(&h[dl][1], sum[1]);
            if (sum[2]) atomicAdd(&h[dl][2], sum[2]);
            atomicAdd(&h[dl][3], (unsigned long long)__popc(peers));
          }
          if (mine) pending = false;
          todo &= ~peers;
        }
      }
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
  // last block to finish chooses the byte (histogram complete): the block's
  // atomics are ordered before its ticket by the barrier and one fence of
  // the thread that takes the ticket (the pattern of a grid barrier)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&st->blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) st->blocks_done = 0;
  if (!done) choose_digit(st, c_bound, pass);
}

// Passes 3 to 7 in one block: they read only the short list of pass 2 (the
// particles matching the two chosen bytes), so one block of 1024 threads
// histograms each byte in shared memory and its first 256 threads choose the
// byte (the same inclusive scan and rule as choose_digit), five passes in
// one launch instead of five launches of mostly idle blocks.
__global__ void __launch_bounds__(1024) k_reduce_tail(const double* __restrict__ g, ReduceState* __restrict__ st,
                                                      const int* __restrict__ sub) {
  __shared__ unsigned long long h[256][4];
  __shared__ unsigned long long s_lo[8], s_hi[8];
  __shared__ int s_sel;
  const int b = threadIdx.x;
  const int n = st->n_sub;
  const int E = exponent_of_key(st->amax_bits);
  for (int pass = 3; pass < 8; ++pass) {
    if (st->done) return;  // uniform: written by thread 255 before the last barrier
    for (int k = b; k < 256; k += blockDim.x) h[k][0] = h[k][1] = h[k][2] = h[k][3] = 0;
    __syncthreads();
    const unsigned long long prefix = st->prefix;
    const int shift = 56 - 8 * pass;
    const int lane = b & 31;
    // whole warps step through the list; lanes holding the same byte merge
    // their limb sums first (a list of equal keys would otherwise serialise
    // on one shared address)
    for (int base = b & ~31; base < n; base += blockDim.x) {
      const int t = base + lane;
      bool pending = false;
      int d = 0;
      unsigned long long lim[3] = {0, 0, 0};
      if (t < n) {
        const unsigned long long key = (unsigned long long)__double_as_longlong(g[sub[t]]) & 0x7FFFFFFFFFFFFFFFull;
        if ((key >> (shift + 8)) == prefix) {
          pending = true;
          d = (int)((key >> shift) & 0xFF);
          const u128 q = q_of_key(key, E);
          lim[0] = (unsigned long long)(q & 0xFFFFFFFFull);
          lim[1] = (unsigned long long)((q >> 32) & 0xFFFFFFFFull);
          lim[2] = (unsigned long long)(q >> 64);
        }
      }
      unsigned todo = __ballot_sync(0xffffffffu, pending);
      while (todo) {
        const int leader = __ffs(todo) - 1;
        const int dl = __shfl_sync(0xffffffffu, d, leader);
        const bool mine = pending && d == dl;
        const unsigned peers = __ballot_sync(0xffffffffu, mine);
        // 16-bit halves of the 32-bit limbs: sums of 32 lanes stay below 2^21
        unsigned long long sum[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const unsigned lo = mine ? (unsigned)(lim[k] & 0xFFFFu) : 0u;
          const unsigned hi = mine ? (unsigned)(lim[k] >> 16) : 0u;
          sum[k] = (unsigned long long)__reduce_add_sync(0xffffffffu, lo) +
                   ((unsigned long long)__reduce_add_sync(0xffffffffu, hi) << 16);
        }
        if (lane == leader) {
          if (sum[0]) atomicAdd(&h[dl][0], sum[0]);
          if (sum[1]) atomicAdd(&h[dl][1], sum[1]);
          if (sum[2]) atomicAdd(&h[dl][2], sum[2]);
          atomicAdd(&h[dl][3], (unsigned long long)__popc(peers));
        }
        if (mine) pending = false;
        todo &= ~peers;
      }
    }
    __syncthreads();
    // inclusive scan of the 128-bit bucket sums over the first 256 threads
    // (warps 0..7): shuffles within each warp, then the warps' totals
    u128 v = 0, acc = 0;
    if (b < 256) {
      v = (u128)h[b][0] + ((u128)h[b][1] << 32) + ((u128)h[b][2] << 64);
      acc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long lo = __shfl_up_sync(0xffffffffu, (unsigned long long)acc, o);
        const unsigned long long hi = __shfl_up_sync(0xffffffffu, (unsigned long long)(acc >> 64), o);
        if (lane >= o) acc += ((u128)hi << 64) | (u128)lo;
      }
      if (lane == 31) {
        s_lo[b >> 5] = (unsigned long long)acc;
        s_hi[b >> 5] = (unsigned long long)(acc >> 64);
      }
    }
    if (b == 0) s_sel = 255;
    __syncthreads();
    if (b < 256)
      for (int k = 0; k < (b >> 5); ++k) acc += ((u128)s_hi[k] << 64) | (u128)s_lo[k];
    const u128 tau = ((u128)st->tau_hi << 64) | (u128)st->tau_lo;
    const u128 excl = acc - v;
    if (b < 256 && acc > tau && excl <= tau) atomicMin(&s_sel, b);
    __syncthreads();
    if (b == s_sel) {
      const u128 rem = tau - excl;
      st->prefix = (prefix << 8) | (unsigned long long)b;
      st->tau_lo = (unsigned long long)rem;
      st->tau_hi = (unsigned long long)(rem >> 64);
      if (pass == 7) {
        // all particles with key == T have the same q_T > 0; the first k_tie
        // by index fit: k_tie = max k <= count with k q_T <= rem (bisection)
        const unsigned long long T = st->prefix;
        const u128 qT = q_of_key(T, E);
        unsigned long long lo = 0, hi = h[b][3];
        while (lo < hi) {
          const unsigned long long mid = (lo + hi + 1) / 2;
          if ((u128)mid * qT <= rem) lo = mid;
          else hi = mid - 1;
        }
        st->T = T;
        st->k_tie = (int)lo;
        st->done = 1;
      }
    }
    __syncthreads();
  }
}


// diffused[i] = key > T, tie_flag[i] = key == T for i < n (both 0 when
// every particle stays out), diffused[i] = 0 for n <= i < n_bound; each block
// takes whole scan tiles and writes their sums of both flags (the tie scan
// and the diffused list's scan then skip their first pass).
__global__ void __launch_bounds__(kBlock) k_reduce_mark(const double* __restrict__ g, int n_bound,
                                                        const int* __restrict__ n_dev,
                                                        const ReduceState* __restrict__ st,
                                                        uint8_t* __restrict__ diffused, uint8_t* __restrict__ tie_flag,
                                                        int* __restrict__ dflag_ts, int* __restrict__ tie_ts) {
  static_assert(kScanTile % kBlock == 0, "a tile is whole block passes");
  __shared__ int s_d[kBlock / 32], s_t[kBlock / 32];
  const int n = n_dev ? *n_dev : n_bound;
  const int all_out = st->all_out;
  const unsigned long long T = st->T;
  const int ntiles = (n_bound + kScanTile - 1) / kScanTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int sd = 0, stie = 0;
#pragma unroll
    for (int k = 0; k < kScanTile / kBlock; ++k) {
      const long i = (long)tile * kScanTile + k * kBlock + threadIdx.x;
      if (i < n) {
        const unsigned long long key = (unsigned long long)__double_as_longlong(g[i]) & 0x7FFFFFFFFFFFFFFFull;
        uint8_t d = 0, t = 0;
        if (!all_out) {
          d = key > T;
          t = key == T;
        }
        diffused[i] = d;
        tie_flag[i] = t;
        sd += d;
        stie += t;
      } else if (i < n_bound) {
        diffused[i] = 0;
      }
    }
    sd = __reduce_add_sync(0xffffffffu, sd);
    stie = __reduce_add_sync(0xffffffffu, stie);
    if ((threadIdx.x & 31) == 0) {
      s_d[threadIdx.x >> 5] = sd;
      s_t[threadIdx.x >> 5] = stie;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int a = 0, b = 0;
      for (int w = 0; w < kBlock / 32; ++w) {
        a += s_d[w];
        b += s_t[w];
      }
      dflag_ts[tile] = a;
      tie_ts[tile] = b;
    }
    __syncthreads();
  }
}

// The ties that diffuse (rank >= k_tie), added to the diffused flags and
// their tile sums.
__global__ void k_reduce_ties(int n, const int* __restrict__ n_dev, const ReduceState* __restrict__ st,
                              const uint8_t* __restrict__ tie_flag, const int* __restrict__ tie_rank,
                              uint8_t* __restrict__ diffused, int* __restrict__ dflag_ts) {
  if (n_dev) n = *n_dev;
  const int k_tie = st->k_tie;
  const int lane = threadIdx.x & 31;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
       base += (long)gridDim.x * blockDim.x) {
    const long i = base + lane;
    bool up = false;
    if (i < n && tie_flag[i] && tie_rank[i] >= k_tie) {
      diffused[i] = 1;
      up = true;
    }
    tile_sum_add(dflag_ts, up ? i : -1, 1);
  }
}

cudaError_t reduce_select_dev(const double* gamma, int n_bound, const int* n_dev, double c_bound, uint8_t* diffused,
                              ReduceState* st, uint8_t* tie_flag, int* tie_rank, int* scan_tmp, DevStats* ds,
                              cudaStream_t s, int* dflag_ts, int* tie_ts, const double* x, const double* y,
                              unsigned long long* bbox) {
  int blocks = n_bound > 0 ? (n_bound + kBlock - 1) / kBlock : 1;
  int pblocks = blocks < 4 * sm_count() ? blocks : 4 * sm_count();
  // k_absmax keeps one partial maximum per block in the 1024 slots of hist
  if (pblocks > 1024) pblocks = 1024;
  k_absmax<<<pblocks, kBlock, 0, s>>>(gamma, n_bound, n_dev, st, ds, c_bound, x, y, bbox); note_launch();
  for (int pass = 0; pass < 3; ++pass) {
    // pass 2 lists its matches in tie_rank (free until the tie scan)
    k_reduce_pass<<<pblocks, 256, 0, s>>>(gamma, n_bound, n_dev, st, c_bound, pass, tie_rank); note_launch();
  }
  k_reduce_tail<<<1, 1024, 0, s>>>(gamma, st, tie_rank); note_launch();
  k_reduce_mark<<<pblocks, kBlock, 0, s>>>(gamma, n_bound, n_dev, st, diffused, tie_flag, dflag_ts, tie_ts);
  note_launch();
  cudaError_t e = scan_presummed_u8_dev(tie_flag, tie_rank, n_bound, n_dev, tie_ts, s);
  if (e != cudaSuccess) return e;
  k_reduce_ties<<<pblocks, kBlock, 0, s>>>(n_bound, n_dev, st, tie_flag, tie_rank, diffused, dflag_ts);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
