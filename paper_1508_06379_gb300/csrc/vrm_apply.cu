// Operator application (Eq. nsode, reduced operator Eq. reducedop) and the
// forward-Euler update (Sec. 3.3).
//
//   dGamma_j/dt = (nu/h^2) sum_{i in D} f~_ij Gamma_i
//
// computed as a gather, one thread per target j and no floating-point
// atomics: the annulus relation is symmetric (dx and dy only change sign when
// i and j swap, so d2 is bit-identical), hence every source i whose stencil
// contains j is in j's neighbour row (in any order).  The terms are added in
// ascending i with the self term f~_jj Gamma_j at i = j,
// each product and sum rounded separately, which fixes the result bit for
// bit given the weights.  Targets are visited in cell order so that the
// stencils of the neighbours of a warp's targets share cache lines.
#include <climits>

#include "vrm_internal.cuh"

namespace vrm {

// Products and sums of the application: FP64 rounded separately, or the
// mixed precision's fp32 (weights and circulations rounded to fp32 first).
template <typename Acc>
__device__ __forceinline__ Acc mul_acc(double a, double b);
template <>
__device__ __forceinline__ double mul_acc<double>(double a, double b) {
  return __dmul_rn(a, b);
}
template <>
__device__ __forceinline__ float mul_acc<float>(double a, double b) {
  return __fmul_rn(__double2float_rn(a), __double2float_rn(b));
}
__device__ __forceinline__ double add_acc(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_acc(float a, float b) { return __fadd_rn(a, b); }

// Batcher odd-even merge sort of 8 source indices with their terms.
template <typename Acc>
__device__ __forceinline__ void cx_terms(int* k, Acc* v, int p, int q) {
  const bool sw = k[q] < k[p];
  const int k0 = sw ? k[q] : k[p], k1 = sw ? k[p] : k[q];
  const Acc v0 = sw ? v[q] : v[p], v1 = sw ? v[p] : v[q];
  k[p] = k0;
  k[q] = k1;
  v[p] = v0;
  v[q] = v1;
}
template <typename Acc>
__device__ __forceinline__ void sort8_terms(int* k, Acc* v) {
  cx_terms(k, v, 0, 1); cx_terms(k, v, 2, 3); cx_terms(k, v, 4, 5); cx_terms(k, v, 6, 7);
  cx_terms(k, v, 0, 2); cx_terms(k, v, 1, 3); cx_terms(k, v, 4, 6); cx_terms(k, v, 5, 7);
  cx_terms(k, v, 1, 2); cx_terms(k, v, 5, 6);
  cx_terms(k, v, 0, 4); cx_terms(k, v, 1, 5); cx_terms(k, v, 2, 6); cx_terms(k, v, 3, 7);
  cx_terms(k, v, 2, 4); cx_terms(k, v, 3, 5);
  cx_terms(k, v, 1, 2); cx_terms(k, v, 3, 4); cx_terms(k, v, 5, 6);
}

// W: stencil width (8 for n = 1, 12 for n = 2); slot numbers fit 4 bits.
template <typename Acc, int W>
__global__ void __launch_bounds__(kBlock) k_apply(Consts c, int n, const int* __restrict__ n_dev, int n_gamma,
                                                  const int* __restrict__ n_gamma_dev, const double* __restrict__ gamma,
                                                  const uint8_t* __restrict__ diffused,
                                                  const int* __restrict__ nbr_count, const int* __restrict__ nbr_idx,
                                                  const int* __restrict__ cols, const double* __restrict__ f,
                                                  const double* __restrict__ fii, const int* __restrict__ order,
                                                  double* __restrict__ dgamma, double* __restrict__ gamma_out,
                                                  double dt, const double* __restrict__ dt_dev) {
  if (n_dev) n = *n_dev;
  if (n_gamma_dev) n_gamma = *n_gamma_dev;
  if (dt_dev) dt = *dt_dev;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const int j = order ? order[p] : (int)p;
    const int cnt0 = nbr_count[j];
    const int cnt = cnt0 < c.row_cap ? cnt0 : c.row_cap;
    const int* row = nbr_idx + (size_t)j * c.k_cap;
    const bool self_src = j < n_gamma && diffused[j];
    const double gj = j < n_gamma ? gamma[j] : 0.0;
    const Acc selfv = self_src ? mul_acc<Acc>(fii[j], gj) : Acc(0);
    // integer pass: which row entries are sources whose stencil holds j (and
    // in which slot, 4 bits per entry)
    unsigned match = 0;
    unsigned long long slot_lo = 0, slot_hi = 0;
    for (int t = 0; t < cnt; ++t) {
      const int i = row[t];
      if (i >= n_gamma || !diffused[i]) continue;
      const int4* cr = reinterpret_cast<const int4*>(cols + (size_t)i * W);
      int slot = -1;
#pragma unroll
      for (int q = W / 4 - 1; q >= 0; --q) {
        const int4 a = cr[q];
        slot = (a.w == j) ? 4 * q + 3 : slot;
        slot = (a.z == j) ? 4 * q + 2 : slot;
        slot = (a.y == j) ? 4 * q + 1 : slot;
        slot = (a.x == j) ? 4 * q : slot;
      }
      if (slot < 0) continue;
      match |= 1u << t;
      if (t < 16)
        slot_lo |= (unsigned long long)slot << (4 * t);
      else
        slot_hi |= (unsigned long long)slot << (4 * (t - 16));
    }
    // FP64 (or fp32) pass over the matches only, in ascending i (rows may
    // be in visiting order), the self term before the first i > j
    Acc acc = Acc(0);
    bool self_done = !self_src;
    unsigned rest = match;
    if (__popc(match) <= 8) {
      // up to 8 matches (nearly all targets): their terms are loaded at once
      // (the loads of one target overlap instead of queueing), then sorted
      // by source index with the terms as payload and added in that order
      int mi[8];
      Acc term[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        mi[k] = INT_MAX;
        term[k] = Acc(0);
        if (rest) {
          const int t = __ffs(rest) - 1;
          rest &= rest - 1;
          const int i = row[t];
          const int slot = (int)(((t < 16 ? slot_lo >> (4 * t) : slot_hi >> (4 * (t - 16)))) & 15ull);
          mi[k] = i;
          term[k] = mul_acc<Acc>(f[(size_t)i * W + slot], gamma[i]);
        }
      }
      sort8_terms(mi, term);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (mi[k] == INT_MAX) break;
        if (!self_done && mi[k] > j) {
          acc = add_acc(acc, selfv);
          self_done = true;
        }
        acc = add_acc(acc, term[k]);
      }
    }
    for (; rest;) {
      int tb = 0, ib = INT_MAX;
      for (unsigned r2 = rest; r2; r2 &= r2 - 1) {
        const int t = __ffs(r2) - 1;
        const int i = row[t];
        if (i < ib) {
          ib = i;
          tb = t;
        }
      }
      rest &= ~(1u << tb);
      if (!self_done && ib > j) {
        acc = add_acc(acc, selfv);
        self_done = true;
      }
      const int slot = (int)(((tb < 16 ? slot_lo >> (4 * tb) : slot_hi >> (4 * (tb - 16)))) & 15ull);
      acc = add_acc(acc, mul_acc<Acc>(f[(size_t)ib * W + slot], gamma[ib]));
    }
    if (!self_done) acc = add_acc(acc, selfv);
    const double dg = __dmul_rn(c.nu_over_h2, (double)acc);
    if (dgamma) dgamma[j] = dg;
    if (gamma_out) gamma_out[j] = __fma_rn(dt, dg, gj);
  }
}

// ---------------------------------------------------------------------------
// The same application through the transpose of the stencils (the step's
// form), as a compact CSR by target.  k_t_count adds every stencil entry
// (i -> j, f~_ij) of the diffused particles to target j's integer counter
// (atomics whose results nobody waits for); an exclusive scan of the counts
// gives the lists' offsets; k_t_fill takes each entry's place in j's list
// from an integer atomic on j's offset (the counts are exact, the order of a
// list varies; the offset ends at the list's end) and writes the entry as
// one 16-byte record (source, term f~_ij Gamma_i, the product rounded as the
// gather rounds it), so that the lists lie back to back and every sector of
// the array is written whole.  k_apply_t sets each counter back to 0 once it
// has read it, so that the counters are clear for the next application
// without a memset (they start at 0 when allocated).  k_apply_t sorts a
// target's few records by source index and adds the terms in that order
// with the self term at i = j: exactly the sum of k_apply, with no
// neighbour rows and no search of the sources' stencils.  The products are
// taken in k_t_fill (a thread per source, its entries in lockstep, the FP64
// pipe otherwise idle) and not in k_apply_t, whose lanes carry lists of
// uneven length: there every FP64 instruction costs the warp's longest list.
// ---------------------------------------------------------------------------
struct TEntry {
  int i, pad;
  double w;
};

template <int W>
__global__ void __launch_bounds__(kBlock) k_t_count(const int* __restrict__ list, const int* __restrict__ list_count,
                                                    const int* __restrict__ cols, int* __restrict__ tcount) {
  const int m = *list_count;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) {
    const int i = list[t];
    const int4* cr = reinterpret_cast<const int4*>(cols + (size_t)i * W);
    int js[W];
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
      const int4 a = cr[q];
      js[4 * q] = a.x;
      js[4 * q + 1] = a.y;
      js[4 * q + 2] = a.z;
      js[4 * q + 3] = a.w;
    }
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (js[u] >= 0) atomicAdd(&tcount[js[u]], 1);
  }
}

template <typename Acc, int W>
__global__ void __launch_bounds__(kBlock) k_t_fill(const int* __restrict__ list, const int* __restrict__ list_count,
                                                   const int* __restrict__ cols, const double* __restrict__ f,
                                                   const double* __restrict__ gamma, int* __restrict__ toff,
                                                   TEntry* __restrict__ tent) {
  const int m = *list_count;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) {
    const int i = list[t];
    const double gi = gamma[i];
    // the stencil row as vectors (rows of 8 or 12 entries start on 16-byte
    // boundaries), every place requested before any is used (their round
    // trips overlap), then the records
    const int4* cr = reinterpret_cast<const int4*>(cols + (size_t)i * W);
    const double2* fr = reinterpret_cast<const double2*>(f + (size_t)i * W);
    int js[W];
    double fs[W];
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
      const int4 a = cr[q];
      js[4 * q] = a.x;
      js[4 * q + 1] = a.y;
      js[4 * q + 2] = a.z;
      js[4 * q + 3] = a.w;
    }
#pragma unroll
    for (int q = 0; q < W / 2; ++q) {
      const double2 b = fr[q];
      fs[2 * q] = b.x;
      fs[2 * q + 1] = b.y;
    }
    int pos[W];
#pragma unroll
    for (int u = 0; u < W; ++u) pos[u] = js[u] >= 0 ? atomicAdd(&toff[js[u]], 1) : 0;
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (js[u] >= 0) {
        // the term f~_ij Gamma_i as the gather forms it (exact in a double
        // for the fp32 product of the mixed precision)
        const double term = (double)mul_acc<Acc>(fs[u], gi);
        reinterpret_cast<int4*>(tent)[pos[u]] = make_int4(i, 0, __double2loint(term), __double2hiint(term));
      }
  }
}

template <typename Acc>
__global__ void __launch_bounds__(kBlock) k_apply_t(Consts c, int n, const int* __restrict__ n_dev, int n_gamma,
                                                    const int* __restrict__ n_gamma_dev,
                                                    const double* __restrict__ gamma,
                                                    const uint8_t* __restrict__ diffused,
                                                    int* __restrict__ tcount, const int* __restrict__ toff,
                                                    const TEntry* __restrict__ tent, const double* __restrict__ fii,
                                                    double* __restrict__ dgamma, double* __restrict__ gamma_out,
                                                    double dt, const double* __restrict__ dt_dev,
                                                    DevStats* __restrict__ ds) {
  if (n_dev) n = *n_dev;
  if (n_gamma_dev) n_gamma = *n_gamma_dev;
  if (dt_dev) dt = *dt_dev;
  int widest = 0;
  for (long jj = (long)blockIdx.x * blockDim.x + threadIdx.x; jj < n; jj += (long)gridDim.x * blockDim.x) {
    const int j = (int)jj;
    const int cnt = tcount[j];
    if (cnt) tcount[j] = 0;  // clear for the next application
    widest = cnt > widest ? cnt : widest;
    const bool self_src = j < n_gamma && diffused[j];
    const double gj = j < n_gamma ? gamma[j] : 0.0;
    const Acc selfv = self_src ? mul_acc<Acc>(fii[j], gj) : Acc(0);
    // k_t_fill moved the offset to the end of the list
    const int4* rec = reinterpret_cast<const int4*>(tent) + (toff[j] - cnt);
    Acc acc = Acc(0);
    bool self_done = !self_src;
    if (cnt <= 8) {
      // nearly all targets: every term loaded at once, sorted by source
      int mi[8];
      Acc term[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        mi[k] = INT_MAX;
        term[k] = Acc(0);
        if (k < cnt) {
          const int4 r = rec[k];
          mi[k] = r.x;
          term[k] = (Acc)__hiloint2double(r.w, r.z);
        }
      }
      sort8_terms(mi, term);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (mi[k] == INT_MAX) break;
        if (!self_done && mi[k] > j) {
          acc = add_acc(acc, selfv);
          self_done = true;
        }
        acc = add_acc(acc, term[k]);
      }
    } else {
      // long lists: the smallest source not yet added, one at a time
      int last = -1;
      for (int r = 0; r < cnt; ++r) {
        int ib = INT_MAX, kb = 0;
        for (int k = 0; k < cnt; ++k) {
          const int i = rec[k].x;
          if (i > last && i < ib) {
            ib = i;
            kb = k;
          }
        }
        last = ib;
        if (!self_done && ib > j) {
          acc = add_acc(acc, selfv);
          self_done = true;
        }
        const int4 rk = rec[kb];
        acc = add_acc(acc, (Acc)__hiloint2double(rk.w, rk.z));
      }
    }
    if (!self_done) acc = add_acc(acc, selfv);
    const double dg = __dmul_rn(c.nu_over_h2, (double)acc);
    if (dgamma) dgamma[j] = dg;
    if (gamma_out) gamma_out[j] = __fma_rn(dt, dg, gj);
  }
  // a list longer than k_cap (only where some row is wider than k_cap, which
  // the rows of the diffused particles report themselves) makes the step
  // report a capacity error through the widest-row statistic
  widest = (int)__reduce_max_sync(0xffffffffu, (unsigned)widest);
  if ((threadIdx.x & 31) == 0 && widest > c.k_cap) atomicMax(&ds->max_count, widest);
}

cudaError_t apply_transposed_dev(const Consts& c, int n_bound, const int* n_dev, int n_gamma, const int* n_gamma_dev,
                                 const double* gamma, const uint8_t* diffused, const int* list, const int* list_count,
                                 const int* cols, const double* f, const double* fii, int* tcount, int* toff,
                                 void* tent, int* scan_tmp, DevStats* ds, double* dgamma, double* gamma_out, double dt,
                                 const double* dt_dev, cudaStream_t s) {
  if (n_bound <= 0) return cudaSuccess;
  cudaError_t e;
  const int blocks = (int)(((long)n_bound + kBlock - 1) / kBlock);
  if (c.order == 2)
    k_t_count<12><<<blocks, kBlock, 0, s>>>(list, list_count, cols, tcount);
  else
    k_t_count<8><<<blocks, kBlock, 0, s>>>(list, list_count, cols, tcount);
  note_launch();
  if ((e = scan_exclusive_i32_dev(tcount, toff, n_bound, n_dev, scan_tmp, s)) != cudaSuccess) return e;
  TEntry* te = static_cast<TEntry*>(tent);
  const bool mixed = c.precision == VRM_PREC_MIXED;
  if (c.order == 2) {
    if (mixed)
      k_t_fill<float, 12><<<blocks, kBlock, 0, s>>>(list, list_count, cols, f, gamma, toff, te);
    else
      k_t_fill<double, 12><<<blocks, kBlock, 0, s>>>(list, list_count, cols, f, gamma, toff, te);
  } else {
    if (mixed)
      k_t_fill<float, 8><<<blocks, kBlock, 0, s>>>(list, list_count, cols, f, gamma, toff, te);
    else
      k_t_fill<double, 8><<<blocks, kBlock, 0, s>>>(list, list_count, cols, f, gamma, toff, te);
  }
  note_launch();
  const int tb = c.apply_block;
  const int ab = (int)(((long)n_bound + tb - 1) / tb);
  auto kern = c.precision == VRM_PREC_MIXED ? k_apply_t<float> : k_apply_t<double>;
  kern<<<ab, tb, 0, s>>>(c, n_bound, n_dev, n_gamma, n_gamma_dev, gamma, diffused, tcount, toff, te, fii, dgamma,
                         gamma_out, dt, dt_dev, ds);
  note_launch();
  return cudaGetLastError();
}

cudaError_t apply_gather_dev(const Consts& c, int n_bound, const int* n_dev, int n_gamma, const int* n_gamma_dev,
                             const double* gamma, const uint8_t* diffused, const int* nbr_count, const int* nbr_idx,
                             const int* cols, const double* f, const double* fii, const int* order, double* dgamma,
                             double* gamma_out, double dt, const double* dt_dev, cudaStream_t s) {
  if (n_bound <= 0) return cudaSuccess;
  const int tb = c.apply_block;
  const int blocks = (int)(((long)n_bound + tb - 1) / tb);
  auto kern = c.precision == VRM_PREC_MIXED ? (c.order == 2 ? k_apply<float, 12> : k_apply<float, 8>)
                                             : (c.order == 2 ? k_apply<double, 12> : k_apply<double, 8>);
  kern<<<blocks, tb, 0, s>>>(c, n_bound, n_dev, n_gamma, n_gamma_dev, gamma, diffused, nbr_count, nbr_idx, cols, f,
                             fii, order, dgamma, gamma_out, dt, dt_dev);
  note_launch();
  return cudaGetLastError();
}

cudaError_t apply_gather(const Consts& c, int n, int n_gamma, const double* gamma, const uint8_t* diffused,
                         const int* nbr_count, const int* nbr_idx, const int* cols, const double* f, const double* fii,
                         const int* order, double* dgamma, double* gamma_out, double dt, cudaStream_t s) {
  return apply_gather_dev(c, n, nullptr, n_gamma, nullptr, gamma, diffused, nbr_count, nbr_idx, cols, f, fii, order,
                          dgamma, gamma_out, dt, nullptr, s);
}

}  // namespace vrm
