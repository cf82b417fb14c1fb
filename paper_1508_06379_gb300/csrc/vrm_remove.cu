// Particle removal (the outlook of Sec. 6.2): where particles have come closer
// than r h to one another, the one with the smaller key (|Gamma|, index) of
// such a pair is redistributed to its kept neighbours by non-negative
// weights that reproduce the identity's moments of order 0 and 1 (sum g = 1,
// sum g r = 0; the weights come from k_lp_identity in vrm_lp.cu) and removed.
//
//   k_close          candidate flags on the cell grid (FP32 prefilter on
//                    cell-local coordinates, the FP64 definition
//                    dx*dx + dy*dy < (r h)^2 for the undecided pairs)
//   k_remove_gather  Gamma_j + sum_i g_ij Gamma_i for every kept j, the
//                    removed i in ascending order (the annulus relation is
//                    symmetric, so they are all in j's row); no atomics
//   k_remove_out     the kept particles compacted in index order
#include "vrm_internal.cuh"

namespace vrm {

// |Gamma| as bits (non-negative: the bit order is the value order).
__device__ __forceinline__ unsigned long long abs_key(double g) {
  return (unsigned long long)__double_as_longlong(g) & 0x7FFFFFFFFFFFFFFFull;
}

__global__ void __launch_bounds__(kBlock) k_close(Consts c, const Grid* __restrict__ gp,
                                                  const int* __restrict__ cell_start,
                                                  const double2* __restrict__ sxy, const float2* __restrict__ sloc,
                                                  const int* __restrict__ sidx, int n,
                                                  const double* __restrict__ gamma, uint8_t* __restrict__ close) {
  const Grid g = *gp;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const int i = sidx[p];
    const double2 pi = sxy[p];
    const float2 li = sloc[p];
    const int cx = grid_cell_x(g, pi.x), cy = grid_cell_y(g, pi.y);
    const unsigned long long ai = abs_key(gamma[i]);
    bool cl = false;
    for (int by = cy - 1; by <= cy + 1 && !cl; ++by) {
      if (by < 0 || by >= g.ny) continue;
      const float dvb = (float)(by - cy) - li.y;
      for (int bx = cx - 1; bx <= cx + 1 && !cl; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        const float dub = (float)(bx - cx) - li.x;
        const int cell = by * g.nx + bx;
        const int q1 = cell_start[cell + 1];
        for (int q = cell_start[cell]; q < q1; ++q) {
          const float2 lj = sloc[q];
          const float du = dub + lj.x, dv = dvb + lj.y;
          const float d2f = __fmaf_rn(du, du, dv * dv);
          if (d2f > g.lo_in) continue;  // certainly not closer than r h
          const int j = sidx[q];
          if (j == i) continue;
          bool in = d2f < g.lo_out;  // certainly closer
          if (!in) {
            const double2 pj = sxy[q];
            in = dist2(__dsub_rn(pj.x, pi.x), __dsub_rn(pj.y, pi.y)) < c.lo2;
          }
          if (!in) continue;
          const unsigned long long aj = abs_key(gamma[j]);
          if (ai < aj || (ai == aj && i < j)) {
            cl = true;
            break;
          }
        }
      }
    }
    close[i] = cl ? 1 : 0;
  }
}

__global__ void __launch_bounds__(kBlock) k_remove_gather(Consts c, int n, const double* __restrict__ gamma,
                                                          const uint8_t* __restrict__ removed,
                                                          const int* __restrict__ nbr_count,
                                                          const int* __restrict__ nbr_idx,
                                                          const int* __restrict__ cols4,
                                                          const double* __restrict__ w4, double* __restrict__ gnew,
                                                          uint8_t* __restrict__ keep, DevStats* __restrict__ ds) {
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
    const double gj = gamma[j];
    if ((__double_as_longlong(gj) & 0x7FF0000000000000LL) == 0x7FF0000000000000LL) atomicOr(&ds->nonfinite, 1);
    const bool gone = removed[j] != 0;
    keep[j] = gone ? 0 : 1;
    if (gone) continue;
    const int cnt0 = nbr_count[j];
    const int cnt = cnt0 < c.row_cap ? cnt0 : c.row_cap;
    const int* row = nbr_idx + (size_t)j * c.k_cap;
    double acc = gj;
    for (int t = 0; t < cnt; ++t) {
      const int i = row[t];
      if (!removed[i]) continue;
      const int4 cc = reinterpret_cast<const int4*>(cols4)[i];
      int slot = -1;
      slot = (cc.w == j) ? 3 : slot;
      slot = (cc.z == j) ? 2 : slot;
      slot = (cc.y == j) ? 1 : slot;
      slot = (cc.x == j) ? 0 : slot;
      if (slot < 0) continue;
      acc = __dadd_rn(acc, __dmul_rn(w4[(size_t)i * 4 + slot], gamma[i]));
    }
    gnew[j] = acc;
  }
}

__global__ void __launch_bounds__(kBlock) k_remove_out(const int* __restrict__ n_keep, const int* __restrict__ klist,
                                                       const double* __restrict__ x, const double* __restrict__ y,
                                                       const double* __restrict__ gnew, double* __restrict__ x_out,
                                                       double* __restrict__ y_out, double* __restrict__ g_out) {
  const int m = *n_keep;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (long)gridDim.x * blockDim.x) {
    const int i = klist[k];
    x_out[k] = x[i];
    y_out[k] = y[i];
    g_out[k] = gnew[i];
  }
}

namespace {
int blocks_for(int n) {
  long b = ((long)n + kBlock - 1) / kBlock;
  if (b > 8L * sm_count()) b = 8L * sm_count();
  return b < 1 ? 1 : (int)b;
}
}  // namespace

cudaError_t remove_close_flags(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                               const float2* sorted_loc, const int* sorted_idx, int n, const double* gamma,
                               uint8_t* close, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_close<<<blocks_for(n), kBlock, 0, s>>>(c, g, cell_start, sorted_xy, sorted_loc, sorted_idx, n, gamma, close);
  note_launch();
  return cudaGetLastError();
}

cudaError_t remove_gather(const Consts& c, int n, const double* gamma, const uint8_t* removed, const int* nbr_count,
                          const int* nbr_idx, const int* cols4, const double* w4, double* gnew, uint8_t* keep,
                          DevStats* ds, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_remove_gather<<<blocks_for(n), kBlock, 0, s>>>(c, n, gamma, removed, nbr_count, nbr_idx, cols4, w4, gnew, keep,
                                                   ds);
  note_launch();
  return cudaGetLastError();
}

cudaError_t remove_out(int n, const int* n_keep, const int* klist, const double* x, const double* y,
                       const double* gnew, double* x_out, double* y_out, double* g_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_remove_out<<<blocks_for(n), kBlock, 0, s>>>(n_keep, klist, x, y, gnew, x_out, y_out, g_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
