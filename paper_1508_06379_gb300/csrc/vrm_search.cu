// Annulus neighbourhoods (Sec. 2, Eq. neighbourhood), 45-degree segment
// masks (Sec. 4.2) and small neighbourhoods (Sec. 4.3) on the cell grid.
//
// One thread per particle, taken in cell order so that the threads of a warp
// read overlapping cells (coalesced double2 loads of the sorted positions).
// Each thread scans the three grid rows around its cell; the three cells of
// a row are contiguous in the sorted arrays.  A hit j of particle i obeys
//   lo2 <= dx*dx + dy*dy <= hi2,  dx = x_j - x_i,  dy = y_j - y_i
// with every operation rounded separately, exactly as the FP64 definition.
// The row is kept sorted by index in a per-thread buffer (the k_cap smallest
// indices survive); the closest particle of every segment is tracked in
// registers with ties to the smaller index.
#include "vrm_internal.cuh"

namespace vrm {

template <int KCAP>
__global__ void __launch_bounds__(kBlock) k_search_all(Consts c, const Grid* __restrict__ gp,
                                                       const int* __restrict__ cell_start,
                                                       const double2* __restrict__ sxy,
                                                       const int* __restrict__ sidx, int n,
                                                       int* __restrict__ nbr_count, int* __restrict__ nbr_idx,
                                                       uint8_t* __restrict__ seg_mask, int* __restrict__ small,
                                                       DevStats* __restrict__ ds) {
  const Grid g = *gp;
  const int k_cap = c.k_cap;
  int local_max = 0;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const int i = sidx[p];
    const double2 pi = sxy[p];
    const int cx = grid_cell_x(g, pi.x), cy = grid_cell_y(g, pi.y);
    const int c0 = cx > 0 ? cx - 1 : 0, c1 = cx + 1 < g.nx ? cx + 1 : g.nx - 1;
    int list[KCAP];
    int cnt = 0;
    double bd[8];
    int bj[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      bd[t] = 1e300;
      bj[t] = -1;
    }
    unsigned mask = 0;
    for (int by = cy - 1; by <= cy + 1; ++by) {
      if (by < 0 || by >= g.ny) continue;
      const int q0 = cell_start[by * g.nx + c0], q1 = cell_start[by * g.nx + c1 + 1];
      for (int q = q0; q < q1; ++q) {
        const int j = sidx[q];
        if (j == i) continue;
        const double2 pj = sxy[q];
        const double dx = __dsub_rn(pj.x, pi.x), dy = __dsub_rn(pj.y, pi.y);
        const double d2 = dist2(dx, dy);
        if (d2 < c.lo2 || d2 > c.hi2) continue;
        const int s = segment_of(dx, dy);
        mask |= 1u << s;
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (t == s && (d2 < bd[t] || (d2 == bd[t] && j < bj[t]))) {
            bd[t] = d2;
            bj[t] = j;
          }
        if (cnt < k_cap || j < list[k_cap - 1]) {
          int pos = cnt < k_cap ? cnt : k_cap - 1;
          while (pos > 0 && list[pos - 1] > j) {
            list[pos] = list[pos - 1];
            --pos;
          }
          list[pos] = j;
        }
        ++cnt;
      }
    }
    nbr_count[i] = cnt;
    const int m = cnt < k_cap ? cnt : k_cap;
    int* row = nbr_idx + (size_t)i * k_cap;
    for (int t = 0; t < m; ++t) row[t] = list[t];
    seg_mask[i] = (uint8_t)mask;
    int4* sm = reinterpret_cast<int4*>(small + (size_t)i * 8);
    sm[0] = make_int4(bj[0], bj[1], bj[2], bj[3]);
    sm[1] = make_int4(bj[4], bj[5], bj[6], bj[7]);
    local_max = cnt > local_max ? cnt : local_max;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int t = __shfl_xor_sync(0xffffffffu, local_max, o);
    local_max = t > local_max ? t : local_max;
  }
  if ((threadIdx.x & 31) == 0 && local_max > 0) atomicMax(&ds->max_count, local_max);
}

// Segment mask only, for the particles of a list (insertion rounds).
__global__ void __launch_bounds__(kBlock) k_search_masks(Consts c, const Grid* __restrict__ gp,
                                                         const int* __restrict__ cell_start,
                                                         const double2* __restrict__ sxy,
                                                         const int* __restrict__ sidx, const double* __restrict__ x,
                                                         const double* __restrict__ y, const int* __restrict__ list,
                                                         const int* __restrict__ list_count, uint8_t* __restrict__ mask) {
  const Grid g = *gp;
  const int m = *list_count;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) {
    const int i = list[t];
    const double xi = x[i], yi = y[i];
    const int cx = grid_cell_x(g, xi), cy = grid_cell_y(g, yi);
    const int c0 = cx > 0 ? cx - 1 : 0, c1 = cx + 1 < g.nx ? cx + 1 : g.nx - 1;
    unsigned mk = 0;
    for (int by = cy - 1; by <= cy + 1; ++by) {
      if (by < 0 || by >= g.ny) continue;
      const int q0 = cell_start[by * g.nx + c0], q1 = cell_start[by * g.nx + c1 + 1];
      for (int q = q0; q < q1; ++q) {
        const int j = sidx[q];
        if (j == i) continue;
        const double2 pj = sxy[q];
        const double dx = __dsub_rn(pj.x, xi), dy = __dsub_rn(pj.y, yi);
        const double d2 = dist2(dx, dy);
        if (d2 < c.lo2 || d2 > c.hi2) continue;
        mk |= 1u << segment_of(dx, dy);
      }
    }
    mask[i] = (uint8_t)mk;
  }
}

cudaError_t search_all(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                       const int* sorted_idx, int n, int* nbr_count, int* nbr_idx, uint8_t* seg_mask, int* small,
                       DevStats* ds, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (n + kBlock - 1) / kBlock;
  k_search_all<VRM_KCAP_MAX><<<blocks, kBlock, 0, s>>>(c, g, cell_start, sorted_xy, sorted_idx, n, nbr_count,
                                                        nbr_idx, seg_mask, small, ds); note_launch();
  return cudaGetLastError();
}

cudaError_t search_masks(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                         const int* sorted_idx, const double* x, const double* y, const int* list,
                         const int* list_count, int cap, uint8_t* mask, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  int blocks = (cap + kBlock - 1) / kBlock;
  if (blocks > 8 * sm_count()) blocks = 8 * sm_count();
  k_search_masks<<<blocks, kBlock, 0, s>>>(c, g, cell_start, sorted_xy, sorted_idx, x, y, list, list_count, mask); note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
