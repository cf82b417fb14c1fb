// Annulus neighbourhoods (Sec. 2, Eq. neighbourhood), 45-degree segment
// masks (Sec. 4.2) and small neighbourhoods (Sec. 4.3) on the cell grid.
//
// One thread per particle, taken in cell order so that the threads of a warp
// read overlapping cells.  Each thread scans the 3 x 3 cells around its own.
// The annulus test of the method is the FP64 definition
//   lo2 <= dx*dx + dy*dy <= hi2,  dx = x_j - x_i,  dy = y_j - y_i,
// every operation rounded separately.  GB300 runs FP64 at 1/60 of its FP32
// rate, so each pair is first measured in FP32 on cell-local coordinates
// (error below 1e-5 cell^2): a pair outside the bounds by more than the band
// is skipped, a pair inside by more than the band is a member without an FP64
// bound test, and only the hits (which need their FP64 squared distance for
// the small neighbourhood's order) and the pairs in the band take FP64 work.
// Segments are decided in FP32 unless the offset is within seg_eps of a
// decision line.  The result is bit-identical to the FP64 definition.
//
// The row is kept sorted by index in a per-thread buffer (the k_cap smallest
// indices survive); the closest particle of every segment is tracked in
// registers with ties to the smaller index.
#include "vrm_internal.cuh"

namespace vrm {

template <int KCAP>
__global__ void __launch_bounds__(kBlock) k_search_all(Consts c, const Grid* __restrict__ gp,
                                                       const int* __restrict__ cell_start,
                                                       const double2* __restrict__ sxy,
                                                       const float2* __restrict__ sloc,
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
    const float2 li = sloc[p];
    const int cx = grid_cell_x(g, pi.x), cy = grid_cell_y(g, pi.y);
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
      const float dvb = (float)(by - cy) - li.y;
      for (int bx = cx - 1; bx <= cx + 1; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        const float dub = (float)(bx - cx) - li.x;
        const int cell = by * g.nx + bx;
        const int q0 = cell_start[cell], q1 = cell_start[cell + 1];
        for (int q = q0; q < q1; ++q) {
          const float2 lj = sloc[q];
          const float du = dub + lj.x, dv = dvb + lj.y;
          const float d2f = __fmaf_rn(du, du, dv * dv);
          if (d2f < g.lo_out || d2f > g.hi_out) continue;
          const int j = sidx[q];
          if (j == i) continue;
          const double2 pj = sxy[q];
          const double dx = __dsub_rn(pj.x, pi.x), dy = __dsub_rn(pj.y, pi.y);
          const double d2 = dist2(dx, dy);
          if (!(d2f > g.lo_in && d2f < g.hi_in) && (d2 < c.lo2 || d2 > c.hi2)) continue;
          int s = segment_or_ambiguous(du, dv, g.seg_eps);
          if (s < 0) s = segment_of(dx, dy);
          mask |= 1u << s;
          // current best of segment s by register selects, one FP64 compare
          double cb = bd[0];
          int cjb = bj[0];
#pragma unroll
          for (int t = 1; t < 8; ++t) {
            cb = (s == t) ? bd[t] : cb;
            cjb = (s == t) ? bj[t] : cjb;
          }
          if (d2 < cb || (d2 == cb && j < cjb)) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
              bd[t] = (s == t) ? d2 : bd[t];
              bj[t] = (s == t) ? j : bj[t];
            }
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

// Segment mask only, for the particles with flag[i] set (insertion rounds).
// Threads run over the particles in cell order and skip unflagged ones.
__global__ void __launch_bounds__(kBlock) k_search_masks(Consts c, const Grid* __restrict__ gp,
                                                         const int* __restrict__ cell_start,
                                                         const double2* __restrict__ sxy,
                                                         const float2* __restrict__ sloc,
                                                         const int* __restrict__ sidx, int n,
                                                         const uint8_t* __restrict__ flag,
                                                         uint8_t* __restrict__ mask) {
  const Grid g = *gp;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long)gridDim.x * blockDim.x) {
    const int i = sidx[p];
    if (!flag[i]) continue;
    const double2 pi = sxy[p];
    const float2 li = sloc[p];
    const int cx = grid_cell_x(g, pi.x), cy = grid_cell_y(g, pi.y);
    unsigned mk = 0;
    for (int by = cy - 1; by <= cy + 1; ++by) {
      if (by < 0 || by >= g.ny) continue;
      const float dvb = (float)(by - cy) - li.y;
      for (int bx = cx - 1; bx <= cx + 1; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        const float dub = (float)(bx - cx) - li.x;
        const int cell = by * g.nx + bx;
        const int q0 = cell_start[cell], q1 = cell_start[cell + 1];
        for (int q = q0; q < q1; ++q) {
          const float2 lj = sloc[q];
          const float du = dub + lj.x, dv = dvb + lj.y;
          const float d2f = __fmaf_rn(du, du, dv * dv);
          if (d2f < g.lo_out || d2f > g.hi_out) continue;
          int s = -1;
          if (d2f > g.lo_in && d2f < g.hi_in) s = segment_or_ambiguous(du, dv, g.seg_eps);
          if (s < 0) {
            const int j = sidx[q];
            if (j == i) continue;
            const double2 pj = sxy[q];
            const double dx = __dsub_rn(pj.x, pi.x), dy = __dsub_rn(pj.y, pi.y);
            const double d2 = dist2(dx, dy);
            if (d2 < c.lo2 || d2 > c.hi2) continue;
            s = segment_of(dx, dy);
          }
          mk |= 1u << s;
        }
      }
    }
    mask[i] = (uint8_t)mk;
  }
}

cudaError_t search_all(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                       const float2* sorted_loc, const int* sorted_idx, int n, int* nbr_count, int* nbr_idx,
                       uint8_t* seg_mask, int* small, DevStats* ds, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (n + kBlock - 1) / kBlock;
  k_search_all<VRM_KCAP_MAX><<<blocks, kBlock, 0, s>>>(c, g, cell_start, sorted_xy, sorted_loc, sorted_idx, n,
                                                        nbr_count, nbr_idx, seg_mask, small, ds);
  note_launch();
  return cudaGetLastError();
}

cudaError_t search_masks(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                         const float2* sorted_loc, const int* sorted_idx, int n, const uint8_t* flag, uint8_t* mask,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int blocks = (n + kBlock - 1) / kBlock;
  k_search_masks<<<blocks, kBlock, 0, s>>>(c, g, cell_start, sorted_xy, sorted_loc, sorted_idx, n, flag, mask);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
