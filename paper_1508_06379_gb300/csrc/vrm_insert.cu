// Insertion of zero-strength particles (Sec. 2 and Sec. 4.2).
//
// Every diffused particle whose annulus leaves a 45-degree segment empty
// proposes the point at radius 1.5 h on that segment's centre line.  The
// paper describes one insertion at a time; for many at once the rule here is
// a round: all open particles propose at once, a proposal with key (i, s) is
// dropped if a proposal of smaller key lies closer than r h, and the rest are
// appended in key order.  Rounds repeat until nothing is proposed.
//
// One round works on explicit lists:
//   1. the proposals are written in key order (open particles ascending,
//      segments ascending), so a proposal's list index is its key rank;
//   2. the proposals get their own cell grid (cell side >= R h);
//   3. conflict test: each proposal scans the 3 x 3 cells around it for a
//      proposal of smaller list index within r h;
//   4. the accepted ones are appended in list order;
//   5. every open particle ORs into its segment mask the accepted proposals
//      of its annulus, found in the same 3 x 3 cells.
// All threads of a warp do the same kind of work on nearby proposals, and
// every distance is the FP64 definition, so the result is the oracle's.
#include "vrm_internal.cuh"

namespace vrm {

static int blocks_for(int m) {
  int b = m > 0 ? (m + kBlock - 1) / kBlock : 1;
  return b < 8 * sm_count() ? b : 8 * sm_count();
}

__global__ void k_cand_count(const int* __restrict__ open, int n_open, const uint8_t* __restrict__ mask,
                             int* __restrict__ cnt) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x)
    cnt[t] = __popc((~(unsigned)mask[open[t]]) & 0xFFu);
}

__global__ void k_cand_emit(Consts c, const int* __restrict__ open, int n_open, const uint8_t* __restrict__ mask,
                            const int* __restrict__ cpos, const double* __restrict__ x,
                            const double* __restrict__ y, double* __restrict__ cx, double* __restrict__ cy) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x) {
    const int i = open[t];
    const unsigned empty = (~(unsigned)mask[i]) & 0xFFu;
    const double xi = x[i], yi = y[i];
    int pos = cpos[t];
    for (int s = 0; s < 8; ++s)
      if ((empty >> s) & 1u) {
        cx[pos] = __dadd_rn(xi, c.ins_dx[s]);
        cy[pos] = __dadd_rn(yi, c.ins_dy[s]);
        ++pos;
      }
  }
}

// keep[c] = 1 unless a proposal of smaller index lies closer than r h.
// Pairs clearly apart (or clearly too close) are decided in FP32 on the
// cell-local coordinates, the rest by the FP64 distance.
__global__ void __launch_bounds__(kBlock) k_conflict(Consts c, const Grid* __restrict__ gp,
                                                     const int* __restrict__ cell_start,
                                                     const double2* __restrict__ sxy, const float2* __restrict__ sloc,
                                                     const int* __restrict__ sidx, int n_cand,
                                                     uint8_t* __restrict__ keep) {
  const Grid g = *gp;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n_cand; p += (long)gridDim.x * blockDim.x) {
    const int ci = sidx[p];
    const double2 pc = sxy[p];
    const float2 lc = sloc[p];
    const int gx = grid_cell_x(g, pc.x), gy = grid_cell_y(g, pc.y);
    bool ok = true;
    for (int by = gy - 1; by <= gy + 1 && ok; ++by) {
      if (by < 0 || by >= g.ny) continue;
      const float dvb = (float)(by - gy) - lc.y;
      for (int bx = gx - 1; bx <= gx + 1 && ok; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        const float dub = (float)(bx - gx) - lc.x;
        const int cell = by * g.nx + bx;
        const int q0 = cell_start[cell], q1 = cell_start[cell + 1];
        for (int q = q0; q < q1; ++q) {
          const float2 lo = sloc[q];
          const float du = dub + lo.x, dv = dvb + lo.y;
          const float d2f = __fmaf_rn(du, du, dv * dv);
          if (d2f > g.lo_in) continue;
          if (sidx[q] >= ci) continue;
          bool close = d2f < g.lo_out;
          if (!close) {
            const double2 o = sxy[q];
            close = dist2(__dsub_rn(pc.x, o.x), __dsub_rn(pc.y, o.y)) < c.lo2;
          }
          if (close) {
            ok = false;
            break;
          }
        }
      }
    }
    keep[ci] = ok;
  }
}

__global__ void k_append(const double* __restrict__ cx, const double* __restrict__ cy,
                         const uint8_t* __restrict__ keep, const int* __restrict__ apos, int n_cand, int n_cur,
                         double* __restrict__ x, double* __restrict__ y) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_cand; t += (long)gridDim.x * blockDim.x)
    if (keep[t]) {
      x[n_cur + apos[t]] = cx[t];
      y[n_cur + apos[t]] = cy[t];
    }
}

// Segment bits of the accepted proposals in the annulus of every open
// particle; keep_flag[t] = 1 if the mask is still not full.  FP32 filter on
// cell-local coordinates as in the neighbour search.
__global__ void __launch_bounds__(kBlock) k_mask_update(Consts c, const Grid* __restrict__ gp,
                                                        const int* __restrict__ cell_start,
                                                        const double2* __restrict__ sxy,
                                                        const float2* __restrict__ sloc,
                                                        const int* __restrict__ sidx, const uint8_t* __restrict__ keep,
                                                        const double* __restrict__ x, const double* __restrict__ y,
                                                        const int* __restrict__ open, int n_open,
                                                        uint8_t* __restrict__ mask, uint8_t* __restrict__ keep_flag) {
  const Grid g = *gp;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x) {
    const int i = open[t];
    const double xi = x[i], yi = y[i];
    const int gx = grid_cell_x(g, xi), gy = grid_cell_y(g, yi);
    const float ux = grid_local_x(g, xi, gx), uy = grid_local_y(g, yi, gy);
    unsigned mk = mask[i];
    for (int by = gy - 1; by <= gy + 1; ++by) {
      if (by < 0 || by >= g.ny) continue;
      const float dvb = (float)(by - gy) - uy;
      for (int bx = gx - 1; bx <= gx + 1; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        const float dub = (float)(bx - gx) - ux;
        const int cell = by * g.nx + bx;
        const int q0 = cell_start[cell], q1 = cell_start[cell + 1];
        for (int q = q0; q < q1; ++q) {
          const float2 lo = sloc[q];
          const float du = dub + lo.x, dv = dvb + lo.y;
          const float d2f = __fmaf_rn(du, du, dv * dv);
          if (d2f < g.lo_out || d2f > g.hi_out) continue;
          if (!keep[sidx[q]]) continue;
          int s = -1;
          if (d2f > g.lo_in && d2f < g.hi_in) s = segment_or_ambiguous(du, dv, g.seg_eps);
          if (s < 0) {
            const double2 o = sxy[q];
            const double dx = __dsub_rn(o.x, xi), dy = __dsub_rn(o.y, yi);
            const double d2 = dist2(dx, dy);
            if (d2 < c.lo2 || d2 > c.hi2) continue;
            s = segment_of(dx, dy);
          }
          mk |= 1u << s;
        }
      }
    }
    mask[i] = (uint8_t)mk;
    keep_flag[t] = mk != 0xFFu;
  }
}

// out[k] = list[t] for the k-th flagged t (order kept); *count = total.
__global__ void k_compact_list(const int* __restrict__ list, const uint8_t* __restrict__ flag,
                               const int* __restrict__ pos, int m, int* __restrict__ out, int* __restrict__ count) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x)
    if (flag[t]) out[pos[t]] = list[t];
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = pos[m];
}

// Empty segments left on the open list (reported when max_rounds is hit).
__global__ void k_count_open_segments(const int* __restrict__ open, int n_open, const uint8_t* __restrict__ mask,
                                      int* __restrict__ out) {
  int s = 0;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x)
    s += __popc((~(unsigned)mask[open[t]]) & 0xFFu);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// Open list of round 1: diffused particles whose mask is not full.
__global__ void k_open_flags(const int* __restrict__ list, const int* __restrict__ list_count,
                             const uint8_t* __restrict__ mask, uint8_t* __restrict__ flag, int cap) {
  const int m = *list_count;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < cap; t += (long)gridDim.x * blockDim.x)
    flag[t] = t < m ? (mask[list[t]] != 0xFFu) : 0;
}

cudaError_t open_list(const int* dlist, const int* dcount, int cap, const uint8_t* mask, uint8_t* flag, int* pos,
                      int* open, int* n_open, int* scan_tmp, cudaStream_t s) {
  int b = blocks_for(cap);
  k_open_flags<<<b, kBlock, 0, s>>>(dlist, dcount, mask, flag, cap); note_launch();
  cudaError_t e = scan_exclusive_u8(flag, pos, cap, scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_compact_list<<<b, kBlock, 0, s>>>(dlist, flag, pos, cap, open, n_open); note_launch();
  return cudaGetLastError();
}

cudaError_t insert_count(const int* open, int n_open, const uint8_t* mask, int* cnt, int* cpos, int* scan_tmp,
                         cudaStream_t s) {
  k_cand_count<<<blocks_for(n_open), kBlock, 0, s>>>(open, n_open, mask, cnt); note_launch();
  return scan_exclusive_i32(cnt, cpos, n_open, scan_tmp, s);  // cpos[n_open] = proposals
}

cudaError_t insert_propose(const Consts& c, const int* open, int n_open, const uint8_t* mask, const int* cpos,
                           const double* x, const double* y, double* cx, double* cy, int n_cand, int ncell_cap,
                           const CandGrid& cg, uint8_t* keep, int* apos, int* scan_tmp, cudaStream_t s) {
  k_cand_emit<<<blocks_for(n_open), kBlock, 0, s>>>(c, open, n_open, mask, cpos, x, y, cx, cy); note_launch();
  cudaError_t e = grid_build(cx, cy, n_cand, c.Rh, c.lo2, c.hi2, ncell_cap, cg.grid, cg.cell_key, cg.cell_rank,
                             cg.cell_count, cg.cell_start, cg.sorted_xy, cg.sorted_loc, cg.sorted_idx, cg.bbox,
                             scan_tmp, s);
  if (e != cudaSuccess) return e;
  int b = n_cand > 0 ? (n_cand + kBlock - 1) / kBlock : 1;
  k_conflict<<<b, kBlock, 0, s>>>(c, cg.grid, cg.cell_start, cg.sorted_xy, cg.sorted_loc, cg.sorted_idx, n_cand,
                                   keep);
  note_launch();
  return scan_exclusive_u8(keep, apos, n_cand, scan_tmp, s);  // apos[n_cand] = accepted
}

cudaError_t insert_commit(const Consts& c, const int* open, int n_open, const double* cx, const double* cy,
                          int n_cand, const CandGrid& cg, const uint8_t* keep, const int* apos, int n_cur, double* x,
                          double* y, uint8_t* mask, uint8_t* keep_flag, int* keep_pos, int* open_next, int* n_next,
                          int* scan_tmp, cudaStream_t s) {
  k_append<<<blocks_for(n_cand), kBlock, 0, s>>>(cx, cy, keep, apos, n_cand, n_cur, x, y); note_launch();
  int b = n_open > 0 ? (n_open + kBlock - 1) / kBlock : 1;
  k_mask_update<<<b, kBlock, 0, s>>>(c, cg.grid, cg.cell_start, cg.sorted_xy, cg.sorted_loc, cg.sorted_idx, keep,
                                      x, y, open, n_open, mask, keep_flag);
  note_launch();
  cudaError_t e = scan_exclusive_u8(keep_flag, keep_pos, n_open, scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_compact_list<<<blocks_for(n_open), kBlock, 0, s>>>(open, keep_flag, keep_pos, n_open, open_next, n_next);
  note_launch();
  return cudaGetLastError();
}

cudaError_t count_open_segments(const int* open, int n_open, const uint8_t* mask, int* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_count_open_segments<<<blocks_for(n_open), kBlock, 0, s>>>(open, n_open, mask, out); note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
