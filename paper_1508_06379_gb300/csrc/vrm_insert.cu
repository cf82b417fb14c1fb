// Insertion of zero-strength particles (Sec. 2 and Sec. 4.2).
//
// Every diffused particle whose annulus leaves a 45-degree segment empty
// proposes the point at radius 1.5 h on that segment's centre line.  The
// paper describes one insertion at a time; for many at once the rule here is
// a round: all open particles propose at once, a proposal with key (i, s) is
// dropped if a proposal of smaller key lies closer than r h, and the rest are
// appended in key order.  Rounds repeat until nothing is proposed.
//
// Work per round is proportional to the open list, not to the cloud: the
// proposals of particle i and of every particle i' that can conflict with
// them lie within 1.5h of their origins, so the origins are within 3.5 h and
// are found in the 5 x 5 cells (cell side >= 2 h) of the grid of the original
// particles.  Masks are updated incrementally with the points accepted in the
// round: a mask only gains bits.
#include "vrm_internal.cuh"

namespace vrm {

__global__ void k_cand(const int* __restrict__ open, int n_open, const uint8_t* __restrict__ mask,
                       uint8_t* __restrict__ cand) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x) {
    int i = open[t];
    cand[i] = (uint8_t)(~mask[i]);
  }
}

__global__ void k_accept(Consts c, const Grid* __restrict__ gp, const int* __restrict__ cell_start,
                         const double2* __restrict__ sxy, const int* __restrict__ sidx,
                         const double* __restrict__ x, const double* __restrict__ y, const int* __restrict__ open,
                         int n_open, const uint8_t* __restrict__ cand, uint8_t* __restrict__ acc,
                         int* __restrict__ acc_count) {
  const Grid g = *gp;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x) {
    const int i = open[t];
    const double xi = x[i], yi = y[i];
    const unsigned mine = cand[i];
    const int cx = grid_cell_x(g, xi), cy = grid_cell_y(g, yi);
    const int c0 = cx > 1 ? cx - 2 : 0, c1 = cx + 2 < g.nx ? cx + 2 : g.nx - 1;
    unsigned keep = 0;
    for (int s = 0; s < 8; ++s) {
      if (!((mine >> s) & 1u)) continue;
      const double px = __dadd_rn(xi, c.ins_dx[s]), py = __dadd_rn(yi, c.ins_dy[s]);
      bool ok = true;
      for (int by = cy - 2; by <= cy + 2 && ok; ++by) {
        if (by < 0 || by >= g.ny) continue;
        const int q0 = cell_start[by * g.nx + c0], q1 = cell_start[by * g.nx + c1 + 1];
        for (int q = q0; q < q1 && ok; ++q) {
          const int ip = sidx[q];
          if (ip > i) continue;
          unsigned cb = cand[ip];
          if (ip == i) cb &= (1u << s) - 1u;
          if (!cb) continue;
          const double2 op = sxy[q];
          for (int sp = 0; sp < 8; ++sp) {
            if (!((cb >> sp) & 1u)) continue;
            const double qx = __dadd_rn(op.x, c.ins_dx[sp]), qy = __dadd_rn(op.y, c.ins_dy[sp]);
            const double d2 = dist2(__dsub_rn(px, qx), __dsub_rn(py, qy));
            if (d2 < c.lo2) {
              ok = false;
              break;
            }
          }
        }
      }
      if (ok) keep |= 1u << s;
    }
    acc[i] = (uint8_t)keep;
    acc_count[t] = __popc(keep);
  }
}

__global__ void k_append(Consts c, const int* __restrict__ open, int n_open, const uint8_t* __restrict__ acc,
                         const int* __restrict__ acc_pos, int n_cur, double* __restrict__ x, double* __restrict__ y) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x) {
    const int i = open[t];
    const unsigned a = acc[i];
    if (!a) continue;
    const double xi = x[i], yi = y[i];
    int pos = n_cur + acc_pos[t];
    for (int s = 0; s < 8; ++s)
      if ((a >> s) & 1u) {
        x[pos] = __dadd_rn(xi, c.ins_dx[s]);
        y[pos] = __dadd_rn(yi, c.ins_dy[s]);
        ++pos;
      }
  }
}

__global__ void k_mask_update(Consts c, const Grid* __restrict__ gp, const int* __restrict__ cell_start,
                              const double2* __restrict__ sxy, const int* __restrict__ sidx,
                              const double* __restrict__ x, const double* __restrict__ y,
                              const int* __restrict__ open, int n_open, const uint8_t* __restrict__ acc,
                              uint8_t* __restrict__ mask, uint8_t* __restrict__ keep_flag) {
  const Grid g = *gp;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x) {
    const int i = open[t];
    const double xi = x[i], yi = y[i];
    const int cx = grid_cell_x(g, xi), cy = grid_cell_y(g, yi);
    const int c0 = cx > 1 ? cx - 2 : 0, c1 = cx + 2 < g.nx ? cx + 2 : g.nx - 1;
    unsigned mk = mask[i];
    for (int by = cy - 2; by <= cy + 2; ++by) {
      if (by < 0 || by >= g.ny) continue;
      const int q0 = cell_start[by * g.nx + c0], q1 = cell_start[by * g.nx + c1 + 1];
      for (int q = q0; q < q1; ++q) {
        const unsigned a = acc[sidx[q]];
        if (!a) continue;
        const double2 op = sxy[q];
        for (int sp = 0; sp < 8; ++sp) {
          if (!((a >> sp) & 1u)) continue;
          const double qx = __dadd_rn(op.x, c.ins_dx[sp]), qy = __dadd_rn(op.y, c.ins_dy[sp]);
          const double dx = __dsub_rn(qx, xi), dy = __dsub_rn(qy, yi);
          const double d2 = dist2(dx, dy);
          if (d2 < c.lo2 || d2 > c.hi2) continue;
          mk |= 1u << segment_of(dx, dy);
        }
      }
    }
    mask[i] = (uint8_t)mk;
    keep_flag[t] = mk != 0xFFu;
  }
}

__global__ void k_clear_round(const int* __restrict__ open, int n_open, uint8_t* __restrict__ cand,
                              uint8_t* __restrict__ acc) {
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x) {
    int i = open[t];
    cand[i] = 0;
    acc[i] = 0;
  }
}

// open[k] = list[k'] for the k-th flagged entry (order kept).
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

static int blocks_for(int m) {
  int b = m > 0 ? (m + kBlock - 1) / kBlock : 1;
  return b < 8 * sm_count() ? b : 8 * sm_count();
}

cudaError_t insert_round_accept(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                                const int* sorted_idx, const double* x, const double* y, const int* open,
                                int n_open, const uint8_t* mask, uint8_t* cand, uint8_t* acc, int* acc_count,
                                int* acc_pos, int* scan_tmp, cudaStream_t s) {
  int b = blocks_for(n_open);
  k_cand<<<b, kBlock, 0, s>>>(open, n_open, mask, cand); note_launch();
  k_accept<<<b, kBlock, 0, s>>>(c, g, cell_start, sorted_xy, sorted_idx, x, y, open, n_open, cand, acc, acc_count); note_launch();
  return scan_exclusive_i32(acc_count, acc_pos, n_open, scan_tmp, s);  // acc_pos[n_open] = accepted
}

cudaError_t insert_round_commit(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                                const int* sorted_idx, double* x, double* y, int n_cur, const int* open, int n_open,
                                uint8_t* mask, uint8_t* cand, uint8_t* acc, const int* acc_pos, int* open_next,
                                uint8_t* keep_flag, int* keep_pos, int* n_next, int* scan_tmp, cudaStream_t s) {
  int b = blocks_for(n_open);
  k_append<<<b, kBlock, 0, s>>>(c, open, n_open, acc, acc_pos, n_cur, x, y); note_launch();
  k_mask_update<<<b, kBlock, 0, s>>>(c, g, cell_start, sorted_xy, sorted_idx, x, y, open, n_open, acc, mask,
                                     keep_flag); note_launch();
  k_clear_round<<<b, kBlock, 0, s>>>(open, n_open, cand, acc); note_launch();
  cudaError_t e = scan_exclusive_u8(keep_flag, keep_pos, n_open, scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_compact_list<<<b, kBlock, 0, s>>>(open, keep_flag, keep_pos, n_open, open_next, n_next); note_launch();
  return cudaGetLastError();
}

cudaError_t count_open_segments(const int* open, int n_open, const uint8_t* mask, int* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_count_open_segments<<<blocks_for(n_open), kBlock, 0, s>>>(open, n_open, mask, out); note_launch();
  return cudaGetLastError();
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

}  // namespace vrm
