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

// Proposal at sorted position p: 1 unless a proposal of smaller index lies
// closer than r h.  Pairs clearly apart (or clearly too close) are decided in
// FP32 on the cell-local coordinates, the rest by the FP64 distance.
__device__ __forceinline__ bool conflict_keep(const Consts& c, const Grid& g, const int* __restrict__ cell_start,
                                              const double2* __restrict__ sxy, const float2* __restrict__ sloc,
                                              const int* __restrict__ sidx, int ci, int key, long p) {
  const double2 pc = sxy[p];
  const float2 lc = sloc[p];
  const int gy = key / g.nx, gx = key - gy * g.nx;
  for (int by = gy - 1; by <= gy + 1; ++by) {
    if (by < 0 || by >= g.ny) continue;
    const float dvb = (float)(by - gy) - lc.y;
    for (int bx = gx - 1; bx <= gx + 1; ++bx) {
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
        if (close) return false;
      }
    }
  }
  return true;
}

// keep[c] = conflict_keep of every proposal.
__global__ void __launch_bounds__(kBlock) k_conflict(Consts c, const Grid* __restrict__ gp,
                                                     const int* __restrict__ cell_start,
                                                     const double2* __restrict__ sxy, const float2* __restrict__ sloc,
                                                     const int* __restrict__ sidx, const int* __restrict__ cell_key,
                                                     const int* __restrict__ n_cand_dev, uint8_t* __restrict__ keep) {
  const int n_cand = *n_cand_dev;
  const Grid g = *gp;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n_cand; p += (long)gridDim.x * blockDim.x) {
    const int ci = sidx[p];
    // the proposal's cell as binned (integer ops, no FP64)
    keep[ci] = conflict_keep(c, g, cell_start, sxy, sloc, sidx, ci, cell_key[ci], p);
  }
}

// Segment bits of the accepted proposals in the annulus of open particle i,
// ORed into mask[i]; returns true if the mask is still not full.  FP32
// filter on cell-local coordinates as in the neighbour search.  The open
// particle's cell and cell-local position come from the particle grid (the
// proposal grid has the same geometry): integer ops and one load instead of
// FP64 arithmetic.
__device__ __forceinline__ bool mask_update_one(const Consts& c, const Grid& g, const int* __restrict__ cell_start,
                                                const double2* __restrict__ sxy, const float2* __restrict__ sloc,
                                                const int* __restrict__ sidx, const uint8_t* __restrict__ keep,
                                                const double* __restrict__ x, const double* __restrict__ y,
                                                const PartCells& pcells, int i, uint8_t* __restrict__ mask) {
  const int key = pcells.cell_key[i];
  const float2 li = pcells.sorted_loc[pcells.cell_start[key] + pcells.cell_rank[i]];
  const int gy = key / g.nx, gx = key - gy * g.nx;
  const float ux = li.x, uy = li.y;
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
          const double dx = __dsub_rn(o.x, x[i]), dy = __dsub_rn(o.y, y[i]);
          const double d2 = dist2(dx, dy);
          if (d2 < c.lo2 || d2 > c.hi2) continue;
          s = segment_of(dx, dy);
        }
        mk |= 1u << s;
      }
    }
  }
  mask[i] = (uint8_t)mk;
  return mk != 0xFFu;
}

// mask_update_one for every open particle; keep_flag[t] = still open.
__global__ void __launch_bounds__(kBlock) k_mask_update(Consts c, const Grid* __restrict__ gp,
                                                        const int* __restrict__ cell_start,
                                                        const double2* __restrict__ sxy,
                                                        const float2* __restrict__ sloc,
                                                        const int* __restrict__ sidx, const uint8_t* __restrict__ keep,
                                                        const double* __restrict__ x, const double* __restrict__ y,
                                                        PartCells pcells, const int* __restrict__ open,
                                                        const int* __restrict__ n_open_dev,
                                                        uint8_t* __restrict__ mask, uint8_t* __restrict__ keep_flag) {
  const int n_open = *n_open_dev;
  const Grid g = *gp;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x)
    keep_flag[t] = mask_update_one(c, g, cell_start, sxy, sloc, sidx, keep, x, y, pcells, open[t], mask);
}

// out[k] = list[t] for the k-th flagged t (order kept); *count = total.
__global__ void k_compact_list(const int* __restrict__ list, const uint8_t* __restrict__ flag,
                               const int* __restrict__ pos, int m, const int* __restrict__ m_dev,
                               int* __restrict__ out, int* __restrict__ count) {
  if (m_dev) m = *m_dev;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x)
    if (flag[t]) out[pos[t]] = list[t];
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = pos[m];
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
  k_compact_list<<<b, kBlock, 0, s>>>(dlist, flag, pos, cap, nullptr, open, n_open); note_launch();
  return cudaGetLastError();
}

// ---- device-resident rounds (no host round trips; graph-capturable) ----------

__global__ void k_rounds_init(StepState* st, const int* __restrict__ n_open_src, cudaGraphConditionalHandle h,
                              int graph) {
  st->n_open = *n_open_src;
  st->round = 0;
  st->rounds_appended = 0;
  st->overflow = 0;
  st->n_needed = 0;
  st->open_segments = 0;
  st->n_cur = st->n;
  // with max_rounds = 0 no round runs and the open list stays as it is: its
  // empty segments are the ones reported
  const int go = st->n_open > 0 && st->max_rounds > 0;
  if (graph) cudaGraphSetConditional(h, go);
}

__global__ void k_cand_count_dev(const int* __restrict__ open, const StepState* __restrict__ st,
                                 const uint8_t* __restrict__ mask, int* __restrict__ cnt) {
  const int n_open = st->n_open;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x)
    cnt[t] = __popc((~(unsigned)mask[open[t]]) & 0xFFu);
}

// The proposals of open particle i (its empty segments, ascending) from
// list position pos on.
__device__ __forceinline__ void emit_one(const Consts& c, int i, unsigned empty, const double* __restrict__ x,
                                         const double* __restrict__ y, int pos, double* __restrict__ cx,
                                         double* __restrict__ cy) {
  const double xi = x[i], yi = y[i];
  for (int s = 0; s < 8; ++s)
    if ((empty >> s) & 1u) {
      cx[pos] = __dadd_rn(xi, c.ins_dx[s]);
      cy[pos] = __dadd_rn(yi, c.ins_dy[s]);
      ++pos;
    }
}

__global__ void k_cand_emit_dev(Consts c, const int* __restrict__ open, const StepState* __restrict__ st,
                                const uint8_t* __restrict__ mask, const int* __restrict__ cpos,
                                const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ cx,
                                double* __restrict__ cy) {
  const int n_open = st->n_open;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x) {
    const int i = open[t];
    emit_one(c, i, (~(unsigned)mask[i]) & 0xFFu, x, y, cpos[t], cx, cy);
  }
}

// Appends the accepted proposals.  Every block checks the capacity itself
// (accepted count apos[n_cand]); block 0 records the count and, when the
// cloud would outgrow its buffers, the overflow flag (then the round appends
// nothing and the loop stops).
__global__ void k_append_dev(const double* __restrict__ cx, const double* __restrict__ cy,
                             const uint8_t* __restrict__ keep, const int* __restrict__ apos,
                             StepState* __restrict__ st, double* __restrict__ x, double* __restrict__ y) {
  const int n_cand = st->n_cand, n_cur = st->n_cur;
  const int a = apos[n_cand];
  const bool over = (long)n_cur + a > st->capacity;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->accepted = a;
    if (over) {
      st->overflow = 1;
      st->n_needed = n_cur + a;
    }
  }
  if (over) return;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_cand; t += (long)gridDim.x * blockDim.x)
    if (keep[t]) {
      x[n_cur + apos[t]] = cx[t];
      y[n_cur + apos[t]] = cy[t];
    }
}

__global__ void k_copy_list(const int* __restrict__ src, int* __restrict__ dst, const StepState* __restrict__ st) {
  const int m = st->n_next;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) dst[t] = src[t];
}

__global__ void k_round_end(StepState* st, cudaGraphConditionalHandle h, int graph) {
  if (st->n_open > 0) {
    if (!st->overflow) {
      st->n_cur += st->accepted;
      if (st->accepted > 0) st->rounds_appended += 1;
    }
    st->round += 1;
    st->n_open = st->overflow ? 0 : st->n_next;
  }
  // rounds stop at max_rounds with the open list kept for the statistics
  const int go = !st->overflow && st->n_open > 0 && st->round < st->max_rounds;
  if (graph) cudaGraphSetConditional(h, go);
}

// Empty segments left (only when max_rounds ended the loop with open particles).
__global__ void k_rounds_finish(StepState* st, const int* __restrict__ open, const uint8_t* __restrict__ mask) {
  const int n_open = (st->overflow || st->round < st->max_rounds) ? 0 : st->n_open;
  int s = 0;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_open; t += (long)gridDim.x * blockDim.x)
    s += __popc((~(unsigned)mask[open[t]]) & 0xFFu);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(&st->open_segments, s);
}

cudaError_t rounds_init(StepState* st, const int* n_open_src, cudaGraphConditionalHandle handle, bool graph,
                        cudaStream_t s) {
  k_rounds_init<<<1, 1, 0, s>>>(st, n_open_src, handle, graph ? 1 : 0); note_launch();
  return cudaGetLastError();
}

cudaError_t round_body(const Consts& c, StepState* st, const Grid* pgrid, const PartCells& pcells, const RoundBufs& rb,
                       int cap, uint8_t* mask, double* x, double* y, cudaGraphConditionalHandle handle, bool graph,
                       cudaStream_t s) {
  const int bo = blocks_for(cap);
  const long cand_cap = 8L * cap;
  const int bc = blocks_for((int)(cand_cap < 0x7FFFFFFF ? cand_cap : 0x7FFFFFFF));
  k_cand_count_dev<<<bo, kBlock, 0, s>>>(rb.open, st, mask, rb.cnt); note_launch();
  cudaError_t e = scan_exclusive_i32_dev(rb.cnt, rb.cpos, cap, &st->n_open, rb.scan_tmp, s, &st->n_cand);
  if (e != cudaSuccess) return e;
  k_cand_emit_dev<<<bo, kBlock, 0, s>>>(c, rb.open, st, mask, rb.cpos, x, y, rb.cx, rb.cy); note_launch();
  // proposals binned on the particle grid's geometry (cells >= R h; points
  // outside it clamp into the edge cells, which keeps 3 x 3 scans complete)
  e = grid_bin_dev(rb.cx, rb.cy, (int)cand_cap, &st->n_cand, rb.ncell_cap, pgrid, rb.cg.cell_key,
                   rb.cg.cell_rank, rb.cg.cell_count, rb.cg.cell_start, rb.cg.sorted_xy, rb.cg.sorted_loc,
                   rb.cg.sorted_idx, rb.scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_conflict<<<bc, kBlock, 0, s>>>(c, pgrid, rb.cg.cell_start, rb.cg.sorted_xy, rb.cg.sorted_loc,
                                   rb.cg.sorted_idx, rb.cg.cell_key, &st->n_cand, rb.keep);
  note_launch();
  e = scan_exclusive_u8_dev(rb.keep, rb.apos, (int)cand_cap, &st->n_cand, rb.scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_append_dev<<<bc, kBlock, 0, s>>>(rb.cx, rb.cy, rb.keep, rb.apos, st, x, y); note_launch();
  k_mask_update<<<bo, kBlock, 0, s>>>(c, pgrid, rb.cg.cell_start, rb.cg.sorted_xy, rb.cg.sorted_loc,
                                      rb.cg.sorted_idx, rb.keep, x, y, pcells, rb.open, &st->n_open, mask,
                                      rb.keep_flag);
  note_launch();
  e = scan_exclusive_u8_dev(rb.keep_flag, rb.keep_pos, cap, &st->n_open, rb.scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_compact_list<<<bo, kBlock, 0, s>>>(rb.open, rb.keep_flag, rb.keep_pos, cap, &st->n_open, rb.open_next,
                                       &st->n_next);
  note_launch();
  k_copy_list<<<bo, kBlock, 0, s>>>(rb.open_next, rb.open, st); note_launch();
  k_round_end<<<1, 1, 0, s>>>(st, handle, graph ? 1 : 0); note_launch();
  return cudaGetLastError();
}

cudaError_t rounds_finish(StepState* st, const int* open, const uint8_t* mask, int cap, cudaStream_t s) {
  k_rounds_finish<<<blocks_for(cap), kBlock, 0, s>>>(st, open, mask); note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
