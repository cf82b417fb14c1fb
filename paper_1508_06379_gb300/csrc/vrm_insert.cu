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
//      segments ascending), so a proposal's list index is its key rank, and
//      binned into their own cell grid (cell side >= R h);
//   2. conflict test: each proposal scans the 3 x 3 cells around it for a
//      proposal of smaller list index within r h;
//   3. the accepted ones are appended in list order;
//   4. every open particle ORs into its segment mask the accepted proposals
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

// keep[c] = conflict_keep of every proposal, the same flag by sorted
// position (keep_s, for the mask update, which visits the proposals in cell
// order), and the tile sums of keep (keep_ts, 0 on entry) for the scan that
// numbers the accepted ones.
__global__ void __launch_bounds__(kBlock) k_conflict(Consts c, const Grid* __restrict__ gp,
                                                     const int* __restrict__ cell_start,
                                                     const double2* __restrict__ sxy, const float2* __restrict__ sloc,
                                                     const int* __restrict__ sidx, const int* __restrict__ cell_key,
                                                     const int* __restrict__ n_cand_dev, uint8_t* __restrict__ keep,
                                                     uint8_t* __restrict__ keep_s, int* __restrict__ keep_ts) {
  const int n_cand = *n_cand_dev;
  const Grid g = *gp;
  const int lane = threadIdx.x & 31;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_cand;
       base += (long)gridDim.x * blockDim.x) {
    const long p = base + lane;
    int ci = -1;
    bool ok = false;
    if (p < n_cand) {
      ci = sidx[p];
      // the proposal's cell as binned (integer ops, no FP64)
      ok = conflict_keep(c, g, cell_start, sxy, sloc, sidx, ci, cell_key[ci], p);
      keep[ci] = ok;
      keep_s[p] = ok;
    }
    tile_sum_add(keep_ts, ok ? ci : -1, 1);
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
                                                const uint8_t* __restrict__ keep_s, const double* __restrict__ x,
                                                const double* __restrict__ y, const PartCells& pcells, int i,
                                                uint8_t* __restrict__ mask) {
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
        if (!keep_s[q]) continue;
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

// out[k] = list[t] for the k-th flagged t (order kept); *count = total.
__global__ void k_compact_list(const int* __restrict__ list, const uint8_t* __restrict__ flag,
                               const int* __restrict__ pos, int m, const int* __restrict__ m_dev,
                               int* __restrict__ out, int* __restrict__ count) {
  if (m_dev) m = *m_dev;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x)
    if (flag[t]) out[pos[t]] = list[t];
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = pos[m];
}

// Open list of round 1: diffused particles whose mask is not full.  Each
// block takes whole scan tiles of the diffused list and writes their sums.
__global__ void __launch_bounds__(kBlock) k_open_flags(const int* __restrict__ list,
                                                       const int* __restrict__ list_count,
                                                       const uint8_t* __restrict__ mask, uint8_t* __restrict__ flag,
                                                       int* __restrict__ flag_ts) {
  static_assert(kScanTile % kBlock == 0, "a tile is whole block passes");
  __shared__ int s_w[kBlock / 32];
  const int m = *list_count;
  const int ntiles = (m + kScanTile - 1) / kScanTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanTile / kBlock; ++k) {
      const long t = (long)tile * kScanTile + k * kBlock + threadIdx.x;
      if (t < m) {
        const uint8_t f = mask[list[t]] != 0xFFu;
        flag[t] = f;
        sum += f;
      }
    }
    sum = __reduce_add_sync(0xffffffffu, sum);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < kBlock / 32; ++w) tot += s_w[w];
      flag_ts[tile] = tot;
    }
    __syncthreads();
  }
}

cudaError_t open_list(const int* dlist, const int* dcount, int cap, const uint8_t* mask, uint8_t* flag, int* pos,
                      int* open, int* n_open, int* flag_ts, cudaStream_t s) {
  const int tiles = (cap + kScanTile - 1) / kScanTile;
  k_open_flags<<<tiles < 8 * sm_count() ? tiles : 8 * sm_count(), kBlock, 0, s>>>(dlist, dcount, mask, flag, flag_ts);
  note_launch();
  cudaError_t e = scan_presummed_u8_dev(flag, pos, cap, dcount, flag_ts, s);
  if (e != cudaSuccess) return e;
  k_compact_list<<<blocks_for(cap), kBlock, 0, s>>>(dlist, flag, pos, cap, dcount, open, n_open); note_launch();
  return cudaGetLastError();
}

// ---- device-resident rounds (no host round trips; graph-capturable) ----------
//
// Every round works on the open list of the first round (open[0 .. n_list),
// ascending): cnt[t] is the number of empty segments of open particle t while
// it is open and 0 once its mask is full, so the proposals of all open
// particles, numbered by the exclusive scan of cnt, come out in key order
// without compacting the list between rounds.  The positions t still open
// are also kept unordered in act0 / act1 (even / odd rounds; appended with
// warp-aggregated atomics), so that the per-particle work of a round visits
// only them.  Per round: scan of cnt, proposals written and binned
// (k_emit_bin), scan of the cell counts, scatter into cell order
// (k_cand_scatter, which also empties the cells again for the next round),
// conflict test, scan of the accepted flags, and k_round_update: append,
// mask update, next counts and active positions, and the round's end.

__global__ void k_rounds_init(StepState* st, const int* __restrict__ n_open_src, cudaGraphConditionalHandle h,
                              int graph) {
  st->n_open = *n_open_src;
  st->n_list = st->n_open;
  st->round = 0;
  st->rounds_appended = 0;
  st->overflow = 0;
  st->n_needed = 0;
  st->open_segments = 0;
  st->n_next = 0;
  st->n_act[0] = st->n_open;
  st->n_act[1] = 0;
  st->blocks_done = 0;
  st->n_cur = st->n;
  // with max_rounds = 0 no round runs and the open list stays as it is: its
  // empty segments are the ones reported
  const int go = st->n_open > 0 && st->max_rounds > 0;
  if (graph) cudaGraphSetConditional(h, go);
}

// cnt[t] of the first round (every position active) and its tile sums:
// each block takes whole scan tiles.
__global__ void __launch_bounds__(kBlock) k_cand_count_dev(const int* __restrict__ open,
                                                           const int* __restrict__ n_open_src,
                                                           const uint8_t* __restrict__ mask, int* __restrict__ cnt,
                                                           int* __restrict__ act0, int* __restrict__ cnt_ts) {
  static_assert(kScanTile % kBlock == 0, "a tile is whole block passes");
  __shared__ int s_w[kBlock / 32];
  const int n_open = *n_open_src;
  const int ntiles = (n_open + kScanTile - 1) / kScanTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanTile / kBlock; ++k) {
      const long t = (long)tile * kScanTile + k * kBlock + threadIdx.x;
      if (t < n_open) {
        const int ct = __popc((~(unsigned)mask[open[t]]) & 0xFFu);
        cnt[t] = ct;
        act0[t] = (int)t;
        sum += ct;
      }
    }
    sum = __reduce_add_sync(0xffffffffu, sum);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < kBlock / 32; ++w) tot += s_w[w];
      cnt_ts[tile] = tot;
    }
    __syncthreads();
  }
}

// Proposals of every open particle written at their key rank and binned on
// the particle grid's geometry (cells >= R h; points outside it clamp into
// the edge cells, which keeps 3 x 3 scans complete).  Each warp takes 32
// active positions and spreads their proposals over its lanes, so that the
// FP64 position and cell arithmetic runs on full warps.  The cell counts are
// 0 on entry.
__global__ void k_emit_bin(Consts c, const int* __restrict__ open, const StepState* __restrict__ st,
                           const int* __restrict__ act0, const int* __restrict__ act1,
                           const uint8_t* __restrict__ mask, const int* __restrict__ cpos,
                           const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ cx,
                           double* __restrict__ cy, const Grid* __restrict__ gp, int* __restrict__ cell_key,
                           int* __restrict__ cell_rank, int* __restrict__ cell_count, int* __restrict__ cell_ts) {
  const int par = st->round & 1;
  const int* act = par ? act1 : act0;
  const int n_act = st->n_act[par];
  const Grid g = *gp;
  const int lane = threadIdx.x & 31;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_act; base += stride) {
    const long k = base + lane;
    int i = 0, pos0 = 0;
    unsigned empty = 0;
    double xi = 0.0, yi = 0.0;
    if (k < n_act) {
      const int t = act[k];
      i = open[t];
      empty = (~(unsigned)mask[i]) & 0xFFu;
      pos0 = cpos[t];
      xi = x[i];
      yi = y[i];
    }
    // inclusive prefix of the proposal counts over the warp
    const int cntl = __popc(empty);
    int incl = cntl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int q0 = 0; q0 < total; q0 += 32) {
      const int q = q0 + lane;
      // owner: the first lane whose inclusive prefix exceeds q
      int owner = 0;
#pragma unroll
      for (int l = 0; l < 32; ++l) {
        const int il = __shfl_sync(0xffffffffu, incl, l);
        owner += (il <= q) ? 1 : 0;
      }
      owner = owner < 31 ? owner : 31;
      const unsigned emp_o = __shfl_sync(0xffffffffu, empty, owner);
      const int excl_o = __shfl_sync(0xffffffffu, incl - cntl, owner);
      const int pos_o = __shfl_sync(0xffffffffu, pos0, owner);
      const double xo = __shfl_sync(0xffffffffu, xi, owner), yo = __shfl_sync(0xffffffffu, yi, owner);
      int key = -1;
      if (q < total) {
        const int r = q - excl_o;  // the owner's r-th empty segment (from 0), ascending
        int sg = 0, seen = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const bool e = (emp_o >> b) & 1u;
          sg = (e && seen == r) ? b : sg;
          seen += e;
        }
        const int pos = pos_o + r;
        const double xp = __dadd_rn(xo, c.ins_dx[sg]), yp = __dadd_rn(yo, c.ins_dy[sg]);
        cx[pos] = xp;
        cy[pos] = yp;
        key = grid_cell_y(g, yp) * g.nx + grid_cell_x(g, xp);
        cell_key[pos] = key;
        cell_rank[pos] = atomicAdd(&cell_count[key], 1);
      }
      tile_sum_add(cell_ts, key, 1);
    }
  }
}

// Proposals into cell order (sorted_xy, sorted_loc, sorted_idx), and their
// cells' counts set back to 0; block 0 clears the cell tile sums (read by
// the scan before) and the tile sums of keep (for the conflict test after).
__global__ void k_cand_scatter(const double* __restrict__ cx, const double* __restrict__ cy,
                               const StepState* __restrict__ st, const Grid* __restrict__ gp,
                               const int* __restrict__ cell_key, const int* __restrict__ cell_rank,
                               const int* __restrict__ cell_start, int* __restrict__ cell_count,
                               double2* __restrict__ sorted_xy, float2* __restrict__ sorted_loc,
                               int* __restrict__ sorted_idx, int* __restrict__ cell_ts, int* __restrict__ keep_ts) {
  const int n_cand = st->n_cand;
  const Grid g = *gp;
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k <= g.ncell / kScanTile; k += blockDim.x) cell_ts[k] = 0;
    for (int k = threadIdx.x; k <= n_cand / kScanTile; k += blockDim.x) keep_ts[k] = 0;
  }
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n_cand; p += (long)gridDim.x * blockDim.x) {
    const int key = cell_key[p];
    const int q = cell_start[key] + cell_rank[p];
    const double xp = cx[p], yp = cy[p];
    sorted_xy[q] = make_double2(xp, yp);
    sorted_loc[q] = make_float2(grid_local_x(g, xp, key % g.nx), grid_local_y(g, yp, key / g.nx));
    sorted_idx[q] = (int)p;
    cell_count[key] = 0;
  }
}

// Appends the accepted proposals in key order, unless the cloud would
// outgrow its buffers (then nothing is appended; k_round_update sets the
// overflow flag and the loop stops).
__global__ void k_append_dev(const double* __restrict__ cx, const double* __restrict__ cy,
                             const uint8_t* __restrict__ keep, const int* __restrict__ apos,
                             const StepState* __restrict__ st, double* __restrict__ x, double* __restrict__ y) {
  const int n_cand = st->n_cand, n_cur = st->n_cur;
  if ((long)n_cur + apos[n_cand] > st->capacity) return;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < n_cand; p += (long)gridDim.x * blockDim.x)
    if (keep[p]) {
      x[n_cur + apos[p]] = cx[p];
      y[n_cur + apos[p]] = cy[p];
    }
}

// The end of a round: every open particle's mask ORed with the accepted
// proposals of its annulus (positions [0, n_cur) of x, y, untouched by the
// append), its count for the next round set (0 once the mask is full) and,
// if still open, its position appended to the next active list; the last
// block to finish records the round's counters and the loop condition.
__global__ void __launch_bounds__(kBlock) k_round_update(
    Consts c, const Grid* __restrict__ gp, const int* __restrict__ cell_start, const double2* __restrict__ sxy,
    const float2* __restrict__ sloc, const uint8_t* __restrict__ keep_s, const int* __restrict__ apos,
    const int* __restrict__ open, int* __restrict__ cnt, int* __restrict__ cnt_ts,
    int* __restrict__ act0, int* __restrict__ act1, PartCells pcells, StepState* __restrict__ st, const double* __restrict__ x,
    const double* __restrict__ y, uint8_t* __restrict__ mask, cudaGraphConditionalHandle h, int graph) {
  const int n_cand = st->n_cand, n_cur = st->n_cur;
  const int a = apos[n_cand];
  const bool over = (long)n_cur + a > st->capacity;
  const Grid g = *gp;
  const long stride = (long)gridDim.x * blockDim.x;
  // whole warps step through the active list so that the ones still open
  // are appended to the next list with one atomic per warp
  const int par = st->round & 1;
  const int* act = par ? act1 : act0;
  int* act_next = par ? act0 : act1;
  const int n_act = st->n_act[par];
  const int lane = threadIdx.x & 31;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_act; base += stride) {
    const long k = base + lane;
    bool still = false;
    int t = 0, dc = 0;
    if (k < n_act) {
      t = act[k];
      const int i = open[t];
      still = mask_update_one(c, g, cell_start, sxy, sloc, keep_s, x, y, pcells, i, mask);
      const int cn = still ? __popc((~(unsigned)mask[i]) & 0xFFu) : 0;
      dc = cn - cnt[t];
      cnt[t] = cn;
    }
    tile_sum_add(cnt_ts, dc ? t : -1, dc);
    const unsigned sb = __ballot_sync(0xffffffffu, still);
    if (sb) {
      const int lead = __ffs(sb) - 1;
      int slot0 = 0;
      if (lane == lead) slot0 = atomicAdd(&st->n_act[par ^ 1], __popc(sb));
      slot0 = __shfl_sync(0xffffffffu, slot0, lead);
      if (still) act_next[slot0 + __popc(sb & ((1u << lane) - 1u))] = t;
    }
  }
  // the last block to finish ends the round (no shared memory in this
  // kernel: a shared flag would take L1 capacity from its lookups)
  __syncthreads();
  if (threadIdx.x != 0) return;
  __threadfence();
  if (atomicAdd(&st->blocks_done, 1u) != gridDim.x - 1) return;
  __threadfence();
  const int n_next = *(volatile int*)&st->n_act[par ^ 1];
  st->n_act[par] = 0;  // the list this round read becomes the next round's output
  st->n_next = n_next;
  st->blocks_done = 0;
  st->accepted = a;
  if (over) {
    st->overflow = 1;
    st->n_needed = n_cur + a;
  }
  if (st->n_open > 0) {
    if (!over) {
      st->n_cur = n_cur + a;
      if (a > 0) st->rounds_appended += 1;
    }
    st->round += 1;
    st->n_open = over ? 0 : n_next;
  }
  // rounds stop at max_rounds with the open particles kept for the statistics
  const int go = !over && st->n_open > 0 && st->round < st->max_rounds;
  if (graph) cudaGraphSetConditional(h, go);
}

// Empty segments left (only when max_rounds ended the loop with open
// particles): the sum of the counts.
__global__ void k_rounds_finish(StepState* st, const int* __restrict__ cnt) {
  const int n_list = (st->overflow || st->round < st->max_rounds || st->n_open == 0) ? 0 : st->n_list;
  int s = 0;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_list; t += (long)gridDim.x * blockDim.x)
    s += cnt[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(&st->open_segments, s);
}

cudaError_t rounds_init(StepState* st, const int* n_open_src, const RoundBufs& rb, const uint8_t* mask, int cap,
                        cudaGraphConditionalHandle handle, bool graph, cudaStream_t s) {
  k_rounds_init<<<1, 1, 0, s>>>(st, n_open_src, handle, graph ? 1 : 0); note_launch();
  const int tiles = (cap + kScanTile - 1) / kScanTile;
  k_cand_count_dev<<<tiles < 8 * sm_count() ? tiles : 8 * sm_count(), kBlock, 0, s>>>(rb.open, n_open_src, mask, rb.cnt,
                                                                                    rb.act0, rb.cnt_ts);
  note_launch();
  return cudaGetLastError();
}

cudaError_t round_body(const Consts& c, StepState* st, const Grid* pgrid, const PartCells& pcells, const RoundBufs& rb,
                       int cap, uint8_t* mask, double* x, double* y, cudaGraphConditionalHandle handle, bool graph,
                       cudaStream_t s) {
  const int bo = blocks_for(cap);
  const long cand_cap = 8L * cap;
  const int bc = blocks_for((int)(cand_cap < 0x7FFFFFFF ? cand_cap : 0x7FFFFFFF));
  const CandGrid& cg = rb.cg;
  const int* ncell_dev = reinterpret_cast<const int*>(reinterpret_cast<const char*>(pgrid) + offsetof(Grid, ncell));
  // the three scans of a round get their tile sums from the kernels that
  // write their inputs (k_cand_count_dev / k_round_update, k_emit_bin,
  // k_conflict)
  cudaError_t e = scan_presummed_i32_dev(rb.cnt, rb.cpos, cap, &st->n_list, rb.cnt_ts, s, &st->n_cand);
  if (e != cudaSuccess) return e;
  k_emit_bin<<<bc, kBlock, 0, s>>>(c, rb.open, st, rb.act0, rb.act1, mask, rb.cpos, x, y, rb.cx, rb.cy, pgrid,
                                   cg.cell_key, cg.cell_rank, cg.cell_count, rb.cell_ts);
  note_launch();
  e = scan_presummed_i32_dev(cg.cell_count, cg.cell_start, rb.ncell_cap, ncell_dev, rb.cell_ts, s);
  if (e != cudaSuccess) return e;
  k_cand_scatter<<<bc, kBlock, 0, s>>>(rb.cx, rb.cy, st, pgrid, cg.cell_key, cg.cell_rank, cg.cell_start,
                                       cg.cell_count, cg.sorted_xy, cg.sorted_loc, cg.sorted_idx, rb.cell_ts,
                                       rb.keep_ts);
  note_launch();
  k_conflict<<<bc, kBlock, 0, s>>>(c, pgrid, cg.cell_start, cg.sorted_xy, cg.sorted_loc, cg.sorted_idx, cg.cell_key,
                                   &st->n_cand, rb.keep, rb.keep_s, rb.keep_ts);
  note_launch();
  e = scan_presummed_u8_dev(rb.keep, rb.apos, (int)cand_cap, &st->n_cand, rb.keep_ts, s);
  if (e != cudaSuccess) return e;
  k_append_dev<<<bc, kBlock, 0, s>>>(rb.cx, rb.cy, rb.keep, rb.apos, st, x, y); note_launch();
  k_round_update<<<bo, kBlock, 0, s>>>(c, pgrid, cg.cell_start, cg.sorted_xy, cg.sorted_loc, rb.keep_s, rb.apos,
                                       rb.open, rb.cnt, rb.cnt_ts, rb.act0, rb.act1, pcells, st, x, y, mask,
                                       handle, graph ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t rounds_finish(StepState* st, const RoundBufs& rb, int cap, cudaStream_t s) {
  k_rounds_finish<<<blocks_for(cap), kBlock, 0, s>>>(st, rb.cnt); note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
