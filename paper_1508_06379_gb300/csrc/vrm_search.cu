// Annulus neighbourhoods (Sec. 2, Eq. neighbourhood), 45-degree segment
// masks (Sec. 4.2) and small neighbourhoods (Sec. 4.3) on the cell grid.
//
// One thread per particle, taken in cell order so that the threads of a warp
// read overlapping cells.  Each thread scans the 3 x 3 cells around its own.
// The annulus test of the method is the FP64 definition
//   lo2 <= dx*dx + dy*dy <= hi2,  dx = x_j - x_i,  dy = y_j - y_i,
// every operation rounded separately.  GB300 runs FP64 at 1/60 of its FP32
// rate, so each pair is measured in FP32 on cell-local coordinates (error
// below 1e-5 cell^2): a pair further than the band from both bounds is
// decided in FP32; segments are decided in FP32 unless the offset lies within
// seg_eps of a decision line; the closest member of a segment is chosen in
// FP32 unless another member lies within two bands of it.  Only the
// undecided cases (rare on jittered clouds, frequent on exact lattices) take
// the FP64 definition, so the result is bit-identical to it.
//
// The row is kept in a per-thread buffer of KCAP entries (rows are k_cap
// apart): sorted by index for the library's neighbourhood calls, in visiting
// order inside a step (SORTED = false: the application orders the few
// matches itself, and a sorted insertion per member was a third of the
// kernel); a row that overflows keeps the row_cap smallest indices either
// way, except in the step's form over the diffused list (LIST), which
// writes members straight to the row and cuts it at row_cap: the step
// then repeats with whole rows or reports the capacity error.  The closest particle of every segment is tracked in shared memory
// with ties to the smaller index.
#include "vrm_internal.cuh"

namespace vrm {

// Exact member test and segment of one candidate pair, for the rare pairs
// the FP32 measure cannot decide.  Returns the segment, or -1 if j is not in
// the annulus of i.
__device__ __forceinline__ int exact_member(const Consts& c, const double2& pi, const double2& pj, bool certain_in,
                                            double* d2_out) {
  const double dx = __dsub_rn(pj.x, pi.x), dy = __dsub_rn(pj.y, pi.y);
  const double d2 = dist2(dx, dy);
  *d2_out = d2;
  if (!certain_in && (d2 < c.lo2 || d2 > c.hi2)) return -1;
  return segment_of(dx, dy);
}

// Small neighbourhood bookkeeping: per segment the smallest FP32 squared
// distance and its particle, and a flag `amb` set when another member of
// the segment lies within 2 bands of it (then the FP32 order may differ from
// the FP64 order, and a second pass decides that segment exactly).
//
// LIST = true: only the particles of `list` (list_count of them; the step's
// diffused set, the only particles whose rows the step reads), each located
// in the sorted arrays through its cell key and rank; threads follow the
// list's order.  Rows are then padded with -1 to the end of their last
// 32-byte sector, so that the sector is written whole.
// ROWS = false (list form only): the rows are not written (the count, mask
// and small neighbourhood are).
template <int KCAP, bool SORTED, bool LIST = false, bool ROWS = true>
__global__ void __launch_bounds__(kBlock) k_search_all(Consts c, const Grid* __restrict__ gp,
                                                       const int* __restrict__ cell_start,
                                                       const double2* __restrict__ sxy,
                                                       const float2* __restrict__ sloc,
                                                       const int* __restrict__ sidx, int n,
                                                       const int* __restrict__ n_dev,
                                                       int* __restrict__ nbr_count, int* __restrict__ nbr_idx,
                                                       uint8_t* __restrict__ seg_mask, int* __restrict__ small,
                                                       DevStats* __restrict__ ds,
                                                       const int* __restrict__ list = nullptr,
                                                       const int* __restrict__ cell_key = nullptr,
                                                       const int* __restrict__ cell_rank = nullptr) {
  if (n_dev) n = *n_dev;
  const Grid g = *gp;
  const int k_cap = c.row_cap < KCAP ? c.row_cap : KCAP;  // entries kept
  const size_t stride = (size_t)c.k_cap;
  const float tie = 2.f * kBand;
  int local_max = 0;
  // closest member of every segment so far (FP32 squared distance, index),
  // one column per thread: read and written with a dynamic segment index
  // (conflict-free: the row stride, the block size, is a multiple of 32
  // words).  Sized by the launch (8 + 8 words per thread), so that a small
  // block leaves the rest of the SM's shared memory to L1.
  extern __shared__ int s_search[];
  const int nb = blockDim.x;
  float* const s_bf = reinterpret_cast<float*>(s_search);
  int* const s_bj = s_search + 8 * nb;
  const int tx = threadIdx.x;
  for (long t0 = (long)blockIdx.x * blockDim.x + threadIdx.x; t0 < n; t0 += (long)gridDim.x * blockDim.x) {
    int i, cx, cy;
    long p;
    if (LIST) {
      i = list[t0];
      const int key = cell_key[i];
      p = cell_start[key] + cell_rank[i];
      cy = key / g.nx;
      cx = key - cy * g.nx;
    } else {
      p = t0;
      i = sidx[p];
    }
    const double2 pi = sxy[p];
    const float2 li = sloc[p];
    if (!LIST) {
      cx = grid_cell_x(g, pi.x);
      cy = grid_cell_y(g, pi.y);
    }
    // LIST: members go straight to the row in visiting order (a row longer
    // than row_cap is cut; the step then repeats with whole rows or reports
    // the capacity error, so no smallest-index rule is needed); otherwise
    // they are collected in a per-thread buffer first
    int list[LIST ? 1 : KCAP];
    int* const row_out = nbr_idx + (size_t)i * stride;
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      s_bf[t * nb + tx] = 3e38f;
      s_bj[t * nb + tx] = -1;
    }
    unsigned mask = 0, amb = 0;
    for (int by = cy - 1; by <= cy + 1; ++by) {
      if (by < 0 || by >= g.ny) continue;
      const float dvb = (float)(by - cy) - li.y;
      for (int bx = cx - 1; bx <= cx + 1; ++bx) {
        if (bx < 0 || bx >= g.nx) continue;
        const float dub = (float)(bx - cx) - li.x;
        const int cell = by * g.nx + bx;
        const int q0 = cell_start[cell], q1 = cell_start[cell + 1];
        // the next candidate's coordinates and index are loaded while this
        // one is tested (the loop is bound by load latency)
        float2 lnext = q0 < q1 ? sloc[q0] : make_float2(0.f, 0.f);
        int jnext = q0 < q1 ? sidx[q0] : 0;
        for (int q = q0; q < q1; ++q) {
          const float2 lj = lnext;
          const int j = jnext;
          if (q + 1 < q1) {
            lnext = sloc[q + 1];
            jnext = sidx[q + 1];
          }
          const float du = dub + lj.x, dv = dvb + lj.y;
          const float d2f = __fmaf_rn(du, du, dv * dv);
          if (d2f < g.lo_out || d2f > g.hi_out) continue;
          if (j == i) continue;
          const bool certain_in = d2f > g.lo_in && d2f < g.hi_in;
          int s = certain_in ? segment_or_ambiguous(du, dv, g.seg_eps) : -1;
          if (s < 0) {
            double d2;
            s = exact_member(c, pi, sxy[q], certain_in, &d2);
            if (s < 0) continue;
          }
          mask |= 1u << s;
          const float cb = s_bf[s * nb + tx];
          const int cjb = s_bj[s * nb + tx];
          const bool take = cjb < 0 || d2f < cb || (d2f == cb && j < cjb);
          // conservative: the displaced or the new member is close to the best
          const bool close = cjb >= 0 && fabsf(d2f - cb) <= tie;
          if (close) amb |= 1u << s;
          if (take) {
            s_bf[s * nb + tx] = d2f;
            s_bj[s * nb + tx] = j;
          }
          if (LIST) {
            if (ROWS && cnt < k_cap) row_out[cnt] = j;
          } else if (SORTED || cnt >= k_cap) {
            if (!SORTED && cnt == k_cap) {
              // the row overflows (rare): order the entries kept so far, so
              // that it keeps the k_cap smallest indices like a sorted row
              for (int a = 1; a < k_cap; ++a) {
                const int v = list[a];
                int b = a;
                while (b > 0 && list[b - 1] > v) {
                  list[b] = list[b - 1];
                  --b;
                }
                list[b] = v;
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
          } else {
            list[cnt] = j;  // unsorted row: append in visiting order
          }
          ++cnt;
        }
      }
    }
    int bj[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) bj[t] = s_bj[t * nb + tx];
    if (amb) {
      // exact FP64 order (ties to the smaller index) for the flagged segments
      double bd[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        bd[t] = 1e300;
        if ((amb >> t) & 1u) bj[t] = -1;
      }
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
            const bool certain_in = d2f > g.lo_in && d2f < g.hi_in;
            double d2;
            const int s = exact_member(c, pi, sxy[q], certain_in, &d2);
            if (s < 0 || !((amb >> s) & 1u)) continue;
            double cb = bd[0];
            int cjb = bj[0];
#pragma unroll
            for (int t = 1; t < 8; ++t) {
              cb = (s == t) ? bd[t] : cb;
              cjb = (s == t) ? bj[t] : cjb;
            }
            if (cjb < 0 || d2 < cb || (d2 == cb && j < cjb)) {
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                bd[t] = (s == t) ? d2 : bd[t];
                bj[t] = (s == t) ? j : bj[t];
              }
            }
          }
        }
      }
    }
    nbr_count[i] = cnt;
    const int m = cnt < k_cap ? cnt : k_cap;
    int* row = nbr_idx + (size_t)i * stride;
    if (!LIST)
      for (int t = 0; t < m; ++t) row[t] = list[t];
    if (LIST && ROWS) {
      const int pad = ((m + 7) & ~7) < (int)stride ? ((m + 7) & ~7) : (int)stride;
      for (int t = m; t < pad; ++t) row[t] = -1;
    }
    seg_mask[i] = (uint8_t)mask;
    int4* sm = reinterpret_cast<int4*>(small + (size_t)i * 8);
    sm[0] = make_int4(bj[0], bj[1], bj[2], bj[3]);
    sm[1] = make_int4(bj[4], bj[5], bj[6], bj[7]);
    local_max = cnt > local_max ? cnt : local_max;
  }
  // one atomic per block (one per warp on a single address serialises at L2)
  local_max = (int)__reduce_max_sync(0xffffffffu, (unsigned)local_max);
  __shared__ int w_max[kBlock / 32];
  if ((threadIdx.x & 31) == 0) w_max[threadIdx.x >> 5] = local_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) local_max = w_max[w] > local_max ? w_max[w] : local_max;
    if (local_max > 0) atomicMax(&ds->max_count, local_max);
  }
}

// Segment masks of the listed particles (the diffused list, in index order:
// lattice order keeps a warp's particles neighbours), each located in the
// sorted arrays through its cell key and rank: FP32 distances on the
// cell-local coordinates, the FP64 definition only for the pairs within the
// band of an annulus bound or a segment line.
__global__ void __launch_bounds__(kBlock) k_search_masks_list(Consts c, const Grid* __restrict__ gp,
                                                              const int* __restrict__ cell_start,
                                                              const double2* __restrict__ sxy,
                                                              const float2* __restrict__ sloc,
                                                              const int* __restrict__ sidx,
                                                              const int* __restrict__ cell_key,
                                                              const int* __restrict__ cell_rank,
                                                              const int* __restrict__ list,
                                                              const int* __restrict__ list_count,
                                                              uint8_t* __restrict__ mask) {
  const int m = *list_count;
  const Grid g = *gp;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x) {
    const int i = list[t];
    const int key = cell_key[i];
    const int p = cell_start[key] + cell_rank[i];
    const double2 pi = sxy[p];
    const float2 li = sloc[p];
    const int cy = key / g.nx, cx = key - cy * g.nx;
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

cudaError_t search_masks_list_dev(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                                  const float2* sorted_loc, const int* sorted_idx, const int* cell_key,
                                  const int* cell_rank, const int* list, const int* list_count, int m_bound,
                                  uint8_t* mask, cudaStream_t s) {
  if (m_bound <= 0) return cudaSuccess;
  const int blocks = (m_bound + kBlock - 1) / kBlock;
  k_search_masks_list<<<blocks, kBlock, 0, s>>>(c, g, cell_start, sorted_xy, sorted_loc, sorted_idx, cell_key,
                                                cell_rank, list, list_count, mask);
  note_launch();
  return cudaGetLastError();
}

// Dynamic shared memory of k_search_all: a segment's best distance and
// index per thread, eight segments.
static size_t search_smem(int tb) { return (size_t)tb * 8 * (sizeof(float) + sizeof(int)); }

cudaError_t search_all_dev(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                           const float2* sorted_loc, const int* sorted_idx, int n_bound, const int* n_dev,
                           int* nbr_count, int* nbr_idx, uint8_t* seg_mask, int* small, DevStats* ds,
                           cudaStream_t s, bool sorted) {
  if (n_bound <= 0) return cudaSuccess;
  const int tb = c.search_block;
  const int blocks = (int)(((long)n_bound + tb - 1) / tb);
#define VRM_SEARCH_LAUNCH(K, S)                                                                                     \
  k_search_all<K, S><<<blocks, tb, search_smem(tb), s>>>(c, g, cell_start, sorted_xy, sorted_loc, sorted_idx,      \
                                                         n_bound, n_dev, nbr_count, nbr_idx, seg_mask, small, ds)
  if (c.row_cap <= 16) {
    if (sorted) VRM_SEARCH_LAUNCH(16, true); else VRM_SEARCH_LAUNCH(16, false);
  } else if (c.row_cap <= 24) {
    if (sorted) VRM_SEARCH_LAUNCH(24, true); else VRM_SEARCH_LAUNCH(24, false);
  } else {
    if (sorted) VRM_SEARCH_LAUNCH(VRM_KCAP_MAX, true); else VRM_SEARCH_LAUNCH(VRM_KCAP_MAX, false);
  }
#undef VRM_SEARCH_LAUNCH
  note_launch();
  return cudaGetLastError();
}

cudaError_t search_list_dev(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                            const float2* sorted_loc, const int* sorted_idx, const int* cell_key,
                            const int* cell_rank, const int* list, const int* list_count, int m_bound,
                            int* nbr_count, int* nbr_idx, uint8_t* seg_mask, int* small, DevStats* ds,
                            cudaStream_t s, bool rows) {
  if (m_bound <= 0) return cudaSuccess;
  const int tb = c.search_block;
  const int blocks = (int)(((long)m_bound + tb - 1) / tb);
#define VRM_SEARCH_LAUNCH(K, R)                                                                                    \
  k_search_all<K, false, true, R><<<blocks, tb, search_smem(tb), s>>>(                                            \
      c, g, cell_start, sorted_xy, sorted_loc, sorted_idx, m_bound, list_count, nbr_count, nbr_idx, seg_mask, small, \
      ds, list, cell_key, cell_rank)
  if (!rows)
    VRM_SEARCH_LAUNCH(VRM_KCAP_MAX, false);  // rows not written: the cap only bounds the count
  else if (c.row_cap <= 16)
    VRM_SEARCH_LAUNCH(16, true);
  else if (c.row_cap <= 24)
    VRM_SEARCH_LAUNCH(24, true);
  else
    VRM_SEARCH_LAUNCH(VRM_KCAP_MAX, true);
#undef VRM_SEARCH_LAUNCH
  note_launch();
  return cudaGetLastError();
}

cudaError_t search_all(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                       const float2* sorted_loc, const int* sorted_idx, int n, int* nbr_count, int* nbr_idx,
                       uint8_t* seg_mask, int* small, DevStats* ds, cudaStream_t s) {
  return search_all_dev(c, g, cell_start, sorted_xy, sorted_loc, sorted_idx, n, nullptr, nbr_count, nbr_idx,
                        seg_mask, small, ds, s, true);
}

}  // namespace vrm
