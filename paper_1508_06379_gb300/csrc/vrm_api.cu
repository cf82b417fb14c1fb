// C ABI of the VRM library: parameter checks, context scratch, and the
// order of the stages of one operator evaluation (Sec. 3.3, 3.5, 4):
// growth control -> insertion -> neighbourhoods -> weights -> application.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "vrm_internal.cuh"

using namespace vrm;

namespace {

struct Buf {
  void* p = nullptr;
};

}  // namespace

struct vrm::Scratch {
  int cap = 0;        // particles the buffers hold
  int ncell_cap = 0;  // cells of the grid
  // grid
  Grid* grid = nullptr;
  int *cell_key = nullptr, *cell_rank = nullptr, *cell_count = nullptr, *cell_start = nullptr;
  double2* sorted_xy = nullptr;
  float2* sorted_loc = nullptr;
  int* sorted_idx = nullptr;
  unsigned long long* bbox = nullptr;
  int *scan_tmp = nullptr, *pos = nullptr;
  // growth control
  ReduceState* rstate = nullptr;
  uint8_t* tie_flag = nullptr;
  int* tie_rank = nullptr;
  uint8_t* diffused = nullptr;
  int* dlist = nullptr;
  // insertion
  uint8_t *mask = nullptr, *keep_flag = nullptr;
  int *open_a = nullptr, *open_b = nullptr, *keep_pos = nullptr, *ccnt = nullptr, *ccpos = nullptr;
  // proposals of one insertion round (grown on demand)
  int cand_cap = 0, cand_ncell_cap = 0;
  double *cx = nullptr, *cy = nullptr;
  uint8_t* ckeep = nullptr;
  int *capos = nullptr, *cscan_tmp = nullptr;
  CandGrid cg = {};
  // neighbourhoods and weights of vrm_step
  int *nbr_count = nullptr, *nbr_idx = nullptr, *small = nullptr, *cols = nullptr, *fail_list = nullptr;
  uint8_t *seg_mask = nullptr, *status = nullptr;
  double *f = nullptr, *fii = nullptr;
  // counters
  DevStats* ds = nullptr;
  int* counters = nullptr;  // [0] |D|, [1] n_open, [2] n_next, [3] open segments
  DevStats* h_ds = nullptr;  // pinned
  int* h_counters = nullptr; // pinned
  Grid* h_grid = nullptr;    // pinned
};

struct vrm_ctx {
  vrm_params p;
  Consts c;
  int device = 0;
  Scratch s;
  // per-stage timing: ev[k] is recorded where stage k starts, ev[k+1] where it ends
  int timing = 0;
  int events_ready = 0;
  int stage_done[VRM_STAGE_COUNT] = {0};
  cudaEvent_t ev[VRM_STAGE_COUNT + 1];
};

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

void free_cand(Scratch& s) {
  void* ptrs[] = {s.cx, s.cy, s.ckeep, s.capos, s.cscan_tmp, s.cg.grid, s.cg.cell_key, s.cg.cell_rank,
                  s.cg.cell_count, s.cg.cell_start, s.cg.sorted_idx, s.cg.sorted_xy, s.cg.sorted_loc, s.cg.bbox};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  s.cx = s.cy = nullptr;
  s.ckeep = nullptr;
  s.capos = s.cscan_tmp = nullptr;
  s.cg = CandGrid{};
  s.cand_cap = s.cand_ncell_cap = 0;
}

void free_scratch(Scratch& s) {
  free_cand(s);
  void* ptrs[] = {s.grid, s.cell_key, s.cell_rank, s.cell_count, s.cell_start, s.sorted_xy, s.sorted_loc,
                  s.sorted_idx, s.bbox,
                  s.scan_tmp, s.pos, s.rstate, s.tie_flag, s.tie_rank, s.diffused, s.dlist, s.mask, s.keep_flag,
                  s.open_a, s.open_b, s.keep_pos, s.ccnt, s.ccpos, s.nbr_count, s.nbr_idx, s.small, s.cols,
                  s.fail_list, s.seg_mask, s.status, s.f, s.fii, s.ds, s.counters};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s.h_ds) cudaFreeHost(s.h_ds);
  if (s.h_counters) cudaFreeHost(s.h_counters);
  if (s.h_grid) cudaFreeHost(s.h_grid);
  Scratch empty;
  s = empty;
}

// Scratch for `cap` particles (grown by 25% steps, never shrunk).
cudaError_t ensure_scratch(vrm_ctx* ctx, int cap, cudaStream_t st) {
  Scratch& s = ctx->s;
  if (cap <= s.cap && s.ds) return cudaSuccess;
  cudaStreamSynchronize(st);
  long want = cap;
  if (s.cap > 0 && want < (long)s.cap + s.cap / 4) want = (long)s.cap + s.cap / 4;
  if (want < 1024) want = 1024;
  if (want > 0x7FFFFFF0L) want = 0x7FFFFFF0L;
  free_scratch(s);
  const int n = (int)want;
  const int k = ctx->p.k_cap;
  const long ncell = 2 * (long)n + 1024;
  s.cap = n;
  s.ncell_cap = (int)ncell;
  cudaError_t e = cudaSuccess;
#define VRM_ALLOC(ptr, count) \
  if (e == cudaSuccess) e = dalloc(&(ptr), (size_t)(count))
  VRM_ALLOC(s.grid, 1);
  VRM_ALLOC(s.cell_key, n);
  VRM_ALLOC(s.cell_rank, n);
  VRM_ALLOC(s.cell_count, ncell);
  VRM_ALLOC(s.cell_start, ncell + 1);
  VRM_ALLOC(s.sorted_xy, n);
  VRM_ALLOC(s.sorted_loc, n);
  VRM_ALLOC(s.sorted_idx, n);
  VRM_ALLOC(s.bbox, 8);
  VRM_ALLOC(s.scan_tmp, scan_tmp_ints((int)(ncell > n ? ncell : n)) + 16);
  VRM_ALLOC(s.pos, (long)n + 1);
  VRM_ALLOC(s.rstate, 1);
  VRM_ALLOC(s.tie_flag, n);
  VRM_ALLOC(s.tie_rank, (long)n + 1);
  VRM_ALLOC(s.diffused, n);
  VRM_ALLOC(s.dlist, n);
  VRM_ALLOC(s.mask, n);
  VRM_ALLOC(s.keep_flag, n);
  VRM_ALLOC(s.open_a, n);
  VRM_ALLOC(s.open_b, n);
  VRM_ALLOC(s.keep_pos, (long)n + 1);
  VRM_ALLOC(s.ccnt, n);
  VRM_ALLOC(s.ccpos, (long)n + 1);
  VRM_ALLOC(s.nbr_count, n);
  VRM_ALLOC(s.nbr_idx, (long)n * k);
  VRM_ALLOC(s.small, (long)n * 8);
  VRM_ALLOC(s.cols, (long)n * VRM_STENCIL_W);
  VRM_ALLOC(s.fail_list, n);
  VRM_ALLOC(s.seg_mask, n);
  VRM_ALLOC(s.status, n);
  VRM_ALLOC(s.f, (long)n * VRM_STENCIL_W);
  VRM_ALLOC(s.fii, n);
  VRM_ALLOC(s.ds, 1);
  VRM_ALLOC(s.counters, 8);
#undef VRM_ALLOC
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_ds, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_counters, sizeof(int) * 8);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_grid, sizeof(Grid));
  if (e != cudaSuccess) {
    free_scratch(s);
    cudaGetLastError();
  }
  return e;
}

// Proposal buffers for n_cand proposals (grown by 50% steps, never shrunk).
cudaError_t ensure_cand(Scratch& s, int n_cand, cudaStream_t st) {
  if (n_cand <= s.cand_cap && s.cx) return cudaSuccess;
  cudaStreamSynchronize(st);
  long want = n_cand;
  if (want < (long)s.cand_cap + s.cand_cap / 2) want = (long)s.cand_cap + s.cand_cap / 2;
  if (want < 4096) want = 4096;
  if (want > 0x7FFFFFF0L) want = 0x7FFFFFF0L;
  free_cand(s);
  const long ncell = 2 * want + 1024;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dalloc(&s.cx, want);
  if (e == cudaSuccess) e = dalloc(&s.cy, want);
  if (e == cudaSuccess) e = dalloc(&s.ckeep, want);
  if (e == cudaSuccess) e = dalloc(&s.capos, want + 1);
  if (e == cudaSuccess) e = dalloc(&s.cscan_tmp, scan_tmp_ints((int)ncell) + 16);
  if (e == cudaSuccess) e = dalloc(&s.cg.grid, 1);
  if (e == cudaSuccess) e = dalloc(&s.cg.cell_key, want);
  if (e == cudaSuccess) e = dalloc(&s.cg.cell_rank, want);
  if (e == cudaSuccess) e = dalloc(&s.cg.cell_count, ncell);
  if (e == cudaSuccess) e = dalloc(&s.cg.cell_start, ncell + 1);
  if (e == cudaSuccess) e = dalloc(&s.cg.sorted_idx, want);
  if (e == cudaSuccess) e = dalloc(&s.cg.sorted_xy, want);
  if (e == cudaSuccess) e = dalloc(&s.cg.sorted_loc, want);
  if (e == cudaSuccess) e = dalloc(&s.cg.bbox, 8);
  if (e != cudaSuccess) {
    free_cand(s);
    cudaGetLastError();
    return e;
  }
  s.cand_cap = (int)want;
  s.cand_ncell_cap = (int)ncell;
  return cudaSuccess;
}

#define VRM_CUDA(call)                       \
  do {                                       \
    cudaError_t _e = (call);                 \
    if (_e != cudaSuccess) return VRM_ERR_CUDA; \
  } while (0)

vrm_status check_params(const vrm_params* p) {
  if (!p) return VRM_ERR_ARG;
  if (!(p->h > 0) || !std::isfinite(p->h)) return VRM_ERR_ARG;
  if (!(p->r > 0) || !(p->R > p->r) || !std::isfinite(p->R)) return VRM_ERR_ARG;
  if (!(p->nu >= 0) || !std::isfinite(p->nu)) return VRM_ERR_ARG;
  if (!(p->c_diff >= 0) || !std::isfinite(p->c_diff)) return VRM_ERR_ARG;
  if (p->k_cap < 8 || p->k_cap > VRM_KCAP_MAX) return VRM_ERR_ARG;
  if (p->max_rounds < 0 || p->max_rounds > 1000) return VRM_ERR_ARG;
  if (p->order != 1) return VRM_ERR_UNSUPPORTED;
  if (p->precision != VRM_PREC_FP64) return VRM_ERR_UNSUPPORTED;
  return VRM_OK;
}

void fill_consts(const vrm_params& p, Consts& c) {
  memset(&c, 0, sizeof(c));
  const double h = p.h;
  const double rh = p.r * h, Rh = p.R * h;
  c.h = h;
  c.inv_h = 1.0 / h;
  c.lo2 = rh * rh;
  c.hi2 = Rh * Rh;
  c.lo2f = (float)c.lo2;
  c.hi2f = (float)c.hi2;
  c.Rh = Rh;
  volatile double hh = h * h;  // keep the documented rounding order
  volatile double hhh = hh * h;
  c.c_bound = p.c_diff * hhh;
  c.nu_over_h2 = p.nu / hh;
  // insertion offsets: radius 1.5 h on the segment centre lines (s + 1/2) pi/4,
  // with cos and sin of 22.5 degrees from the half-angle identities
  volatile double r2 = std::sqrt(2.0);
  const double cs = 0.5 * std::sqrt(2.0 + r2), sn = 0.5 * std::sqrt(2.0 - r2);
  const double ux[8] = {cs, sn, -sn, -cs, -cs, -sn, sn, cs};
  const double uy[8] = {sn, cs, cs, sn, -sn, -cs, -cs, -sn};
  volatile double a = 1.5 * h;
  for (int k = 0; k < 8; ++k) {
    c.ins_dx[k] = a * ux[k];
    c.ins_dy[k] = a * uy[k];
  }
  c.k_cap = p.k_cap;
  c.max_rounds = p.max_rounds;
  c.fallback = p.fallback;
  c.precision = p.precision;
}

cudaError_t read_back(vrm_ctx* ctx, cudaStream_t st) {
  Scratch& s = ctx->s;
  cudaError_t e = cudaMemcpyAsync(s.h_ds, s.ds, sizeof(DevStats), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_counters, s.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_grid, s.grid, sizeof(Grid), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

double ratio_from_bits(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
}

cudaError_t mark(vrm_ctx* ctx, int k, cudaStream_t st);

// Growth control + insertion on x, y (capacity entries, n given).  Leaves the
// diffused flags in `diffused` (capacity), the diffused list in s.dlist with
// its count in s.counters[0], and *n_cur = n'.
vrm_status stage_insert_reduce(vrm_ctx* ctx, double* x, double* y, int n, int capacity, const double* gamma,
                               uint8_t* diffused, int* n_cur_out, vrm_stats* acc_stats, cudaStream_t st) {
  Scratch& s = ctx->s;
  const Consts& c = ctx->c;
  VRM_CUDA(mark(ctx, VRM_STAGE_REDUCE, st));
  VRM_CUDA(reduce_select(gamma, n, c.c_bound, diffused, s.rstate, s.tie_flag, s.tie_rank, s.scan_tmp, s.ds, st));
  if (capacity > n) VRM_CUDA(cudaMemsetAsync(diffused + n, 0, (size_t)(capacity - n), st));
  VRM_CUDA(compact_flags(diffused, n, s.dlist, s.counters + 0, s.pos, s.scan_tmp, st));
  VRM_CUDA(mark(ctx, VRM_STAGE_GRID, st));
  VRM_CUDA(grid_build(x, y, n, c.Rh, c.lo2, c.hi2, s.ncell_cap, s.grid, s.cell_key, s.cell_rank, s.cell_count,
                      s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.bbox, s.scan_tmp, st));
  VRM_CUDA(search_masks(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, n, diffused, s.mask, st));
  VRM_CUDA(open_list(s.dlist, s.counters + 0, n, s.mask, s.keep_flag, s.pos, s.open_a, s.counters + 1, s.scan_tmp,
                     st));
  VRM_CUDA(mark(ctx, VRM_STAGE_INSERT, st));
  VRM_CUDA(read_back(ctx, st));
  if (s.h_grid->nonfinite || s.h_ds->nonfinite) return VRM_ERR_ARG;
  int n_open = s.h_counters[1];
  int n_cur = n;
  int rounds = 0;
  long open_segments = 0;
  for (int round = 0; n_open > 0; ++round) {
    if (round == c.max_rounds) {
      VRM_CUDA(count_open_segments(s.open_a, n_open, s.mask, s.counters + 3, st));
      VRM_CUDA(read_back(ctx, st));
      open_segments = s.h_counters[3];
      break;
    }
    VRM_CUDA(insert_count(s.open_a, n_open, s.mask, s.ccnt, s.ccpos, s.scan_tmp, st));
    VRM_CUDA(cudaMemcpyAsync(s.h_counters + 4, s.ccpos + n_open, sizeof(int), cudaMemcpyDeviceToHost, st));
    VRM_CUDA(cudaStreamSynchronize(st));
    const int n_cand = s.h_counters[4];
    VRM_CUDA(ensure_cand(s, n_cand, st));
    VRM_CUDA(insert_propose(c, s.open_a, n_open, s.mask, s.ccpos, x, y, s.cx, s.cy, n_cand, s.cand_ncell_cap, s.cg,
                            s.ckeep, s.capos, s.cscan_tmp, st));
    VRM_CUDA(cudaMemcpyAsync(s.h_counters + 5, s.capos + n_cand, sizeof(int), cudaMemcpyDeviceToHost, st));
    VRM_CUDA(cudaStreamSynchronize(st));
    const int accepted = s.h_counters[5];
    if ((long)n_cur + accepted > capacity) {
      if (acc_stats) acc_stats->n_out = (long)n_cur + accepted;
      return VRM_ERR_CAPACITY;
    }
    VRM_CUDA(insert_commit(c, s.open_a, n_open, s.cx, s.cy, n_cand, s.cg, s.ckeep, s.capos, n_cur, x, y, s.mask,
                           s.keep_flag, s.keep_pos, s.open_b, s.counters + 2, s.scan_tmp, st));
    VRM_CUDA(cudaMemcpyAsync(s.h_counters + 2, s.counters + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    VRM_CUDA(cudaStreamSynchronize(st));
    n_cur += accepted;
    if (accepted > 0) ++rounds;
    int* t = s.open_a;
    s.open_a = s.open_b;
    s.open_b = t;
    n_open = s.h_counters[2];
  }
  if (acc_stats) {
    acc_stats->n_in = n;
    acc_stats->n_out = n_cur;
    acc_stats->n_diffused = s.h_counters[0];
    acc_stats->n_inserted = n_cur - n;
    acc_stats->open_segments = open_segments;
    acc_stats->rounds = rounds;
  }
  *n_cur_out = n_cur;
  return VRM_OK;
}

bool bad_ptr(const void* p, int n) { return n > 0 && p == nullptr; }
// small and cols rows are read as int4 vectors
bool misaligned16(const void* p) { return ((uintptr_t)p & 15u) != 0; }

// Records the boundary event in front of stage k (k = VRM_STAGE_COUNT: end).
cudaError_t mark(vrm_ctx* ctx, int k, cudaStream_t st) {
  if (!ctx->timing) return cudaSuccess;
  if (k > 0 && k <= VRM_STAGE_COUNT) ctx->stage_done[k - 1] = 1;
  return cudaEventRecord(ctx->ev[k], st);
}

}  // namespace

extern "C" {

void vrm_default_params(vrm_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->h = 1.0;
  p->r = 0.5;
  p->R = 2.0;
  p->nu = 1.0;
  p->c_diff = 1.0;
  p->order = 1;
  p->k_cap = 32;
  p->max_rounds = 8;
  p->fallback = 1;
  p->precision = VRM_PREC_FP64;
}

const char* vrm_status_string(vrm_status s) {
  switch (s) {
    case VRM_OK: return "ok";
    case VRM_ERR_ARG: return "invalid argument";
    case VRM_ERR_CAPACITY: return "capacity too small";
    case VRM_ERR_CUDA: return "CUDA error";
    case VRM_ERR_UNSUPPORTED: return "unsupported parameter";
    default: return "unknown status";
  }
}

vrm_status vrm_create(const vrm_params* p, vrm_ctx** out) {
  if (!out) return VRM_ERR_ARG;
  *out = nullptr;
  vrm_status st = check_params(p);
  if (st != VRM_OK) return st;
  vrm_ctx* ctx = new (std::nothrow) vrm_ctx();
  if (!ctx) return VRM_ERR_CUDA;
  ctx->p = *p;
  fill_consts(*p, ctx->c);
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    delete ctx;
    return VRM_ERR_CUDA;
  }
  *out = ctx;
  return VRM_OK;
}

void vrm_destroy(vrm_ctx* ctx) {
  if (!ctx) return;
  free_scratch(ctx->s);
  if (ctx->events_ready)
    for (int k = 0; k <= VRM_STAGE_COUNT; ++k) cudaEventDestroy(ctx->ev[k]);
  delete ctx;
}

vrm_status vrm_set_timing(vrm_ctx* ctx, int32_t enable) {
  if (!ctx) return VRM_ERR_ARG;
  if (enable && !ctx->events_ready) {
    for (int k = 0; k <= VRM_STAGE_COUNT; ++k)
      if (cudaEventCreate(&ctx->ev[k]) != cudaSuccess) return VRM_ERR_CUDA;
    ctx->events_ready = 1;
  }
  ctx->timing = enable ? 1 : 0;
  for (int k = 0; k < VRM_STAGE_COUNT; ++k) ctx->stage_done[k] = 0;
  return VRM_OK;
}

vrm_status vrm_stage_times(vrm_ctx* ctx, float* ms) {
  if (!ctx || !ms) return VRM_ERR_ARG;
  for (int k = 0; k < VRM_STAGE_COUNT; ++k) ms[k] = 0.0f;
  if (!ctx->events_ready) return VRM_OK;
  if (cudaEventSynchronize(ctx->ev[VRM_STAGE_COUNT]) != cudaSuccess) return VRM_ERR_CUDA;
  for (int k = 0; k < VRM_STAGE_COUNT; ++k) {
    if (!ctx->stage_done[k]) continue;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, ctx->ev[k], ctx->ev[k + 1]) != cudaSuccess) return VRM_ERR_CUDA;
    ms[k] = t;
  }
  return VRM_OK;
}

int64_t vrm_launch_count(void) { return (int64_t)launch_count(); }

vrm_status vrm_insert_reduce(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma,
                             uint8_t* diffused, int32_t* n_out, vrm_stats* stats, cudaStream_t stream) {
  if (!ctx || !n_out || n < 0 || capacity < n) return VRM_ERR_ARG;
  if (bad_ptr(x, n) || bad_ptr(y, n) || bad_ptr(gamma, n) || bad_ptr(diffused, capacity)) return VRM_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (n == 0) {
    *n_out = 0;
    return VRM_OK;
  }
  VRM_CUDA(ensure_scratch(ctx, capacity, stream));
  VRM_CUDA(cudaMemsetAsync(ctx->s.ds, 0, sizeof(DevStats), stream));
  int n_cur = n;
  vrm_status st = stage_insert_reduce(ctx, x, y, n, capacity, gamma, diffused, &n_cur, stats, stream);
  if (st != VRM_OK) return st;
  *n_out = n_cur;
  return VRM_OK;
}

vrm_status vrm_build_neighbourhoods(vrm_ctx* ctx, const double* x, const double* y, int32_t n, int32_t* nbr_count,
                                    int32_t* nbr_idx, uint8_t* seg_mask, int32_t* small, int32_t* max_count,
                                    cudaStream_t stream) {
  if (!ctx || n < 0) return VRM_ERR_ARG;
  if (bad_ptr(x, n) || bad_ptr(y, n) || bad_ptr(nbr_count, n) || bad_ptr(nbr_idx, n) || bad_ptr(seg_mask, n) ||
      bad_ptr(small, n) || misaligned16(small))
    return VRM_ERR_ARG;
  if (n == 0) {
    if (max_count) *max_count = 0;
    return VRM_OK;
  }
  Scratch& s = ctx->s;
  VRM_CUDA(ensure_scratch(ctx, n, stream));
  VRM_CUDA(cudaMemsetAsync(s.ds, 0, sizeof(DevStats), stream));
  VRM_CUDA(grid_build(x, y, n, ctx->c.Rh, ctx->c.lo2, ctx->c.hi2, s.ncell_cap, s.grid, s.cell_key, s.cell_rank,
                      s.cell_count, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.bbox, s.scan_tmp, stream));
  VRM_CUDA(search_all(ctx->c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, n, nbr_count, nbr_idx,
                      seg_mask, small, s.ds, stream));
  if (max_count) {
    VRM_CUDA(read_back(ctx, stream));
    if (s.h_grid->nonfinite) return VRM_ERR_ARG;
    *max_count = s.h_ds->max_count;
    if (s.h_ds->max_count > ctx->p.k_cap) return VRM_ERR_CAPACITY;
  }
  return VRM_OK;
}

vrm_status vrm_solve_weights(vrm_ctx* ctx, const double* x, const double* y, int32_t n, const uint8_t* diffused,
                             const int32_t* nbr_count, const int32_t* nbr_idx, const int32_t* small, int32_t* cols,
                             double* f, double* fii, uint8_t* status, vrm_stats* stats, cudaStream_t stream) {
  if (!ctx || n < 0) return VRM_ERR_ARG;
  if (bad_ptr(x, n) || bad_ptr(y, n) || bad_ptr(diffused, n) || bad_ptr(nbr_count, n) || bad_ptr(nbr_idx, n) ||
      bad_ptr(small, n) || bad_ptr(cols, n) || bad_ptr(f, n) || bad_ptr(fii, n) || bad_ptr(status, n) ||
      misaligned16(small))
    return VRM_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (n == 0) return VRM_OK;
  Scratch& s = ctx->s;
  const Consts& c = ctx->c;
  VRM_CUDA(ensure_scratch(ctx, n, stream));
  VRM_CUDA(cudaMemsetAsync(s.ds, 0, sizeof(DevStats), stream));
  VRM_CUDA(compact_flags(diffused, n, s.dlist, s.counters + 0, s.pos, s.scan_tmp, stream));
  VRM_CUDA(lp_clear(n, diffused, cols, f, fii, status, stream));
  VRM_CUDA(lp_small(c, x, y, s.dlist, s.counters + 0, n, small, cols, f, fii, status, s.fail_list, s.ds, 0.0,
                    stream));
  VRM_CUDA(lp_full(c, x, y, s.fail_list, &s.ds->n_fail, n, nbr_count, nbr_idx, cols, f, fii, status, s.ds, 0.0,
                   stream));
  if (stats) {
    VRM_CUDA(read_back(ctx, stream));
    stats->n_in = stats->n_out = n;
    stats->n_diffused = s.h_counters[0];
    stats->small_ok = s.h_ds->small_ok;
    stats->full_ok = s.h_ds->full_ok;
    stats->no_stencil = s.h_ds->no_stencil;
    stats->max_pivots = s.h_ds->max_pivots;
    stats->lp_small_solved = s.h_ds->lp_small_solved;
    stats->lp_small_pivots = (int64_t)s.h_ds->lp_small_pivots;
    stats->lp_full_solved = s.h_ds->lp_full_solved;
    stats->lp_full_pivots = (int64_t)s.h_ds->lp_full_pivots;
  }
  return VRM_OK;
}

vrm_status vrm_apply(vrm_ctx* ctx, int32_t n, int32_t n_gamma, const double* gamma, const uint8_t* diffused,
                     const int32_t* nbr_count, const int32_t* nbr_idx, const int32_t* cols, const double* f,
                     const double* fii, double* dgamma, cudaStream_t stream) {
  if (!ctx || n < 0 || n_gamma < 0) return VRM_ERR_ARG;
  if (bad_ptr(gamma, n_gamma) || bad_ptr(diffused, n) || bad_ptr(nbr_count, n) || bad_ptr(nbr_idx, n) ||
      bad_ptr(cols, n) || bad_ptr(f, n) || bad_ptr(fii, n) || bad_ptr(dgamma, n) || misaligned16(cols))
    return VRM_ERR_ARG;
  if (n == 0) return VRM_OK;
  VRM_CUDA(apply_gather(ctx->c, n, n_gamma, gamma, diffused, nbr_count, nbr_idx, cols, f, fii, nullptr, dgamma,
                        nullptr, 0.0, stream));
  return VRM_OK;
}

vrm_status vrm_step(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma_in,
                    double* gamma_out, double dt, int32_t* n_out, vrm_stats* stats, cudaStream_t stream) {
  if (!ctx || !n_out || n < 0 || capacity < n || !std::isfinite(dt)) return VRM_ERR_ARG;
  if (bad_ptr(x, n) || bad_ptr(y, n) || bad_ptr(gamma_in, n) || bad_ptr(gamma_out, capacity)) return VRM_ERR_ARG;
  if (n > 0 && gamma_out < gamma_in + n && gamma_in < gamma_out + capacity) return VRM_ERR_ARG;
  vrm_stats local;
  vrm_stats* st = stats ? stats : &local;
  memset(st, 0, sizeof(*st));
  if (n == 0) {
    *n_out = 0;
    return VRM_OK;
  }
  Scratch& s = ctx->s;
  const Consts& c = ctx->c;
  VRM_CUDA(ensure_scratch(ctx, capacity, stream));
  VRM_CUDA(cudaMemsetAsync(s.ds, 0, sizeof(DevStats), stream));
  int n2 = n;
  if (ctx->timing)
    for (int k = 0; k < VRM_STAGE_COUNT; ++k) ctx->stage_done[k] = 0;
  vrm_status r = stage_insert_reduce(ctx, x, y, n, capacity, gamma_in, s.diffused, &n2, st, stream);
  if (r != VRM_OK) return r;
  VRM_CUDA(mark(ctx, VRM_STAGE_SEARCH, stream));
  if (n2 > n)
    VRM_CUDA(grid_build(x, y, n2, c.Rh, c.lo2, c.hi2, s.ncell_cap, s.grid, s.cell_key, s.cell_rank, s.cell_count,
                        s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.bbox, s.scan_tmp, stream));
  VRM_CUDA(search_all(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, n2, s.nbr_count, s.nbr_idx,
                      s.seg_mask, s.small, s.ds, stream));
  const double nu_dt = ctx->p.nu * dt;
  VRM_CUDA(mark(ctx, VRM_STAGE_LP_SMALL, stream));
  VRM_CUDA(lp_small(c, x, y, s.dlist, s.counters + 0, n, s.small, s.cols, s.f, s.fii, s.status, s.fail_list, s.ds,
                    nu_dt, stream));
  VRM_CUDA(mark(ctx, VRM_STAGE_LP_FULL, stream));
  VRM_CUDA(lp_full(c, x, y, s.fail_list, &s.ds->n_fail, n, s.nbr_count, s.nbr_idx, s.cols, s.f, s.fii, s.status,
                   s.ds, nu_dt, stream));
  VRM_CUDA(mark(ctx, VRM_STAGE_APPLY, stream));
  VRM_CUDA(apply_gather(c, n2, n, gamma_in, s.diffused, s.nbr_count, s.nbr_idx, s.cols, s.f, s.fii, s.sorted_idx,
                        nullptr, gamma_out, dt, stream));
  VRM_CUDA(mark(ctx, VRM_STAGE_COUNT, stream));
  VRM_CUDA(read_back(ctx, stream));
  st->small_ok = s.h_ds->small_ok;
  st->full_ok = s.h_ds->full_ok;
  st->no_stencil = s.h_ds->no_stencil;
  st->max_pivots = s.h_ds->max_pivots;
  st->max_count = s.h_ds->max_count;
  st->max_dt_ratio = ratio_from_bits(s.h_ds->max_dt_ratio_bits);
  st->lp_small_solved = s.h_ds->lp_small_solved;
  st->lp_small_pivots = (int64_t)s.h_ds->lp_small_pivots;
  st->lp_full_solved = s.h_ds->lp_full_solved;
  st->lp_full_pivots = (int64_t)s.h_ds->lp_full_pivots;
  *n_out = n2;
  if (s.h_ds->max_count > ctx->p.k_cap) return VRM_ERR_CAPACITY;
  return VRM_OK;
}

}  // extern "C"
