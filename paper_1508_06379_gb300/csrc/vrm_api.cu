// C ABI of the VRM library: parameter checks, context scratch, and the
// order of the stages of one operator evaluation (Sec. 3.3, 3.5, 4):
// growth control -> insertion -> neighbourhoods -> weights -> application.
//
// vrm_step runs every stage on the device with the counts kept in device
// memory (StepState), so the whole step is one CUDA graph: it is captured
// once per set of buffers (x, y, gamma_in, gamma_out, capacity), with the
// insertion rounds as a conditional while node whose body is one round, and
// replayed on later calls; n and dt travel in a host-to-device copy at the
// head of the graph.  When graph capture is unavailable the same kernels run
// eagerly, rounds unrolled with a host check between them.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>

#include "vrm_internal.cuh"
#include "vrm_mlp.cuh"

using namespace vrm;

// Buffers of the learned proposal (vrm_set_mlp): input rows, slot map,
// proposals, rejected list, network activations.
struct Learned {
  int cap = 0;
  MlpActs acts;
  int* slots = nullptr;
  float* Y = nullptr;
  int* rlist = nullptr;
  float2* xyf = nullptr;  // fp32 positions
  ProjScratch proj;       // correction rounds
};

struct vrm::Scratch {
  int cap = 0;        // particles the buffers hold
  int ncell_cap = 0;  // cells of the grid
  // particle grid
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
  // tile sums of the scans whose inputs the kernels before them accumulate:
  // the diffused flags, the tie flags, the particle grid's cell counts
  int *dflag_ts = nullptr, *tie_ts = nullptr, *cell_ts = nullptr;
  uint8_t* diffused = nullptr;
  int* dlist = nullptr;
  // insertion: masks and the round buffers (proposals up to 8 per open particle)
  uint8_t* mask = nullptr;
  RoundBufs rb = {};
  // neighbourhoods and weights of vrm_step
  int *nbr_count = nullptr, *nbr_idx = nullptr, *small = nullptr, *cols = nullptr, *fail_list = nullptr;
  int* retry_list = nullptr;  // small LPs re-run in FP64
  uint8_t *seg_mask = nullptr, *status = nullptr;
  double *f = nullptr, *fii = nullptr;
  // the stencils transposed per target (the application's lists, a CSR)
  int *tcount = nullptr, *toff = nullptr;
  double2* tent = nullptr;
  // counters and state
  DevStats* ds = nullptr;
  int* counters = nullptr;  // [0] |D|, [1] first open list length
  StepState* st = nullptr;
  // pinned host mirrors
  DevStats* h_ds = nullptr;
  int* h_counters = nullptr;
  Grid* h_grid = nullptr;
  StepState* h_params = nullptr;  // n, capacity, dt, max_rounds of the next step
  StepState* h_state = nullptr;   // state after the step
};

// The particle grid's cells as the insertion rounds read them.
inline PartCells part_cells(const Scratch& s) {
  return PartCells{s.cell_key, s.cell_rank, s.cell_start, s.sorted_loc};
}

struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  const void *x = nullptr, *y = nullptr, *gi = nullptr, *go = nullptr;
  int cap = 0, timing = 0;
  long long kernels_outer = 0;  // kernel nodes outside the insertion loop
  long long kernels_body = 0;   // kernel nodes of one insertion round
};

struct vrm_ctx {
  vrm_params p;
  Consts c;
  int device = 0;
  Scratch s;
  long long scratch_gen = 0;  // bumped whenever the scratch is reallocated
  // per-stage timing: ev[k] is recorded where stage k starts, ev[k+1] where it ends
  int timing = 0;
  int events_ready = 0;
  int stage_done[VRM_STAGE_COUNT] = {0};
  cudaEvent_t ev[VRM_STAGE_COUNT + 1];
  // graph of vrm_step and the two streams used to capture it
  int use_graph = 1;
  StepGraph graph;
  cudaStream_t cap_stream = nullptr, body_stream = nullptr;
  // learned proposal
  vrm_mlp* mlp = nullptr;
  Learned L;
  // stage buffers of vrm_rk3_step
  int rk_cap = 0;
  double *rk_x1 = nullptr, *rk_y1 = nullptr, *rk_x2 = nullptr, *rk_y2 = nullptr;
  double *rk_g1 = nullptr, *rk_g2 = nullptr, *rk_dg = nullptr, *rk_u = nullptr, *rk_v = nullptr;
  // direct-sum velocity: fp32-split sources and targets
  int bs_src_cap = 0, bs_tgt_cap = 0;
  float4 *bs_src = nullptr, *bs_tgt = nullptr;
  float* bs_g = nullptr;
  // particle removal (vrm_remove_close)
  int rm_cap = 0;
  uint8_t *rm_close = nullptr, *rm_removed = nullptr, *rm_keep = nullptr;
  int *rm_clist = nullptr, *rm_klist = nullptr, *rm_cols4 = nullptr;
  double *rm_w4 = nullptr, *rm_gnew = nullptr;
  // a step enqueued by vrm_step_begin and not yet waited for by vrm_step_end
  struct Pending {
    int active = 0, launched = 0;
    double *x = nullptr, *y = nullptr;
    const double* gi = nullptr;
    double* go = nullptr;
    int n = 0, cap = 0;
    cudaStream_t stream = nullptr;
  } pending;
  cudaEvent_t step_done = nullptr;
};

// What a batch graph was captured for: per cloud the buffers, capacity and
// spacing (n and dt travel in the per-cloud parameter copies).
struct BatchKey {
  const void *x = nullptr, *y = nullptr, *gi = nullptr, *go = nullptr;
  int cap = 0;
  double h = 0.0;
  long long scratch_gen = -1;  // the sub-context's scratch generation
};

struct vrm_batch {
  vrm_params base;
  int max_clouds = 0;
  int use_graph = 1;
  vrm_ctx** sub = nullptr;           // one context per cloud slot
  cudaStream_t* branch = nullptr;    // capture streams, one per cloud slot
  cudaEvent_t* join = nullptr;
  cudaStream_t cap_stream = nullptr, body_stream = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  BatchKey* key = nullptr;           // per slot; cap 0 = slot not in the graph
  long long* kernels_outer = nullptr;
  long long* kernels_body = nullptr;
  vrm_schedule* sched = nullptr;     // per slot; row_cap 0 = default
};

namespace {

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

void drop_graph(vrm_ctx* ctx) {
  if (ctx->graph.exec) cudaGraphExecDestroy(ctx->graph.exec);
  ctx->graph = StepGraph{};
}

void free_scratch(Scratch& s) {
  RoundBufs& r = s.rb;
  void* ptrs[] = {s.grid, s.cell_key, s.cell_rank, s.cell_count, s.cell_start, s.sorted_xy, s.sorted_loc,
                  s.sorted_idx, s.bbox, s.scan_tmp, s.pos, s.rstate, s.tie_flag, s.tie_rank, s.dflag_ts, s.tie_ts,
                  s.cell_ts, s.diffused, s.dlist,
                  s.mask, r.open, r.act0, r.act1, r.cnt, r.cpos, r.cnt_ts, r.cell_ts, r.keep_ts, r.keep_flag, r.cx,
                  r.cy, r.keep, r.keep_s, r.apos,
                  r.cg.grid, r.cg.cell_key, r.cg.cell_rank, r.cg.cell_count, r.cg.cell_start, r.cg.sorted_idx,
                  r.cg.sorted_xy, r.cg.sorted_loc, r.cg.bbox, r.scan_tmp, s.nbr_count, s.nbr_idx, s.small, s.cols,
                  s.fail_list, s.retry_list, s.seg_mask, s.status, s.f, s.fii, s.tcount, s.toff, s.tent, s.ds,
                  s.counters, s.st};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* hp[] = {s.h_ds, s.h_counters, s.h_grid, s.h_params, s.h_state};
  for (void* p : hp)
    if (p) cudaFreeHost(p);
  Scratch empty;
  s = empty;
}

void free_learned(Learned& L) {
  mlp_acts_free(&L.acts);
  if (L.slots) cudaFree(L.slots);
  if (L.Y) cudaFree(L.Y);
  if (L.rlist) cudaFree(L.rlist);
  if (L.xyf) cudaFree(L.xyf);
  proj_free(&L.proj);
  L = Learned{};
}

// Correction-round scratch for m listed particles (the network's stages
// use ensure_learned, which sizes it too).
cudaError_t ensure_proj(vrm_ctx* ctx, int m, cudaStream_t st) {
  ProjScratch& P = ctx->L.proj;
  if (m <= P.cap && P.sel) return cudaSuccess;
  cudaStreamSynchronize(st);
  drop_graph(ctx);
  ++ctx->scratch_gen;
  const cudaError_t e = proj_alloc(&P, m < 128 ? 128 : m);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

// Buffers of the learned proposal for `cap` particles (only with a network).
cudaError_t ensure_learned(vrm_ctx* ctx, int cap, cudaStream_t st) {
  Learned& L = ctx->L;
  if (!ctx->mlp || (cap <= L.cap && L.slots)) return cudaSuccess;
  cudaStreamSynchronize(st);
  drop_graph(ctx);
  ++ctx->scratch_gen;
  free_learned(L);
  const int n = cap < 128 ? 128 : cap;
  cudaError_t e = mlp_acts_alloc(&L.acts, n);
  if (e == cudaSuccess) e = cudaMalloc(&L.slots, sizeof(int) * (size_t)n * 32);
  if (e == cudaSuccess) e = cudaMalloc(&L.Y, sizeof(float) * (size_t)L.acts.rows_pad * 32);
  if (e == cudaSuccess) e = cudaMalloc(&L.rlist, sizeof(int) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&L.xyf, sizeof(float2) * (size_t)n);
  if (e == cudaSuccess) e = proj_alloc(&L.proj, n);
  if (e != cudaSuccess) {
    free_learned(L);
    cudaGetLastError();
    return e;
  }
  L.cap = n;
  return cudaSuccess;
}

// Learned proposal for the listed particles, then the LP for the rejected
// ones (their list and count in L.rlist, counters[2]).
cudaError_t enqueue_learned(vrm_ctx* ctx, const double* x, const double* y, const int* n_dev, const int* list,
                            const int* list_count, int cap, const int* nbr_count, const int* nbr_idx, const int* small, int* cols, double* f,
                            double* fii, uint8_t* status, const double* dt_dev, cudaStream_t st) {
  Scratch& s = ctx->s;
  Learned& L = ctx->L;
  const Consts& c = ctx->c;
  cudaError_t e;
  if ((e = learned_features(c, x, y, cap, n_dev, L.xyf, list, list_count, cap, nbr_count, nbr_idx, L.acts.X, L.slots,
                            st)) != cudaSuccess)
    return e;
  if ((e = mlp_forward(ctx->mlp, L.acts.mX, cap, list_count, L.Y, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(s.counters + 2, 0, sizeof(int), st)) != cudaSuccess) return e;
  return learned_project(c, x, y, list, list_count, cap, L.slots, L.Y, small, cols, f, fii, status, L.rlist,
                         s.counters + 2, s.ds, dt_dev, ctx->p.nu, &L.proj, st);
}

void free_rk(vrm_ctx* ctx) {
  double* ptrs[] = {ctx->rk_x1, ctx->rk_y1, ctx->rk_x2, ctx->rk_y2, ctx->rk_g1, ctx->rk_g2, ctx->rk_dg, ctx->rk_u,
                    ctx->rk_v};
  for (double* p : ptrs)
    if (p) cudaFree(p);
  ctx->rk_x1 = ctx->rk_y1 = ctx->rk_x2 = ctx->rk_y2 = ctx->rk_g1 = ctx->rk_g2 = ctx->rk_dg = nullptr;
  ctx->rk_u = ctx->rk_v = nullptr;
  ctx->rk_cap = 0;
}

void free_bs(vrm_ctx* ctx) {
  if (ctx->bs_src) cudaFree(ctx->bs_src);
  if (ctx->bs_tgt) cudaFree(ctx->bs_tgt);
  if (ctx->bs_g) cudaFree(ctx->bs_g);
  ctx->bs_src = ctx->bs_tgt = nullptr;
  ctx->bs_g = nullptr;
  ctx->bs_src_cap = ctx->bs_tgt_cap = 0;
}

void free_rm(vrm_ctx* ctx) {
  void* ptrs[] = {ctx->rm_close, ctx->rm_removed, ctx->rm_keep, ctx->rm_clist, ctx->rm_klist, ctx->rm_cols4,
                  ctx->rm_w4, ctx->rm_gnew};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  ctx->rm_close = ctx->rm_removed = ctx->rm_keep = nullptr;
  ctx->rm_clist = ctx->rm_klist = ctx->rm_cols4 = nullptr;
  ctx->rm_w4 = ctx->rm_gnew = nullptr;
  ctx->rm_cap = 0;
}

// Buffers of the removal pass for n particles (grown, never shrunk).
cudaError_t ensure_rm(vrm_ctx* ctx, int n, cudaStream_t st) {
  if (n <= ctx->rm_cap && ctx->rm_close) return cudaSuccess;
  cudaStreamSynchronize(st);
  free_rm(ctx);
  const size_t m = (size_t)(n < 1024 ? 1024 : n);
  cudaError_t e = cudaMalloc(&ctx->rm_close, m);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->rm_removed, m);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->rm_keep, m);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->rm_clist, sizeof(int) * m);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->rm_klist, sizeof(int) * m);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->rm_cols4, sizeof(int) * 4 * m);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->rm_w4, sizeof(double) * 4 * m);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->rm_gnew, sizeof(double) * m);
  if (e != cudaSuccess) {
    free_rm(ctx);
    cudaGetLastError();
    return e;
  }
  ctx->rm_cap = (int)m;
  return cudaSuccess;
}

cudaError_t ensure_bs(vrm_ctx* ctx, int n, int m, cudaStream_t st) {
  if (n <= ctx->bs_src_cap && m <= ctx->bs_tgt_cap) return cudaSuccess;
  cudaStreamSynchronize(st);
  const int ns = n > ctx->bs_src_cap ? n : ctx->bs_src_cap;
  const int mt = m > ctx->bs_tgt_cap ? m : ctx->bs_tgt_cap;
  free_bs(ctx);
  cudaError_t e = cudaMalloc(&ctx->bs_src, sizeof(float4) * (size_t)(ns > 0 ? ns : 1));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->bs_g, sizeof(float) * (size_t)(ns > 0 ? ns : 1));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->bs_tgt, sizeof(float4) * (size_t)(mt > 0 ? mt : 1));
  if (e != cudaSuccess) {
    free_bs(ctx);
    cudaGetLastError();
    return e;
  }
  ctx->bs_src_cap = ns;
  ctx->bs_tgt_cap = mt;
  return cudaSuccess;
}

cudaError_t ensure_rk(vrm_ctx* ctx, int cap, cudaStream_t st) {
  if (cap <= ctx->rk_cap) return cudaSuccess;
  cudaStreamSynchronize(st);
  free_rk(ctx);
  cudaError_t e = cudaSuccess;
  double** ptrs[] = {&ctx->rk_x1, &ctx->rk_y1, &ctx->rk_x2, &ctx->rk_y2, &ctx->rk_g1,
                     &ctx->rk_g2, &ctx->rk_dg, &ctx->rk_u,  &ctx->rk_v};
  for (double** p : ptrs)
    if (e == cudaSuccess) e = cudaMalloc((void**)p, sizeof(double) * (size_t)cap);
  if (e != cudaSuccess) {
    free_rk(ctx);
    cudaGetLastError();
    return e;
  }
  ctx->rk_cap = cap;
  return cudaSuccess;
}

// Neighbourhoods and weights of every diffused particle (list s.dlist) at
// positions (x, y) of the n_cur particles: cell grid, search, learned
// proposal (with a network) and LP.
cudaError_t enqueue_stage_weights(vrm_ctx* ctx, const double* x, const double* y, int cap, cudaStream_t st) {
  Scratch& s = ctx->s;
  const Consts& c = ctx->c;
  const int* n_cur = &s.st->n_cur;
  cudaError_t e;
  // the full-neighbourhood queue of this stage starts empty
  if ((e = cudaMemsetAsync(&s.ds->n_fail, 0, sizeof(int), st)) != cudaSuccess) return e;
  if ((e = grid_build_dev(x, y, cap, n_cur, c.Rh, c.lo2, c.hi2, s.ncell_cap, s.grid, s.cell_key, s.cell_rank,
                          s.cell_count, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.bbox, s.scan_tmp,
                          st, s.cell_ts, true)) != cudaSuccess)
    return e;
  // counts, masks and small neighbourhoods of the diffused particles (the
  // LPs read no other particle's); their rows only where the learned slots
  // read them (the full-neighbourhood LP's few particles get theirs below;
  // the application goes through the transposed stencils), in visiting order
  // (the learned slots and the full-neighbourhood LP order their entries
  // themselves)
  const bool rows = ctx->mlp != nullptr;
  if ((e = search_list_dev(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.cell_key, s.cell_rank,
                           s.dlist, s.counters + 0, cap, s.nbr_count, s.nbr_idx, s.seg_mask, s.small, s.ds, st,
                           rows)) != cudaSuccess)
    return e;
  const int* lp_list = s.dlist;
  const int* lp_count = s.counters + 0;
  if (ctx->mlp) {
    if ((e = enqueue_learned(ctx, x, y, n_cur, s.dlist, s.counters + 0, cap, s.nbr_count, s.nbr_idx, s.small, s.cols,
                             s.f, s.fii, s.status, &s.st->dt, st)) != cudaSuccess)
      return e;
    lp_list = ctx->L.rlist;
    lp_count = s.counters + 2;
  }
  if ((e = lp_small(c, x, y, lp_list, lp_count, cap, s.small, s.cols, s.f, s.fii, s.status, s.fail_list, s.retry_list, s.ds,
                    0.0, st, &s.st->dt, ctx->p.nu)) != cudaSuccess)
    return e;
  if (!rows && (e = search_list_dev(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.cell_key,
                                    s.cell_rank, s.fail_list, &s.ds->n_fail, std::min(cap, 32 * sm_count()),
                                    s.nbr_count, s.nbr_idx, s.seg_mask, s.small, s.ds, st, true)) != cudaSuccess)
    return e;
  return lp_full(c, x, y, s.fail_list, &s.ds->n_fail, cap, s.nbr_count, s.nbr_idx, s.cols, s.f, s.fii, s.status,
                 s.ds, 0.0, st, &s.st->dt, ctx->p.nu);
}

// Scratch for `cap` particles (grown by 25% steps, never shrunk).
cudaError_t ensure_scratch(vrm_ctx* ctx, int cap, cudaStream_t st) {
  Scratch& s = ctx->s;
  if (cap <= s.cap && s.ds) return cudaSuccess;
  cudaStreamSynchronize(st);
  drop_graph(ctx);
  ++ctx->scratch_gen;
  long want = cap;
  if (s.cap > 0 && want < (long)s.cap + s.cap / 4) want = (long)s.cap + s.cap / 4;
  if (want < 1024) want = 1024;
  if (want > 0x0FFFFFF0L) want = 0x0FFFFFF0L;  // 8 proposals per particle must fit int32
  free_scratch(s);
  const int n = (int)want;
  const long n8 = 8L * n;
  const int k = ctx->p.k_cap;
  const long ncell = 2 * (long)n + 1024;
  s.cap = n;
  s.ncell_cap = (int)ncell;
  cudaError_t e = cudaSuccess;
  RoundBufs& r = s.rb;
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
  VRM_ALLOC(s.dflag_ts, (long)n / kScanTile + 2);
  VRM_ALLOC(s.tie_ts, (long)n / kScanTile + 2);
  VRM_ALLOC(s.cell_ts, ncell / kScanTile + 2);
  VRM_ALLOC(s.diffused, n);
  VRM_ALLOC(s.dlist, n);
  VRM_ALLOC(s.mask, n);
  VRM_ALLOC(r.open, n);
  VRM_ALLOC(r.act0, n);
  VRM_ALLOC(r.act1, n);
  VRM_ALLOC(r.cnt, n);
  VRM_ALLOC(r.cpos, (long)n + 1);
  VRM_ALLOC(r.cnt_ts, (long)n / kScanTile + 2);
  VRM_ALLOC(r.cell_ts, ncell / kScanTile + 2);
  VRM_ALLOC(r.keep_ts, n8 / kScanTile + 2);
  VRM_ALLOC(r.keep_flag, n);
  VRM_ALLOC(r.cx, n8);
  VRM_ALLOC(r.cy, n8);
  VRM_ALLOC(r.keep, n8);
  VRM_ALLOC(r.keep_s, n8);
  VRM_ALLOC(r.apos, n8 + 1);
  VRM_ALLOC(r.cg.grid, 1);
  VRM_ALLOC(r.cg.cell_key, n8);
  VRM_ALLOC(r.cg.cell_rank, n8);
  VRM_ALLOC(r.cg.cell_count, ncell);
  VRM_ALLOC(r.cg.cell_start, ncell + 1);
  VRM_ALLOC(r.cg.sorted_idx, n8);
  VRM_ALLOC(r.cg.sorted_xy, n8);
  VRM_ALLOC(r.cg.sorted_loc, n8);
  VRM_ALLOC(r.cg.bbox, 8);
  VRM_ALLOC(r.scan_tmp, scan_tmp_ints((int)(n8 > ncell ? n8 : ncell)) + 16);
  r.ncell_cap = (int)ncell;
  VRM_ALLOC(s.nbr_count, n);
  VRM_ALLOC(s.nbr_idx, (long)n * k);
  VRM_ALLOC(s.small, (long)n * 8);
  VRM_ALLOC(s.cols, (long)n * ctx->c.w);
  VRM_ALLOC(s.fail_list, n);
  VRM_ALLOC(s.retry_list, n);
  VRM_ALLOC(s.seg_mask, n);
  VRM_ALLOC(s.status, n);
  VRM_ALLOC(s.f, (long)n * ctx->c.w);
  VRM_ALLOC(s.fii, n);
  VRM_ALLOC(s.tcount, n);
  VRM_ALLOC(s.toff, (long)n + 1);
  VRM_ALLOC(s.tent, (long)n * ctx->c.w);
  VRM_ALLOC(s.ds, 1);
  VRM_ALLOC(s.counters, 8);
  VRM_ALLOC(s.st, 1);
#undef VRM_ALLOC
  // the bounding box starts at its initial values (every grid build leaves it so)
  if (e == cudaSuccess) e = grid_bbox_reset(s.bbox, st);
  // the growth control's pass counter starts at 0 (every pass leaves it so)
  if (e == cudaSuccess) e = cudaMemsetAsync(s.rstate, 0, sizeof(ReduceState), st);
  // the application's per-target counters start at 0 (every application
  // leaves them so)
  if (e == cudaSuccess) e = cudaMemsetAsync(s.tcount, 0, sizeof(int) * (size_t)n, st);
  // the proposal cells (and their tile sums) start empty; every insertion
  // round leaves them empty
  if (e == cudaSuccess) e = cudaMemsetAsync(r.cg.cell_count, 0, sizeof(int) * (size_t)ncell, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(r.cell_ts, 0, sizeof(int) * (size_t)(ncell / kScanTile + 2), st);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_ds, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_counters, sizeof(int) * 8);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_grid, sizeof(Grid));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_params, sizeof(StepState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_state, sizeof(StepState));
  if (e != cudaSuccess) {
    free_scratch(s);
    cudaGetLastError();
  }
  return e;
}

#define VRM_CUDA(call)                          \
  do {                                          \
    cudaError_t _e = (call);                    \
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
  if (p->order != 1 && p->order != 2) return VRM_ERR_UNSUPPORTED;
  if (p->precision != VRM_PREC_FP64 && p->precision != VRM_PREC_MIXED) return VRM_ERR_UNSUPPORTED;
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
  // LP residual certificate: the entries of a basis matrix are offsets and
  // their products, at most max(1, R^2) (offsets within R, up to rounding);
  // max|B| max|x| <= 37 keeps the LU backward error below 0.5e-10 (see
  // lp_finish in vrm_lp.cu)
  volatile double hh = h * h;  // keep the documented rounding order
  volatile double hhh = hh * h;
  volatile double hp = p.order == 2 ? hhh * h : hhh;  // h^{n+2}
  c.c_bound = p.c_diff * hp;
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
  c.order = p.order;
  c.w = vrm_stencil_width(p.order);
  default_schedule(c);
}

cudaError_t read_back(vrm_ctx* ctx, cudaStream_t st) {
  Scratch& s = ctx->s;
  cudaError_t e = cudaMemcpyAsync(s.h_ds, s.ds, sizeof(DevStats), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_counters, s.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_grid, s.grid, sizeof(Grid), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_state, s.st, sizeof(StepState), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

double ratio_from_bits(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
}

bool bad_ptr(const void* p, int n) { return n > 0 && p == nullptr; }

bool block_ok(int b, int hi) { return b >= 32 && b <= hi && b % 32 == 0; }

bool schedule_ok(const vrm_schedule& s, int k_cap) {
  // lp_block 192 and 384: the warp-specialised small LP (4 pivot + 2 finish
  // warps, two blocks per SM; 8 + 4 warps, one block per SM)
  return s.row_cap >= 8 && s.row_cap <= k_cap && block_ok(s.search_block, kBlock) &&
         (block_ok(s.lp_block, 128) || s.lp_block == 192 || s.lp_block == 384) &&
         s.lp_blocks_per_sm >= 1 && s.lp_blocks_per_sm <= 64 && block_ok(s.apply_block, kBlock) &&
         (s.lp_fp64_pivots == 0 || s.lp_fp64_pivots == 1);
}

void put_schedule(Consts& c, const vrm_schedule& s) {
  c.row_cap = s.row_cap;
  c.search_block = s.search_block;
  c.lp_block = s.lp_block;
  c.lp_blocks_per_sm = s.lp_blocks_per_sm;
  c.lp_fp64_pivots = s.lp_fp64_pivots;
  c.apply_block = s.apply_block;
}

// Constants for the stand-alone stage calls: whole rows (row_cap = k_cap).
Consts full_rows(const Consts& c) {
  Consts d = c;
  d.row_cap = d.k_cap;
  return d;
}
// small and cols rows are read as int4 vectors
bool misaligned16(const void* p) { return ((uintptr_t)p & 15u) != 0; }

// Records the boundary event in front of stage k (k = VRM_STAGE_COUNT: end).
// External records so that, inside a captured graph, they become event
// record nodes that the host can time.
cudaError_t mark(vrm_ctx* ctx, int k, cudaStream_t st) {
  if (!ctx->timing) return cudaSuccess;
  if (k > 0 && k <= VRM_STAGE_COUNT) ctx->stage_done[k - 1] = 1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return e;
  if (cap == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ctx->ev[k], st, cudaEventRecordExternal);
  return cudaEventRecord(ctx->ev[k], st);
}

// Growth control, grid of the given cloud, segment masks, first open list
// (the rounds follow).  n is read from s.st->n.
cudaError_t enqueue_front(vrm_ctx* ctx, double* x, double* y, int cap, const double* gamma, uint8_t* diffused,
                          cudaStream_t st) {
  Scratch& s = ctx->s;
  const Consts& c = ctx->c;
  const int* n_dev = &s.st->n;
  cudaError_t e;
  if ((e = mark(ctx, VRM_STAGE_REDUCE, st)) != cudaSuccess) return e;
  // the growth control's first pass also takes the bounding box of the
  // particles for the grid build below
  if ((e = reduce_select_dev(gamma, cap, n_dev, c.c_bound, diffused, s.rstate, s.tie_flag, s.tie_rank, s.scan_tmp,
                             s.ds, st, s.dflag_ts, s.tie_ts, x, y, s.bbox)) != cudaSuccess)
    return e;
  if ((e = compact_flags_dev(diffused, cap, n_dev, s.dlist, s.counters + 0, s.pos, s.scan_tmp, st, s.dflag_ts)) !=
      cudaSuccess)
    return e;
  if ((e = mark(ctx, VRM_STAGE_GRID, st)) != cudaSuccess) return e;
  if ((e = grid_build_dev(x, y, cap, n_dev, c.Rh, c.lo2, c.hi2, s.ncell_cap, s.grid, s.cell_key, s.cell_rank,
                          s.cell_count, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.bbox, s.scan_tmp,
                          st, s.cell_ts, true, true)) != cudaSuccess)
    return e;
  if ((e = search_masks_list_dev(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.cell_key,
                                 s.cell_rank, s.dlist, s.counters + 0, cap, s.mask, st)) != cudaSuccess)
    return e;
  if ((e = open_list(s.dlist, s.counters + 0, cap, s.mask, s.rb.keep_flag, s.pos, s.rb.open, s.counters + 1,
                     s.rb.keep_ts, st)) != cudaSuccess)
    return e;
  return mark(ctx, VRM_STAGE_INSERT, st);
}

// Final grid, neighbourhoods, weights, application + Euler, statistics copy.
cudaError_t enqueue_back(vrm_ctx* ctx, double* x, double* y, int cap, const double* gamma_in, double* gamma_out,
                         cudaStream_t st) {
  Scratch& s = ctx->s;
  const Consts& c = ctx->c;
  const int* n_cur = &s.st->n_cur;
  cudaError_t e;
  if ((e = rounds_finish(s.st, s.rb, cap, st)) != cudaSuccess) return e;
  if ((e = mark(ctx, VRM_STAGE_SEARCH, st)) != cudaSuccess) return e;
  // the grid of the given particles (enqueue_front) extended by the inserted
  // ones, with its geometry kept
  if ((e = grid_extend_dev(x, y, cap, &s.st->n, n_cur, s.ncell_cap, s.grid, s.cell_key, s.cell_rank, s.cell_count,
                           s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.scan_tmp, st, s.cell_ts)) !=
      cudaSuccess)
    return e;
  // counts, masks and small neighbourhoods of the diffused particles (the
  // LPs read no other particle's); their rows only where the learned slots
  // read them (the full-neighbourhood LP's few particles get theirs below;
  // the application goes through the transposed stencils), in visiting order
  // (the learned slots and the full-neighbourhood LP order their entries
  // themselves)
  const bool rows = ctx->mlp != nullptr;
  if ((e = search_list_dev(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.cell_key, s.cell_rank,
                           s.dlist, s.counters + 0, cap, s.nbr_count, s.nbr_idx, s.seg_mask, s.small, s.ds, st,
                           rows)) != cudaSuccess)
    return e;
  if ((e = mark(ctx, VRM_STAGE_LP_SMALL, st)) != cudaSuccess) return e;
  const int* lp_list = s.dlist;
  const int* lp_count = s.counters + 0;
  if (ctx->mlp) {
    if ((e = enqueue_learned(ctx, x, y, &s.st->n_cur, s.dlist, s.counters + 0, cap, s.nbr_count, s.nbr_idx, s.small, s.cols, s.f,
                             s.fii, s.status, &s.st->dt, st)) != cudaSuccess)
      return e;
    lp_list = ctx->L.rlist;
    lp_count = s.counters + 2;
  }
  if ((e = lp_small(c, x, y, lp_list, lp_count, cap, s.small, s.cols, s.f, s.fii, s.status, s.fail_list, s.retry_list, s.ds,
                    0.0, st, &s.st->dt, ctx->p.nu)) != cudaSuccess)
    return e;
  if ((e = mark(ctx, VRM_STAGE_LP_FULL, st)) != cudaSuccess) return e;
  if (!rows && (e = search_list_dev(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.cell_key,
                                    s.cell_rank, s.fail_list, &s.ds->n_fail, std::min(cap, 32 * sm_count()),
                                    s.nbr_count, s.nbr_idx, s.seg_mask, s.small, s.ds, st, true)) != cudaSuccess)
    return e;
  if ((e = lp_full(c, x, y, s.fail_list, &s.ds->n_fail, cap, s.nbr_count, s.nbr_idx, s.cols, s.f, s.fii, s.status,
                   s.ds, 0.0, st, &s.st->dt, ctx->p.nu)) != cudaSuccess)
    return e;
  if ((e = mark(ctx, VRM_STAGE_APPLY, st)) != cudaSuccess) return e;
  if ((e = apply_transposed_dev(c, cap, n_cur, cap, &s.st->n, gamma_in, s.diffused, s.dlist, s.counters + 0, s.cols,
                                s.f, s.fii, s.tcount, s.toff, s.tent, s.scan_tmp, s.ds, nullptr, gamma_out,
                                0.0, &s.st->dt, st)) != cudaSuccess)
    return e;
  if ((e = mark(ctx, VRM_STAGE_COUNT, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(s.h_ds, s.ds, sizeof(DevStats), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(s.h_counters, s.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(s.h_grid, s.grid, sizeof(Grid), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  return cudaMemcpyAsync(s.h_state, s.st, sizeof(StepState), cudaMemcpyDeviceToHost, st);
}

cudaError_t enqueue_head(vrm_ctx* ctx, cudaStream_t st) {
  Scratch& s = ctx->s;
  cudaError_t e = cudaMemcpyAsync(s.st, s.h_params, sizeof(StepState), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.ds, 0, sizeof(DevStats), st);
  return e;
}

// Records one context's whole step into the graph being captured on cs: the
// insertion rounds become a conditional while node whose body is captured on
// body_stream.  Kernel counts of the outer part and of one round are
// returned for the launch accounting.
bool record_step(vrm_ctx* ctx, cudaStream_t cs, cudaStream_t body_stream, double* x, double* y, int cap,
                 const double* gamma_in, double* gamma_out, long long* outer_kernels, long long* body_kernels) {
  Scratch& s = ctx->s;
  const long long l0 = launch_count();
  long long bk = 0;
  bool ok = enqueue_head(ctx, cs) == cudaSuccess;
  ok = ok && enqueue_front(ctx, x, y, cap, gamma_in, s.diffused, cs) == cudaSuccess;
  cudaGraphConditionalHandle handle = 0;
  if (ok) {
    cudaStreamCaptureStatus status;
    cudaGraph_t cg = nullptr;
    ok = cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, nullptr, nullptr, nullptr) == cudaSuccess;
    ok = ok && cudaGraphConditionalHandleCreate(&handle, cg, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  }
  ok = ok && rounds_init(s.st, s.counters + 1, s.rb, s.mask, cap, handle, true, cs) == cudaSuccess;
  if (ok) {
    cudaStreamCaptureStatus status;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    ok = cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, &deps, nullptr, &ndeps) == cudaSuccess;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    ok = ok && cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &cp) == cudaSuccess;
    ok = ok && cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                   cudaSuccess;
    if (ok) {
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      ok = cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
           cudaSuccess;
      if (ok) {
        const long long b0 = launch_count();
        ok = round_body(ctx->c, s.st, s.grid, part_cells(s), s.rb, cap, s.mask, x, y, handle, true, body_stream) ==
             cudaSuccess;
        bk = launch_count() - b0;
        cudaGraph_t got = nullptr;
        const bool ended = cudaStreamEndCapture(body_stream, &got) == cudaSuccess;
        ok = ok && ended;
      }
    }
  }
  ok = ok && enqueue_back(ctx, x, y, cap, gamma_in, gamma_out, cs) == cudaSuccess;
  const long long recorded = launch_count() - l0;
  add_launches(-recorded);  // counted when the graph runs
  *outer_kernels = recorded - bk;
  *body_kernels = bk;
  return ok;
}

// Captures the whole step on the context's streams; the insertion rounds are
// a conditional while node.  Returns false (graph left empty) on failure.
bool capture_step(vrm_ctx* ctx, double* x, double* y, int cap, const double* gamma_in, double* gamma_out) {
  Scratch& s = ctx->s;
  if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return false;
  if (!ctx->body_stream && cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking) != cudaSuccess)
    return false;
  cudaStream_t cs = ctx->cap_stream;
  cudaGraph_t g = nullptr;
  long long outer = 0, body = 0;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  const bool capturing = ok;
  ok = ok && record_step(ctx, cs, ctx->body_stream, x, y, cap, gamma_in, gamma_out, &outer, &body);
  if (capturing) {
    const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
    ok = ok && ended && g;
  }
  cudaGraphExec_t exec = nullptr;
  ok = ok && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    return false;
  }
  drop_graph(ctx);
  ctx->graph.exec = exec;
  ctx->graph.x = x;
  ctx->graph.y = y;
  ctx->graph.gi = gamma_in;
  ctx->graph.go = gamma_out;
  ctx->graph.cap = cap;
  ctx->graph.timing = ctx->timing;
  ctx->graph.kernels_outer = outer;
  ctx->graph.kernels_body = body;
  return true;
}

// The same step without a graph: rounds unrolled, with a host check of the
// open list between rounds.  back = false stops after insertion.
vrm_status run_step_eager(vrm_ctx* ctx, double* x, double* y, int cap, const double* gamma_in, double* gamma_out,
                          uint8_t* diffused, bool back, cudaStream_t st) {
  Scratch& s = ctx->s;
  VRM_CUDA(enqueue_head(ctx, st));
  VRM_CUDA(enqueue_front(ctx, x, y, cap, gamma_in, diffused, st));
  VRM_CUDA(rounds_init(s.st, s.counters + 1, s.rb, s.mask, cap, 0, false, st));
  for (int r = 0; r < ctx->p.max_rounds; ++r) {
    VRM_CUDA(cudaMemcpyAsync(s.h_state, s.st, sizeof(StepState), cudaMemcpyDeviceToHost, st));
    VRM_CUDA(cudaStreamSynchronize(st));
    if (s.h_state->n_open == 0) break;
    VRM_CUDA(round_body(ctx->c, s.st, s.grid, part_cells(s), s.rb, cap, s.mask, x, y, 0, false, st));
  }
  if (back) {
    VRM_CUDA(enqueue_back(ctx, x, y, cap, gamma_in, gamma_out, st));
  } else {
    VRM_CUDA(rounds_finish(s.st, s.rb, cap, st));
  }
  return VRM_OK;
}

void fill_front_stats(vrm_ctx* ctx, int n, vrm_stats* st) {
  const Scratch& s = ctx->s;
  const StepState& S = *s.h_state;
  st->n_in = n;
  st->n_out = S.overflow ? S.n_needed : S.n_cur;
  st->n_diffused = s.h_counters[0];
  st->n_inserted = S.n_cur - n;
  st->open_segments = S.open_segments;
  st->rounds = S.rounds_appended;
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

int32_t vrm_stencil_width(int32_t order) {
  return order == 1 ? VRM_STENCIL_W : order == 2 ? VRM_STENCIL_W2 : -1;
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
  const char* env = getenv("VRM_NO_GRAPH");
  ctx->use_graph = !(env && env[0] == '1');
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    delete ctx;
    return VRM_ERR_CUDA;
  }
  *out = ctx;
  return VRM_OK;
}

void vrm_destroy(vrm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->step_done) {
    cudaEventSynchronize(ctx->step_done);
    cudaEventDestroy(ctx->step_done);
  }
  drop_graph(ctx);
  free_scratch(ctx->s);
  free_learned(ctx->L);
  free_rk(ctx);
  free_bs(ctx);
  free_rm(ctx);
  if (ctx->events_ready)
    for (int k = 0; k <= VRM_STAGE_COUNT; ++k) cudaEventDestroy(ctx->ev[k]);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->body_stream) cudaStreamDestroy(ctx->body_stream);
  delete ctx;
}

vrm_status vrm_remove_close(vrm_ctx* ctx, const double* x, const double* y, const double* gamma, int32_t n,
                            double* x_out, double* y_out, double* gamma_out, int32_t* n_out, vrm_stats* stats,
                            cudaStream_t stream) {
  if (!ctx || n < 0 || !n_out) return VRM_ERR_ARG;
  *n_out = 0;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (bad_ptr(x, n) || bad_ptr(y, n) || bad_ptr(gamma, n) || bad_ptr(x_out, n) || bad_ptr(y_out, n) ||
      bad_ptr(gamma_out, n))
    return VRM_ERR_ARG;
  if (n == 0) return VRM_OK;
  Scratch& s = ctx->s;
  const Consts c = full_rows(ctx->c);
  VRM_CUDA(ensure_scratch(ctx, n, stream));
  VRM_CUDA(ensure_rm(ctx, n, stream));
  VRM_CUDA(cudaMemsetAsync(s.ds, 0, sizeof(DevStats), stream));
  VRM_CUDA(grid_build(x, y, n, c.Rh, c.lo2, c.hi2, s.ncell_cap, s.grid, s.cell_key, s.cell_rank, s.cell_count,
                      s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, s.bbox, s.scan_tmp, stream));
  VRM_CUDA(search_all(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, n, s.nbr_count, s.nbr_idx,
                      s.seg_mask, s.small, s.ds, stream));
  VRM_CUDA(remove_close_flags(c, s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, n, gamma,
                              ctx->rm_close, stream));
  VRM_CUDA(compact_flags(ctx->rm_close, n, ctx->rm_clist, s.counters + 3, s.pos, s.scan_tmp, stream));
  VRM_CUDA(cudaMemsetAsync(ctx->rm_removed, 0, (size_t)n, stream));
  VRM_CUDA(lp_identity(c, x, y, ctx->rm_clist, s.counters + 3, n, s.nbr_count, s.nbr_idx, ctx->rm_close,
                       ctx->rm_removed, ctx->rm_cols4, ctx->rm_w4, stream));
  VRM_CUDA(remove_gather(c, n, gamma, ctx->rm_removed, s.nbr_count, s.nbr_idx, ctx->rm_cols4, ctx->rm_w4,
                         ctx->rm_gnew, ctx->rm_keep, s.ds, stream));
  VRM_CUDA(compact_flags(ctx->rm_keep, n, ctx->rm_klist, s.counters + 4, s.pos, s.scan_tmp, stream));
  VRM_CUDA(remove_out(n, s.counters + 4, ctx->rm_klist, x, y, ctx->rm_gnew, x_out, y_out, gamma_out, stream));
  VRM_CUDA(read_back(ctx, stream));
  if (s.h_grid->nonfinite || s.h_ds->nonfinite) return VRM_ERR_ARG;
  if (stats) {
    stats->n_in = n;
    stats->n_out = s.h_counters[4];
    stats->max_count = s.h_ds->max_count;
    stats->remove_candidates = s.h_counters[3];
  }
  if (s.h_ds->max_count > ctx->p.k_cap) return VRM_ERR_CAPACITY;
  *n_out = s.h_counters[4];
  return VRM_OK;
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
  Scratch& s = ctx->s;
  VRM_CUDA(ensure_scratch(ctx, capacity, stream));
  VRM_CUDA(cudaStreamSynchronize(stream));
  StepState P;
  memset(&P, 0, sizeof(P));
  P.n = n;
  P.capacity = capacity;
  P.max_rounds = ctx->p.max_rounds;
  *s.h_params = P;
  const int timing = ctx->timing;
  ctx->timing = 0;
  vrm_status r = run_step_eager(ctx, x, y, capacity, gamma, nullptr, diffused, false, stream);
  ctx->timing = timing;
  if (r != VRM_OK) return r;
  VRM_CUDA(read_back(ctx, stream));
  if (s.h_grid->nonfinite || s.h_ds->nonfinite) return VRM_ERR_ARG;
  vrm_stats local;
  vrm_stats* st = stats ? stats : &local;
  fill_front_stats(ctx, n, st);
  if (s.h_state->overflow) return VRM_ERR_CAPACITY;
  *n_out = s.h_state->n_cur;
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
  VRM_CUDA(search_all(full_rows(ctx->c), s.grid, s.cell_start, s.sorted_xy, s.sorted_loc, s.sorted_idx, n, nbr_count,
                      nbr_idx, seg_mask, small, s.ds, stream));
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
  const Consts c = full_rows(ctx->c);
  VRM_CUDA(ensure_scratch(ctx, n, stream));
  VRM_CUDA(cudaMemsetAsync(s.ds, 0, sizeof(DevStats), stream));
  VRM_CUDA(ensure_learned(ctx, n, stream));
  VRM_CUDA(compact_flags(diffused, n, s.dlist, s.counters + 0, s.pos, s.scan_tmp, stream));
  VRM_CUDA(lp_clear(n, c.w, diffused, cols, f, fii, status, stream));
  const int* lp_list = s.dlist;
  const int* lp_count = s.counters + 0;
  if (ctx->mlp) {
    const Consts keep = ctx->c;
    ctx->c = c;  // whole rows
    const cudaError_t le = enqueue_learned(ctx, x, y, nullptr, s.dlist, s.counters + 0, n, nbr_count, nbr_idx, small, cols, f,
                                           fii, status, nullptr, stream);
    ctx->c = keep;
    VRM_CUDA(le);
    lp_list = ctx->L.rlist;
    lp_count = s.counters + 2;
  }
  VRM_CUDA(lp_small(c, x, y, lp_list, lp_count, n, small, cols, f, fii, status, s.fail_list, s.retry_list, s.ds,
                      0.0, stream));
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
    stats->lp_full_columns = (int64_t)s.h_ds->lp_full_columns;
    stats->lp_full_column_pivots = (int64_t)s.h_ds->lp_full_column_pivots;
    stats->lp_small_rechecked = (int64_t)s.h_ds->lp_small_retries;
    stats->learned_ok = s.h_ds->learned_ok;
    stats->learned_rejected = s.h_ds->learned_rejected;
    stats->learned_square = s.h_ds->learned_square;
    stats->learned_screens = (int64_t)s.h_ds->learned_screens;
  }
  if (ctx->mlp && vrm_mlp_error(ctx->mlp, stream) != VRM_OK) return VRM_ERR_CUDA;
  return VRM_OK;
}

vrm_status vrm_rk3_step(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma_in,
                        double* gamma_out, double t, double dt, const vrm_velocity* vel, int32_t* n_out,
                        vrm_stats* stats, cudaStream_t stream) {
  if (!ctx || !n_out || n < 0 || capacity < n || !std::isfinite(dt) || !std::isfinite(t)) return VRM_ERR_ARG;
  if (bad_ptr(x, n) || bad_ptr(y, n) || bad_ptr(gamma_in, n) || bad_ptr(gamma_out, capacity)) return VRM_ERR_ARG;
  if (n > 0 && gamma_out < gamma_in + n && gamma_in < gamma_out + capacity) return VRM_ERR_ARG;
  Velocity V;
  memset(&V, 0, sizeof(V));
  V.kind = vel ? vel->kind : VRM_VEL_NONE;
  if (V.kind == VRM_VEL_LAMB_OSEEN) {
    if (!(vel->nu > 0) || !std::isfinite(vel->gamma) || !std::isfinite(vel->x0) || !std::isfinite(vel->y0))
      return VRM_ERR_ARG;
    if (!(t > 0 && t + 0.5 * dt > 0 && t + dt > 0)) return VRM_ERR_ARG;
    V.gamma = vel->gamma;
    V.nu = vel->nu;
    V.x0 = vel->x0;
    V.y0 = vel->y0;
  } else if (V.kind == VRM_VEL_BIOT_SAVART) {
    if (!(vel->eps > 0) || !std::isfinite(vel->eps)) return VRM_ERR_ARG;
  } else if (V.kind != VRM_VEL_NONE) {
    return VRM_ERR_ARG;
  }
  vrm_stats local;
  vrm_stats* st = stats ? stats : &local;
  memset(st, 0, sizeof(*st));
  if (n == 0) {
    *n_out = 0;
    return VRM_OK;
  }
  Scratch& s = ctx->s;
  VRM_CUDA(ensure_scratch(ctx, capacity, stream));
  VRM_CUDA(ensure_learned(ctx, capacity, stream));
  VRM_CUDA(ensure_rk(ctx, capacity, stream));
  if (V.kind == VRM_VEL_BIOT_SAVART) VRM_CUDA(ensure_bs(ctx, capacity, capacity, stream));
  VRM_CUDA(cudaStreamSynchronize(stream));
  StepState P;
  memset(&P, 0, sizeof(P));
  P.n = n;
  P.capacity = capacity;
  P.dt = dt;
  P.max_rounds = ctx->p.max_rounds;
  *s.h_params = P;
  const int timing = ctx->timing;
  ctx->timing = 0;
  // growth control and insertion once, on the step's initial cloud
  vrm_status r = run_step_eager(ctx, x, y, capacity, gamma_in, nullptr, s.diffused, false, stream);
  ctx->timing = timing;
  if (r != VRM_OK) return r;
  VRM_CUDA(read_back(ctx, stream));
  if (s.h_grid->nonfinite || s.h_ds->nonfinite) return VRM_ERR_ARG;
  fill_front_stats(ctx, n, st);
  if (s.h_state->overflow) return VRM_ERR_CAPACITY;
  const int* n_cur = &s.st->n_cur;
  double* Xs[3] = {x, ctx->rk_x1, ctx->rk_x2};
  double* Ys[3] = {y, ctx->rk_y1, ctx->rk_y2};
  const double* Gs[3] = {gamma_in, ctx->rk_g1, ctx->rk_g2};
  double* Xo[3] = {ctx->rk_x1, ctx->rk_x2, x};
  double* Yo[3] = {ctx->rk_y1, ctx->rk_y2, y};
  double* Go[3] = {ctx->rk_g1, ctx->rk_g2, gamma_out};
  const double ts[3] = {t, t + dt, t + 0.5 * dt};
  const bool move = V.kind != VRM_VEL_NONE;
  for (int k = 0; k < 3; ++k) {
    // without a velocity every stage sits at the initial positions
    const double* px = move ? Xs[k] : x;
    const double* py = move ? Ys[k] : y;
    VRM_CUDA(enqueue_stage_weights(ctx, px, py, capacity, stream));
    VRM_CUDA(apply_transposed_dev(ctx->c, capacity, n_cur, k == 0 ? n : capacity, k == 0 ? nullptr : n_cur, Gs[k],
                                  s.diffused, s.dlist, s.counters + 0, s.cols, s.f, s.fii, s.tcount, s.toff,
                                  s.tent, s.scan_tmp, s.ds, ctx->rk_dg, nullptr, 0.0, nullptr, stream));
    const double *us = nullptr, *vs = nullptr;
    if (V.kind == VRM_VEL_BIOT_SAVART) {
      // the stage's own velocity at every stage particle; in the first stage
      // only the n given particles carry circulation (gamma_in holds n)
      if (k == 0) {
        VRM_CUDA(bs_split(px, py, gamma_in, n, nullptr, ctx->bs_src, ctx->bs_g, stream));
        VRM_CUDA(bs_split(px, py, nullptr, capacity, n_cur, ctx->bs_tgt, nullptr, stream));
        VRM_CUDA(bs_direct(ctx->bs_src, ctx->bs_g, n, nullptr, ctx->bs_tgt, capacity, n_cur, vel->eps, ctx->rk_u,
                           ctx->rk_v, stream));
      } else {
        VRM_CUDA(bs_split(px, py, Gs[k], capacity, n_cur, ctx->bs_src, ctx->bs_g, stream));
        VRM_CUDA(bs_direct(ctx->bs_src, ctx->bs_g, capacity, n_cur, ctx->bs_src, capacity, n_cur, vel->eps,
                           ctx->rk_u, ctx->rk_v, stream));
      }
      us = ctx->rk_u;
      vs = ctx->rk_v;
    }
    VRM_CUDA(rk3_stage(k, capacity, n_cur, dt, ts[k], V, x, y, gamma_in, n, px, py, Gs[k], ctx->rk_dg, us, vs, Xo[k],
                       Yo[k], Go[k], stream));
  }
  VRM_CUDA(read_back(ctx, stream));
  if (ctx->mlp && vrm_mlp_error(ctx->mlp, stream) != VRM_OK) return VRM_ERR_CUDA;
  if (s.h_grid->nonfinite || s.h_ds->nonfinite) return VRM_ERR_ARG;
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
  st->lp_full_columns = (int64_t)s.h_ds->lp_full_columns;
  st->lp_full_column_pivots = (int64_t)s.h_ds->lp_full_column_pivots;
  st->lp_small_rechecked = (int64_t)s.h_ds->lp_small_retries;
  st->learned_ok = s.h_ds->learned_ok;
  st->learned_rejected = s.h_ds->learned_rejected;
  st->learned_square = s.h_ds->learned_square;
  st->learned_screens = (int64_t)s.h_ds->learned_screens;
  *n_out = s.h_state->n_cur;
  if (s.h_ds->max_count > ctx->c.row_cap) return VRM_ERR_CAPACITY;
  return VRM_OK;
}

vrm_status vrm_biot_savart(vrm_ctx* ctx, const double* xs, const double* ys, const double* gamma, int32_t n,
                           const double* xt, const double* yt, int32_t m, double eps, double* u, double* v,
                           cudaStream_t stream) {
  if (!ctx || n < 0 || m < 0 || !(eps > 0) || !std::isfinite(eps)) return VRM_ERR_ARG;
  if (bad_ptr(xs, n) || bad_ptr(ys, n) || bad_ptr(gamma, n) || bad_ptr(xt, m) || bad_ptr(yt, m) || bad_ptr(u, m) ||
      bad_ptr(v, m))
    return VRM_ERR_ARG;
  if (m == 0) return VRM_OK;
  if (n == 0) {
    VRM_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * (size_t)m, stream));
    VRM_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * (size_t)m, stream));
    return VRM_OK;
  }
  VRM_CUDA(ensure_bs(ctx, n, m, stream));
  VRM_CUDA(bs_split(xs, ys, gamma, n, nullptr, ctx->bs_src, ctx->bs_g, stream));
  VRM_CUDA(bs_split(xt, yt, nullptr, m, nullptr, ctx->bs_tgt, nullptr, stream));
  VRM_CUDA(bs_direct(ctx->bs_src, ctx->bs_g, n, nullptr, ctx->bs_tgt, m, nullptr, eps, u, v, stream));
  return VRM_OK;
}

vrm_status vrm_set_mlp(vrm_ctx* ctx, vrm_mlp* net) {
  if (!ctx) return VRM_ERR_ARG;
  if (net && ctx->p.order != 1) return VRM_ERR_UNSUPPORTED;  // the network proposes n = 1 stencils
  if (ctx->mlp != net) {
    ctx->mlp = net;
    drop_graph(ctx);
    ++ctx->scratch_gen;
  }
  return VRM_OK;
}

vrm_status vrm_learned_features(vrm_ctx* ctx, const double* x, const double* y, int32_t n, const int32_t* list,
                                int32_t m, const int32_t* nbr_count, const int32_t* nbr_idx, uint16_t* X,
                                int32_t* slots, cudaStream_t stream) {
  if (!ctx || m < 0 || n < 0) return VRM_ERR_ARG;
  if (m == 0) return VRM_OK;
  if (!x || !y || n == 0 || !nbr_count || !nbr_idx || !X || !slots || misaligned16(X)) return VRM_ERR_ARG;
  if (!list && m > n) return VRM_ERR_ARG;
  VRM_CUDA(ensure_scratch(ctx, n, stream));
  // the fp32 position copy lives in the step's weight scratch (8 doubles per particle)
  VRM_CUDA(learned_features(full_rows(ctx->c), x, y, n, nullptr, reinterpret_cast<float2*>(ctx->s.f), list, nullptr,
                            m, nbr_count, nbr_idx, reinterpret_cast<__nv_bfloat16*>(X), slots, stream));
  return VRM_OK;
}

vrm_status vrm_learned_project(vrm_ctx* ctx, const double* x, const double* y, const int32_t* list, int32_t m,
                               const int32_t* slots, const float* f0, const int32_t* small, int32_t* cols, double* f,
                               double* fii, uint8_t* status, int32_t* n_accepted, cudaStream_t stream) {
  if (!ctx || m < 0) return VRM_ERR_ARG;
  if (n_accepted) *n_accepted = 0;
  if (m == 0) return VRM_OK;
  if (!x || !y || !slots || !f0 || !small || !cols || !f || !fii || !status || misaligned16(small)) return VRM_ERR_ARG;
  if (ctx->p.order != 1) return VRM_ERR_UNSUPPORTED;
  Scratch& s = ctx->s;
  VRM_CUDA(ensure_scratch(ctx, m, stream));
  VRM_CUDA(ensure_proj(ctx, m, stream));
  VRM_CUDA(cudaMemsetAsync(s.ds, 0, sizeof(DevStats), stream));
  VRM_CUDA(learned_project(ctx->c, x, y, list, nullptr, m, slots, f0, small, cols, f, fii, status, nullptr, nullptr,
                           s.ds, nullptr, ctx->p.nu, &ctx->L.proj, stream));
  VRM_CUDA(read_back(ctx, stream));
  if (n_accepted) *n_accepted = s.h_ds->learned_ok;
  return VRM_OK;
}

vrm_status vrm_learned_targets(const int32_t* list, int32_t m, const int32_t* slots, const int32_t* cols,
                               const double* f, float* T, cudaStream_t stream) {
  if (m < 0) return VRM_ERR_ARG;
  if (m == 0) return VRM_OK;
  if (!list || !slots || !cols || !f || !T) return VRM_ERR_ARG;
  VRM_CUDA(learned_targets(list, m, slots, cols, f, T, stream));
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
  VRM_CUDA(apply_gather(full_rows(ctx->c), n, n_gamma, gamma, diffused, nbr_count, nbr_idx, cols, f, fii, nullptr, dgamma,
                        nullptr, 0.0, stream));
  return VRM_OK;
}

// Enqueues one attempt of the step (the captured graph, or the kernels one
// by one when graphs are off) on the stream.
static vrm_status step_launch(vrm_ctx* ctx, bool* launched) {
  Scratch& s = ctx->s;
  const vrm_ctx::Pending& P = ctx->pending;
  if (ctx->timing)
    for (int k = 0; k < VRM_STAGE_COUNT; ++k) ctx->stage_done[k] = 0;
  *launched = false;
  if (ctx->use_graph) {
    const StepGraph& G = ctx->graph;
    const bool hit = G.exec && G.x == P.x && G.y == P.y && G.gi == P.gi && G.go == P.go && G.cap == P.cap &&
                     G.timing == ctx->timing;
    if (!hit && !capture_step(ctx, P.x, P.y, P.cap, P.gi, P.go)) ctx->use_graph = 0;
    if (ctx->use_graph) {
      // the captured event nodes record every stage boundary
      if (ctx->timing)
        for (int k = 0; k < VRM_STAGE_COUNT; ++k) ctx->stage_done[k] = 1;
      VRM_CUDA(cudaGraphLaunch(ctx->graph.exec, P.stream));
      *launched = true;
    }
  }
  if (!*launched) {
    vrm_status r = run_step_eager(ctx, P.x, P.y, P.cap, P.gi, P.go, s.diffused, true, P.stream);
    if (r != VRM_OK) return r;
  }
  VRM_CUDA(cudaEventRecord(ctx->step_done, P.stream));
  return VRM_OK;
}

vrm_status vrm_step_begin(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma_in,
                          double* gamma_out, double dt, cudaStream_t stream) {
  if (!ctx || n < 0 || capacity < n || !std::isfinite(dt)) return VRM_ERR_ARG;
  if (ctx->pending.active) return VRM_ERR_ARG;
  if (bad_ptr(x, n) || bad_ptr(y, n) || bad_ptr(gamma_in, n) || bad_ptr(gamma_out, capacity)) return VRM_ERR_ARG;
  if (n > 0 && gamma_out < gamma_in + n && gamma_in < gamma_out + capacity) return VRM_ERR_ARG;
  vrm_ctx::Pending& P = ctx->pending;
  P = vrm_ctx::Pending{};
  P.x = x;
  P.y = y;
  P.gi = gamma_in;
  P.go = gamma_out;
  P.n = n;
  P.cap = capacity;
  P.stream = stream;
  if (n == 0) {
    P.active = 1;
    return VRM_OK;
  }
  Scratch& s = ctx->s;
  VRM_CUDA(ensure_scratch(ctx, capacity, stream));
  VRM_CUDA(ensure_learned(ctx, capacity, stream));
  if (!ctx->step_done) VRM_CUDA(cudaEventCreateWithFlags(&ctx->step_done, cudaEventDisableTiming));
  // the pinned parameter block is read by the step's head copy; the last
  // step of this context has ended (vrm_step_end waited for it), so it is
  // free to rewrite
  StepState S;
  memset(&S, 0, sizeof(S));
  S.n = n;
  S.capacity = capacity;
  S.dt = dt;
  S.max_rounds = ctx->p.max_rounds;
  *s.h_params = S;
  bool launched = false;
  vrm_status r = step_launch(ctx, &launched);
  if (r != VRM_OK) return r;
  P.launched = launched;
  P.active = 1;
  return VRM_OK;
}

vrm_status vrm_step_end(vrm_ctx* ctx, int32_t* n_out, vrm_stats* stats) {
  if (!ctx || !n_out || !ctx->pending.active) return VRM_ERR_ARG;
  vrm_ctx::Pending& P = ctx->pending;
  P.active = 0;
  vrm_stats local;
  vrm_stats* st = stats ? stats : &local;
  memset(st, 0, sizeof(*st));
  if (P.n == 0) {
    *n_out = 0;
    return VRM_OK;
  }
  Scratch& s = ctx->s;
  const int n = P.n;
  VRM_CUDA(cudaEventSynchronize(ctx->step_done));
  for (int attempt = 0;; ++attempt) {
    if (P.launched) add_launches(ctx->graph.kernels_outer + ctx->graph.kernels_body * s.h_state->round);
    // rows cut by a row_cap below k_cap: the step is repeated with whole rows
    // (it reads only [0, n) of x, y and gamma_in, so the repeat is exact)
    const bool cut = !s.h_grid->nonfinite && !s.h_ds->nonfinite && !s.h_state->overflow &&
                     s.h_ds->max_count > ctx->c.row_cap && ctx->c.row_cap < ctx->p.k_cap;
    if (!cut || attempt > 0) break;
    ctx->c.row_cap = ctx->p.k_cap;
    drop_graph(ctx);
    bool launched = false;
    vrm_status r = step_launch(ctx, &launched);
    if (r != VRM_OK) return r;
    P.launched = launched;
    VRM_CUDA(cudaEventSynchronize(ctx->step_done));
  }
  if (ctx->mlp && vrm_mlp_error(ctx->mlp, P.stream) != VRM_OK) return VRM_ERR_CUDA;
  if (s.h_grid->nonfinite || s.h_ds->nonfinite) return VRM_ERR_ARG;
  fill_front_stats(ctx, n, st);
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
  st->lp_full_columns = (int64_t)s.h_ds->lp_full_columns;
  st->lp_full_column_pivots = (int64_t)s.h_ds->lp_full_column_pivots;
  st->lp_small_rechecked = (int64_t)s.h_ds->lp_small_retries;
  st->learned_ok = s.h_ds->learned_ok;
  st->learned_rejected = s.h_ds->learned_rejected;
  st->learned_square = s.h_ds->learned_square;
  st->learned_screens = (int64_t)s.h_ds->learned_screens;
  if (s.h_state->overflow) return VRM_ERR_CAPACITY;
  *n_out = s.h_state->n_cur;
  if (s.h_ds->max_count > ctx->p.k_cap) return VRM_ERR_CAPACITY;
  return VRM_OK;
}

vrm_status vrm_step(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma_in,
                    double* gamma_out, double dt, int32_t* n_out, vrm_stats* stats, cudaStream_t stream) {
  if (!ctx || !n_out) return VRM_ERR_ARG;
  if (ctx->pending.active) return VRM_ERR_ARG;
  // the head copy of an earlier step on this stream may still read the
  // pinned parameter block: wait for the stream before rewriting it
  if (n > 0) VRM_CUDA(cudaStreamSynchronize(stream));
  vrm_status r = vrm_step_begin(ctx, x, y, n, capacity, gamma_in, gamma_out, dt, stream);
  if (r != VRM_OK) return r;
  return vrm_step_end(ctx, n_out, stats);
}

vrm_status vrm_batch_create(const vrm_params* p, int32_t max_clouds, vrm_batch** out) {
  if (!out) return VRM_ERR_ARG;
  *out = nullptr;
  if (max_clouds < 1 || max_clouds > 4096) return VRM_ERR_ARG;
  vrm_status st = check_params(p);
  if (st != VRM_OK) return st;
  vrm_batch* b = new (std::nothrow) vrm_batch();
  if (!b) return VRM_ERR_CUDA;
  b->base = *p;
  b->max_clouds = max_clouds;
  const char* env = getenv("VRM_NO_GRAPH");
  b->use_graph = !(env && env[0] == '1');
  b->sub = new (std::nothrow) vrm_ctx*[max_clouds]();
  b->branch = new (std::nothrow) cudaStream_t[max_clouds]();
  b->join = new (std::nothrow) cudaEvent_t[max_clouds]();
  b->key = new (std::nothrow) BatchKey[max_clouds]();
  b->kernels_outer = new (std::nothrow) long long[max_clouds]();
  b->kernels_body = new (std::nothrow) long long[max_clouds]();
  b->sched = new (std::nothrow) vrm_schedule[max_clouds]();
  if (!b->sub || !b->branch || !b->join || !b->key || !b->kernels_outer || !b->kernels_body || !b->sched) {
    vrm_batch_destroy(b);
    return VRM_ERR_CUDA;
  }
  *out = b;
  return VRM_OK;
}

void vrm_batch_destroy(vrm_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (int c = 0; c < b->max_clouds; ++c) {
    if (b->sub && b->sub[c]) vrm_destroy(b->sub[c]);
    if (b->branch && b->branch[c]) cudaStreamDestroy(b->branch[c]);
    if (b->join && b->join[c]) cudaEventDestroy(b->join[c]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->body_stream) cudaStreamDestroy(b->body_stream);
  delete[] b->sub;
  delete[] b->branch;
  delete[] b->join;
  delete[] b->key;
  delete[] b->kernels_outer;
  delete[] b->kernels_body;
  delete[] b->sched;
  delete b;
}

vrm_status vrm_batch_set_schedule(vrm_batch* b, int32_t slot, const vrm_schedule* s) {
  if (!b || !s || slot < 0 || slot >= b->max_clouds || !schedule_ok(*s, b->base.k_cap)) return VRM_ERR_ARG;
  b->sched[slot] = *s;
  if (b->sub[slot]) {
    put_schedule(b->sub[slot]->c, *s);
    drop_graph(b->sub[slot]);
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  return VRM_OK;
}

vrm_status vrm_get_schedule(const vrm_ctx* ctx, vrm_schedule* out) {
  if (!ctx || !out) return VRM_ERR_ARG;
  memset(out, 0, sizeof(*out));
  out->row_cap = ctx->c.row_cap;
  out->search_block = ctx->c.search_block;
  out->lp_block = ctx->c.lp_block;
  out->lp_blocks_per_sm = ctx->c.lp_blocks_per_sm;
  out->lp_fp64_pivots = ctx->c.lp_fp64_pivots;
  out->apply_block = ctx->c.apply_block;
  return VRM_OK;
}

vrm_status vrm_set_schedule(vrm_ctx* ctx, const vrm_schedule* s) {
  if (!ctx || !s || !schedule_ok(*s, ctx->p.k_cap)) return VRM_ERR_ARG;
  put_schedule(ctx->c, *s);
  drop_graph(ctx);
  return VRM_OK;
}

}  // extern "C"

namespace {

// Captures every active cloud's step as one branch of one graph: a fork
// event on the capture stream, each cloud's whole step (with its own
// insertion while node) on its own branch stream, and joins back.
bool capture_batch(vrm_batch* b, const vrm_cloud* clouds, int n_clouds, const bool* active) {
  if (!b->cap_stream && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (!b->body_stream && cudaStreamCreateWithFlags(&b->body_stream, cudaStreamNonBlocking) != cudaSuccess)
    return false;
  if (!b->fork && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return false;
  for (int c = 0; c < n_clouds; ++c) {
    if (!active[c]) continue;
    if (!b->branch[c] && cudaStreamCreateWithFlags(&b->branch[c], cudaStreamNonBlocking) != cudaSuccess) return false;
    if (!b->join[c] && cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming) != cudaSuccess) return false;
  }
  cudaStream_t cs = b->cap_stream;
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  const bool capturing = ok;
  ok = ok && cudaEventRecord(b->fork, cs) == cudaSuccess;
  for (int c = 0; c < n_clouds && ok; ++c) {
    if (!active[c]) continue;
    const vrm_cloud& C = clouds[c];
    ok = cudaStreamWaitEvent(b->branch[c], b->fork, 0) == cudaSuccess;
    ok = ok && record_step(b->sub[c], b->branch[c], b->body_stream, C.x, C.y, C.capacity, C.gamma_in, C.gamma_out,
                           &b->kernels_outer[c], &b->kernels_body[c]);
    ok = ok && cudaEventRecord(b->join[c], b->branch[c]) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(cs, b->join[c], 0) == cudaSuccess;
  }
  if (capturing) {
    const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
    ok = ok && ended && g;
  }
  cudaGraphExec_t exec = nullptr;
  ok = ok && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  for (int c = 0; c < b->max_clouds; ++c) b->key[c] = BatchKey{};
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    return false;
  }
  b->exec = exec;
  for (int c = 0; c < n_clouds; ++c) {
    if (!active[c]) continue;
    const vrm_cloud& C = clouds[c];
    b->key[c] = BatchKey{C.x, C.y, C.gamma_in, C.gamma_out, C.capacity, C.h, b->sub[c]->scratch_gen};
  }
  return true;
}

// Outcome of one cloud's step from its pinned mirrors (as in vrm_step).
vrm_status finish_cloud(vrm_ctx* ctx, vrm_cloud& C, vrm_stats* st) {
  Scratch& s = ctx->s;
  memset(st, 0, sizeof(*st));
  if (s.h_grid->nonfinite || s.h_ds->nonfinite) return VRM_ERR_ARG;
  fill_front_stats(ctx, C.n, st);
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
  st->lp_full_columns = (int64_t)s.h_ds->lp_full_columns;
  st->lp_full_column_pivots = (int64_t)s.h_ds->lp_full_column_pivots;
  st->lp_small_rechecked = (int64_t)s.h_ds->lp_small_retries;
  st->learned_ok = s.h_ds->learned_ok;
  st->learned_rejected = s.h_ds->learned_rejected;
  st->learned_square = s.h_ds->learned_square;
  st->learned_screens = (int64_t)s.h_ds->learned_screens;
  C.n_out = st->n_out;
  if (s.h_state->overflow) return VRM_ERR_CAPACITY;
  if (s.h_ds->max_count > ctx->p.k_cap) return VRM_ERR_CAPACITY;
  return VRM_OK;
}

void add_stats(vrm_stats* t, const vrm_stats& a) {
  t->n_in += a.n_in;
  t->n_out += a.n_out;
  t->n_diffused += a.n_diffused;
  t->n_inserted += a.n_inserted;
  t->open_segments += a.open_segments;
  t->small_ok += a.small_ok;
  t->full_ok += a.full_ok;
  t->no_stencil += a.no_stencil;
  if (a.rounds > t->rounds) t->rounds = a.rounds;
  if (a.max_pivots > t->max_pivots) t->max_pivots = a.max_pivots;
  if (a.max_count > t->max_count) t->max_count = a.max_count;
  if (a.max_dt_ratio > t->max_dt_ratio) t->max_dt_ratio = a.max_dt_ratio;
  t->lp_small_solved += a.lp_small_solved;
  t->lp_small_pivots += a.lp_small_pivots;
  t->lp_full_solved += a.lp_full_solved;
  t->lp_full_pivots += a.lp_full_pivots;
  t->lp_full_columns += a.lp_full_columns;
  t->lp_full_column_pivots += a.lp_full_column_pivots;
  t->lp_small_rechecked += a.lp_small_rechecked;
  t->learned_ok += a.learned_ok;
  t->learned_rejected += a.learned_rejected;
  t->learned_square += a.learned_square;
  t->learned_screens += a.learned_screens;
}

}  // namespace

extern "C" vrm_status vrm_step_batched(vrm_batch* b, vrm_cloud* clouds, int32_t n_clouds, vrm_stats* stats,
                                       cudaStream_t stream) {
  if (!b || n_clouds < 0 || n_clouds > b->max_clouds || (n_clouds > 0 && !clouds)) return VRM_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  // argument checks of every cloud before any work
  for (int c = 0; c < n_clouds; ++c) {
    vrm_cloud& C = clouds[c];
    C.n_out = 0;
    C.status = VRM_OK;
    const int n = C.n, cap = C.capacity;
    bool bad = n < 0 || cap < n || !std::isfinite(C.dt) || !(C.h > 0) || !std::isfinite(C.h);
    bad = bad || bad_ptr(C.x, n) || bad_ptr(C.y, n) || bad_ptr(C.gamma_in, n) || bad_ptr(C.gamma_out, cap);
    bad = bad || (n > 0 && C.gamma_out < C.gamma_in + n && C.gamma_in < C.gamma_out + cap);
    if (bad) C.status = VRM_ERR_ARG;
  }
  for (int c = 0; c < n_clouds; ++c)
    if (clouds[c].status != VRM_OK) return VRM_ERR_ARG;
  bool* active = new (std::nothrow) bool[n_clouds > 0 ? n_clouds : 1];
  if (!active) return VRM_ERR_CUDA;
  vrm_status result = VRM_OK;
  bool hit = b->exec != nullptr;
  VRM_CUDA(cudaStreamSynchronize(stream));
  for (int c = 0; c < n_clouds && result == VRM_OK; ++c) {
    vrm_cloud& C = clouds[c];
    active[c] = C.n > 0;
    if (!active[c]) {
      hit = hit && b->key[c].cap == 0;
      continue;
    }
    vrm_params p = b->base;
    p.h = C.h;
    bool fresh = false;
    if (!b->sub[c]) {
      if (vrm_create(&p, &b->sub[c]) != VRM_OK) result = VRM_ERR_CUDA;
      fresh = true;
    } else if (b->sub[c]->p.h != C.h) {
      b->sub[c]->p = p;
      fill_consts(p, b->sub[c]->c);
      drop_graph(b->sub[c]);
      fresh = true;
    }
    if (result != VRM_OK) break;
    vrm_ctx* ctx = b->sub[c];
    if (fresh && b->sched[c].row_cap) put_schedule(ctx->c, b->sched[c]);
    if (ensure_scratch(ctx, C.capacity, stream) != cudaSuccess) {
      result = VRM_ERR_CUDA;
      break;
    }
    StepState P;
    memset(&P, 0, sizeof(P));
    P.n = C.n;
    P.capacity = C.capacity;
    P.dt = C.dt;
    P.max_rounds = ctx->p.max_rounds;
    *ctx->s.h_params = P;
    const BatchKey& K = b->key[c];
    hit = hit && K.x == C.x && K.y == C.y && K.gi == C.gamma_in && K.go == C.gamma_out && K.cap == C.capacity &&
          K.h == C.h && K.scratch_gen == ctx->scratch_gen;
  }
  for (int c = n_clouds; c < b->max_clouds && hit; ++c) hit = b->key[c].cap == 0;
  if (result != VRM_OK) {
    delete[] active;
    return result;
  }
  bool launched = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    launched = false;
    if (b->use_graph) {
      if (!hit && !capture_batch(b, clouds, n_clouds, active)) b->use_graph = 0;
      if (b->use_graph) {
        if (cudaGraphLaunch(b->exec, stream) != cudaSuccess) {
          delete[] active;
          return VRM_ERR_CUDA;
        }
        launched = true;
      }
    }
    if (!launched) {
      // one cloud after the other, each step eager
      for (int c = 0; c < n_clouds && result == VRM_OK; ++c) {
        if (!active[c]) continue;
        const vrm_cloud& C = clouds[c];
        result = run_step_eager(b->sub[c], C.x, C.y, C.capacity, C.gamma_in, C.gamma_out, b->sub[c]->s.diffused,
                                true, stream);
      }
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) result = VRM_ERR_CUDA;
    if (result != VRM_OK) {
      delete[] active;
      return result;
    }
    if (launched)
      for (int c = 0; c < n_clouds; ++c)
        if (active[c]) add_launches(b->kernels_outer[c] + b->kernels_body[c] * b->sub[c]->s.h_state->round);
    // clouds whose rows were cut by a row_cap below k_cap: repeat the batch
    // once with whole rows for them (every step reads only its inputs)
    bool cut = false;
    for (int c = 0; c < n_clouds; ++c) {
      if (!active[c]) continue;
      vrm_ctx* ctx = b->sub[c];
      const Scratch& s = ctx->s;
      if (!s.h_grid->nonfinite && !s.h_ds->nonfinite && !s.h_state->overflow && s.h_ds->max_count > ctx->c.row_cap &&
          ctx->c.row_cap < ctx->p.k_cap) {
        ctx->c.row_cap = ctx->p.k_cap;
        b->sched[c].row_cap = ctx->p.k_cap;
        cut = true;
      }
    }
    if (!cut) break;
    hit = false;
  }
  vrm_status first_bad = VRM_OK;
  for (int c = 0; c < n_clouds; ++c) {
    if (!active[c]) continue;
    vrm_ctx* ctx = b->sub[c];
    vrm_stats one;
    const vrm_status r = finish_cloud(ctx, clouds[c], &one);
    clouds[c].status = r;
    if (r != VRM_OK && first_bad == VRM_OK) first_bad = r;
    if (stats) add_stats(stats, one);
  }
  delete[] active;
  return first_bad;
}
