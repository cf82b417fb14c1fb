// Internal declarations of the VRM CUDA library (not part of the C ABI).
//
// Layout of the work (one context, one stream):
//   vrm_grid.cu    bounding box, cell binning, scans and compaction
//   vrm_reduce.cu  growth control (Sec. 3.5): exact radix select on |Gamma|
//   vrm_search.cu  annulus neighbourhoods, segment masks, small neighbourhoods
//   vrm_insert.cu  insertion rounds (Sec. 4.2)
//   vrm_lp.cu      phase-I simplex per particle (Sec. 4.1, 4.3)
//   vrm_apply.cu   gather-form operator application and Euler update
//   vrm_api.cu     the C ABI: argument checks, scratch, orchestration
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vrm.h"

namespace vrm {

typedef unsigned __int128 u128;

// Threads per block for the streaming kernels, and the persistent grid size
// (a multiple of the SM count) used for grid-stride loops.
constexpr int kBlock = 256;

// Constants every kernel may need, passed by value.
struct Consts {
  double h, inv_h, lo2, hi2, Rh, c_bound, nu_over_h2;
  float lo2f, hi2f;
  double ins_dx[8], ins_dy[8];  // insertion offsets 1.5h (cos, sin)((s+1/2) pi/4)
  int k_cap;      // neighbour row stride
  int max_rounds;
  int fallback;
  int precision;
  int order;      // consistency order n (1 or 2)
  int w;          // stencil width: 8 for n = 1, 12 for n = 2
  // launch schedule (vrm_schedule); results do not depend on it
  int row_cap;           // neighbour entries kept per row (<= k_cap)
  int search_block;      // threads per block of k_search_all
  int lp_block;          // threads per block of k_lp_small
  int lp_blocks_per_sm;  // grid cap of k_lp_small
  int lp_fp64_pivots;    // 1: small LPs pivot in FP64; 0: certified binary32 pivots, FP64 re-runs
  int apply_block;       // threads per block of k_apply
};

// The schedule every context starts with.
inline void default_schedule(Consts& c) {
  c.row_cap = c.k_cap;
  c.search_block = 256;
  c.lp_block = 128;
  c.lp_blocks_per_sm = 16;
  c.lp_fp64_pivots = 0;
  c.apply_block = 256;
}

// Uniform cell grid, device resident (written by grid_build).
// Besides FP64 positions, the sorted arrays hold FP32 cell-local coordinates
// u - floor(u) with u = (x - x0)/cs.  In cell units the offset of two
// particles is (cell difference) + (local difference), within 5e-7 of the
// exact value (|offset| < 2 cells), so an FP32 squared distance is within
// 1e-5 of the exact one: pairs further than `band` from an annulus bound are
// decided in FP32, the rest by the FP64 definition.
struct Grid {
  double x0, y0, inv_cs;
  int nx, ny, ncell;
  int nonfinite;          // set if a position was NaN/Inf
  float lo_out, lo_in;    // (r h / cs)^2 -/+ band
  float hi_in, hi_out;    // (R h / cs)^2 -/+ band
  float seg_eps;          // FP32 segment decisions need this margin (cell units)
};
constexpr float kBand = 2e-5f;
constexpr float kSegEps = 4e-6f;

// Device-side counters of one step.
struct DevStats {
  int n_diffused;
  int n_open;          // open particles of the current insertion round
  int n_accepted;      // points accepted in the current round
  int small_ok, full_ok, no_stencil;
  int max_pivots;
  int max_count;
  int n_fail;          // particles queued for the full-neighbourhood LP
  int nonfinite;       // set if a circulation was NaN/Inf
  unsigned long long max_dt_ratio_bits;  // positive double, as bits
  unsigned long long lp_small_pivots, lp_full_pivots;
  int lp_small_solved, lp_full_solved;
  int learned_ok, learned_rejected, learned_square;
  unsigned long long learned_screens;        // supports screened by the learned path
  unsigned long long lp_full_columns;        // columns summed over the full-neighbourhood LPs
  unsigned long long lp_full_column_pivots;  // columns x pivots summed over them
  int n_retry;                               // retry list of the current small-LP pass (FP64 re-runs)
  unsigned long long lp_small_retries;       // small LPs re-run in FP64 (uncertain binary32 decision)
};

// Growth-control selection state (device resident).
struct ReduceState {
  unsigned long long amax_bits;  // max |Gamma| as bits
  int E;                         // max |Gamma| < 2^E
  int done;                      // 1: no particle diffuses / selection finished early
  unsigned long long prefix;     // high key bits matched so far
  unsigned long long tau_lo, tau_hi;  // remaining budget (u128)
  unsigned long long T;          // threshold key (bits of |Gamma|)
  int k_tie;                     // particles with key == T that stay out (lowest indices)
  int all_out;                   // 1: every particle stays out (sum within bound)
  unsigned int blocks_done;      // blocks of the current pass that have merged their histogram
  int n_sub;                     // particles matching the first two chosen bytes (listed by pass 2)
  unsigned long long hist[256][4];  // per digit: limb sums (3 x 32-bit limbs) and count
};

// Device-resident state of one vrm_step (so that the step runs without host
// round trips and can be captured in a CUDA graph).
struct StepState {
  int n;               // particles given
  int capacity;        // room in x, y, gamma_out
  double dt;           // Euler step
  int n_cur;           // particles now (grows with insertion)
  int n_open;          // open particles of the current insertion round
  int n_cand;          // proposals of the current round
  int accepted;        // proposals accepted in the current round
  int n_next;          // open particles left after the round
  int round;           // insertion rounds run
  int rounds_appended; // rounds that appended particles
  int overflow;        // 1: an insertion would exceed the capacity
  int n_needed;        // particles that would have been needed then
  int open_segments;   // empty segments left when max_rounds is reached
  int max_rounds;
  int n_list;          // length of the first round's open list (every round works on it)
  int n_act[2];        // lengths of RoundBufs::act0 / act1
  unsigned blocks_done;  // blocks of the round's last kernel that have finished
};

struct Scratch;  // defined in vrm_api.cu

// ---- device helpers --------------------------------------------------------

// Segment k covers [k pi/4, (k+1) pi/4) counter-clockwise from +x, decided by
// comparisons only (seg(-r) = seg(r) + 4 mod 8 exactly).
template <typename T>
__device__ __forceinline__ int segment_of(T dx, T dy) {
  int s;
  if (dx > T(0) && dy >= T(0)) s = dy < dx ? 0 : 1;
  else if (dx <= T(0) && dy > T(0)) s = dy > -dx ? 2 : 3;
  else if (dx < T(0) && dy <= T(0)) s = dy > dx ? 4 : 5;
  else s = -dy > dx ? 6 : 7;
  return s;
}

// Squared distance with separate roundings (no contraction).
__device__ __forceinline__ double dist2(double dx, double dy) {
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}
__device__ __forceinline__ float dist2f(float dx, float dy) {
  return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Order-preserving map of doubles to u64 (for atomic min/max).
__device__ __forceinline__ unsigned long long ordered_bits(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered_bits(unsigned long long b) {
  b = (b >> 63) ? (b & 0x7FFFFFFFFFFFFFFFull) : ~b;
  return __longlong_as_double((long long)b);
}

__device__ __forceinline__ int grid_cell_x(const Grid& g, double x) {
  int c = (int)floor(__dmul_rn(__dsub_rn(x, g.x0), g.inv_cs));
  return c < 0 ? 0 : (c >= g.nx ? g.nx - 1 : c);
}
__device__ __forceinline__ int grid_cell_y(const Grid& g, double y) {
  int c = (int)floor(__dmul_rn(__dsub_rn(y, g.y0), g.inv_cs));
  return c < 0 ? 0 : (c >= g.ny ? g.ny - 1 : c);
}
// Cell-local FP32 coordinate of x in a cell of index cx.
__device__ __forceinline__ float grid_local_x(const Grid& g, double x, int cx) {
  return __double2float_rn(__dsub_rn(__dmul_rn(__dsub_rn(x, g.x0), g.inv_cs), (double)cx));
}
__device__ __forceinline__ float grid_local_y(const Grid& g, double y, int cy) {
  return __double2float_rn(__dsub_rn(__dmul_rn(__dsub_rn(y, g.y0), g.inv_cs), (double)cy));
}
// Segment of an FP32 cell-unit offset, or -1 when it lies within seg_eps of a
// decision line (then the FP64 classifier decides).
__device__ __forceinline__ int segment_or_ambiguous(float du, float dv, float eps) {
  if (fabsf(du) <= eps || fabsf(dv) <= eps || fabsf(dv - du) <= 2.f * eps || fabsf(dv + du) <= 2.f * eps) return -1;
  return segment_of(du, dv);
}

// Analytic velocity of the RK3 step (vrm_velocity).
struct Velocity {
  int kind;
  double gamma, nu, x0, y0;
};

// ---- launch helpers (host) -----------------------------------------------

int persistent_blocks(int block_threads, int per_sm);
int sm_count();
// Counts kernel launches of the library (vrm_launch_count).
void note_launch();
void add_launches(long long k);
long long launch_count();

// vrm_grid.cu
// Builds the cell grid over n particles: bbox, cell size (>= Rh (1+1e-6),
// doubled while the cell count exceeds ncell_cap), keys, exclusive scan of
// the cell counts (cell_start, ncell_cap + 1 entries), sorted positions and
// indices.  Grid g is written on the device.
cudaError_t grid_build(const double* x, const double* y, int n, double Rh, double lo2, double hi2, int ncell_cap,
                       Grid* g, int* cell_key, int* cell_rank, int* cell_count, int* cell_start, double2* sorted_xy,
                       float2* sorted_loc, int* sorted_idx, unsigned long long* bbox_tmp, int* scan_tmp,
                       cudaStream_t s);
// Same with the count read from device memory (*n_dev <= n_bound); the
// cell grid is then binned with the geometry already in g (grid_bin_dev).
cudaError_t grid_build_dev(const double* x, const double* y, int n_bound, const int* n_dev, double Rh, double lo2,
                           double hi2, int ncell_cap, Grid* g, int* cell_key, int* cell_rank, int* cell_count,
                           int* cell_start, double2* sorted_xy, float2* sorted_loc, int* sorted_idx,
                           unsigned long long* bbox_tmp, int* scan_tmp, cudaStream_t s, int* cell_ts = nullptr,
                           bool bbox_ready = false, bool bbox_done = false);
// Sets the bounding-box accumulators to their initial values (every grid
// build leaves them so; a build with bbox_ready = true relies on it).  A
// build with bbox_done = true finds the box of its particles already
// accumulated (reduce_select_dev with x, y and bbox) and skips k_bbox.
cudaError_t grid_bbox_reset(unsigned long long* bbox_tmp, cudaStream_t s);
// cell_ts (optional, ncell_cap / kScanTile + 2 ints): the binning kernel
// accumulates the tile sums of the cell counts there, and the scan of the
// counts is one launch.
cudaError_t grid_bin_dev(const double* x, const double* y, int n_bound, const int* n_dev, int ncell_cap, const Grid* g,
                         int* cell_key, int* cell_rank, int* cell_count, int* cell_start, double2* sorted_xy,
                         float2* sorted_loc, int* sorted_idx, int* scan_tmp, cudaStream_t s, int* cell_ts = nullptr);
// Grid g, built over [0, *n0_dev), extended to [0, *n1_dev) with the same
// geometry: the new particles are binned onto the existing counts (points
// outside the grid clamp into its edge cells; cells are >= R h, so the 3 x 3
// scans stay complete), then the counts are scanned and every particle is
// scattered again.  cell_count must still hold the counts of [0, *n0_dev).
cudaError_t grid_extend_dev(const double* x, const double* y, int n_bound, const int* n0_dev, const int* n1_dev,
                            int ncell_cap, const Grid* g, int* cell_key, int* cell_rank, int* cell_count,
                            int* cell_start, double2* sorted_xy, float2* sorted_loc, int* sorted_idx, int* scan_tmp,
                            cudaStream_t s, int* cell_ts = nullptr);
// Scans work on tiles of kScanTile elements.  A kernel that produces the
// input can accumulate the tiles' sums itself (tile_sum_add); the scan then
// skips its first pass (scan_presummed_*).
constexpr int kScanTileLog = 10;
constexpr int kScanTile = 1 << kScanTileLog;
// tsum[idx >> kScanTileLog] += v with one atomic per distinct tile of the
// warp.  Every lane of the warp must call it; a lane without a value passes
// idx < 0 or v = 0.
__device__ __forceinline__ void tile_sum_add(int* tsum, long idx, int v) {
  const int tile = (idx >= 0 && v != 0) ? (int)(idx >> kScanTileLog) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, tile);
  const int sum = __reduce_add_sync(peers, v);
  if (tile >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&tsum[tile], sum);
}
// Exclusive scan of *n_dev (<= n_bound) ints or bytes whose tile sums are
// already in tile_sums (ceil(n / kScanTile) of them): out[0..n], out[n] =
// total (also written to total_out when given).  One launch.
cudaError_t scan_presummed_i32_dev(const int* in, int* out, int n_bound, const int* n_dev, const int* tile_sums,
                                   cudaStream_t s, int* total_out = nullptr);
cudaError_t scan_presummed_u8_dev(const uint8_t* in, int* out, int n_bound, const int* n_dev, const int* tile_sums,
                                  cudaStream_t s);
// Exclusive scan of n ints into out[0..n] (out[n] = total).
cudaError_t scan_exclusive_i32(const int* in, int* out, int n, int* tmp, cudaStream_t s);
// Scans and compaction with the count in device memory (*n_dev <= n_bound).
// total_out (optional, device): receives the total, as out[n] does.
cudaError_t scan_exclusive_i32_dev(const int* in, int* out, int n_bound, const int* n_dev, int* tmp, cudaStream_t s,
                                   int* total_out = nullptr);
cudaError_t scan_exclusive_u8_dev(const uint8_t* in, int* out, int n_bound, const int* n_dev, int* tmp,
                                  cudaStream_t s);
// flag_ts (optional): the flags' tile sums, already accumulated by their
// producer (the scan is then one launch).
cudaError_t compact_flags_dev(const uint8_t* flags, int n_bound, const int* n_dev, int* list, int* count, int* pos,
                              int* tmp, cudaStream_t s, const int* flag_ts = nullptr);
// Exclusive scan of n bytes (0/1) into out[0..n].
cudaError_t scan_exclusive_u8(const uint8_t* in, int* out, int n, int* tmp, cudaStream_t s);
// list[k] = the k-th index with flag set (ascending); count written to *count
// (device).  pos is scratch of n+1 ints.
cudaError_t compact_flags(const uint8_t* flags, int n, int* list, int* count, int* pos, int* tmp, cudaStream_t s);
size_t scan_tmp_ints(int n);

// vrm_reduce.cu
// Growth control over *n_dev (<= n_bound) particles: diffused[i] for i < n,
// 0 on [n, n_bound).  dflag_ts and tie_ts (n_bound / kScanTile + 2 ints
// each) receive the tile sums of diffused and of the tie flags.
// With x, y and bbox given, the first pass over Gamma also accumulates the
// bounding box of the same particles into bbox, as k_bbox does (for a grid
// build with bbox_done = true).
cudaError_t reduce_select_dev(const double* gamma, int n_bound, const int* n_dev, double c_bound, uint8_t* diffused,
                              ReduceState* st, uint8_t* tie_flag, int* tie_rank, int* scan_tmp, DevStats* ds,
                              cudaStream_t s, int* dflag_ts, int* tie_ts, const double* x = nullptr,
                              const double* y = nullptr, unsigned long long* bbox = nullptr);

// vrm_search.cu
cudaError_t search_all(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                       const float2* sorted_loc, const int* sorted_idx, int n, int* nbr_count, int* nbr_idx,
                       uint8_t* seg_mask, int* small, DevStats* ds, cudaStream_t s);
cudaError_t search_all_dev(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                           const float2* sorted_loc, const int* sorted_idx, int n_bound, const int* n_dev,
                           int* nbr_count, int* nbr_idx, uint8_t* seg_mask, int* small, DevStats* ds,
                           cudaStream_t s, bool sorted = true);
// Rows, masks and small neighbourhoods of the listed particles only (rows in
// visiting order, padded to whole 32-byte sectors); rows = false leaves the
// rows unwritten (counts, masks and small neighbourhoods still are).
cudaError_t search_list_dev(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                            const float2* sorted_loc, const int* sorted_idx, const int* cell_key,
                            const int* cell_rank, const int* list, const int* list_count, int m_bound,
                            int* nbr_count, int* nbr_idx, uint8_t* seg_mask, int* small, DevStats* ds,
                            cudaStream_t s, bool rows = true);
cudaError_t search_masks_list_dev(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                                  const float2* sorted_loc, const int* sorted_idx, const int* cell_key,
                                  const int* cell_rank, const int* list, const int* list_count, int m_bound,
                                  uint8_t* mask, cudaStream_t s);
// Segment masks of the particles flagged in `flag` (n entries), in cell order.

// vrm_insert.cu
// Cell grid of the insertion proposals of one round.
struct CandGrid {
  Grid* grid;
  int *cell_key, *cell_rank, *cell_count, *cell_start, *sorted_idx;
  double2* sorted_xy;
  float2* sorted_loc;
  unsigned long long* bbox;
};
// Open list of round 1: the diffused particles (dlist, ascending) whose
// segment mask is not full; open[] ascending, *n_open on the device.
cudaError_t open_list(const int* dlist, const int* dcount, int cap, const uint8_t* mask, uint8_t* flag, int* pos,
                      int* open, int* n_open, int* flag_ts, cudaStream_t s);

// Buffers of the device-resident insertion rounds (proposal capacity 8 n).
struct RoundBufs {
  int* open;           // open list (cap)
  int* act0;           // open-list positions still open in the round, unordered (cap):
  int* act1;           // act0 for even rounds, act1 for odd ones
  int *cnt, *cpos;     // proposals per open particle and their offsets (cap, cap+1)
  int* cnt_ts;         // tile sums of cnt (kept up to date by the round kernels)
  int* cell_ts;        // tile sums of the proposal cell counts (0 between rounds)
  int* keep_ts;        // tile sums of keep (0 before each conflict test)
  uint8_t *keep_flag;  // open particle still open (cap)
  double *cx, *cy;     // proposals (8 cap)
  uint8_t* keep;       // proposal accepted (8 cap)
  uint8_t* keep_s;     // the same flags by position in the proposal grid's cell order (8 cap)
  int* apos;           // offsets of accepted proposals (8 cap + 1)
  int ncell_cap;       // cells of the proposal grid
  CandGrid cg;         // proposal cell grid (geometry copied from the particle grid)
  int* scan_tmp;       // scan workspace for 8 cap entries
};
// The particle grid's per-particle cell keys and ranks and its sorted
// cell-local coordinates (an open particle's cell and local position come
// from there instead of FP64 arithmetic on its coordinates).
struct PartCells {
  const int* cell_key;
  const int* cell_rank;
  const int* cell_start;
  const float2* sorted_loc;
};
// Round state initialisation after the open list exists (rb.open, *n_open_src
// entries): the counts of the first round's proposals (rb.cnt); sets the
// loop condition (handle may be 0 when not capturing).  rb.cg.cell_count
// must be all 0 (it is after allocation and after every round).
cudaError_t rounds_init(StepState* st, const int* n_open_src, const RoundBufs& rb, const uint8_t* mask, int cap,
                        cudaGraphConditionalHandle handle, bool graph, cudaStream_t s);
// One insertion round on device-resident counts; a no-op once the state has
// no open particle.  The last kernel updates the state and, in a graph, sets
// the while-loop condition.
cudaError_t round_body(const Consts& c, StepState* st, const Grid* pgrid, const PartCells& pcells, const RoundBufs& rb,
                       int cap, uint8_t* mask, double* x, double* y, cudaGraphConditionalHandle handle, bool graph,
                       cudaStream_t s);
cudaError_t rounds_finish(StepState* st, const RoundBufs& rb, int cap, cudaStream_t s);

// vrm_lp.cu
// nu_dt = nu * dt for the stability statistic; with dt_dev it is nu * *dt_dev.
cudaError_t lp_small(const Consts& c, const double* x, const double* y, const int* list, const int* list_count,
                     int cap, const int* small, int* cols, double* f, double* fii, uint8_t* status, int* fail_list,
                     int* retry_list,
                     DevStats* ds, double nu_dt, cudaStream_t s, const double* dt_dev = nullptr, double nu = 0.0);
cudaError_t lp_full(const Consts& c, const double* x, const double* y, const int* fail_list, const int* fail_count,
                    int cap, const int* nbr_count, const int* nbr_idx, int* cols, double* f, double* fii,
                    uint8_t* status, DevStats* ds, double nu_dt, cudaStream_t s, const double* dt_dev = nullptr,
                    double nu = 0.0);
// Identity weights of the removal candidates (list, *list_count on the
// device): removed[i], cols4/w4 [n x 4] (vrm_remove.cu drives it).
cudaError_t lp_identity(const Consts& c, const double* x, const double* y, const int* list, const int* list_count,
                        int cap, const int* nbr_count, const int* nbr_idx, const uint8_t* close, uint8_t* removed,
                        int* cols4, double* w4, cudaStream_t s);
cudaError_t lp_clear(int n, int w, const uint8_t* diffused, int* cols, double* f, double* fii, uint8_t* status,
                     cudaStream_t s);

// vrm_apply.cu
cudaError_t apply_gather(const Consts& c, int n, int n_gamma, const double* gamma, const uint8_t* diffused,
                         const int* nbr_count, const int* nbr_idx, const int* cols, const double* f, const double* fii,
                         const int* order, double* dgamma, double* gamma_out, double dt, cudaStream_t s);
// The step's application: the stencils of the listed (diffused) particles
// transposed into a CSR by target (tcount[n_bound], all 0 on entry and left
// so; toff[n_bound + 1]; tent n_bound x w records of 16 bytes), then the same
// sums as apply_gather.
cudaError_t apply_transposed_dev(const Consts& c, int n_bound, const int* n_dev, int n_gamma, const int* n_gamma_dev,
                                 const double* gamma, const uint8_t* diffused, const int* list, const int* list_count,
                                 const int* cols, const double* f, const double* fii, int* tcount, int* toff,
                                 void* tent, int* scan_tmp, DevStats* ds, double* dgamma, double* gamma_out, double dt,
                                 const double* dt_dev, cudaStream_t s);
cudaError_t apply_gather_dev(const Consts& c, int n_bound, const int* n_dev, int n_gamma, const int* n_gamma_dev,
                             const double* gamma, const uint8_t* diffused, const int* nbr_count, const int* nbr_idx,
                             const int* cols, const double* f, const double* fii, const int* order, double* dgamma,
                             double* gamma_out, double dt, const double* dt_dev, cudaStream_t s);

// vrm_remove.cu: particle removal (candidates, gather, compaction).
cudaError_t remove_close_flags(const Consts& c, const Grid* g, const int* cell_start, const double2* sorted_xy,
                               const float2* sorted_loc, const int* sorted_idx, int n, const double* gamma,
                               uint8_t* close, cudaStream_t s);
cudaError_t remove_gather(const Consts& c, int n, const double* gamma, const uint8_t* removed, const int* nbr_count,
                          const int* nbr_idx, const int* cols4, const double* w4, double* gnew, uint8_t* keep,
                          DevStats* ds, cudaStream_t s);
cudaError_t remove_out(int n, const int* n_keep, const int* klist, const double* x, const double* y,
                       const double* gnew, double* x_out, double* y_out, double* g_out, cudaStream_t s);

// vrm_rk3.cu
// One stage update of the SSP-RK3 step (positions by the velocity, circulations
// by the stage's dGamma), for n particles (*n_dev if given).
// us, vs: precomputed stage velocities (or null: the analytic field of vel).
cudaError_t rk3_stage(int stage, int n_bound, const int* n_dev, double dt, double t_s, const Velocity& vel,
                      const double* X0, const double* Y0, const double* G0, int n_g0, const double* Xs,
                      const double* Ys, const double* Gs, const double* dg, const double* us, const double* vs,
                      double* Xo, double* Yo, double* Go, cudaStream_t s);

// vrm_bs.cu: smoothed Biot-Savart velocity by direct summation.
// Splits FP64 positions into fp32 hi/lo pairs (and circulations to fp32).
cudaError_t bs_split(const double* x, const double* y, const double* g, int n_bound, const int* n_dev, float4* pos,
                     float* gf, cudaStream_t s);
// u, v at the m targets from the n sources (counts on the device if given).
cudaError_t bs_direct(const float4* src, const float* gs, int n_bound, const int* n_dev, const float4* tgt,
                      int m_bound, const int* m_dev, double eps, double* u, double* v, cudaStream_t s);

}  // namespace vrm
