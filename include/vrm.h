/*
 * vrm.h: C ABI of the GB300 (sm_103a) implementation of the diffusion
 * operator of the splitting-free vorticity redistribution method (VRM),
 * M. Kirchhart and S. Obi, arXiv 1508.06379.
 *
 * A 2-D vortex-particle cloud carries circulations Gamma_i at positions x_i
 * (Sec. 1, Eq. vfield).  The operator approximates nu * Laplacian of the
 * vorticity by redistribution weights f_ij (Sec. 2):
 *     dGamma_j/dt = nu sum_i f_ij Gamma_i                  (Eq. nsode)
 * with f_ij >= 0 for j != i, f_ii = -sum_{j != i} f_ij (Eq. fii), chosen per
 * particle so that the moment conditions V_i f_i = b hold (Eq. momcondmv).
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers owned by the caller, unless a
 *     comment says "host".  The library never frees or keeps them.
 *   - Positions are FP64, structure of arrays: x[i], y[i].
 *   - Indices are int32 (particle counts below 2^31).
 *   - Neighbour rows are "ELL" rows of width k_cap: row i occupies
 *     nbr_idx[i*k_cap .. i*k_cap + min(nbr_count[i], k_cap)), ascending
 *     global indices; entries past the count are not written.
 *   - Stencils have width W = vrm_stencil_width(order) (VRM_STENCIL_W = 8
 *     for n = 1, VRM_STENCIL_W2 = 12 for n = 2): stencil i occupies
 *     cols[i*W .. i*W+W), f[i*W .. i*W+W): the nonzero h-scaled weights
 *     f~_ij = h^2 f_ij in the LP's column order, padded with -1 / 0.0;
 *     fii[i] = f~_ii.
 *   - small (n*8 int32) and cols (n*W int32) must start on a 16-byte
 *     boundary (their rows are read as 16-byte vectors); a misaligned
 *     pointer gives VRM_ERR_ARG.
 *   - Every call is asynchronous on the given stream, except that a call
 *     which returns a size or statistics to a host pointer synchronises the
 *     stream before it returns.
 *   - Every call returns a vrm_status; no call aborts or throws.  On
 *     VRM_ERR_CUDA the stream's work may be incomplete; on any error the
 *     output arrays are unspecified.
 *   - Derived constants are computed once in vrm_create, in FP64, as
 *       lo2 = (r h)^2, hi2 = (R h)^2         annulus bounds (Eq. neighbourhood)
 *       c_bound = C_diff * ((h*h)*h)         growth-control bound h^{n+2} (Eq. reduced_bound), n = 1
 *       c_bound = C_diff * (((h*h)*h)*h)                                                      n = 2
 *       nu_over_h2 = nu / (h*h)
 *       inv_h = 1 / h
 *     so that a caller can reproduce every decision bit for bit.
 */
#ifndef VRM_H
#define VRM_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef int vrm_status;
#define VRM_OK 0
#define VRM_ERR_ARG 1        /* bad parameter, null pointer, NaN/Inf input */
#define VRM_ERR_CAPACITY 2   /* an output or scratch capacity is too small */
#define VRM_ERR_CUDA 3       /* a CUDA runtime call failed */
#define VRM_ERR_UNSUPPORTED 4 /* a parameter value this build does not support */

/* Stencil width: columns kept per particle.  A basic solution of the m-row
   LP has at most m nonzero weights: m = 5 for n = 1 (the small neighbourhood's
   8 columns fit), m = 9 for n = 2 (Eq. momcondmv). */
#define VRM_STENCIL_W 8   /* n = 1 */
#define VRM_STENCIL_W2 12 /* n = 2 */
/* Largest neighbour-row width (k_cap) the library accepts. */
#define VRM_KCAP_MAX 32

/* Per-particle LP outcome codes (status arrays). */
#define VRM_LP_NOT_DIFFUSED 0
#define VRM_LP_SMALL 1   /* solved on the small neighbourhood (Sec. 4.3) */
#define VRM_LP_FULL 2    /* solved on the full neighbourhood after a retry */
#define VRM_LP_NONE 3    /* no non-negative stencil found: zero stencil */
#define VRM_LP_LEARNED 4 /* the network's proposal, corrected and accepted (vrm_set_mlp) */

/* Precision of the step.  The neighbourhoods are always those of the FP64
   definition (FP32 measures with an exact fallback), the LP and the
   corrections always FP64. */
#define VRM_PREC_FP64 0  /* FP64 application: bit-identical to the FP64 oracle */
#define VRM_PREC_MIXED 1 /* the application (Eq. nsode) accumulates fp32 products
                            of fp32-rounded weights and circulations; dGamma is
                            within 1e-5 (nu/h^2) sum_i |f~_ij Gamma_i| of the FP64
                            value; the Euler update stays FP64 */

/* ---- parameters ---------------------------------------------------------- */
typedef struct vrm_params {
  double h;          /* mean particle spacing (length units) */
  double r;          /* inner annulus radius in units of h (paper: 1/2) */
  double R;          /* outer annulus radius in units of h (paper: 2) */
  double nu;         /* kinematic viscosity */
  double c_diff;     /* growth-control constant C_diff (Eq. reduced_bound) */
  int32_t order;     /* consistency order n: 1 (m = 5 moment rows) or 2 (m = 9, cubic
                        moments added; Eqs. cond_two, cond_alpha) */
  int32_t k_cap;     /* neighbour-row width, 8 <= k_cap <= VRM_KCAP_MAX */
  int32_t max_rounds;/* insertion rounds per step (Sec. 4.2), >= 0 */
  int32_t fallback;  /* 1: retry failed small neighbourhoods on the full one (Sec. 4.3) */
  int32_t precision; /* VRM_PREC_FP64 or VRM_PREC_MIXED */
  int32_t reserved;
} vrm_params;

/* Counters of one call.  Filled only when a stats pointer is given (host). */
typedef struct vrm_stats {
  int64_t n_in;          /* particles given */
  int64_t n_out;         /* particles after insertion */
  int64_t n_diffused;    /* |D|: particles that diffuse (Sec. 3.5) */
  int64_t n_inserted;    /* zero-strength particles appended (Sec. 4.2) */
  int64_t open_segments; /* empty segments of diffused particles left after max_rounds */
  int64_t small_ok;      /* stencils from the small neighbourhood */
  int64_t full_ok;       /* stencils from the full-neighbourhood retry */
  int64_t no_stencil;    /* diffused particles left with a zero stencil */
  int32_t rounds;        /* insertion rounds that appended particles */
  int32_t max_pivots;    /* largest pivot count of one LP */
  int32_t max_count;     /* largest neighbour count (> k_cap means rows were cut) */
  int32_t reserved;
  double max_dt_ratio;   /* max over diffused i of nu*dt*(-f~_ii)/h^2; > 1 breaks
                            the a-posteriori stability bound (Thm. stability) */
  int64_t lp_small_solved; /* LPs run on small neighbourhoods (= |D|) */
  int64_t lp_small_pivots; /* pivots summed over those LPs */
  int64_t lp_full_solved;  /* LPs run on full neighbourhoods */
  int64_t lp_full_pivots;  /* pivots summed over those LPs */
  int64_t learned_ok;      /* stencils from the learned proposal (vrm_set_mlp) */
  int64_t learned_rejected; /* proposals rejected (then solved by the LP) */
  int64_t learned_square;  /* of learned_ok: accepted on the first support tried (the network's top five) */
  int64_t lp_full_columns;       /* columns summed over the full-neighbourhood LPs */
  int64_t lp_full_column_pivots; /* columns x pivots summed over them (their algorithmic work) */
  int64_t learned_screens; /* five-slot supports screened by the learned path (binary32 solves) */
  int64_t remove_candidates; /* vrm_remove_close: particles closer than r h to one of larger key */
  int64_t lp_small_rechecked; /* of lp_small_solved: LPs whose binary32 pivot decisions were not all
                                 certain and that were re-run with FP64 pivots (same result either way) */
} vrm_stats;

/* Stages of vrm_step, for vrm_stage_times. */
#define VRM_STAGE_REDUCE 0   /* growth control, diffused list */
#define VRM_STAGE_GRID 1     /* cell grid of the given cloud, segment masks */
#define VRM_STAGE_INSERT 2   /* insertion rounds */
#define VRM_STAGE_SEARCH 3   /* cell grid of the final cloud, neighbourhoods */
#define VRM_STAGE_LP_SMALL 4 /* LP on small neighbourhoods */
#define VRM_STAGE_LP_FULL 5  /* LP retry on full neighbourhoods */
#define VRM_STAGE_APPLY 6    /* application and Euler update */
#define VRM_STAGE_COUNT 7

typedef struct vrm_ctx vrm_ctx;

/* Paper defaults: r = 1/2, R = 2, n = 1, C_diff = 1 (Sec. 4.2, 6), k_cap = 32,
   8 insertion rounds, fallback on, FP64; h and nu set to 1. */
void vrm_default_params(vrm_params* p);

/* Stencil width W of consistency order n (8 for n = 1, 12 for n = 2, -1
   otherwise): the row length of cols and f in every call below. */
int32_t vrm_stencil_width(int32_t order);

/* Text of a status code (static storage). */
const char* vrm_status_string(vrm_status s);

/* Create a context on the current CUDA device.  Checks the parameters
   (VRM_ERR_ARG / VRM_ERR_UNSUPPORTED) and computes the derived constants.
   The context owns its scratch memory, grown on demand by the calls below;
   one context must not be used by two streams at once. */
vrm_status vrm_create(const vrm_params* p, vrm_ctx** out);
void vrm_destroy(vrm_ctx* ctx);

/*
 * Growth control and insertion (Sec. 3.5 and Sec. 4.2).
 *   1. D = the particles that diffuse: the complement of the longest prefix I
 *      of the particles sorted by (|Gamma_i|, i) with
 *      sum_I |Gamma_i| <= C_diff h^{n+2} ||Gamma||_1 (Eq. reduced_bound),
 *      the sums taken exactly on |Gamma_i| 2^(96-E) truncated to integers.
 *   2. Insertion rounds: every i in D whose annulus r h <= |x_j - x_i| <= R h
 *      leaves a 45-degree segment s empty proposes x_i + 1.5 h (cos, sin)
 *      ((s + 1/2) pi/4); a proposal is dropped if a proposal of smaller key
 *      (i, s) lies closer than r h; the rest are appended in key order.
 *      Rounds repeat until none is proposed, at most max_rounds times.
 * x, y:      capacity entries; [0, n) given, appended points written at [n, n').
 * gamma:     n circulations (read only).
 * diffused:  capacity bytes out: 1 for i in D, 0 otherwise (also 0 on [n, n')).
 * n_out:     host; receives n'.  Synchronises the stream.
 * Errors: VRM_ERR_ARG on null pointers, n < 0, n > capacity or non-finite
 * input; VRM_ERR_CAPACITY when n' would exceed capacity (stats->n_out, if
 * given, then holds the count after the first round that did not fit: a
 * lower bound of the capacity needed, since later rounds were not run).
 */
vrm_status vrm_insert_reduce(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma,
                             uint8_t* diffused, int32_t* n_out, vrm_stats* stats, cudaStream_t stream);

/*
 * Neighbourhoods (Eq. neighbourhood), segment masks and small neighbourhoods
 * (Sec. 4.2, 4.3) of n particles, by a cell-list search.
 * nbr_count: n out, |N_i \ {i}| (the true count, also above k_cap).
 * nbr_idx:   n*k_cap out, ELL rows (see top); rows above k_cap keep their
 *            k_cap smallest indices.
 * seg_mask:  n out, bit s set iff segment s of the annulus holds a particle;
 *            segment s is the half-open angle [s pi/4, (s+1) pi/4) of r_ij.
 * small:     n*8 out, small[i*8+s] = the particle of segment s with the
 *            smallest distance (ties: smaller index), -1 if empty.
 * max_count: host, optional (may be NULL); receives max_i nbr_count[i] and
 *            synchronises.  Without it the call is fully asynchronous.
 * Errors: VRM_ERR_ARG; VRM_ERR_CAPACITY if max_count is requested and some
 * row exceeds k_cap (the outputs are still written, cut as described).
 */
vrm_status vrm_build_neighbourhoods(vrm_ctx* ctx, const double* x, const double* y, int32_t n, int32_t* nbr_count,
                                    int32_t* nbr_idx, uint8_t* seg_mask, int32_t* small, int32_t* max_count,
                                    cudaStream_t stream);

/*
 * Redistribution weights (Sec. 2 Eq. momcondmv, Sec. 4.1, 4.3) of every
 * particle with diffused[i] = 1: the phase-I simplex on the small
 * neighbourhood (columns ordered by (|r_ij|^2, j)), rows
 * (1,0) (0,1) (2,0) (1,1) (0,2) in xi = r_ij / h with b = (0,0,2,0,2), for
 * n = 2 followed by (3,0) (2,1) (1,2) (0,3) with b = 0, each monomial a
 * product of separately rounded factors ((xi xi) xi, (xi xi) eta,
 * xi (eta eta), (eta eta) eta);
 * artificials start the basis; entering column = lowest index with reduced
 * cost < -1e-9; leaving row = minimum ratio over pivots > 1e-9 (basic values
 * <= 1e-11 count as zero), ties within 1e-12 max(1, ratio) to the lowest
 * basic variable (artificials first); at
 * most 64 pivots; feasible iff phase-I objective <= 1e-10 and
 * max |V f~ - b| <= 1e-10; basic values <= 1e-11 are zeros.  If infeasible
 * and fallback is on, the same LP on the full row (its k_cap first entries,
 * ordered by (|r_ij|^2, j)); if that fails too the stencil is zero.
 * f~_ii = -sum_j f~_ij in column order.
 * Inputs are the outputs of vrm_build_neighbourhoods on the same x, y, n.
 * cols, f:  n*W out (W = vrm_stencil_width(order)); fii: n out; status: n
 *           out (VRM_LP_*).
 * stats:    host, optional; fills small_ok, full_ok, no_stencil, max_pivots,
 *           n_diffused and synchronises.
 */
vrm_status vrm_solve_weights(vrm_ctx* ctx, const double* x, const double* y, int32_t n, const uint8_t* diffused,
                             const int32_t* nbr_count, const int32_t* nbr_idx, const int32_t* small, int32_t* cols,
                             double* f, double* fii, uint8_t* status, vrm_stats* stats, cudaStream_t stream);

/*
 * Operator application (Eq. nsode, reduced form Eq. reducedop):
 *   dgamma[j] = (nu/h^2) * sum_{i in D} f~_ij Gamma_i
 * for j in [0, n), as a gather over the neighbour rows (the annulus relation
 * is symmetric, so every i with j in its stencil is in row j): terms in
 * ascending i with the self term f~_jj Gamma_j at i = j, products and sums
 * rounded separately, no atomics.  Particles i >= n_gamma carry Gamma = 0.
 * gamma: n_gamma values; diffused, nbr_*, cols, f, fii as produced above.
 */
vrm_status vrm_apply(vrm_ctx* ctx, int32_t n, int32_t n_gamma, const double* gamma, const uint8_t* diffused,
                     const int32_t* nbr_count, const int32_t* nbr_idx, const int32_t* cols, const double* f,
                     const double* fii, double* dgamma, cudaStream_t stream);

/*
 * One forward-Euler step of the heat equation with the VRM operator
 * (Sec. 3.3): growth control, insertion, neighbourhoods, weights, then
 *   gamma_out[j] = fma(dt, dgamma[j], gamma_in[j])   (gamma_in = 0 for j >= n)
 * for j in [0, n').  Scratch lives in the context.
 * x, y:      capacity entries; inserted points appended at [n, n').
 * gamma_in:  n values (read only); gamma_out: capacity entries, must not
 *            overlap gamma_in.  Repeating a call with the same n and
 *            gamma_in gives the same result (x, y beyond n are overwritten
 *            with the same points).
 * n_out:     host; receives n'.  Synchronises the stream.
 * stats:     host, optional.
 * Errors: as vrm_insert_reduce and vrm_build_neighbourhoods; a row above
 * k_cap gives VRM_ERR_CAPACITY (stats->max_count holds the width needed).
 */
vrm_status vrm_step(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma_in,
                    double* gamma_out, double dt, int32_t* n_out, vrm_stats* stats, cudaStream_t stream);

/*
 * vrm_step in two halves, so that a caller can keep the GPU busy with a
 * stream of steps (no runtime counterpart in the paper).  vrm_step_begin
 * enqueues the step on the stream and returns at once (the first step on a
 * new set of buffers, or after the capacity grew, builds the context's
 * scratch and captured step first, and synchronises then); vrm_step_end
 * waits for it and returns n_out and the statistics, repeating the step with
 * whole rows if the schedule's row_cap cut one (as vrm_step does).
 * Arguments as vrm_step.  Between the two calls the context and its buffers
 * belong to the pending step: no other call on the context (VRM_ERR_ARG for
 * a second vrm_step_begin or a vrm_step), and no change of its inputs.  Two
 * contexts let a caller enqueue step k + 1 before waiting for step k.
 */
vrm_status vrm_step_begin(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma_in,
                          double* gamma_out, double dt, cudaStream_t stream);
vrm_status vrm_step_end(vrm_ctx* ctx, int32_t* n_out, vrm_stats* stats);

/*
 * Batched steps: many independent clouds (each with its own spacing h and
 * step dt) advanced by one call.  The clouds' steps are captured once as
 * parallel branches of one CUDA graph (per-cloud insertion loops included)
 * and replayed while the clouds' buffers, capacities and spacings stay the
 * same, so uneven clouds share the GPU.  Every cloud gets exactly the result
 * of vrm_step on it with the batch's parameters and its own h.
 */
typedef struct vrm_cloud {
  double* x;              /* device, capacity entries; inserted points appended */
  double* y;
  const double* gamma_in; /* device, n entries (read only) */
  double* gamma_out;      /* device, capacity entries, not overlapping gamma_in */
  int32_t n;              /* particles given */
  int32_t capacity;
  double h;               /* particle spacing of this cloud */
  double dt;              /* Euler step of this cloud */
  int32_t n_out;          /* out: particles after insertion (on VRM_ERR_CAPACITY: the count after the
                             first round that did not fit, a lower bound of the capacity needed) */
  int32_t status;         /* out: VRM_OK, VRM_ERR_ARG or VRM_ERR_CAPACITY for this cloud */
} vrm_cloud;

typedef struct vrm_batch vrm_batch;

/*
 * Launch schedule of the step's three largest kernels.  No field changes any
 * result (every schedule gives bit-identical output); they trade occupancy,
 * registers and tail effects, and the best choice depends on the cloud's size.
 * An autotuner (paper_1508_06379_gb300.autotune) times the candidates and
 * caches the fastest per size bucket.
 *   row_cap:          neighbour entries the search keeps per row: 16, 24 or
 *                     up to k_cap (32 by default).  A step whose rows need
 *                     more than row_cap but at most k_cap is repeated once
 *                     with row_cap = k_cap, which the context then keeps.
 *   search_block:     threads per block of the neighbourhood search (32..256, multiple of 32).
 *   lp_block:         threads per block of the small-neighbourhood LP, one particle per thread (32..128, multiple of 32);
 *                     192 and 384 select the warp-specialised form of the binary32 LP (4 pivot and 2 FP64 warps
 *                     per block, two blocks per SM; 8 pivot and 4 FP64 warps, one block per SM).
 *   lp_blocks_per_sm: the small LP's grid is capped at this many blocks per SM (1..64).
 *   apply_block:      threads per block of the application (32..256, multiple of 32).
 *   lp_fp64_pivots:   0 (default): the small-neighbourhood LPs (n = 1) pivot
 *                     in binary32 with certified decisions, and the few whose
 *                     decisions are not all certain are re-run with FP64
 *                     pivots; 1: every LP pivots in FP64.  The final basis,
 *                     hence every weight, is the same bit for bit.
 * Setting a schedule drops any captured step graph; VRM_ERR_ARG if a field
 * is out of range.
 */
typedef struct vrm_schedule {
  int32_t row_cap;
  int32_t search_block;
  int32_t lp_block;
  int32_t lp_blocks_per_sm;
  int32_t apply_block;
  int32_t lp_fp64_pivots;
  int32_t reserved[2];
} vrm_schedule;

vrm_status vrm_get_schedule(const vrm_ctx* ctx, vrm_schedule* out);
vrm_status vrm_set_schedule(vrm_ctx* ctx, const vrm_schedule* s);
/* The schedule of cloud slot `slot` of a batch (used from the next vrm_step_batched on). */
vrm_status vrm_batch_set_schedule(vrm_batch* b, int32_t slot, const vrm_schedule* s);

/* A batch for up to max_clouds clouds; p gives every parameter but h. */
vrm_status vrm_batch_create(const vrm_params* p, int32_t max_clouds, vrm_batch** out);
void vrm_batch_destroy(vrm_batch* b);
/* One step of every cloud.  Synchronises the stream.  Returns VRM_OK when
   every cloud succeeded, else the first failing cloud's status (each cloud's
   own status is in clouds[c].status).  stats (host, optional) receives the
   sums over the clouds (maxima for the max_* fields). */
vrm_status vrm_step_batched(vrm_batch* b, vrm_cloud* clouds, int32_t n_clouds, vrm_stats* stats, cudaStream_t stream);

/*
 * The weight-proposal network of the learned path (not in the paper: the
 * paper solves every stencil with the LP of Sec. 4.1).  A proposal is kept
 * only if, after the least-change correction onto the moment conditions
 * (Eqs. momcondmv, cond_two, cond_alpha), every weight is non-negative and
 * the residual is at most 1e-12; otherwise the LP decides, so the network
 * changes speed, never validity.
 *
 * Input rows: 128 bf16 per particle: xi_x of the 32 neighbour slots, xi_y,
 * the slot mask (1/0), then 32 zeros.  Slots hold the annulus neighbours
 * ordered by (45-degree segment, squared distance, index), xi = (x_j - x_i)/h.
 * Output rows: 32 fp32 proposals f~ (Eq. momcondmv scaling f~ = h^2 f).
 * Network 96 -> 256 -> 256 -> 256 -> 32, GELU (tanh form) on the hidden
 * layers; parameters one fp32 vector of VRM_MLP_PARAMS entries in the order
 * W1 (256 x 96, row-major [out][in]), b1, W2 (256 x 256), b2, W3, b3,
 * W4 (32 x 256), b4.  Products run on the tensor cores with bf16 weights and
 * activations and fp32 accumulation.
 *
 * Training: vrm_mlp_train_step gathers rows batch_idx[0..rows) of a data set
 * (X_all bf16 [N x 128], T_all fp32 [N x 32] targets, device), runs the
 * forward and backward passes of the masked mean squared error
 * sum(mask (Y - T)^2) / sum(mask) and one AdamW step (decoupled weight decay)
 * with bias corrections for step t >= 1.  rows <= batch_rows; missing rows
 * are zero and add nothing.  All calls are asynchronous except where noted;
 * a tensor-core wait that gives up (about a second) makes the synchronous
 * calls return VRM_ERR_CUDA.
 */
#define VRM_MLP_PARAMS 164640
#define VRM_MLP_IN 128
#define VRM_MLP_OUT 32
typedef struct vrm_mlp vrm_mlp;
typedef struct vrm_adamw {
  float lr, beta1, beta2, eps, weight_decay;
  int32_t reserved[3];
} vrm_adamw;
/* batch_rows: training batch, a multiple of 128 (<= 2^20).  VRM_ERR_UNSUPPORTED
   when the driver offers no tensor-map encoder. */
vrm_status vrm_mlp_create(int32_t batch_rows, vrm_mlp** out);
void vrm_mlp_destroy(vrm_mlp* net);
/* theta: VRM_MLP_PARAMS floats (host or device); resets the AdamW moments. */
vrm_status vrm_mlp_set_params(vrm_mlp* net, const float* theta, cudaStream_t stream);
vrm_status vrm_mlp_get_params(const vrm_mlp* net, float* theta, cudaStream_t stream);
/* Y[rows x 32] = network(X).  X: device bf16 rows of VRM_MLP_IN, allocated for
   rows rounded up to a multiple of 128, 16-byte aligned.  Synchronises. */
vrm_status vrm_mlp_forward(vrm_mlp* net, const uint16_t* X, int32_t rows, float* Y, cudaStream_t stream);
/* Gradient (VRM_MLP_PARAMS floats) and loss[0..1] = (loss, sum of the mask)
   of rows X, T (device) without an update.  Synchronises. */
vrm_status vrm_mlp_grads(vrm_mlp* net, const uint16_t* X, const float* T, int32_t rows, float* grad, float* loss,
                         cudaStream_t stream);
/* One training step on rows batch_idx (device int32, or NULL for rows 0..rows-1). */
vrm_status vrm_mlp_train_step(vrm_mlp* net, const uint16_t* X_all, const float* T_all, const int32_t* batch_idx,
                              int32_t rows, const vrm_adamw* hp, int32_t t, float* loss, cudaStream_t stream);
/* One AdamW step with a given gradient (device, VRM_MLP_PARAMS floats). */
vrm_status vrm_mlp_adamw(vrm_mlp* net, const float* grad, const vrm_adamw* hp, int32_t t, cudaStream_t stream);
/* VRM_ERR_CUDA if a tensor-core wait of an earlier asynchronous call gave up.  Synchronises. */
vrm_status vrm_mlp_error(vrm_mlp* net, cudaStream_t stream);

/*
 * The learned proposal in the step.  With a network set, vrm_step and
 * vrm_solve_weights first build the input rows of every diffused particle,
 * run the network, correct each proposal onto the moment conditions and
 * accept it under the test above; only the rejected particles run the LP
 * (small neighbourhood, then the full-neighbourhood retry).  The network must
 * outlive its use; its weights may change between steps (training).  NULL
 * restores the LP for every particle.  The network's time counts in the
 * VRM_STAGE_LP_SMALL stage.  The network proposes n = 1 stencils: a context
 * of order 2 gives VRM_ERR_UNSUPPORTED for a non-NULL net.
 */
vrm_status vrm_set_mlp(vrm_ctx* ctx, vrm_mlp* net);

/* Input rows of the listed particles of an n-particle cloud (list: device
 * int32 [m], or NULL for 0..m-1) from their neighbour rows: X bf16 [m rounded
 * up to 128][128] and slots int32 [m][32] (particle index of each slot, -1
 * empty).  Offsets are taken between fp32-rounded positions. */
vrm_status vrm_learned_features(vrm_ctx* ctx, const double* x, const double* y, int32_t n, const int32_t* list,
                                int32_t m, const int32_t* nbr_count, const int32_t* nbr_idx, uint16_t* X,
                                int32_t* slots, cudaStream_t stream);
/* Correction and acceptance of given proposals f0 (device fp32 [m][32]) for
 * the listed particles; the candidates are the slots holding the small
 * neighbourhood (small: device int32 [n][8] as from vrm_build_neighbourhoods,
 * 16-byte aligned): accepted stencils are written as by the LP (status
 * VRM_LP_LEARNED), rejected ones get VRM_LP_NONE and a zero stencil.
 * *n_accepted (host) receives the count.  Synchronises.  n = 1 only
 * (VRM_ERR_UNSUPPORTED for a context of order 2); stencil width 8. */
vrm_status vrm_learned_project(vrm_ctx* ctx, const double* x, const double* y, const int32_t* list, int32_t m,
                               const int32_t* slots, const float* f0, const int32_t* small, int32_t* cols, double* f,
                               double* fii, uint8_t* status, int32_t* n_accepted, cudaStream_t stream);
/* Training targets: T fp32 [m][32], the weight f~ of each listed particle's
 * stencil (cols, f as written by vrm_solve_weights for n = 1, width 8) at
 * each slot's particle. */
vrm_status vrm_learned_targets(const int32_t* list, int32_t m, const int32_t* slots, const int32_t* cols,
                               const double* f, float* T, cudaStream_t stream);

/*
 * One SSP-RK3 (Shu-Osher) step of the viscous particle method: positions
 * move with an analytic velocity, circulations follow the diffusion operator
 * (the heat part of Sec. 3; the velocity of Sec. 5's Lamb-Oseen test case
 * stands in for the Biot-Savart law).  Growth control and insertion run once,
 * on the step's initial cloud; neighbourhoods and weights (LP, or the learned
 * proposal with vrm_set_mlp) are rebuilt at each of the three stages:
 *   X1 = X0 + dt u(X0, t),                        G1 = G0 + dt L(X0) G0
 *   X2 = 3/4 X0 + 1/4 (X1 + dt u(X1, t + dt)),    G2 = 3/4 G0 + 1/4 (G1 + dt L(X1) G1)
 *   X3 = 1/3 X0 + 2/3 (X2 + dt u(X2, t + dt/2)),  G3 = 1/3 G0 + 2/3 (G2 + dt L(X2) G2)
 * products and sums rounded separately.  x, y (capacity entries) receive X3
 * (inserted particles appended), gamma_out receives G3; t is the field time
 * of the state.  Without a velocity (vel NULL or kind VRM_VEL_NONE) the
 * positions stay.  Stats sum over the three stages (n_in, n_out, insertion
 * and growth-control counts are the step's).  Errors as vrm_step.
 */
#define VRM_VEL_NONE 0
#define VRM_VEL_LAMB_OSEEN 1 /* u_theta = gamma/(2 pi r) (1 - exp(-r^2/(4 nu t))) about (x0, y0) */
#define VRM_VEL_BIOT_SAVART 2 /* the particles' own smoothed velocity (vrm_biot_savart, core eps) */
typedef struct vrm_velocity {
  int32_t kind;
  int32_t reserved;
  double gamma, nu, x0, y0;
  double eps;
} vrm_velocity;

/*
 * Smoothed Biot-Savart velocity by direct summation (Sec. 5, Eq.
 * smoothkernel): u_h(x) = sum_j Gamma_j K_eps(x - x_j) with
 * K_eps(x) = (-y, x)/(2 pi |x|^2) (1 - exp(-|x/eps|^2)), K_eps(0) = 0, at the m
 * targets (xt, yt) from the n sources (xs, ys, gamma); all device pointers,
 * u and v receive m values.  Pair terms in fp32 on hi/lo-split positions,
 * tile sums in FP64: relative error about 1e-6 of sum_j |Gamma_j K_eps|.
 * O(n m) work (the fast multipole method of the paper is not part of this
 * library).  Asynchronous.
 */
vrm_status vrm_biot_savart(vrm_ctx* ctx, const double* xs, const double* ys, const double* gamma, int32_t n,
                           const double* xt, const double* yt, int32_t m, double eps, double* u, double* v,
                           cudaStream_t stream);
vrm_status vrm_rk3_step(vrm_ctx* ctx, double* x, double* y, int32_t n, int32_t capacity, const double* gamma_in,
                        double* gamma_out, double t, double dt, const vrm_velocity* vel, int32_t* n_out,
                        vrm_stats* stats, cudaStream_t stream);

/* Per-stage timing of vrm_step with CUDA events recorded on the call's
   stream between the stages.  Off by default; enable != 0 turns it on. */
vrm_status vrm_set_timing(vrm_ctx* ctx, int32_t enable);
/* ms[VRM_STAGE_COUNT] (host) receives the stage durations in milliseconds of
   the last vrm_step made with timing on (0 for stages it skipped).  Waits for
   that step's events. */
vrm_status vrm_stage_times(vrm_ctx* ctx, float* ms);

/* Kernels launched by this library in this process so far (all contexts),
   kernels run by replays of a captured step graph included. */
int64_t vrm_launch_count(void);

/*
 * Peak FMA probe (no paper counterpart: the roofline denominator of the LP
 * kernels, which are bound by FP64 and binary32 arithmetic).  Enqueues one
 * kernel of `blocks` blocks of 256 threads, each thread running 8
 * independent chains of fused multiply-adds for iters x 16 steps, in FP64
 * (fp64 != 0) or FP32.  sink: device buffer of blocks + 1 elements of that
 * type (written, contents meaningless).  *flops = the floating-point
 * operations the launch performs (2 per FMA); the caller times the launch
 * on `stream` (divide *flops by the duration).  VRM_ERR_ARG for
 * non-positive sizes or null pointers.
 */
vrm_status vrm_fma_probe(int32_t fp64, int32_t blocks, int32_t iters, void* sink, double* flops,
                         cudaStream_t stream);

/*
 * Particle removal (the outlook of Sec. 6.2): where particles have come closer
 * than r h to one another (inside the inner bound of Eq. neighbourhood),
 * redistribute one of each such pair to its neighbours by an approximation
 * of the identity operator and remove it.
 *   1. Candidates: i with a particle j != i at dx*dx + dy*dy < (r h)^2 (FP64,
 *      separately rounded) whose key (|Gamma_j|, j) is larger than i's.
 *   2. Weights: on the closest non-candidate particle of every 45-degree
 *      segment of i's annulus (ties to the smaller index; columns ordered by
 *      (|r_ij|^2, j)), the phase-I simplex of vrm_solve_weights with rows
 *      (0,0) (1,0) (0,1) in xi = r_ij / h and b = (1, 0, 0): sum_j g_ij = 1,
 *      sum_j g_ij r_ij = 0, g_ij >= 0 (circulation and its first moments are
 *      kept; non-negative weights cannot also keep the second moments).  A
 *      candidate without such weights is kept.
 *   3. gamma_out of a kept j: Gamma_j + sum_i g_ij Gamma_i over the removed i
 *      in ascending order, products and sums rounded separately.
 *   4. The kept particles are written to x_out, y_out, gamma_out in index
 *      order; *n_out (host) receives their number.  Synchronises.
 * x, y, gamma: n inputs (device, read only); the outputs hold n entries and
 * must not overlap the inputs.  stats (host, optional): n_in, n_out,
 * max_count, remove_candidates.
 * Errors: VRM_ERR_ARG (null pointers, NaN/Inf input); VRM_ERR_CAPACITY if a
 * neighbour row exceeds k_cap (outputs unspecified).
 */
vrm_status vrm_remove_close(vrm_ctx* ctx, const double* x, const double* y, const double* gamma, int32_t n,
                            double* x_out, double* y_out, double* gamma_out, int32_t* n_out, vrm_stats* stats,
                            cudaStream_t stream);

/* Largest cloud vrm_build_neighbourhoods_noalloc accepts. */
#define VRM_NOALLOC_MAX_N 65536

/*
 * The neighbourhood search of vrm_build_neighbourhoods (same outputs, bit for
 * bit) for callers that cannot allocate device memory when they need
 * neighbourhoods: applications that hand all device memory to their own pool
 * at start-up and forbid allocations afterwards (for instance a host program
 * that loads this library as a plug-in and owns every buffer), and real-time
 * loops whose latency budget has no room for cudaMalloc/cudaFree, which can
 * take milliseconds and synchronise the device.  The paper has no
 * counterpart; it is a service of this library.
 *
 * It takes the parameters instead of a context and calls no cudaMalloc,
 * cudaFree or other allocating routine.  Its scratch is one fixed device
 * array of about 3.4 MB inside this library, which every GPU that loads the
 * library holds until the process exits; it serves clouds of at most
 * VRM_NOALLOC_MAX_N particles and returns VRM_ERR_CAPACITY above that.
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress, once per device, with that device current).  Every
 * call shares the array
 * and overwrites what the previous call left there (the counters it needs
 * at zero are cleared on the stream at the start of each call), so calls
 * whose work overlaps on the GPU (two streams, or two host threads) race:
 * serialise them.  Arguments, outputs and errors are as for
 * vrm_build_neighbourhoods; only r, R, h and k_cap of *p are used.  With
 * max_count non-NULL the call copies two small records to the host and waits
 * for the stream (it also then reports NaN/Inf input and rows wider than
 * k_cap); with max_count NULL it only enqueues work on the stream.
 */
vrm_status vrm_build_neighbourhoods_noalloc(const vrm_params* p, const double* x, const double* y, int32_t n,
                                            int32_t* nbr_count, int32_t* nbr_idx, uint8_t* seg_mask, int32_t* small,
                                            int32_t* max_count, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* VRM_H */
