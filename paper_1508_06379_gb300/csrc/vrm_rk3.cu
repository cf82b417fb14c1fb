// Stage update of the SSP-RK3 (Shu-Osher) step with an analytic velocity
// (the viscous Lamb-Oseen run of Sec. 5 with advection): positions follow
// dx/dt = u(x, t), circulations dGamma/dt = L(x) Gamma with the operator of
// the current stage.
//
//   stage 0: X1 = X0 + dt u(X0, t),            G1 = G0 + dt dG(X0)
//   stage 1: X2 = 3/4 X0 + 1/4 (X1 + dt u(X1, t + dt)),    G2 likewise
//   stage 2: X3 = 1/3 X0 + 2/3 (X2 + dt u(X2, t + dt/2)),  G3 likewise
//
// Products and sums are rounded separately; without a velocity the positions
// stay those of the step's start.  With the particles' own velocity (direct
// sum, vrm_bs.cu) the stage velocities come precomputed.  The Lamb-Oseen velocity is
// (u, v) = (-(y - y0), x - x0) k, k = Gamma / (2 pi r^2) (1 - exp(-r^2/(4 nu t))),
// k = 0 at r = 0, with 1 - exp(-a) by a fixed sequence of separately rounded
// operations (so that every platform gets the same bits): the series
// a (1 - a/2 (1 - a/3 (... (1 - a/16)))) for a <= 1/4, otherwise Cody and
// Waite's range reduction exp(-a) = 2^-k exp(-r), k = floor(a / ln 2 + 1/2),
// r = (a - k ln2_hi) - k ln2_lo, exp(-r) by its Taylor series to degree 18
// (Horner), and 1 - that; 1 for a > 700.
#include "vrm_internal.cuh"

namespace vrm {

namespace {
__device__ constexpr double kInvK[19] = {0.0,        1.0 / 1,  1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,
                                         1.0 / 7,    1.0 / 8,  1.0 / 9,  1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13,
                                         1.0 / 14,   1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18};
constexpr double kLn2Hi = 6.93147180369123816490e-01;
constexpr double kLn2Lo = 1.90821492927058770002e-10;
constexpr double kInvLn2 = 1.44269504088896338700e+00;
}  // namespace

__device__ __forceinline__ double one_minus_exp_neg(double a) {
  if (a <= 0.25) {
    double p = 1.0;
#pragma unroll
    for (int k = 16; k >= 2; --k) p = __dsub_rn(1.0, __dmul_rn(__dmul_rn(a, kInvK[k]), p));
    return __dmul_rn(a, p);
  }
  if (a > 700.0) return 1.0;
  const double kk = floor(__dadd_rn(__dmul_rn(a, kInvLn2), 0.5));
  const double r = __dsub_rn(__dsub_rn(a, __dmul_rn(kk, kLn2Hi)), __dmul_rn(kk, kLn2Lo));
  const double mr = -r;
  double q = 1.0;
#pragma unroll
  for (int k = 18; k >= 1; --k) q = __dadd_rn(1.0, __dmul_rn(__dmul_rn(mr, kInvK[k]), q));
  return __dsub_rn(1.0, ldexp(q, -(int)kk));
}

__device__ __forceinline__ void lamb_oseen_uv(const Velocity& v, double x, double y, double t, double* u,
                                              double* w) {
  const double dx = __dsub_rn(x, v.x0), dy = __dsub_rn(y, v.y0);
  const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  double k = 0.0;
  if (r2 > 0.0) {
    const double a = __ddiv_rn(r2, __dmul_rn(__dmul_rn(4.0, v.nu), t));
    k = __dmul_rn(__ddiv_rn(v.gamma, __dmul_rn(2.0 * 3.141592653589793, r2)), one_minus_exp_neg(a));
  }
  *u = __dmul_rn(-dy, k);
  *w = __dmul_rn(dx, k);
}

__global__ void k_rk3_stage(int stage, int n_bound, const int* __restrict__ n_dev, double dt, double t_s, Velocity vel,
                            const double* X0, const double* Y0, const double* __restrict__ G0, int n_g0,
                            const double* Xs, const double* Ys, const double* Gs, const double* __restrict__ dg,
                            const double* __restrict__ us, const double* __restrict__ vs, double* Xo, double* Yo,
                            double* Go) {
  const int n = n_dev ? *n_dev : n_bound;
  const double third = 1.0 / 3.0, two_thirds = 2.0 / 3.0;
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
    const double g0 = j < n_g0 ? G0[j] : 0.0;
    const double gs = stage == 0 ? g0 : Gs[j];
    const double ge = __dadd_rn(gs, __dmul_rn(dt, dg[j]));
    double xe = 0.0, ye = 0.0;
    const bool move = vel.kind != VRM_VEL_NONE;
    if (move) {
      double u, w;
      if (us) {
        u = us[j];
        w = vs[j];
      } else {
        lamb_oseen_uv(vel, Xs[j], Ys[j], t_s, &u, &w);
      }
      xe = __dadd_rn(Xs[j], __dmul_rn(dt, u));
      ye = __dadd_rn(Ys[j], __dmul_rn(dt, w));
    }
    if (stage == 0) {
      Go[j] = ge;
      if (move) {
        Xo[j] = xe;
        Yo[j] = ye;
      }
    } else {
      const double a = stage == 1 ? 0.75 : third, b = stage == 1 ? 0.25 : two_thirds;
      const double x0 = X0[j], y0 = Y0[j];
      Go[j] = __dadd_rn(__dmul_rn(a, g0), __dmul_rn(b, ge));
      if (move) {
        Xo[j] = __dadd_rn(__dmul_rn(a, x0), __dmul_rn(b, xe));
        Yo[j] = __dadd_rn(__dmul_rn(a, y0), __dmul_rn(b, ye));
      }
    }
  }
}

cudaError_t rk3_stage(int stage, int n_bound, const int* n_dev, double dt, double t_s, const Velocity& vel,
                      const double* X0, const double* Y0, const double* G0, int n_g0, const double* Xs,
                      const double* Ys, const double* Gs, const double* dg, const double* us, const double* vs,
                      double* Xo, double* Yo, double* Go, cudaStream_t s) {
  if (n_bound <= 0) return cudaSuccess;
  int blocks = (n_bound + kBlock - 1) / kBlock;
  if (blocks > 8 * sm_count()) blocks = 8 * sm_count();
  k_rk3_stage<<<blocks, kBlock, 0, s>>>(stage, n_bound, n_dev, dt, t_s, vel, X0, Y0, G0, n_g0, Xs, Ys, Gs, dg, us, vs,
                                        Xo, Yo, Go);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
