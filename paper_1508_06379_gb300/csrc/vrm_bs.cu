// Smoothed Biot-Savart velocity by direct summation (Sec. 5, Eq.
// smoothkernel): u_h(x) = sum_j Gamma_j K_eps(x - x_j),
//   K_eps(x) = (-y, x) / (2 pi |x|^2) (1 - exp(-|x/eps|^2)),
// written as K_eps(x) = (-y, x) phi(q) / (2 pi eps^2), q = |x|^2/eps^2,
// phi(q) = (1 - exp(-q))/q (phi(0) = 1, so a particle does not move itself).
//
// GB300 runs FP32 at 62x its FP64 rate, so the pair terms are FP32: every
// position is split into an fp32 pair hi + lo (hi = fp32(x), lo =
// fp32(x - hi)), the offset is (hi_t - hi_s) + (lo_t - lo_s), accurate to
// about 1e-14 of |x| like an FP64 difference; phi by its Taylor series
// 1 - q/2 + q^2/6 - q^3/24 + q^4/120 - q^5/720 for q < 0.1 (truncation below
// 2e-10) and (1 - expf(-q)) / q above; terms summed in fp32 over tiles of
// 256 sources, tile sums added in FP64.  Relative error of a velocity about
// 1e-6 of sum_j |Gamma_j K_eps|.
//
// One thread per target; the block stages tiles of 256 sources in shared
// memory.
#include "vrm_internal.cuh"

namespace vrm {

namespace {
constexpr int kTile = 256;
}

__global__ void k_bs_split(const double* __restrict__ x, const double* __restrict__ y,
                           const double* __restrict__ g, int n_bound, const int* __restrict__ n_dev,
                           float4* __restrict__ pos, float* __restrict__ gf) {
  const int n = n_dev ? *n_dev : n_bound;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double xi = x[i], yi = y[i];
    const float xh = __double2float_rn(xi), yh = __double2float_rn(yi);
    const float xl = __double2float_rn(xi - (double)xh), yl = __double2float_rn(yi - (double)yh);
    pos[i] = make_float4(xh, yh, xl, yl);
    if (gf) gf[i] = g ? __double2float_rn(g[i]) : 0.0f;
  }
}

__device__ __forceinline__ float phi_of(float q) {
  if (q < 0.1f) {
    float p = fmaf(q, -1.0f / 720.0f, 1.0f / 120.0f);
    p = fmaf(q, p, -1.0f / 24.0f);
    p = fmaf(q, p, 1.0f / 6.0f);
    p = fmaf(q, p, -0.5f);
    return fmaf(q, p, 1.0f);
  }
  return (1.0f - expf(-q)) * __frcp_rn(q);
}

__global__ void __launch_bounds__(kTile) k_bs_direct(const float4* __restrict__ src, const float* __restrict__ gs,
                                                     int n_bound, const int* __restrict__ n_dev,
                                                     const float4* __restrict__ tgt, int m_bound,
                                                     const int* __restrict__ m_dev, float inv_eps2, double c0,
                                                     double* __restrict__ u, double* __restrict__ v) {
  __shared__ float4 sp[kTile];
  __shared__ float sg[kTile];
  const int n = n_dev ? *n_dev : n_bound;
  const int m = m_dev ? *m_dev : m_bound;
  for (long base = (long)blockIdx.x * kTile; base < m; base += (long)gridDim.x * kTile) {
    const long t = base + threadIdx.x;
    const float4 pt = t < m ? tgt[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    double U = 0.0, V = 0.0;
    for (int s0 = 0; s0 < n; s0 += kTile) {
      __syncthreads();
      const int s = s0 + threadIdx.x;
      sp[threadIdx.x] = s < n ? src[s] : make_float4(0.f, 0.f, 0.f, 0.f);
      sg[threadIdx.x] = s < n ? gs[s] : 0.0f;
      __syncthreads();
      float au = 0.0f, av = 0.0f;
      const int cnt = n - s0 < kTile ? n - s0 : kTile;
#pragma unroll 4
      for (int k = 0; k < cnt; ++k) {
        const float4 ps = sp[k];
        const float dx = (pt.x - ps.x) + (pt.z - ps.z);
        const float dy = (pt.y - ps.y) + (pt.w - ps.w);
        const float q = fmaf(dx, dx, dy * dy) * inv_eps2;
        const float w = sg[k] * phi_of(q);
        au = fmaf(-dy, w, au);
        av = fmaf(dx, w, av);
      }
      U += (double)au;
      V += (double)av;
    }
    if (t < m) {
      u[t] = U * c0;
      v[t] = V * c0;
    }
  }
}

cudaError_t bs_split(const double* x, const double* y, const double* g, int n_bound, const int* n_dev, float4* pos,
                     float* gf, cudaStream_t s) {
  if (n_bound <= 0) return cudaSuccess;
  int blocks = (n_bound + kBlock - 1) / kBlock;
  if (blocks > 8 * sm_count()) blocks = 8 * sm_count();
  k_bs_split<<<blocks, kBlock, 0, s>>>(x, y, g, n_bound, n_dev, pos, gf);
  note_launch();
  return cudaGetLastError();
}

cudaError_t bs_direct(const float4* src, const float* gs, int n_bound, const int* n_dev, const float4* tgt,
                      int m_bound, const int* m_dev, double eps, double* u, double* v, cudaStream_t s) {
  if (m_bound <= 0) return cudaSuccess;
  int blocks = (m_bound + kTile - 1) / kTile;
  if (blocks > 16 * sm_count()) blocks = 16 * sm_count();
  const float inv_eps2 = (float)(1.0 / (eps * eps));
  const double c0 = 1.0 / (2.0 * 3.141592653589793 * eps * eps);
  k_bs_direct<<<blocks, kTile, 0, s>>>(src, gs, n_bound, n_dev, tgt, m_bound, m_dev, inv_eps2, c0, u, v);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
