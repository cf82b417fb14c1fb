// Peak FMA throughput probe: the roofline denominator of the LP kernels.
//
// The LP stage is bound by FP64 (and binary32) arithmetic, so its roofline
// fraction needs the rate at which this GPU retires FP64 and FP32 fused
// multiply-adds.  k_fma_probe runs, in every thread, kChains independent
// dependency chains a <- a * b + c of kUnroll FMAs per loop iteration; with
// enough warps per SM the FMA pipes stay busy and the kernel's duration gives
// the peak: flops = 2 * kChains * kUnroll * iters * threads.
#include "vrm_internal.cuh"

namespace vrm {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kProbeBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeBlock) k_fma_probe(int iters, T b, T c, T* __restrict__ sink) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  // one store per block keeps the chains alive without measurable traffic
  if (s == (T)-1.2345) sink[blockIdx.x] = s;
  if (threadIdx.x == 0 && blockIdx.x == 0) sink[gridDim.x] = s;
}

}  // namespace
}  // namespace vrm

extern "C" vrm_status vrm_fma_probe(int32_t fp64, int32_t blocks, int32_t iters, void* sink, double* flops,
                                    cudaStream_t stream) {
  if (blocks <= 0 || iters <= 0 || !sink || !flops) return VRM_ERR_ARG;
  if (fp64)
    vrm::k_fma_probe<double><<<blocks, vrm::kProbeBlock, 0, stream>>>(iters, 0.9999999, 1e-7,
                                                                      static_cast<double*>(sink));
  else
    vrm::k_fma_probe<float><<<blocks, vrm::kProbeBlock, 0, stream>>>(iters, 0.9999999f, 1e-7f,
                                                                     static_cast<float*>(sink));
  vrm::note_launch();
  if (cudaGetLastError() != cudaSuccess) return VRM_ERR_CUDA;
  *flops = 2.0 * vrm::kChains * vrm::kUnroll * (double)iters * (double)blocks * vrm::kProbeBlock;
  return VRM_OK;
}
