// The weight-proposal network of the learned path and its training, on the
// tensor cores (tcgen05, bf16 operands, fp32 accumulators in TMEM).
//
// Network: 96 inputs (the K = 32 neighbour slots' scaled offsets xi_x, xi_y
// and mask; padded to 128 columns with zeros) -> 256 -> 256 -> 256 -> 32,
// GELU (tanh form) after each hidden layer.  Parameters are kept as one fp32
// vector [W1 (256x96), b1, W2 (256x256), b2, W3, b3, W4 (32x256), b4]; the
// GEMMs read bf16 copies (W1 padded to 256x128) and, for the backward pass,
// transposed bf16 copies.
//
// Every product is one kernel, k_gemm<NT>: C[M x N] = A[M x K] B[N x K]^T with
// A and B K-major bf16 in global memory.  A CTA of 4 warps owns a 128-row
// tile of C and NT columns: thread 0 streams 64-column slabs of A and B into
// a 4-stage shared-memory ring with TMA and issues the MMAs (M = 128, N = NT,
// K = 16) into a TMEM accumulator; all four warps then read the accumulator
// (one TMEM lane = one row per thread) and run the fused epilogue (bias,
// GELU, GELU derivative, bf16 rounding, transposed copies for the next
// product).  Weight gradients split K (the batch) across CTAs and sum the
// partials in a fixed order, so training is deterministic.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "vrm_internal.cuh"
#include "vrm_mlp.cuh"
#include "vrm_umma.cuh"

using namespace vrm;
using bf16 = __nv_bfloat16;

namespace {

constexpr int kIn = 96;       // features
constexpr int kInPad = 128;   // feature row stride
constexpr int kHid = 256;
constexpr int kOut = 32;
constexpr int kOutPad = 64;   // dY row stride (one K slab)
constexpr int kBM = 128;      // rows per tile
constexpr int kBK = 64;       // K per slab
constexpr int kStages = 4;
constexpr long long kWaitCycles = 2000000000LL;  // about one second

constexpr long kOffW1 = 0, kOffB1 = kOffW1 + (long)kHid * kIn;
constexpr long kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + (long)kHid * kHid;
constexpr long kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + (long)kHid * kHid;
constexpr long kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + (long)kOut * kHid;
constexpr long kParams = kOffB4 + kOut;
static_assert(kParams == VRM_MLP_PARAMS, "parameter count");

enum EpiMode { EPI_BIAS_GELU = 0, EPI_BIAS_F32 = 1, EPI_F32 = 2, EPI_GELU_BWD = 3 };

struct Epi {
  int mode;
  int M, N;              // logical output rows and columns (stores are guarded)
  const int* m_dev;      // optional device row count (< M)
  int k_slabs;           // K slabs of 64 per CTA
  const float* bias;     // [N]
  const float* z_in;     // EPI_GELU_BWD: pre-activations, ld_zin
  int ld_zin;
  float* out_f32;        // EPI_BIAS_F32 / EPI_F32 (+ blockIdx.z * split_stride)
  int ld_f32;
  long long split_stride;
  bf16* out_bf16;        // row-major, ld_bf16
  int ld_bf16;
  bf16* out_t;           // transposed copy out_t[col * ld_t + row], optional
  int ld_t;
  float* out_z;          // EPI_BIAS_GELU: pre-activation store, optional
  int ld_z;
  int* error;            // set on a wait that gave up
};

// GELU in its tanh form, 0.5 z (1 + tanh(c (z + a z^3))) with c = sqrt(2/pi),
// a = 0.044715, on the hardware tanh (tanh.approx.f32, relative error about
// 2^-11, below the bf16 rounding of the activations).
constexpr float kGeluC = 0.7978845608028654f, kGeluA = 0.044715f;
__device__ __forceinline__ float tanh_hw(float u) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return t;
}
// c (z + a z^3) as z (c + (c a) z^2): five fp32 operations and the tanh.
constexpr float kGeluCA = kGeluC * kGeluA;
__device__ __forceinline__ float gelu(float z) {
  const float u = z * fmaf(kGeluCA, z * z, kGeluC);
  const float hz = 0.5f * z;
  return fmaf(hz, tanh_hw(u), hz);
}
// d/dz of the same: 0.5 (1 + t) + 0.5 z (1 - t^2) c (1 + 3 a z^2).
__device__ __forceinline__ float gelu_grad(float z) {
  const float z2 = z * z;
  const float t = tanh_hw(kGeluC * fmaf(kGeluA * z, z2, z));
  const float du = kGeluC * fmaf(3.0f * kGeluA, z2, 1.0f);
  return fmaf(0.5f * z * du, fmaf(-t, t, 1.0f), 0.5f * (1.0f + t));
}

template <int NT>
constexpr size_t gemm_smem_bytes() {
  return 1024 + (size_t)kStages * (kBM * kBK * 2 + NT * kBK * 2) + 256;
}

template <int NT>
__global__ void __launch_bounds__(128, 1) k_gemm(const __grid_constant__ CUtensorMap tma_a,
                                                 const __grid_constant__ CUtensorMap tma_b, Epi e) {
  static_assert(NT == 32 || NT == 64 || NT == 128 || NT == 256, "tile width");
  extern __shared__ uint8_t smem_raw[];
  const int m0 = blockIdx.x * kBM;
  const int n0 = blockIdx.y * NT;
  int m_limit = e.M;
  if (e.m_dev) {
    const int md = *e.m_dev;
    m_limit = md < m_limit ? md : m_limit;
  }
  if (m0 >= m_limit) return;  // the whole CTA leaves before any barrier or TMEM use

  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sa = base;                                   // kStages x 16 KB
  uint8_t* sb = base + (size_t)kStages * kBM * kBK * 2;  // kStages x NT*128 B
  uint64_t* bars = (uint64_t*)(sb + (size_t)kStages * NT * kBK * 2);
  uint64_t* full = bars;                // TMA -> MMA
  uint64_t* empty = bars + kStages;     // MMA -> TMA
  uint64_t* done = bars + 2 * kStages;  // MMA -> epilogue
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * kStages + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < kStages; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(done, 1);
    umma::fence_barrier_init();
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, NT);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int nk = e.k_slabs;
  const int kslab0 = blockIdx.z * nk;
  constexpr uint32_t kStageBytes = kBM * kBK * 2 + NT * kBK * 2;
  if (threadIdx.x == 0) {
    bool ok = true;
    const uint32_t idesc = umma::idesc_bf16(kBM, NT);
    auto load = [&](int stage, int kb) {
      umma::mbar_arrive_expect_tx(&full[stage], kStageBytes);
      umma::tma_load_2d(sa + (size_t)stage * kBM * kBK * 2, &tma_a, &full[stage], (kslab0 + kb) * kBK, m0);
      umma::tma_load_2d(sb + (size_t)stage * NT * kBK * 2, &tma_b, &full[stage], (kslab0 + kb) * kBK, n0);
    };
    for (int s = 0; s < kStages && s < nk; ++s) load(s, s);
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % kStages;
      if (!umma::mbar_wait(&full[s], (uint32_t)(kb / kStages) & 1u, kWaitCycles)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      const uint64_t da = umma::desc_sw128(umma::smem_u32(sa + (size_t)s * kBM * kBK * 2));
      const uint64_t db = umma::desc_sw128(umma::smem_u32(sb + (size_t)s * NT * kBK * 2));
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k)  // +32 bytes per K step (encoded >> 4)
        umma::mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
      umma::mma_commit(&empty[s]);
      const int kp = kb - 1;  // refill the slot read one slab earlier
      if (kp >= 0 && kp + kStages < nk) {
        const int sp = kp % kStages;
        if (!umma::mbar_wait(&empty[sp], (uint32_t)(kp / kStages) & 1u, kWaitCycles)) {
          ok = false;
          break;
        }
        load(sp, kp + kStages);
      }
    }
    umma::mma_commit(done);
    if (!ok) s_fail = 1;
  }
  const bool got = umma::mbar_wait(done, 0, 2 * kWaitCycles);
  umma::fence_after_sync();
  const bool failed = __syncthreads_or(!got || s_fail) != 0;  // uniform: the TMEM loads below are warp-wide
  if (failed) {
    if (threadIdx.x == 0 && e.error) atomicExch(e.error, 1);
  } else {
    // epilogue: this thread's TMEM lane is row m0 + 32 warp + lane
    const int row = m0 + warp * 32 + lane;
    const bool row_ok = row < m_limit;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < NT; c0 += 16) {
      float v[16];
      umma::tmem_ld16(trow + (uint32_t)c0, v);
      const int col0 = n0 + c0;
      if (!row_ok || col0 >= e.N) continue;
      if (e.mode == EPI_BIAS_GELU) {
        __align__(16) bf16 hv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float z = v[i] + e.bias[col0 + i];
          if (e.out_z) e.out_z[(size_t)row * e.ld_z + col0 + i] = z;
          hv[i] = __float2bfloat16_rn(gelu(z));
        }
        uint4* dst = reinterpret_cast<uint4*>(e.out_bf16 + (size_t)row * e.ld_bf16 + col0);
        dst[0] = *reinterpret_cast<uint4*>(&hv[0]);
        dst[1] = *reinterpret_cast<uint4*>(&hv[8]);
        if (e.out_t) {
#pragma unroll
          for (int i = 0; i < 16; ++i) e.out_t[(size_t)(col0 + i) * e.ld_t + row] = hv[i];
        }
      } else if (e.mode == EPI_BIAS_F32) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (col0 + i < e.N) e.out_f32[(size_t)row * e.ld_f32 + col0 + i] = v[i] + e.bias[col0 + i];
      } else if (e.mode == EPI_F32) {
        float* dst = e.out_f32 + (size_t)blockIdx.z * e.split_stride + (size_t)row * e.ld_f32 + col0;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (col0 + i < e.N) dst[i] = v[i];
      } else {  // EPI_GELU_BWD
        __align__(16) bf16 hv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float z = e.z_in[(size_t)row * e.ld_zin + col0 + i];
          hv[i] = __float2bfloat16_rn(v[i] * gelu_grad(z));
        }
        uint4* dst = reinterpret_cast<uint4*>(e.out_bf16 + (size_t)row * e.ld_bf16 + col0);
        dst[0] = *reinterpret_cast<uint4*>(&hv[0]);
        dst[1] = *reinterpret_cast<uint4*>(&hv[8]);
        if (e.out_t) {
#pragma unroll
          for (int i = 0; i < 16; ++i) e.out_t[(size_t)(col0 + i) * e.ld_t + row] = hv[i];
        }
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, NT);
  }
}

// ---- fused inference ------------------------------------------------------------------
//
// The whole network for 128-row tiles in one persistent kernel; a tile's
// activations never leave shared memory.  Two tiles are in flight per CTA
// (slots 0 and 1: activation tiles H[0], H[1], TMEM columns 0-255 and
// 256-511) so that the MMAs of one overlap the epilogue of the other:
//   warp 16 (one thread): streams the weight slabs (64 input columns of one
//     layer: W1, W2, W3 with 256 rows, W4 with 32) through a 3-stage ring
//     with TMA, loads the input tiles, and issues the MMAs layer by layer,
//     alternating the slots (a weight slab is loaded once per slot);
//   warps 0-15: the epilogue of each (slot, layer) as its accumulator
//     completes: warp w reads TMEM lanes 32 (w mod 4), columns 64 (w div 4),
//     adds the bias, applies GELU and writes bf16 back into the slot's
//     activation tile in the MMA operand layout (128-byte swizzle), which the
//     next layer reads as A; the last layer writes the 32 proposals.
// Barriers per slot: xfull (input tile loaded), accf (the layer's MMAs are
// complete: commit), actr (the layer's epilogue is done: 16 warp arrivals,
// so the next layer may overwrite TMEM and read the activations), hfree (the
// last layer's MMAs are complete: the next input may replace the tile).
// Every wait is bounded; one that gives up raises a shared abort flag that
// every role checks before its next wait, and the error flag in global
// memory.

constexpr int kEpiWarps = 16;
constexpr int kFusedThreads = (kEpiWarps + 1) * 32;
constexpr int kRing = 3;
constexpr int kSlabsPerTile = 14;  // W1: 2, W2: 4, W3: 4, W4: 4
constexpr int kSlabsPerPair = 2 * kSlabsPerTile;
constexpr uint32_t kSlabBytes = kBM * kBK * 2;  // one 128-row activation slab
constexpr uint32_t kRingBytes = 256 * kBK * 2;  // one 256-row weight slab
constexpr size_t kFusedSmem = 1024 + 2 * 4 * (size_t)kSlabBytes + (size_t)kRing * kRingBytes + 256;

// Layer and K slab of the g-th weight slab a single tile consumes.
__device__ __forceinline__ void slab_of(int s, int* layer, int* kb) {
  if (s < 2) {
    *layer = 0, *kb = s;
  } else if (s < 6) {
    *layer = 1, *kb = s - 2;
  } else if (s < 10) {
    *layer = 2, *kb = s - 6;
  } else {
    *layer = 3, *kb = s - 10;
  }
}

// Layer and K slab of the g-th weight slab the producer consumes: whole
// pairs of tiles take each layer's slabs twice (slot 0, then slot 1); a
// last unpaired tile takes them once.
__device__ __forceinline__ void slab_at(int g, int pairs, int* layer, int* kb) {
  if (g < pairs * kSlabsPerPair) {
    const int r = g % kSlabsPerPair;
    if (r < 4) {
      *layer = 0, *kb = r & 1;
    } else if (r < 12) {
      *layer = 1, *kb = (r - 4) & 3;
    } else if (r < 20) {
      *layer = 2, *kb = (r - 12) & 3;
    } else {
      *layer = 3, *kb = (r - 20) & 3;
    }
  } else {
    slab_of(g - pairs * kSlabsPerPair, layer, kb);
  }
}

struct FusedArgs {
  const float* bias;  // theta: b1, b2, b3, b4 at their offsets
  float* Y;           // [rows x 32]
  int rows;           // bound
  const int* rows_dev;
  int* error;
};

__global__ void __launch_bounds__(kFusedThreads, 1)
    k_mlp_fused(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tw1,
                const __grid_constant__ CUtensorMap tw2, const __grid_constant__ CUtensorMap tw3,
                const __grid_constant__ CUtensorMap tw4, FusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  int rows = a.rows;
  if (a.rows_dev) {
    const int r = *a.rows_dev;
    rows = r < rows ? r : rows;
  }
  const int ntiles = (rows + kBM - 1) / kBM;
  if ((int)blockIdx.x >= ntiles) return;
  const int my_tiles = (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;
  const int pairs_full = my_tiles / 2;
  const int npairs = (my_tiles + 1) / 2;
  const int total = pairs_full * kSlabsPerPair + (my_tiles & 1) * kSlabsPerTile;

  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* H = base;                         // 2 slots x 4 slabs x 16 KB
  uint8_t* ring = base + 8 * (size_t)kSlabBytes;  // kRing x 32 KB
  uint64_t* bars = (uint64_t*)(ring + (size_t)kRing * kRingBytes);
  uint64_t* xfull = bars;
  uint64_t* accf = bars + 2;
  uint64_t* actr = bars + 4;
  uint64_t* hfree = bars + 6;
  uint64_t* wfull = bars + 8;
  uint64_t* wempty = bars + 8 + kRing;
  uint64_t* drain = bars + 8 + 2 * kRing;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      umma::mbar_init(&xfull[s], 1);
      umma::mbar_init(&accf[s], 1);
      umma::mbar_init(&actr[s], kEpiWarps);
      umma::mbar_init(&hfree[s], 1);
    }
    for (int s = 0; s < kRing; ++s) {
      umma::mbar_init(&wfull[s], 1);
      umma::mbar_init(&wempty[s], 1);
    }
    umma::mbar_init(drain, 1);
    *abort_flag = 0;
    umma::fence_barrier_init();
  }
  if (warp == 0) umma::tmem_alloc(tmem_slot, 512);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == kEpiWarps) {
    // ---- producer / MMA issue (one thread) ----
    if (lane == 0) {
      const CUtensorMap* wmap[4] = {&tw1, &tw2, &tw3, &tw4};
      auto load_w = [&](int gl) {
        int layer, kb;
        slab_at(gl, pairs_full, &layer, &kb);
        const int st = gl % kRing;
        umma::mbar_arrive_expect_tx(&wfull[st], layer == 3 ? (uint32_t)kOut * kBK * 2 : kRingBytes);
        umma::tma_load_2d(ring + (size_t)st * kRingBytes, wmap[layer], &wfull[st], kb * kBK, 0);
      };
      auto load_x = [&](int s, int tile) {
        uint8_t* h = H + (size_t)s * 4 * kSlabBytes;
        umma::mbar_arrive_expect_tx(&xfull[s], 2u * kSlabBytes);
        umma::tma_load_2d(h, &tx, &xfull[s], 0, tile * kBM);
        umma::tma_load_2d(h + kSlabBytes, &tx, &xfull[s], kBK, tile * kBM);
      };
      load_x(0, blockIdx.x);
      if (my_tiles > 1) load_x(1, blockIdx.x + gridDim.x);
      int g_load = 0;
      for (; g_load < kRing && g_load < total; ++g_load) load_w(g_load);
      bool fail = false;
      int g = 0;
      for (int p = 0; p < npairs && !fail; ++p) {
        const int nslot = (2 * p + 1 < my_tiles) ? 2 : 1;
        for (int l = 0; l < 4 && !fail; ++l) {
          for (int s = 0; s < nslot && !fail; ++s) {
            if (*abort_flag) {
              fail = true;
              break;
            }
            if (l == 0 && !umma::mbar_wait(&xfull[s], (uint32_t)p & 1u, kWaitCycles)) {
              fail = true;
              break;
            }
            const int e = 4 * p + l;  // epilogues of this slot that must be done
            if (e > 0 && !umma::mbar_wait(&actr[s], (uint32_t)(e - 1) & 1u, kWaitCycles)) {
              fail = true;
              break;
            }
            umma::fence_after_sync();
            const uint32_t idesc = umma::idesc_bf16(kBM, l == 3 ? kOut : kHid);
            const int nk = l == 0 ? 2 : 4;
            uint8_t* h = H + (size_t)s * 4 * kSlabBytes;
            for (int kb = 0; kb < nk; ++kb, ++g) {
              const int st = g % kRing;
              if (!umma::mbar_wait(&wfull[st], (uint32_t)(g / kRing) & 1u, kWaitCycles)) {
                fail = true;
                break;
              }
              umma::fence_after_sync();
              const uint64_t da = umma::desc_sw128(umma::smem_u32(h + (size_t)kb * kSlabBytes));
              const uint64_t db = umma::desc_sw128(umma::smem_u32(ring + (size_t)st * kRingBytes));
#pragma unroll
              for (int k = 0; k < kBK / 16; ++k)
                umma::mma_bf16(tmem + (uint32_t)(s * 256), da + 2 * k, db + 2 * k, idesc, (kb | k) != 0);
              umma::mma_commit(&wempty[st]);
              // refill the slot of the previous slab (its MMAs were issued earlier)
              const int gp = g - 1;
              if (gp >= 0 && gp + kRing < total && g_load == gp + kRing) {
                if (!umma::mbar_wait(&wempty[gp % kRing], (uint32_t)(gp / kRing) & 1u, kWaitCycles)) {
                  fail = true;
                  break;
                }
                load_w(g_load++);
              }
            }
            if (fail) break;
            umma::mma_commit(&accf[s]);
            if (l == 3) umma::mma_commit(&hfree[s]);
          }
        }
        // the next inputs, once the last layer's MMAs of a slot have read its tile
        for (int s = 0; s < nslot && !fail; ++s) {
          const int nt = 2 * (p + 1) + s;
          if (nt >= my_tiles) continue;
          if (!umma::mbar_wait(&hfree[s], (uint32_t)p & 1u, kWaitCycles)) {
            fail = true;
            break;
          }
          load_x(s, blockIdx.x + nt * gridDim.x);
        }
      }
      if (fail) *abort_flag = 1;
      // every MMA issued completes before the TMEM is released
      umma::mma_commit(drain);
      if (!umma::mbar_wait(drain, 0u, kWaitCycles)) *abort_flag = 1;
    }
  } else {
    // ---- epilogue warps ----
    const int q = warp & 3, cg = warp >> 2;
    const int r = q * 32 + lane;  // row within the tile
    bool stop = false;
    for (int p = 0; p < npairs && !stop; ++p) {
      const int nslot = (2 * p + 1 < my_tiles) ? 2 : 1;
      for (int l = 0; l < 4 && !stop; ++l) {
        for (int s = 0; s < nslot; ++s) {
          if (*abort_flag) {
            stop = true;
            break;
          }
          if (!umma::mbar_wait(&accf[s], (uint32_t)(4 * p + l) & 1u, 2 * kWaitCycles)) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          umma::fence_after_sync();
          const uint32_t trow = tmem + (uint32_t)(s * 256) + ((uint32_t)(q * 32) << 16);
          uint8_t* h = H + (size_t)s * 4 * kSlabBytes;
          if (l < 3) {
            const float* b = a.bias + (l == 0 ? kOffB1 : l == 1 ? kOffB2 : kOffB3);
#pragma unroll 1
            for (int c0 = cg * 64; c0 < cg * 64 + 64; c0 += 32) {
              float v[32];
              umma::tmem_ld32(trow + (uint32_t)c0, v);
              __align__(16) __nv_bfloat162 hv[16];
#pragma unroll
              for (int i = 0; i < 16; ++i)
                hv[i] = __floats2bfloat162_rn(gelu(v[2 * i] + __ldg(b + c0 + 2 * i)),
                                              gelu(v[2 * i + 1] + __ldg(b + c0 + 2 * i + 1)));
              uint8_t* slab = h + (size_t)(c0 >> 6) * kSlabBytes + (size_t)r * 128;
              const int ch = (c0 & 63) >> 3;
#pragma unroll
              for (int u = 0; u < 4; ++u)
                *reinterpret_cast<uint4*>(slab + (((ch + u) ^ (r & 7)) << 4)) = *reinterpret_cast<uint4*>(&hv[4 * u]);
            }
          } else if (cg < 2) {
            const int c0 = cg * 16;
            float v[16];
            umma::tmem_ld16(trow + (uint32_t)c0, v);
            const int row = (blockIdx.x + (2 * p + s) * gridDim.x) * kBM + r;
            if (row < rows) {
              const float* b = a.bias + kOffB4 + c0;
              float4* dst = reinterpret_cast<float4*>(a.Y + (size_t)row * kOut + c0);
#pragma unroll
              for (int i = 0; i < 4; ++i)
                dst[i] = make_float4(v[4 * i] + __ldg(b + 4 * i), v[4 * i + 1] + __ldg(b + 4 * i + 1),
                                     v[4 * i + 2] + __ldg(b + 4 * i + 2), v[4 * i + 3] + __ldg(b + 4 * i + 3));
            }
          }
          umma::fence_proxy_async_smem();  // the activation writes feed the next MMAs (async proxy)
          umma::fence_before_sync();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(&actr[s]);
        }
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag && a.error) atomicExch(a.error, 1);
  if (warp == 0) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, 512);
  }
}

// ---- small kernels -----------------------------------------------------------------

// Batch assembly: rows idx[r] (or r) of the data set into X [B x 128],
// X^T [128 x B] and T [B x 32]; rows >= rows are zero (their mask is 0, so
// they add nothing to the loss or the gradients).
__global__ void k_gather(const bf16* __restrict__ X_all, const float* __restrict__ T_all,
                         const int* __restrict__ idx, int rows, int B, bf16* __restrict__ Xb, bf16* __restrict__ Xbt,
                         float* __restrict__ Tb) {
  const long total = (long)B * kInPad;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int r = (int)(t / kInPad), c = (int)(t % kInPad);
    bf16 v = __float2bfloat16_rn(0.0f);
    if (r < rows) {
      const long src = idx ? idx[r] : r;
      v = X_all[src * kInPad + c];
      if (c < kOut) Tb[(size_t)r * kOut + c] = T_all[src * kOut + c];
    } else if (c < kOut) {
      Tb[(size_t)r * kOut + c] = 0.0f;
    }
    Xb[(size_t)r * kInPad + c] = v;
    Xbt[(size_t)c * B + r] = v;
  }
}

// Masked mean squared error and its gradient, one block, fixed summation
// order: dY = 2 M (Y - T) / sum(M), written as bf16 [B x 64] (columns >= 32
// zero) and transposed [128 x B] (rows >= 32 zero).
__global__ void __launch_bounds__(1024) k_loss(const float* __restrict__ Y, const float* __restrict__ T,
                                               const bf16* __restrict__ Xb, int B, bf16* __restrict__ dY,
                                               bf16* __restrict__ dYt, float* __restrict__ loss) {
  __shared__ float red[32];
  const int tid = threadIdx.x;
  const long total = (long)B * kOut;
  auto block_sum = [&](float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    float s = 0.0f;
    if (tid < 32) {
      s = tid < (int)(blockDim.x >> 5) ? red[tid] : 0.0f;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    if (tid == 0) red[0] = s;
    __syncthreads();
    const float r = red[0];
    __syncthreads();
    return r;
  };
  float cnt = 0.0f;
  for (long t = tid; t < total; t += blockDim.x) {
    const int r = (int)(t / kOut), k = (int)(t % kOut);
    cnt += __bfloat162float(Xb[(size_t)r * kInPad + 2 * kOut + k]);
  }
  cnt = block_sum(cnt);
  const float inv = 1.0f / fmaxf(cnt, 1.0f);
  float l = 0.0f;
  for (long t = tid; t < total; t += blockDim.x) {
    const int r = (int)(t / kOut), k = (int)(t % kOut);
    const float m = __bfloat162float(Xb[(size_t)r * kInPad + 2 * kOut + k]);
    const float d = m * (Y[t] - T[t]);
    l += d * d;
    const bf16 g = __float2bfloat16_rn(2.0f * d * inv);
    dY[(size_t)r * kOutPad + k] = g;
    dY[(size_t)r * kOutPad + kOut + k] = __float2bfloat16_rn(0.0f);
    dYt[(size_t)k * B + r] = g;
  }
  l = block_sum(l);
  if (tid == 0) {
    loss[0] = l * inv;
    loss[1] = cnt;
  }
}

// out[n] = sum over the B entries of row n of a bf16 [N x B] matrix (one
// warp per row, fixed order).
__global__ void k_rowsum(const bf16* __restrict__ m, int N, int B, float* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= N) return;
  float s = 0.0f;
  for (int r = lane; r < B; r += 32) s += __bfloat162float(m[(size_t)w * B + r]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[w] = s;
}

// g[r * cols + c] = sum_s part[s][r * ld + c] for r < rows, c < cols.
__global__ void k_split_sum(const float* __restrict__ part, int splits, long long stride, int rows, int cols, int ld,
                            float* __restrict__ g) {
  const long total = (long)rows * cols;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int r = (int)(t / cols), c = (int)(t % cols);
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * stride + (size_t)r * ld + c];
    g[t] = s;
  }
}

// AdamW (decoupled weight decay): c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void k_adamw(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                        const float* __restrict__ g, long n, float lr, float b1, float b2, float eps, float wd,
                        float c1, float c2) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    theta[i] = theta[i] - lr * (mh / (sqrtf(vh) + eps) + wd * theta[i]);
  }
}

// bf16 weights for the GEMMs from the fp32 parameters: W1 padded to 256 x 128,
// W2, W3, W4, and transposed copies W2^T, W3^T (256 x 256), W4^T (256 x 64).
__global__ void k_refresh(const float* __restrict__ th, bf16* __restrict__ W1, bf16* __restrict__ W2,
                          bf16* __restrict__ W3, bf16* __restrict__ W4, bf16* __restrict__ W2t,
                          bf16* __restrict__ W3t, bf16* __restrict__ W4t) {
  const long n1 = (long)kHid * kInPad, n2 = (long)kHid * kHid, n4 = (long)kHid * kOutPad;
  const long total = n1 + 2 * n2 + n4;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    if (t < n1) {
      const int r = (int)(t / kInPad), c = (int)(t % kInPad);
      W1[t] = __float2bfloat16_rn(c < kIn ? th[kOffW1 + (long)r * kIn + c] : 0.0f);
    } else if (t < n1 + n2) {
      const long u = t - n1;
      const int r = (int)(u / kHid), c = (int)(u % kHid);
      const bf16 w = __float2bfloat16_rn(th[kOffW2 + u]);
      W2[u] = w;
      W2t[(long)c * kHid + r] = w;
    } else if (t < n1 + 2 * n2) {
      const long u = t - n1 - n2;
      const int r = (int)(u / kHid), c = (int)(u % kHid);
      const bf16 w = __float2bfloat16_rn(th[kOffW3 + u]);
      W3[u] = w;
      W3t[(long)c * kHid + r] = w;
    } else {
      const long u = t - n1 - 2 * n2;  // W4^T entry (c, r): c < 256, r < 64
      const int c = (int)(u / kOutPad), r = (int)(u % kOutPad);
      const bf16 w = __float2bfloat16_rn(r < kOut ? th[kOffW4 + (long)r * kHid + c] : 0.0f);
      W4t[u] = w;
      if (r < kOut) W4[(long)r * kHid + c] = w;
    }
  }
}

// ---- host side ----------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// Tensor map of a row-major bf16 matrix [rows x cols] read in boxes of
// 64 columns x box_rows rows with 128-byte swizzle.  The caller keeps every
// box inside the matrix (rows a multiple of box_rows, cols of 64).
bool make_map(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !ptr || ((uintptr_t)ptr & 15u) || cols % 64 || rows % box_rows) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT>
cudaError_t launch_gemm_nt(const CUtensorMap& a, const CUtensorMap& b, int m_tiles, int n_tiles, int splits,
                           const Epi& e, cudaStream_t s) {
  static bool attr_set = false;
  const size_t smem = gemm_smem_bytes<NT>();
  if (!attr_set) {
    cudaError_t r = cudaFuncSetAttribute(k_gemm<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r != cudaSuccess) return r;
    attr_set = true;
  }
  dim3 grid(m_tiles, n_tiles, splits);
  k_gemm<NT><<<grid, 128, smem, s>>>(a, b, e);
  note_launch();
  return cudaGetLastError();
}

// C[M x N] = A[M x K] B[N x K]^T with K split `splits` ways (K / 64 divisible).
cudaError_t gemm(const CUtensorMap& a, const CUtensorMap& b, int nt, int m_bound, int N, int K, int splits, Epi e,
                 cudaStream_t s) {
  if (K % kBK || (K / kBK) % splits) return cudaErrorInvalidValue;
  e.k_slabs = K / kBK / splits;
  const int m_tiles = (m_bound + kBM - 1) / kBM;
  const int n_tiles = (N + nt - 1) / nt;
  switch (nt) {
    case 32: return launch_gemm_nt<32>(a, b, m_tiles, n_tiles, splits, e, s);
    case 64: return launch_gemm_nt<64>(a, b, m_tiles, n_tiles, splits, e, s);
    case 128: return launch_gemm_nt<128>(a, b, m_tiles, n_tiles, splits, e, s);
    case 256: return launch_gemm_nt<256>(a, b, m_tiles, n_tiles, splits, e, s);
    default: return cudaErrorInvalidValue;
  }
}

Epi epi(int mode, int M, int N) {
  Epi e;
  memset(&e, 0, sizeof(e));
  e.mode = mode;
  e.M = M;
  e.N = N;
  return e;
}

int blocks_for_n(long n, int threads) {
  long b = (n + threads - 1) / threads;
  const long cap = 8L * sm_count();
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

struct vrm_mlp {
  int B = 0;       // training batch rows (multiple of 128)
  int splits = 1;  // K splits of the weight-gradient products
  int* err = nullptr;
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *part = nullptr, *loss = nullptr;
  bf16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W4 = nullptr, *W2t = nullptr, *W3t = nullptr, *W4t = nullptr;
  bf16 *Xb = nullptr, *Xbt = nullptr;
  float* Tb = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *Y = nullptr;
  bf16 *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *H1t = nullptr, *H2t = nullptr, *H3t = nullptr;
  bf16 *dY = nullptr, *dYt = nullptr;
  bf16 *dZ1 = nullptr, *dZ2 = nullptr, *dZ3 = nullptr, *dZ1t = nullptr, *dZ2t = nullptr, *dZ3t = nullptr;
  CUtensorMap mW1, mW2, mW3, mW4, mW2t, mW3t, mW4t;  // weights as B operands
  CUtensorMap mX, mXt, mH1, mH2, mH3, mH1t, mH2t, mH3t, mdY, mdYt, mdZ1t, mdZ2, mdZ2t, mdZ3, mdZ3t;
};

namespace vrm {

cudaError_t mlp_acts_alloc(MlpActs* a, int rows) {
  mlp_acts_free(a);
  const int rp = (rows + kBM - 1) / kBM * kBM;
  cudaError_t e = cudaMalloc(&a->X, (size_t)rp * kInPad * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMemset(a->X, 0, (size_t)rp * kInPad * sizeof(bf16));
  if (e != cudaSuccess) {
    mlp_acts_free(a);
    return e;
  }
  if (!make_map(&a->mX, a->X, rp, kInPad, kBM)) {
    mlp_acts_free(a);
    return cudaErrorInvalidValue;
  }
  a->rows_pad = rp;
  return cudaSuccess;
}

void mlp_acts_free(MlpActs* a) {
  if (a->X) cudaFree(a->X);
  a->X = nullptr;
  a->rows_pad = 0;
}

bool mlp_input_map(CUtensorMap* m, const bf16* X, int rows_pad) { return make_map(m, X, rows_pad, kInPad, kBM); }

cudaError_t mlp_forward(vrm_mlp* net, const CUtensorMap& mX, int rows, const int* rows_dev, float* Y,
                        cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t r = cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmem);
    if (r != cudaSuccess) return r;
    attr_set = true;
  }
  const int ntiles = (rows + kBM - 1) / kBM;
  const int grid = ntiles < sm_count() ? ntiles : sm_count();
  FusedArgs fa;
  fa.bias = net->theta;
  fa.Y = Y;
  fa.rows = rows;
  fa.rows_dev = rows_dev;
  fa.error = net->err;
  k_mlp_fused<<<grid, kFusedThreads, kFusedSmem, s>>>(mX, net->mW1, net->mW2, net->mW3, net->mW4, fa);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vrm

namespace {

void free_mlp(vrm_mlp* n) {
  void* ptrs[] = {n->err, n->theta, n->m, n->v, n->grad, n->part, n->loss, n->W1, n->W2, n->W3, n->W4, n->W2t,
                  n->W3t, n->W4t, n->Xb, n->Xbt, n->Tb, n->Z1, n->Z2, n->Z3, n->Y, n->H1, n->H2, n->H3, n->H1t,
                  n->H2t, n->H3t, n->dY, n->dYt, n->dZ1, n->dZ2, n->dZ3, n->dZ1t, n->dZ2t, n->dZ3t};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

template <typename T>
cudaError_t zalloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e == cudaSuccess) e = cudaMemset(*p, 0, sizeof(T) * count);
  return e;
}

// Forward and backward of the current batch (Xb, Xbt, Tb): loss -> net->loss,
// gradient -> net->grad.
cudaError_t forward_backward(vrm_mlp* n, cudaStream_t s) {
  const int B = n->B;
  cudaError_t r;
  // forward, keeping pre-activations and transposed activations
  Epi e = epi(EPI_BIAS_GELU, B, kHid);
  e.error = n->err;
  e.ld_bf16 = kHid;
  e.ld_t = B;
  e.ld_z = kHid;
  e.bias = n->theta + kOffB1, e.out_bf16 = n->H1, e.out_t = n->H1t, e.out_z = n->Z1;
  if ((r = gemm(n->mX, n->mW1, 256, B, kHid, kInPad, 1, e, s)) != cudaSuccess) return r;
  e.bias = n->theta + kOffB2, e.out_bf16 = n->H2, e.out_t = n->H2t, e.out_z = n->Z2;
  if ((r = gemm(n->mH1, n->mW2, 256, B, kHid, kHid, 1, e, s)) != cudaSuccess) return r;
  e.bias = n->theta + kOffB3, e.out_bf16 = n->H3, e.out_t = n->H3t, e.out_z = n->Z3;
  if ((r = gemm(n->mH2, n->mW3, 256, B, kHid, kHid, 1, e, s)) != cudaSuccess) return r;
  Epi f = epi(EPI_BIAS_F32, B, kOut);
  f.error = n->err;
  f.bias = n->theta + kOffB4, f.out_f32 = n->Y, f.ld_f32 = kOut;
  if ((r = gemm(n->mH3, n->mW4, 32, B, kOut, kHid, 1, f, s)) != cudaSuccess) return r;
  k_loss<<<1, 1024, 0, s>>>(n->Y, n->Tb, n->Xb, B, n->dY, n->dYt, n->loss);
  note_launch();
  // backward
  const long long pstride = (long long)kHid * kHid;
  Epi w = epi(EPI_F32, kOut, kHid);  // dW4 = dY^T H3
  w.error = n->err;
  w.out_f32 = n->part, w.ld_f32 = kHid, w.split_stride = pstride;
  if ((r = gemm(n->mdYt, n->mH3t, 256, kOut, kHid, B, n->splits, w, s)) != cudaSuccess) return r;
  k_split_sum<<<blocks_for_n((long)kOut * kHid, 256), 256, 0, s>>>(n->part, n->splits, pstride, kOut, kHid, kHid,
                                                                    n->grad + kOffW4);
  note_launch();
  k_rowsum<<<(kOut * 32 + 255) / 256, 256, 0, s>>>(n->dYt, kOut, B, n->grad + kOffB4);
  note_launch();
  Epi d = epi(EPI_GELU_BWD, B, kHid);  // dZ3 = (dY W4) * gelu'(Z3)
  d.error = n->err;
  d.ld_bf16 = kHid, d.ld_t = B, d.ld_zin = kHid;
  d.z_in = n->Z3, d.out_bf16 = n->dZ3, d.out_t = n->dZ3t;
  if ((r = gemm(n->mdY, n->mW4t, 256, B, kHid, kOutPad, 1, d, s)) != cudaSuccess) return r;
  w = epi(EPI_F32, kHid, kHid);  // dW3 = dZ3^T H2
  w.error = n->err;
  w.out_f32 = n->part, w.ld_f32 = kHid, w.split_stride = pstride;
  if ((r = gemm(n->mdZ3t, n->mH2t, 256, kHid, kHid, B, n->splits, w, s)) != cudaSuccess) return r;
  k_split_sum<<<blocks_for_n(pstride, 256), 256, 0, s>>>(n->part, n->splits, pstride, kHid, kHid, kHid,
                                                          n->grad + kOffW3);
  note_launch();
  k_rowsum<<<(kHid * 32 + 255) / 256, 256, 0, s>>>(n->dZ3t, kHid, B, n->grad + kOffB3);
  note_launch();
  d.z_in = n->Z2, d.out_bf16 = n->dZ2, d.out_t = n->dZ2t;  // dZ2 = (dZ3 W3) * gelu'(Z2)
  if ((r = gemm(n->mdZ3, n->mW3t, 256, B, kHid, kHid, 1, d, s)) != cudaSuccess) return r;
  if ((r = gemm(n->mdZ2t, n->mH1t, 256, kHid, kHid, B, n->splits, w, s)) != cudaSuccess) return r;  // dW2
  k_split_sum<<<blocks_for_n(pstride, 256), 256, 0, s>>>(n->part, n->splits, pstride, kHid, kHid, kHid,
                                                          n->grad + kOffW2);
  note_launch();
  k_rowsum<<<(kHid * 32 + 255) / 256, 256, 0, s>>>(n->dZ2t, kHid, B, n->grad + kOffB2);
  note_launch();
  d.z_in = n->Z1, d.out_bf16 = n->dZ1, d.out_t = n->dZ1t;  // dZ1 = (dZ2 W2) * gelu'(Z1)
  if ((r = gemm(n->mdZ2, n->mW2t, 256, B, kHid, kHid, 1, d, s)) != cudaSuccess) return r;
  w = epi(EPI_F32, kHid, kInPad);  // dW1 = dZ1^T X (padded input columns dropped in the sum)
  w.error = n->err;
  w.out_f32 = n->part, w.ld_f32 = kInPad, w.split_stride = pstride;
  if ((r = gemm(n->mdZ1t, n->mXt, 128, kHid, kInPad, B, n->splits, w, s)) != cudaSuccess) return r;
  k_split_sum<<<blocks_for_n((long)kHid * kIn, 256), 256, 0, s>>>(n->part, n->splits, pstride, kHid, kIn, kInPad,
                                                                    n->grad + kOffW1);
  note_launch();
  k_rowsum<<<(kHid * 32 + 255) / 256, 256, 0, s>>>(n->dZ1t, kHid, B, n->grad + kOffB1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t refresh(vrm_mlp* n, cudaStream_t s) {
  const long total = (long)kHid * kInPad + 2L * kHid * kHid + (long)kHid * kOutPad;
  k_refresh<<<blocks_for_n(total, 256), 256, 0, s>>>(n->theta, n->W1, n->W2, n->W3, n->W4, n->W2t, n->W3t, n->W4t);
  note_launch();
  return cudaGetLastError();
}

cudaError_t gather(vrm_mlp* n, const bf16* X, const float* T, const int* idx, int rows, cudaStream_t s) {
  k_gather<<<blocks_for_n((long)n->B * kInPad, 256), 256, 0, s>>>(X, T, idx, rows, n->B, n->Xb, n->Xbt, n->Tb);
  note_launch();
  return cudaGetLastError();
}

vrm_status check_err(vrm_mlp* n, cudaStream_t s) {
  int h = 0;
  if (cudaMemcpyAsync(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VRM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return VRM_ERR_CUDA;
  return h ? VRM_ERR_CUDA : VRM_OK;
}

bool adamw_ok(const vrm_adamw* a) {
  return a && a->lr >= 0 && a->beta1 >= 0 && a->beta1 < 1 && a->beta2 >= 0 && a->beta2 < 1 && a->eps >= 0 &&
         a->weight_decay >= 0 && std::isfinite(a->lr);
}

vrm_status run_adamw(vrm_mlp* n, const float* grad, const vrm_adamw* a, int32_t t, cudaStream_t s) {
  const double c1 = 1.0 - std::pow((double)a->beta1, (double)t);
  const double c2 = 1.0 - std::pow((double)a->beta2, (double)t);
  k_adamw<<<blocks_for_n(kParams, 256), 256, 0, s>>>(n->theta, n->m, n->v, grad, kParams, a->lr, a->beta1, a->beta2,
                                                      a->eps, a->weight_decay, (float)c1, (float)c2);
  note_launch();
  if (refresh(n, s) != cudaSuccess) return VRM_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? VRM_OK : VRM_ERR_CUDA;
}

}  // namespace

extern "C" {

vrm_status vrm_mlp_create(int32_t batch_rows, vrm_mlp** out) {
  if (!out) return VRM_ERR_ARG;
  *out = nullptr;
  if (batch_rows < kBM || batch_rows % kBM || batch_rows > (1 << 20)) return VRM_ERR_ARG;
  if (!encode_fn()) return VRM_ERR_UNSUPPORTED;
  vrm_mlp* n = new (std::nothrow) vrm_mlp();
  if (!n) return VRM_ERR_CUDA;
  const int B = batch_rows;
  n->B = B;
  // weight-gradient products: K = B split in at most 64 equal pieces of whole
  // 128-row blocks
  int splits = 1;
  for (int d = 64; d >= 1; --d)
    if ((B / 128) % d == 0) {
      splits = d;
      break;
    }
  n->splits = splits;
  cudaError_t e = cudaSuccess;
#define MLP_ALLOC(p, cnt) \
  if (e == cudaSuccess) e = zalloc(&(n->p), (size_t)(cnt))
  MLP_ALLOC(err, 1);
  MLP_ALLOC(theta, kParams);
  MLP_ALLOC(m, kParams);
  MLP_ALLOC(v, kParams);
  MLP_ALLOC(grad, kParams);
  MLP_ALLOC(part, (size_t)splits * kHid * kHid);
  MLP_ALLOC(loss, 2);
  MLP_ALLOC(W1, (size_t)kHid * kInPad);
  MLP_ALLOC(W2, (size_t)kHid * kHid);
  MLP_ALLOC(W3, (size_t)kHid * kHid);
  MLP_ALLOC(W4, (size_t)kOut * kHid);
  MLP_ALLOC(W2t, (size_t)kHid * kHid);
  MLP_ALLOC(W3t, (size_t)kHid * kHid);
  MLP_ALLOC(W4t, (size_t)kHid * kOutPad);
  MLP_ALLOC(Xb, (size_t)B * kInPad);
  MLP_ALLOC(Xbt, (size_t)kInPad * B);
  MLP_ALLOC(Tb, (size_t)B * kOut);
  MLP_ALLOC(Z1, (size_t)B * kHid);
  MLP_ALLOC(Z2, (size_t)B * kHid);
  MLP_ALLOC(Z3, (size_t)B * kHid);
  MLP_ALLOC(Y, (size_t)B * kOut);
  MLP_ALLOC(H1, (size_t)B * kHid);
  MLP_ALLOC(H2, (size_t)B * kHid);
  MLP_ALLOC(H3, (size_t)B * kHid);
  MLP_ALLOC(H1t, (size_t)kHid * B);
  MLP_ALLOC(H2t, (size_t)kHid * B);
  MLP_ALLOC(H3t, (size_t)kHid * B);
  MLP_ALLOC(dY, (size_t)B * kOutPad);
  MLP_ALLOC(dYt, (size_t)kBM * B);
  MLP_ALLOC(dZ1, (size_t)B * kHid);
  MLP_ALLOC(dZ2, (size_t)B * kHid);
  MLP_ALLOC(dZ3, (size_t)B * kHid);
  MLP_ALLOC(dZ1t, (size_t)kHid * B);
  MLP_ALLOC(dZ2t, (size_t)kHid * B);
  MLP_ALLOC(dZ3t, (size_t)kHid * B);
#undef MLP_ALLOC
  bool ok = e == cudaSuccess;
  // B operands (weights): boxes of NT rows; A operands: 128-row boxes
  ok = ok && make_map(&n->mW1, n->W1, kHid, kInPad, 256) && make_map(&n->mW2, n->W2, kHid, kHid, 256) &&
       make_map(&n->mW3, n->W3, kHid, kHid, 256) && make_map(&n->mW4, n->W4, kOut, kHid, 32) &&
       make_map(&n->mW2t, n->W2t, kHid, kHid, 256) && make_map(&n->mW3t, n->W3t, kHid, kHid, 256) &&
       make_map(&n->mW4t, n->W4t, kHid, kOutPad, 256);
  ok = ok && make_map(&n->mX, n->Xb, B, kInPad, kBM) && make_map(&n->mXt, n->Xbt, kInPad, B, 128) &&
       make_map(&n->mH1, n->H1, B, kHid, kBM) && make_map(&n->mH2, n->H2, B, kHid, kBM) &&
       make_map(&n->mH3, n->H3, B, kHid, kBM) && make_map(&n->mH1t, n->H1t, kHid, B, 256) &&
       make_map(&n->mH2t, n->H2t, kHid, B, 256) && make_map(&n->mH3t, n->H3t, kHid, B, 256) &&
       make_map(&n->mdY, n->dY, B, kOutPad, kBM) && make_map(&n->mdYt, n->dYt, kBM, B, kBM) &&
       make_map(&n->mdZ1t, n->dZ1t, kHid, B, kBM) && make_map(&n->mdZ2, n->dZ2, B, kHid, kBM) &&
       make_map(&n->mdZ2t, n->dZ2t, kHid, B, kBM) && make_map(&n->mdZ3, n->dZ3, B, kHid, kBM) &&
       make_map(&n->mdZ3t, n->dZ3t, kHid, B, kBM);
  if (!ok) {
    free_mlp(n);
    delete n;
    cudaGetLastError();
    return e == cudaSuccess ? VRM_ERR_UNSUPPORTED : VRM_ERR_CUDA;
  }
  *out = n;
  return VRM_OK;
}

void vrm_mlp_destroy(vrm_mlp* n) {
  if (!n) return;
  free_mlp(n);
  delete n;
}

vrm_status vrm_mlp_set_params(vrm_mlp* n, const float* theta, cudaStream_t s) {
  if (!n || !theta) return VRM_ERR_ARG;
  if (cudaMemcpyAsync(n->theta, theta, sizeof(float) * kParams, cudaMemcpyDefault, s) != cudaSuccess)
    return VRM_ERR_CUDA;
  if (cudaMemsetAsync(n->m, 0, sizeof(float) * kParams, s) != cudaSuccess) return VRM_ERR_CUDA;
  if (cudaMemsetAsync(n->v, 0, sizeof(float) * kParams, s) != cudaSuccess) return VRM_ERR_CUDA;
  if (refresh(n, s) != cudaSuccess) return VRM_ERR_CUDA;
  return VRM_OK;
}

vrm_status vrm_mlp_get_params(const vrm_mlp* n, float* theta, cudaStream_t s) {
  if (!n || !theta) return VRM_ERR_ARG;
  if (cudaMemcpyAsync(theta, n->theta, sizeof(float) * kParams, cudaMemcpyDefault, s) != cudaSuccess)
    return VRM_ERR_CUDA;
  return VRM_OK;
}

vrm_status vrm_mlp_forward(vrm_mlp* n, const uint16_t* X, int32_t rows, float* Y, cudaStream_t s) {
  if (!n || rows < 0 || (rows > 0 && (!X || !Y)) || ((uintptr_t)X & 15u)) return VRM_ERR_ARG;
  if (rows == 0) return VRM_OK;
  const int rp = (rows + kBM - 1) / kBM * kBM;
  CUtensorMap mX;
  if (!vrm::mlp_input_map(&mX, reinterpret_cast<const bf16*>(X), rp)) return VRM_ERR_ARG;
  if (vrm::mlp_forward(n, mX, rows, nullptr, Y, s) != cudaSuccess) return VRM_ERR_CUDA;
  return check_err(n, s);
}

vrm_status vrm_mlp_grads(vrm_mlp* n, const uint16_t* X, const float* T, int32_t rows, float* grad, float* loss,
                         cudaStream_t s) {
  if (!n || !X || !T || rows < 1 || rows > n->B) return VRM_ERR_ARG;
  if (gather(n, reinterpret_cast<const bf16*>(X), T, nullptr, rows, s) != cudaSuccess) return VRM_ERR_CUDA;
  if (forward_backward(n, s) != cudaSuccess) return VRM_ERR_CUDA;
  if (grad && cudaMemcpyAsync(grad, n->grad, sizeof(float) * kParams, cudaMemcpyDefault, s) != cudaSuccess)
    return VRM_ERR_CUDA;
  if (loss && cudaMemcpyAsync(loss, n->loss, sizeof(float) * 2, cudaMemcpyDefault, s) != cudaSuccess)
    return VRM_ERR_CUDA;
  return check_err(n, s);
}

vrm_status vrm_mlp_train_step(vrm_mlp* n, const uint16_t* X_all, const float* T_all, const int32_t* batch_idx,
                              int32_t rows, const vrm_adamw* hp, int32_t t, float* loss, cudaStream_t s) {
  if (!n || !X_all || !T_all || rows < 1 || rows > n->B || t < 1 || !adamw_ok(hp)) return VRM_ERR_ARG;
  if (gather(n, reinterpret_cast<const bf16*>(X_all), T_all, batch_idx, rows, s) != cudaSuccess) return VRM_ERR_CUDA;
  if (forward_backward(n, s) != cudaSuccess) return VRM_ERR_CUDA;
  if (loss && cudaMemcpyAsync(loss, n->loss, sizeof(float) * 2, cudaMemcpyDefault, s) != cudaSuccess)
    return VRM_ERR_CUDA;
  return run_adamw(n, n->grad, hp, t, s);
}

vrm_status vrm_mlp_adamw(vrm_mlp* n, const float* grad, const vrm_adamw* hp, int32_t t, cudaStream_t s) {
  if (!n || !grad || t < 1 || !adamw_ok(hp)) return VRM_ERR_ARG;
  return run_adamw(n, grad, hp, t, s);
}

vrm_status vrm_mlp_error(vrm_mlp* n, cudaStream_t s) {
  if (!n) return VRM_ERR_ARG;
  return check_err(n, s);
}

}  // extern "C"
