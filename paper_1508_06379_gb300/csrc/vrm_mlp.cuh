// Inference side of the weight-proposal network (vrm_mlp.cu) as used by the
// step (vrm_api.cu): the input-row buffer with its tensor map, owned by the
// caller so that a captured graph keeps valid pointers (the activations stay
// in shared memory).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "vrm_internal.cuh"

namespace vrm {

struct MlpActs {
  int rows_pad = 0;            // rows the buffer holds (multiple of 128)
  __nv_bfloat16* X = nullptr;  // input rows [rows_pad x 128]
  CUtensorMap mX;
};

// Input rows for `rows` rows (rounded up to 128).
cudaError_t mlp_acts_alloc(MlpActs* a, int rows);
void mlp_acts_free(MlpActs* a);
// Tensor map of caller-owned input rows X [rows_pad x 128].
bool mlp_input_map(CUtensorMap* m, const __nv_bfloat16* X, int rows_pad);
// Y[rows x 32] = network(X) for rows_bound rows (or *rows_dev <= rows_bound);
// X (through its tensor map) holds rows_bound rounded up to 128 rows.
cudaError_t mlp_forward(vrm_mlp* net, const CUtensorMap& mX, int rows_bound, const int* rows_dev, float* Y,
                        cudaStream_t s);

// vrm_learned.cu
// Input rows and slot maps of the listed particles; xyf (n_bound entries)
// receives the fp32 positions first.
cudaError_t learned_features(const Consts& c, const double* x, const double* y, int n_bound, const int* n_dev,
                             float2* xyf, const int* list, const int* list_count, int m_bound, const int* nbr_count,
                             const int* nbr_idx, __nv_bfloat16* X, int* slots, cudaStream_t s);
// Scratch of the correction rounds: per listed particle the screened
// support, two work lists and the rounds' list sizes.
constexpr int kProjRounds = 7;
struct ProjScratch {
  int cap = 0;
  void* sel = nullptr;  // ProjSel[cap] (vrm_learned.cu)
  int* list_s = nullptr;  // the round's particles with a support to solve
  int* list_r = nullptr;  // the next round's particles (two, alternating)
  int* list_p = nullptr;
  int* counts = nullptr;  // [2 * kProjRounds]
};
cudaError_t proj_alloc(ProjScratch* p, int cap);
void proj_free(ProjScratch* p);
cudaError_t learned_project(const Consts& c, const double* x, const double* y, const int* list, const int* list_count,
                            int m_bound, const int* slots, const float* f0, const int* small, int* cols, double* f,
                            double* fii, uint8_t* status, int* reject_list, int* reject_count, DevStats* ds,
                            const double* dt_dev, double nu, ProjScratch* ps, cudaStream_t s);
cudaError_t learned_targets(const int* list, int m, const int* slots, const int* cols, const double* f, float* T,
                            cudaStream_t s);

}  // namespace vrm
