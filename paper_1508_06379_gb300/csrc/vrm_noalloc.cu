// vrm_build_neighbourhoods_noalloc: the neighbourhood search of
// vrm_build_neighbourhoods for callers that must not allocate memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need neighbourhoods: applications that hand all device memory to
// their own pool up front and forbid allocations afterwards (a host program
// that loads this library as a plug-in and owns every buffer), and real-time
// loops whose latency budget has no room for allocator calls, which can take
// milliseconds and synchronise the device.  This entry point needs no context
// and allocates nothing: its scratch (cell grid, sorted copies of the cloud,
// scan workspace) lives in one file-scope device array of fixed size, which
// every GPU that loads this library holds until the process exits.  The
// caller still passes the inputs and outputs.
#include <cstring>
#include <mutex>

#include "vrm_internal.cuh"

namespace {

// Largest cloud the static scratch holds, and the scratch itself.
constexpr int kNoAllocMaxN = VRM_NOALLOC_MAX_N;
constexpr long kNoAllocCells = 2L * kNoAllocMaxN + 1024;
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kScanInts = (size_t)((kNoAllocCells + 1023) / 1024) + 18;
constexpr size_t kScratchBytes =
    align256(sizeof(vrm::Grid)) + align256(sizeof(vrm::DevStats)) + align256(8 * sizeof(unsigned long long)) +
    2 * align256(sizeof(int) * kNoAllocMaxN) +           // cell_key, cell_rank
    align256(sizeof(int) * kNoAllocCells) +              // cell_count
    align256(sizeof(int) * (kNoAllocCells + 1)) +        // cell_start
    align256(sizeof(double2) * kNoAllocMaxN) +           // sorted_xy
    align256(sizeof(float2) * kNoAllocMaxN) +            // sorted_loc
    align256(sizeof(int) * kNoAllocMaxN) +               // sorted_idx
    align256(sizeof(int) * kScanInts);                   // scan workspace

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device (the host-side symbol is only
// a stand-in; the address must come from cudaGetSymbolAddress with that
// device current).
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return cudaSuccess;
}

template <typename T>
T* carve(unsigned char*& cur, size_t count) {
  T* p = reinterpret_cast<T*>(cur);
  cur += align256(sizeof(T) * count);
  return p;
}

}  // namespace

extern "C" vrm_status vrm_build_neighbourhoods_noalloc(const vrm_params* p, const double* x, const double* y,
                                                       int32_t n, int32_t* nbr_count, int32_t* nbr_idx,
                                                       uint8_t* seg_mask, int32_t* small, int32_t* max_count,
                                                       cudaStream_t stream) {
  if (!p || n < 0) return VRM_ERR_ARG;
  if (!(p->h > 0) || !(p->r > 0) || !(p->R > p->r) || p->k_cap < 8 || p->k_cap > VRM_KCAP_MAX) return VRM_ERR_ARG;
  if (n > kNoAllocMaxN) return VRM_ERR_CAPACITY;
  if (n > 0 && (!x || !y || !nbr_count || !nbr_idx || !seg_mask || !small)) return VRM_ERR_ARG;
  if (((uintptr_t)small & 15u) != 0) return VRM_ERR_ARG;
  unsigned char* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) return VRM_ERR_CUDA;
  if (n == 0) {
    if (max_count) *max_count = 0;
    return VRM_OK;
  }
  // the same derived constants as vrm_create
  vrm::Consts c;
  memset(&c, 0, sizeof(c));
  const double rh = p->r * p->h, Rh = p->R * p->h;
  c.h = p->h;
  c.inv_h = 1.0 / p->h;
  c.lo2 = rh * rh;
  c.hi2 = Rh * Rh;
  c.Rh = Rh;
  c.k_cap = p->k_cap;
  vrm::default_schedule(c);
  unsigned char* cur = base;
  vrm::Grid* grid = carve<vrm::Grid>(cur, 1);
  vrm::DevStats* ds = carve<vrm::DevStats>(cur, 1);
  unsigned long long* bbox = carve<unsigned long long>(cur, 8);
  int* cell_key = carve<int>(cur, kNoAllocMaxN);
  int* cell_rank = carve<int>(cur, kNoAllocMaxN);
  int* cell_count = carve<int>(cur, kNoAllocCells);
  int* cell_start = carve<int>(cur, kNoAllocCells + 1);
  double2* sorted_xy = carve<double2>(cur, kNoAllocMaxN);
  float2* sorted_loc = carve<float2>(cur, kNoAllocMaxN);
  int* sorted_idx = carve<int>(cur, kNoAllocMaxN);
  int* scan_tmp = carve<int>(cur, kScanInts);
  // the array keeps the previous call's contents: the counters start at zero
  if (cudaMemsetAsync(ds, 0, sizeof(vrm::DevStats), stream) != cudaSuccess) return VRM_ERR_CUDA;
  if (vrm::grid_build(x, y, n, c.Rh, c.lo2, c.hi2, (int)kNoAllocCells, grid, cell_key, cell_rank, cell_count,
                      cell_start, sorted_xy, sorted_loc, sorted_idx, bbox, scan_tmp, stream) != cudaSuccess)
    return VRM_ERR_CUDA;
  if (vrm::search_all(c, grid, cell_start, sorted_xy, sorted_loc, sorted_idx, n, nbr_count, nbr_idx, seg_mask, small,
                      ds, stream) != cudaSuccess)
    return VRM_ERR_CUDA;
  if (max_count) {
    vrm::DevStats h_ds;
    vrm::Grid h_grid;
    if (cudaMemcpyAsync(&h_ds, ds, sizeof(h_ds), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return VRM_ERR_CUDA;
    if (cudaMemcpyAsync(&h_grid, grid, sizeof(h_grid), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
      return VRM_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return VRM_ERR_CUDA;
    if (h_grid.nonfinite) return VRM_ERR_ARG;
    *max_count = h_ds.max_count;
    if (h_ds.max_count > p->k_cap) return VRM_ERR_CAPACITY;
  }
  return VRM_OK;
}
