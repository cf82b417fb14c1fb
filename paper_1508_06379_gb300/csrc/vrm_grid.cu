// Cell grid, scans and compaction for the VRM library.
//
// The neighbour search (Sec. 2, Eq. neighbourhood) runs on a uniform cell
// grid whose cell side is at least R h, so that the annulus of a particle lies
// in the 3 x 3 cells around it.  Particles are binned by a counting sort:
// an atomic count per cell gives every particle its rank inside its cell, an
// exclusive scan gives the cell starts, and a scatter writes positions and
// indices in cell order (row-major cells, so the three cells of one grid row
// are contiguous in memory).  The order inside a cell is not deterministic;
// no result depends on it (neighbour rows are sorted by index afterwards).
#include <atomic>

#include <cstddef>

#include "vrm_internal.cuh"

namespace vrm {

static int g_sm_count = 0;
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 1;
  }
  return g_sm_count;
}

int persistent_blocks(int block_threads, int per_sm) {
  (void)block_threads;
  return sm_count() * per_sm;
}

// ---- scans -------------------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
static_assert(kScanThreads * kScanItems == kScanTile, "scan tile");

size_t scan_tmp_ints(int n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 2; }

template <typename T>
__device__ __forceinline__ int load_count(const T* in, long i, int n) {
  return i < n ? (int)in[i] : 0;
}

// Block-wide exclusive scan of one int per thread; returns the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[kScanThreads / 32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  int r = incl - v + warp_sums[warp];
  __syncthreads();
  return r;
}

// Tile sums; tiles are visited grid-stride so that the grid can be sized by
// an upper bound while the count itself comes from device memory (n_dev).
template <typename T>
__global__ void k_tile_sums(const T* __restrict__ in, int n, const int* __restrict__ n_dev,
                            int* __restrict__ tile_sums) {
  if (n_dev) n = *n_dev;
  const int ntiles = (n + kScanTile - 1) / kScanTile;
  __shared__ int total;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    long base = (long)t * kScanTile + (long)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += load_count(in, base + k, n);
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) tile_sums[t] = total;
    __syncthreads();
  }
}

// Tile scan that forms each tile's exclusive prefix itself from the tile
// totals of k_tile_sums (no separate scan of the tile sums and no launch
// for it).  out[n] = the total.
template <typename T>
__global__ void k_tile_scan_fused(const T* __restrict__ in, int n, const int* __restrict__ n_dev,
                                  const int* __restrict__ tile_sums, int* __restrict__ out,
                                  int* __restrict__ total_out) {
  if (n_dev) n = *n_dev;
  const int ntiles = (n + kScanTile - 1) / kScanTile;
  __shared__ int total;
  if (ntiles == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = 0;
    if (total_out) *total_out = 0;
  }
  // a block's tiles ascend, so the prefix of tile t is carried forward from
  // the block's previous tile: every block reads the tile sums once in all
  int pre = 0, upto = 0;  // pre = sum of tile_sums[0 .. upto)
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int part = 0;
    for (int k = upto + threadIdx.x; k < t; k += kScanThreads) part += tile_sums[k];
    block_exclusive_scan(part, &total);
    pre += total;
    upto = t;
    long base = (long)t * kScanTile + (long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = load_count(in, base + k, n);
      s += v[k];
    }
    int ex = block_exclusive_scan(s, &total) + pre;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (base + k < n) out[base + k] = ex;
      ex += v[k];
    }
    if (t == ntiles - 1 && threadIdx.x == 0) {
      out[n] = pre + total;
      if (total_out) *total_out = pre + total;
    }
    __syncthreads();
  }
}

// Up to 8 blocks per SM: a scan of a million entries (about 1,300 tiles)
// then runs nearly one tile per block in one wave (two tiles per block in
// turn at 4 per SM cost about 0.5 us per scan).
static int scan_grid(int n_bound) {
  int ntiles = (n_bound + kScanTile - 1) / kScanTile;
  int cap = 8 * sm_count();
  return ntiles < 1 ? 1 : (ntiles < cap ? ntiles : cap);
}

template <typename T>
static cudaError_t scan_impl(const T* in, int* out, int n, const int* n_dev, int* tmp, cudaStream_t s,
                             int* total_out = nullptr) {
  if (!n_dev && n <= 0) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int), s);
    if (e == cudaSuccess && total_out) e = cudaMemsetAsync(total_out, 0, sizeof(int), s);
    return e;
  }
  const int g = scan_grid(n);
  k_tile_sums<T><<<g, kScanThreads, 0, s>>>(in, n, n_dev, tmp); note_launch();
  k_tile_scan_fused<T><<<g, kScanThreads, 0, s>>>(in, n, n_dev, tmp, out, total_out); note_launch();
  return cudaGetLastError();
}

cudaError_t scan_presummed_i32_dev(const int* in, int* out, int n_bound, const int* n_dev, const int* tile_sums,
                                   cudaStream_t s, int* total_out) {
  k_tile_scan_fused<int><<<scan_grid(n_bound), kScanThreads, 0, s>>>(in, n_bound, n_dev, tile_sums, out, total_out);
  note_launch();
  return cudaGetLastError();
}
cudaError_t scan_presummed_u8_dev(const uint8_t* in, int* out, int n_bound, const int* n_dev, const int* tile_sums,
                                  cudaStream_t s) {
  k_tile_scan_fused<uint8_t><<<scan_grid(n_bound), kScanThreads, 0, s>>>(in, n_bound, n_dev, tile_sums, out,
                                                                          nullptr);
  note_launch();
  return cudaGetLastError();
}

cudaError_t scan_exclusive_i32(const int* in, int* out, int n, int* tmp, cudaStream_t s) {
  return scan_impl<int>(in, out, n, nullptr, tmp, s);
}
cudaError_t scan_exclusive_u8(const uint8_t* in, int* out, int n, int* tmp, cudaStream_t s) {
  return scan_impl<uint8_t>(in, out, n, nullptr, tmp, s);
}
cudaError_t scan_exclusive_i32_dev(const int* in, int* out, int n_bound, const int* n_dev, int* tmp, cudaStream_t s,
                                   int* total_out) {
  return scan_impl<int>(in, out, n_bound, n_dev, tmp, s, total_out);
}
cudaError_t scan_exclusive_u8_dev(const uint8_t* in, int* out, int n_bound, const int* n_dev, int* tmp,
                                  cudaStream_t s) {
  return scan_impl<uint8_t>(in, out, n_bound, n_dev, tmp, s);
}

__global__ void k_compact(const uint8_t* __restrict__ flags, int n, const int* __restrict__ pos,
                          int* __restrict__ list, int* __restrict__ count) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (flags[i]) list[pos[i]] = (int)i;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = pos[n];
}

cudaError_t compact_flags(const uint8_t* flags, int n, int* list, int* count, int* pos, int* tmp, cudaStream_t s) {
  cudaError_t e = scan_exclusive_u8(flags, pos, n, tmp, s);
  if (e != cudaSuccess) return e;
  int blocks = n > 0 ? (n + kBlock - 1) / kBlock : 1;
  if (blocks > 8 * sm_count()) blocks = 8 * sm_count();
  k_compact<<<blocks, kBlock, 0, s>>>(flags, n, pos, list, count); note_launch();
  return cudaGetLastError();
}

// ---- grid ----------------------------------------------------------------------

__global__ void k_bbox_init(unsigned long long* bb) {
  bb[0] = ~0ull;  // min x (ordered)
  bb[1] = 0ull;   // max x
  bb[2] = ~0ull;  // min y
  bb[3] = 0ull;   // max y
  bb[4] = 0ull;   // non-finite flag
}

__global__ void k_bbox(const double* __restrict__ x, const double* __restrict__ y, int n, const int* __restrict__ n_dev,
                       unsigned long long* __restrict__ bb) {
  if (n_dev) n = *n_dev;
  unsigned long long mnx = ~0ull, mxx = 0, mny = ~0ull, mxy = 0;
  int bad = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double a = x[i], b = y[i];
    if (!isfinite(a) || !isfinite(b)) {
      bad = 1;
      continue;
    }
    unsigned long long oa = ordered_bits(a), ob = ordered_bits(b);
    mnx = oa < mnx ? oa : mnx;
    mxx = oa > mxx ? oa : mxx;
    mny = ob < mny ? ob : mny;
    mxy = ob > mxy ? ob : mxy;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t;
    t = __shfl_xor_sync(0xffffffffu, mnx, o);
    mnx = t < mnx ? t : mnx;
    t = __shfl_xor_sync(0xffffffffu, mxx, o);
    mxx = t > mxx ? t : mxx;
    t = __shfl_xor_sync(0xffffffffu, mny, o);
    mny = t < mny ? t : mny;
    t = __shfl_xor_sync(0xffffffffu, mxy, o);
    mxy = t > mxy ? t : mxy;
  }
  bad = __any_sync(0xffffffffu, bad);
  // one atomic per block and quantity (per-warp atomics on four addresses
  // serialise at L2)
  __shared__ unsigned long long w_mn[2][32], w_mx[2][32];
  __shared__ int w_bad[32];
  const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    w_mn[0][warp] = mnx;
    w_mx[0][warp] = mxx;
    w_mn[1][warp] = mny;
    w_mx[1][warp] = mxy;
    w_bad[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      mnx = w_mn[0][w] < mnx ? w_mn[0][w] : mnx;
      mxx = w_mx[0][w] > mxx ? w_mx[0][w] : mxx;
      mny = w_mn[1][w] < mny ? w_mn[1][w] : mny;
      mxy = w_mx[1][w] > mxy ? w_mx[1][w] : mxy;
      bad |= w_bad[w];
    }
    if (mnx != ~0ull) atomicMin(&bb[0], mnx);
    if (mxx) atomicMax(&bb[1], mxx);
    if (mny != ~0ull) atomicMin(&bb[2], mny);
    if (mxy) atomicMax(&bb[3], mxy);
    if (bad) atomicOr(&bb[4], 1ull);
  }
}

// Also puts the bounding-box accumulators back to their initial values once
// read, so that the next grid build may skip k_bbox_init.
__global__ void k_grid_finalize(unsigned long long* __restrict__ bb, int n, const int* __restrict__ n_dev,
                                double Rh, double lo2, double hi2, int ncell_cap, Grid* __restrict__ g) {
  if (n_dev) n = *n_dev;
  Grid G;
  G.nonfinite = (int)bb[4];
  double x0 = 0, x1 = 0, y0 = 0, y1 = 0;
  if (n > 0 && bb[0] != ~0ull) {
    x0 = from_ordered_bits(bb[0]);
    x1 = from_ordered_bits(bb[1]);
    y0 = from_ordered_bits(bb[2]);
    y1 = from_ordered_bits(bb[3]);
  }
  double cs = Rh * (1.0 + 1e-6);
  double w = x1 - x0, hgt = y1 - y0;
  // keep nx * ny within the cell capacity for very sparse clouds
  while ((floor(w / cs) + 1.0) * (floor(hgt / cs) + 1.0) > (double)ncell_cap) cs *= 2.0;
  G.x0 = x0;
  G.y0 = y0;
  G.inv_cs = 1.0 / cs;
  G.nx = (int)floor(w * G.inv_cs) + 1;
  G.ny = (int)floor(hgt * G.inv_cs) + 1;
  if ((long)G.nx * G.ny > ncell_cap) {  // rounding at the limit: enlarge once more
    G.inv_cs *= 0.5;
    G.nx = (int)floor(w * G.inv_cs) + 1;
    G.ny = (int)floor(hgt * G.inv_cs) + 1;
  }
  G.ncell = G.nx * G.ny;
  const double s2 = G.inv_cs * G.inv_cs;
  const float lo2c = (float)(lo2 * s2), hi2c = (float)(hi2 * s2);
  G.lo_out = lo2c - kBand;
  G.lo_in = lo2c + kBand;
  G.hi_in = hi2c - kBand;
  G.hi_out = hi2c + kBand;
  G.seg_eps = kSegEps;
  *g = G;
  bb[0] = ~0ull;
  bb[1] = 0ull;
  bb[2] = ~0ull;
  bb[3] = 0ull;
  bb[4] = 0ull;
}

// Keys and ranks of particles [n0, n1); with cell_ts the scan's tile sums
// of the cell counts are accumulated too.  Whole warps step through the
// particles (tile_sum_add needs every lane).
__device__ __forceinline__ void bin_range(const double* __restrict__ x, const double* __restrict__ y, long n0,
                                          long n1, const Grid& g, int* __restrict__ cell_key,
                                          int* __restrict__ cell_rank, int* __restrict__ cell_count,
                                          int* __restrict__ cell_ts) {
  const int lane = threadIdx.x & 31;
  for (long base = n0 + (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n1;
       base += (long)gridDim.x * blockDim.x) {
    const long i = base + lane;
    int key = -1;
    if (i < n1) {
      key = grid_cell_y(g, y[i]) * g.nx + grid_cell_x(g, x[i]);
      cell_key[i] = key;
      cell_rank[i] = atomicAdd(&cell_count[key], 1);
    }
    if (cell_ts) tile_sum_add(cell_ts, key, 1);
  }
}

__global__ void k_bin(const double* __restrict__ x, const double* __restrict__ y, int n, const int* __restrict__ n_dev,
                      const Grid* __restrict__ gp, int* __restrict__ cell_key, int* __restrict__ cell_rank,
                      int* __restrict__ cell_count, int* __restrict__ cell_ts) {
  if (n_dev) n = *n_dev;
  const Grid g = *gp;
  bin_range(x, y, 0, n, g, cell_key, cell_rank, cell_count, cell_ts);
}

__global__ void k_scatter(const double* __restrict__ x, const double* __restrict__ y, int n,
                          const int* __restrict__ n_dev, const Grid* __restrict__ gp,
                          const int* __restrict__ cell_key, const int* __restrict__ cell_rank,
                          const int* __restrict__ cell_start, double2* __restrict__ sorted_xy,
                          float2* __restrict__ sorted_loc, int* __restrict__ sorted_idx) {
  if (n_dev) n = *n_dev;
  const Grid g = *gp;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int key = cell_key[i];
    const int p = cell_start[key] + cell_rank[i];
    const double xi = x[i], yi = y[i];
    sorted_xy[p] = make_double2(xi, yi);
    sorted_loc[p] = make_float2(grid_local_x(g, xi, key % g.nx), grid_local_y(g, yi, key / g.nx));
    sorted_idx[p] = (int)i;
  }
}

static int stream_grid(int n_bound, int per_sm) {
  int b = n_bound > 0 ? (n_bound + kBlock - 1) / kBlock : 1;
  int cap = per_sm * sm_count();
  return b < cap ? b : cap;
}

cudaError_t grid_build_dev(const double* x, const double* y, int n_bound, const int* n_dev, double Rh, double lo2,
                           double hi2, int ncell_cap, Grid* g, int* cell_key, int* cell_rank, int* cell_count,
                           int* cell_start, double2* sorted_xy, float2* sorted_loc, int* sorted_idx,
                           unsigned long long* bbox_tmp, int* scan_tmp, cudaStream_t s, int* cell_ts,
                           bool bbox_ready, bool bbox_done) {
  if (!bbox_done) {
    if (!bbox_ready) {
      k_bbox_init<<<1, 1, 0, s>>>(bbox_tmp);
      note_launch();
    }
    k_bbox<<<stream_grid(n_bound, 4), kBlock, 0, s>>>(x, y, n_bound, n_dev, bbox_tmp); note_launch();
  }
  k_grid_finalize<<<1, 1, 0, s>>>(bbox_tmp, n_bound, n_dev, Rh, lo2, hi2, ncell_cap, g); note_launch();
  return grid_bin_dev(x, y, n_bound, n_dev, ncell_cap, g, cell_key, cell_rank, cell_count, cell_start, sorted_xy,
                      sorted_loc, sorted_idx, scan_tmp, s, cell_ts);
}

// Zeroes the counts of the grid's own cells (g->ncell of them, at most the
// capacity the buffers were sized for) and, when given, their tile sums.
__global__ void k_zero_cells(const Grid* __restrict__ g, int* __restrict__ cell_count, int* __restrict__ cell_ts) {
  const int m = g->ncell;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (long)gridDim.x * blockDim.x)
    cell_count[t] = 0;
  if (cell_ts)
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t <= m / kScanTile; t += (long)gridDim.x * blockDim.x)
      cell_ts[t] = 0;
}

cudaError_t grid_bin_dev(const double* x, const double* y, int n_bound, const int* n_dev, int ncell_cap, const Grid* g,
                         int* cell_key, int* cell_rank, int* cell_count, int* cell_start, double2* sorted_xy,
                         float2* sorted_loc, int* sorted_idx, int* scan_tmp, cudaStream_t s, int* cell_ts) {
  // only the grid's own cells (g->ncell, known on the device) are counted
  // and scanned, not the whole capacity: a cloud of spacing h has about
  // (extent / 2h)^2 cells, far fewer than the capacity's 2 per particle
  const int* ncell_dev = reinterpret_cast<const int*>(reinterpret_cast<const char*>(g) + offsetof(Grid, ncell));
  k_zero_cells<<<stream_grid(ncell_cap, 4), kBlock, 0, s>>>(g, cell_count, cell_ts); note_launch();
  const int b = stream_grid(n_bound, 8);
  k_bin<<<b, kBlock, 0, s>>>(x, y, n_bound, n_dev, g, cell_key, cell_rank, cell_count, cell_ts); note_launch();
  cudaError_t e = cell_ts ? scan_presummed_i32_dev(cell_count, cell_start, ncell_cap, ncell_dev, cell_ts, s)
                          : scan_exclusive_i32_dev(cell_count, cell_start, ncell_cap, ncell_dev, scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_scatter<<<b, kBlock, 0, s>>>(x, y, n_bound, n_dev, g, cell_key, cell_rank, cell_start, sorted_xy, sorted_loc,
                                 sorted_idx);
  note_launch();
  return cudaGetLastError();
}

// Particles [*n0_dev, *n1_dev) binned onto the counts of a grid that holds
// [0, *n0_dev) already (their ranks follow the ones there).
__global__ void k_bin_range(const double* __restrict__ x, const double* __restrict__ y,
                            const int* __restrict__ n0_dev, const int* __restrict__ n1_dev,
                            const Grid* __restrict__ gp, int* __restrict__ cell_key, int* __restrict__ cell_rank,
                            int* __restrict__ cell_count, int* __restrict__ cell_ts) {
  const Grid g = *gp;
  bin_range(x, y, *n0_dev, *n1_dev, g, cell_key, cell_rank, cell_count, cell_ts);
}

cudaError_t grid_extend_dev(const double* x, const double* y, int n_bound, const int* n0_dev, const int* n1_dev,
                            int ncell_cap, const Grid* g, int* cell_key, int* cell_rank, int* cell_count,
                            int* cell_start, double2* sorted_xy, float2* sorted_loc, int* sorted_idx, int* scan_tmp,
                            cudaStream_t s, int* cell_ts) {
  const int* ncell_dev = reinterpret_cast<const int*>(reinterpret_cast<const char*>(g) + offsetof(Grid, ncell));
  const int b = stream_grid(n_bound, 8);
  k_bin_range<<<b, kBlock, 0, s>>>(x, y, n0_dev, n1_dev, g, cell_key, cell_rank, cell_count, cell_ts); note_launch();
  cudaError_t e = cell_ts ? scan_presummed_i32_dev(cell_count, cell_start, ncell_cap, ncell_dev, cell_ts, s)
                          : scan_exclusive_i32_dev(cell_count, cell_start, ncell_cap, ncell_dev, scan_tmp, s);
  if (e != cudaSuccess) return e;
  k_scatter<<<b, kBlock, 0, s>>>(x, y, n_bound, n1_dev, g, cell_key, cell_rank, cell_start, sorted_xy, sorted_loc,
                                 sorted_idx);
  note_launch();
  return cudaGetLastError();
}

cudaError_t grid_bbox_reset(unsigned long long* bbox_tmp, cudaStream_t s) {
  k_bbox_init<<<1, 1, 0, s>>>(bbox_tmp);
  note_launch();
  return cudaGetLastError();
}

cudaError_t grid_build(const double* x, const double* y, int n, double Rh, double lo2, double hi2, int ncell_cap,
                       Grid* g, int* cell_key, int* cell_rank, int* cell_count, int* cell_start, double2* sorted_xy,
                       float2* sorted_loc, int* sorted_idx, unsigned long long* bbox_tmp, int* scan_tmp,
                       cudaStream_t s) {
  return grid_build_dev(x, y, n, nullptr, Rh, lo2, hi2, ncell_cap, g, cell_key, cell_rank, cell_count, cell_start,
                        sorted_xy, sorted_loc, sorted_idx, bbox_tmp, scan_tmp, s);
}

// list[k] = the k-th index with flag set; the count comes from n_dev.
__global__ void k_compact_dev(const uint8_t* __restrict__ flags, int n, const int* __restrict__ n_dev,
                              const int* __restrict__ pos, int* __restrict__ list, int* __restrict__ count) {
  if (n_dev) n = *n_dev;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (flags[i]) list[pos[i]] = (int)i;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = pos[n];
}

cudaError_t compact_flags_dev(const uint8_t* flags, int n_bound, const int* n_dev, int* list, int* count, int* pos,
                              int* tmp, cudaStream_t s, const int* flag_ts) {
  cudaError_t e = flag_ts ? scan_presummed_u8_dev(flags, pos, n_bound, n_dev, flag_ts, s)
                          : scan_exclusive_u8_dev(flags, pos, n_bound, n_dev, tmp, s);
  if (e != cudaSuccess) return e;
  k_compact_dev<<<stream_grid(n_bound, 8), kBlock, 0, s>>>(flags, n_bound, n_dev, pos, list, count); note_launch();
  return cudaGetLastError();
}

}  // namespace vrm
