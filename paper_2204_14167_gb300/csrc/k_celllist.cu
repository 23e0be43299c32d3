// Cell list for the near-field neighbour sets of Sec. II.B.1 (Eq. fullElectro):
// binning by the integer rule cell = min(floor(x) div k, nc - 1), a
// warp-aggregated counting sort (histogram, exclusive scan, scatter), a
// per-cell sort by ion index that makes the order deterministic, and a gather
// of the ions into cell order.
#include "internal.h"

namespace discos {

namespace {

constexpr int kScanTile = 1024;

template <typename T>
__device__ __forceinline__ int cell_coord(T v, int k, int nc) {
  int c = (int)floor(v);
  c = c < 0 ? 0 : c / k;
  return c < nc ? c : nc - 1;
}

template <typename T>
__global__ void k_bin(const T* __restrict__ x, int N, Params P, int* __restrict__ cell_of,
                      int* __restrict__ counts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int cid = -1;
  if (i < N) {
    int cx = cell_coord(x[i], P.k_cell, P.ncx);
    int cy = cell_coord(x[N + i], P.k_cell, P.ncy);
    int cz = cell_coord(x[2 * N + i], P.k_cell, P.ncz);
    cid = (cz * P.ncy + cy) * P.ncx + cx;
    cell_of[i] = cid;
  }
  // warp aggregation: one atomic per distinct cell in the warp
  unsigned peers = __match_any_sync(0xffffffffu, cid);
  int leader = __ffs(peers) - 1;
  if (cid >= 0 && (int)lane_id() == leader) atomicAdd(&counts[cid], __popc(peers));
}

// Exclusive scan in three passes over tiles of kScanTile counts.
__global__ void k_tile_sums(const int* __restrict__ counts, int n, int* __restrict__ tile_sums) {
  __shared__ int red[32];
  int base = blockIdx.x * kScanTile;
  int s = 0;
  for (int t = threadIdx.x; t < kScanTile; t += blockDim.x) {
    int g = base + t;
    s += g < n ? counts[g] : 0;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane_id() == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = v;
  }
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024).
__device__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_tot[32];
  int lane = lane_id(), wid = threadIdx.x >> 5;
  int inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    int t = lane < nw ? warp_tot[lane] : 0;
    int ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == 31 && total) *total = ti;
  }
  __syncthreads();
  int r = inc - v + warp_tot[wid];
  __syncthreads();
  return r;
}

__global__ void k_scan_tiles(int* __restrict__ tile_sums, int ntiles) {
  __shared__ int total;
  int carry = 0;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    int t = base + threadIdx.x;
    int v = t < ntiles ? tile_sums[t] : 0;
    int ex = block_exclusive_scan(v, &total);
    if (t < ntiles) tile_sums[t] = ex + carry;
    __syncthreads();
    carry += total;
    __syncthreads();
  }
}

__global__ void k_scan_apply(const int* __restrict__ counts, int n, const int* __restrict__ tile_off,
                             int* __restrict__ start, int N) {
  // one thread per count, blockDim.x == kScanTile
  int g = blockIdx.x * kScanTile + threadIdx.x;
  int v = g < n ? counts[g] : 0;
  int ex = block_exclusive_scan(v, nullptr);
  if (g < n) start[g] = ex + tile_off[blockIdx.x];
  if (g == 0) start[n] = N;
}

__global__ void k_scatter(const int* __restrict__ cell_of, int N, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int cid = i < N ? cell_of[i] : -1;
  unsigned peers = __match_any_sync(0xffffffffu, cid);
  int leader = __ffs(peers) - 1;
  int lane = lane_id();
  int base = 0;
  if (cid >= 0 && lane == leader) base = atomicAdd(&fill[cid], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  int rank = __popc(peers & ((1u << lane) - 1u));
  if (cid >= 0) perm[start[cid] + base + rank] = i;
}

__global__ void k_sort_cells(const int* __restrict__ start, int n_cells, int* __restrict__ perm) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  int b = start[c], e = start[c + 1];
  for (int a = b + 1; a < e; ++a) {
    int v = perm[a];
    int j = a - 1;
    while (j >= b && perm[j] > v) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = v;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_cell_list(const Params& P, Workspace& W, const T* x, int N, cudaStream_t s) {
  int n = W.n_cells;
  cudaMemsetAsync(W.counts, 0, sizeof(int) * n, s);
  cudaMemsetAsync(W.fill, 0, sizeof(int) * n, s);
  int bs = 256;
  int nb = (N + bs - 1) / bs;
  if (nb > 0) {
    k_bin<T><<<nb, bs, 0, s>>>(x, N, P, W.cell_of, W.counts);
    count_launches(1);
  }
  int ntiles = (n + kScanTile - 1) / kScanTile;
  k_tile_sums<<<ntiles, 256, 0, s>>>(W.counts, n, W.tile_sums);
  count_launches(1);
  k_scan_tiles<<<1, 1024, 0, s>>>(W.tile_sums, ntiles);
  count_launches(1);
  k_scan_apply<<<ntiles, kScanTile, 0, s>>>(W.counts, n, W.tile_sums, W.cell_start, N);
  count_launches(1);
  if (nb > 0) {
    k_scatter<<<nb, bs, 0, s>>>(W.cell_of, N, W.cell_start, W.fill, W.perm);
    count_launches(1);
  }
  k_sort_cells<<<(n + 255) / 256, 256, 0, s>>>(W.cell_start, n, W.perm);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_cell_list<float>(const Params&, Workspace&, const float*, int, cudaStream_t);
template cudaError_t launch_cell_list<double>(const Params&, Workspace&, const double*, int, cudaStream_t);

}  // namespace discos
