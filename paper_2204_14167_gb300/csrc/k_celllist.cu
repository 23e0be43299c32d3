// Cell list for the near-field neighbour sets of Sec. II.B.1 (Eq. fullElectro):
// binning by the integer rule cell = min(floor(x) div k, nc - 1), a
// warp-aggregated counting sort (histogram, exclusive scan, scatter), a
// per-cell sort by ion index that makes the order deterministic, and a gather
// of the ions into cell order.
#include <mutex>
#include "physics.cuh"

namespace discos {

namespace {

constexpr int kScanTile = 1024;

// x and z are periodic: a position outside [0, L) is binned where its
// periodic image inside the box lies (the sorted copies hold that image).
template <typename T>
__global__ void k_bin(const T* __restrict__ x, int N, Params P, int* __restrict__ cell_of,
                      int* __restrict__ counts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int cid = -1;
  if (i < N) {
    const T px = wrap_coord(x[i], P.Nx), py = x[N + i], pz = wrap_coord(x[2 * N + i], P.Nz);
    int cx = cell_coord(px, P.k_cell, P.ncx);
    int cy = cell_coord(py, P.k_cell, P.ncy);
    int cz = cell_coord(pz, P.k_cell, P.ncz);
    cid = (cz * P.ncy + cy) * P.ncx + cx;
    cell_of[i] = cid;
    // positions that would pile into the edge cells are flagged here, before
    // the per-cell work that such a pile-up would make quadratic
    if (P.fault) {
      if (!(isfinite(px) && isfinite(py) && isfinite(pz))) atomicOr(P.fault, 1u);
      else if (py < T(0) || py > T(P.Ny)) atomicOr(P.fault, 2u);
    }
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

__global__ void k_sort_cells(const int* __restrict__ start, int n_cells, int* __restrict__ perm,
                             const unsigned* __restrict__ fault = nullptr) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  // a flagged run may have every ion in one cell: the order no longer matters
  if (fault && *reinterpret_cast<const volatile unsigned*>(fault)) return;
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
  probe_begin(PROBE_CELL_LIST, s);
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
  k_sort_cells<<<(n + 255) / 256, 256, 0, s>>>(W.cell_start, n, W.perm, P.fault);
  count_launches(1);
  probe_end(PROBE_CELL_LIST, s);
  return cudaGetLastError();
}

template cudaError_t launch_cell_list<float>(const Params&, Workspace&, const float*, int, cudaStream_t);
template cudaError_t launch_cell_list<double>(const Params&, Workspace&, const double*, int, cudaStream_t);

}  // namespace discos

// ---------------------------------------------------------------------------
// Allocation-free cell list.
//
// Some callers cannot allocate device memory when they need a cell list: code
// that runs while its stream is being captured into a CUDA graph (an
// allocation there is either illegal or escapes the graph), code embedded in a
// host framework whose caching allocator has already reserved the device
// memory, and fixed-latency loops that are not allowed to call into the
// allocator at all.  For them discos_cell_list_noalloc builds the same cell
// list as discos_cell_list without a handle and without any allocation: its
// scratch (per-ion cell ids, per-cell counts and fill counters, scan tile sums)
// lives in the file-scope device array below, which every GPU that loads this
// library holds until the process exits.
namespace discos {

namespace {

constexpr int kNoAllocMaxIons = 1 << 20;      // ions per call
constexpr int kNoAllocMaxCells = 1 << 18;     // list cells per call
constexpr int kNoAllocMaxTiles = kNoAllocMaxCells / kScanTile + 1;
// cell ids, counts, fill counters, scan tile sums, and one fault word
constexpr size_t kNoAllocInts = (size_t)kNoAllocMaxIons + 2 * (size_t)kNoAllocMaxCells + kNoAllocMaxTiles + 1;

static __device__ __align__(256) int g_noalloc_scratch[kNoAllocInts];

constexpr int kMaxDevices = 64;
int* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

}  // namespace

}  // namespace discos

extern "C" discos_status discos_cell_list_noalloc(const discos_config* cfg, const void* x, int N, int* cell_start,
                                                  int* perm, int* n_cells_out, void* stream) {
  using namespace discos;
  if (!cfg) {
    set_error("discos_cell_list_noalloc: null config");
    return DISCOS_ERR_INVALID_ARG;
  }
  const discos_config& c = *cfg;
  if (c.Nx < 1 || c.Ny < 1 || c.Nz < 1 || !(c.psi > 0.0) || c.nspecies < 1 || c.nspecies > DISCOS_MAX_SPECIES ||
      (c.precision != DISCOS_FP64 && c.precision != DISCOS_MIXED)) {
    set_error("discos_cell_list_noalloc: bad configuration");
    return DISCOS_ERR_INVALID_ARG;
  }
  double rcmax = c.psi;
  for (int a = 0; a < c.nspecies; ++a)
    for (int b = 0; b < c.nspecies; ++b) rcmax = rcmax > c.lj_rc[a][b] ? rcmax : c.lj_rc[a][b];
  int k = (int)ceil(rcmax - 1e-12);
  if (k < 1) k = 1;
  Params P{};
  P.Nx = c.Nx;
  P.Ny = c.Ny;
  P.Nz = c.Nz;
  P.k_cell = k;
  P.ncx = c.Nx / k;
  P.ncy = c.Ny / k > 1 ? c.Ny / k : 1;
  P.ncz = c.Nz / k;
  if (P.ncx < 1 || P.ncz < 1) {
    set_error("discos_cell_list_noalloc: cutoff larger than the box");
    return DISCOS_ERR_INVALID_ARG;
  }
  const long long n_cells = (long long)P.ncx * P.ncy * P.ncz;
  if (n_cells_out) *n_cells_out = (int)(n_cells <= kNoAllocMaxCells ? n_cells : -1);
  if (N < 0 || N > kNoAllocMaxIons || n_cells > kNoAllocMaxCells) {
    set_error("discos_cell_list_noalloc: at most 1048576 ions and 262144 list cells per call");
    return DISCOS_ERR_INVALID_ARG;
  }
  if ((N > 0 && (!x || !perm)) || !cell_start) {
    set_error("discos_cell_list_noalloc: null pointer");
    return DISCOS_ERR_INVALID_ARG;
  }
  // one-time set-up per device: the device address of the scratch array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "discos_cell_list_noalloc");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("discos_cell_list_noalloc: device index out of range");
    return DISCOS_ERR_INVALID_ARG;
  }
  int* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_status(e, "discos_cell_list_noalloc: cudaGetSymbolAddress");
      g_noalloc_ptr[dev] = static_cast<int*>(ptr);
    }
    base = g_noalloc_ptr[dev];
  }
  int* cell_of = base;
  int* counts = cell_of + kNoAllocMaxIons;
  int* fill = counts + kNoAllocMaxCells;
  int* tile_sums = fill + kNoAllocMaxCells;
  // positions that are not finite or leave the channel in y set this word in
  // the binning; the per-cell sort then stands down (such ions can all share
  // one cell, which would make it quadratic)
  unsigned* fault = reinterpret_cast<unsigned*>(tile_sums + kNoAllocMaxTiles);
  P.fault = fault;
  const int n = (int)n_cells;
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear what must start at zero
  e = cudaMemsetAsync(counts, 0, sizeof(int) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fill, 0, sizeof(int) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(fault, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_status(e, "discos_cell_list_noalloc");
  const int bs = 256;
  const int nb = (N + bs - 1) / bs;
  const int ntiles = (n + kScanTile - 1) / kScanTile;
  if (nb > 0) {
    if (c.precision == DISCOS_MIXED) k_bin<float><<<nb, bs, 0, s>>>((const float*)x, N, P, cell_of, counts);
    else k_bin<double><<<nb, bs, 0, s>>>((const double*)x, N, P, cell_of, counts);
    count_launches(1);
  }
  k_tile_sums<<<ntiles, 256, 0, s>>>(counts, n, tile_sums);
  k_scan_tiles<<<1, 1024, 0, s>>>(tile_sums, ntiles);
  k_scan_apply<<<ntiles, kScanTile, 0, s>>>(counts, n, tile_sums, cell_start, N);
  count_launches(3);
  if (nb > 0) {
    k_scatter<<<nb, bs, 0, s>>>(cell_of, N, cell_start, fill, perm);
    count_launches(1);
  }
  k_sort_cells<<<(n + 255) / 256, 256, 0, s>>>(cell_start, n, perm, fault);
  count_launches(1);
  return cuda_status(cudaGetLastError(), "discos_cell_list_noalloc");
}
