// Dispatch of the batched step (k_batched.cuh) by stencil width, its
// shared-memory size and the queue reset that starts a run.
#include "internal.h"

namespace discos {
namespace batched {
template <int W>
cudaError_t launch_w(const Params& P, const BatchArgs& B, int grid, size_t smem, cudaStream_t s, bool launch);
}  // namespace batched

namespace {

__global__ void k_batched_reset(int* queue, long long* dstep, long long step0) {
  queue[0] = 0;
  queue[1] = 0;
  *dstep = step0;
}

cudaError_t dispatch(const Params& P, const BatchArgs& B, int grid, cudaStream_t s, bool launch) {
  const size_t smem = batched_smem_bytes(P.Ny, B.n_cells, P.n_tab);
  if (P.kes.w == 4) return batched::launch_w<4>(P, B, grid, smem, s, launch);
  if (P.kes.w == 6) return batched::launch_w<6>(P, B, grid, smem, s, launch);
  return cudaErrorInvalidValue;
}

}  // namespace

size_t batched_smem_bytes(int Ny, int n_cells, int n_tab) {
  const size_t plane = 32 * 33, maxn = 512;
  return sizeof(float) * ((size_t)Ny * plane + 7 * maxn) + sizeof(int) * (3 * maxn + n_cells + 1) +
         sizeof(float) * (n_tab + 1);
}

bool batched_supported(const Params& P) { return (P.kes.w == 4 || P.kes.w == 6) && (P.Ny == 16 || P.Ny == 32); }

cudaError_t batched_prepare(const Params& P, int n_cells) {
  BatchArgs B{};
  B.n_cells = n_cells;
  return dispatch(P, B, 0, nullptr, false);
}

cudaError_t launch_batched_reset(int* queue, long long* dstep, long long step0, cudaStream_t s) {
  k_batched_reset<<<1, 1, 0, s>>>(queue, dstep, step0);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batched_step(const Params& P, const BatchArgs& B, int grid, cudaStream_t s) {
  cudaError_t e = dispatch(P, B, grid, s, true);
  count_launches(1);
  return e;
}

}  // namespace discos
