// Batched step kernels for stencil width 6 (Ny = 16 and 32); the kernel is in k_batched.cuh.
#include "k_batched.cuh"

namespace discos {
namespace batched {
template cudaError_t launch_w<6>(const Params&, const BatchArgs&, int, size_t, cudaStream_t, bool);
}  // namespace batched
}  // namespace discos
