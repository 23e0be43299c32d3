// Position updates of Sec. II.D.
//  * dry part of Eq. ions3 over one step (Euler-Maruyama):
//      dt (D^dry Gamma F / kT + div D^dry) + sqrt(2 dt D^dry Gamma) W,
//    with the near-wall tensor Gamma = (gamma^tot D^tot - gamma^wet D^wet) / D^dry
//    of Eqs. diff1-diff2 from the fit of Eq. fitfunction in the distance to the
//    nearest wall, and the Ito drift D^dry dGamma_perp/dy along y;
//  * plus, on the wet path, dt J(x*) v (Eq. step2);
//  * the midpoint predictor x* = x + dt/2 J(x) v of Eq. step1.
// Positions are wrapped in x, z and reflected specularly at the walls.
#include "physics.cuh"

namespace discos {

namespace {

template <typename T>
__global__ void k_dry_update(T* __restrict__ x, const int* __restrict__ species, const T* __restrict__ F,
                             const T* __restrict__ V, int N, Params P, long long step) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int sp = species ? species[i] : 0;
  T p[3] = {x[i], x[N + i], x[2 * N + i]};
  T W[4];
  normals4(u32x4{(uint32_t)i, (uint32_t)step, 0u, (uint32_t)TAG_DRY}, P.seed, W);
  const T f[3] = {F[i], F[N + i], F[2 * N + i]};
  T v[3] = {T(0), T(0), T(0)};
  if (V) { v[0] = V[i]; v[1] = V[N + i]; v[2] = V[2 * N + i]; }
  dry_move(P, sp, p, f, V ? v : nullptr, W);
  check_position(P, p);
  x[i] = p[0];
  x[N + i] = p[1];
  x[2 * N + i] = p[2];
}

template <typename T>
__global__ void k_midpoint(const T* __restrict__ x, const T* __restrict__ V, int N, T half_dt, T* __restrict__ xs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * N) return;
  xs[i] = x[i] + half_dt * V[i];
}

}  // namespace

template <typename T>
cudaError_t launch_dry_update(const Params& P, T* x, const int* species, const T* F, const T* V, int N,
                              int64_t step, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  probe_begin(PROBE_UPDATE, s);
  k_dry_update<T><<<(N + 127) / 128, 128, 0, s>>>(x, species, F, V, N, P, (long long)step);
  count_launches(1);
  probe_end(PROBE_UPDATE, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_midpoint(const Params& P, const T* x, const T* V, int N, T* xstar, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_midpoint<T><<<(3 * N + 255) / 256, 256, 0, s>>>(x, V, N, T(0.5 * P.dt), xstar);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_dry_update<float>(const Params&, float*, const int*, const float*, const float*, int, int64_t, cudaStream_t);
template cudaError_t launch_dry_update<double>(const Params&, double*, const int*, const double*, const double*, int, int64_t, cudaStream_t);
template cudaError_t launch_midpoint<float>(const Params&, const float*, const float*, int, float*, cudaStream_t);
template cudaError_t launch_midpoint<double>(const Params&, const double*, const double*, int, double*, cudaStream_t);

}  // namespace discos
