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

// Ion s of the input order (positions xin, forces F, velocities V, species)
// is ion index[s] of the caller's order (index NULL: the same order): its
// noise is keyed by that index and its new position written there.
template <typename T>
__global__ void k_dry_update(T* __restrict__ x, const T* __restrict__ xin, const int* __restrict__ species,
                             const T* __restrict__ F, const T* __restrict__ V, int N, Params P, long long step,
                             const int* __restrict__ index) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int i = index ? index[s] : s;
  const int sp = species ? species[s] : 0;
  T p[3] = {xin[s], xin[N + s], xin[2 * N + s]};
  T W[4];
  normals4(u32x4{(uint32_t)i, (uint32_t)step, 0u, (uint32_t)TAG_DRY}, P.seed, W);
  const T f[3] = {F[s], F[N + s], F[2 * N + s]};
  T v[3] = {T(0), T(0), T(0)};
  if (V) { v[0] = V[s]; v[1] = V[N + s]; v[2] = V[2 * N + s]; }
  dry_move(P, sp, p, f, V ? v : nullptr, W);
  check_position(P, p);
  x[i] = p[0];
  x[N + i] = p[1];
  x[2 * N + i] = p[2];
}

// dst[:, index[s]] = src[:, s] for the three rows of an ion array.
template <typename T>
__global__ void k_scatter3(const T* __restrict__ src, const int* __restrict__ index, int N, T* __restrict__ dst) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int i = index[s];
  dst[i] = src[s];
  dst[N + i] = src[N + s];
  dst[2 * N + i] = src[2 * N + s];
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
                              int64_t step, cudaStream_t s, const T* xin, const int* index) {
  if (N <= 0) return cudaSuccess;
  probe_begin(PROBE_UPDATE, s);
  k_dry_update<T><<<(N + 127) / 128, 128, 0, s>>>(x, xin ? xin : x, species, F, V, N, P, (long long)step, index);
  count_launches(1);
  probe_end(PROBE_UPDATE, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter3(const T* src, const int* index, int N, T* dst, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_scatter3<T><<<(N + 255) / 256, 256, 0, s>>>(src, index, N, dst);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_midpoint(const Params& P, const T* x, const T* V, int N, T* xstar, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  k_midpoint<T><<<(3 * N + 255) / 256, 256, 0, s>>>(x, V, N, T(0.5 * P.dt), xstar);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_dry_update<float>(const Params&, float*, const int*, const float*, const float*, int, int64_t, cudaStream_t, const float*, const int*);
template cudaError_t launch_dry_update<double>(const Params&, double*, const int*, const double*, const double*, int, int64_t, cudaStream_t, const double*, const int*);
template cudaError_t launch_scatter3<float>(const float*, const int*, int, float*, cudaStream_t);
template cudaError_t launch_scatter3<double>(const double*, const int*, int, double*, cudaStream_t);
template cudaError_t launch_midpoint<float>(const Params&, const float*, const float*, int, float*, cudaStream_t);
template cudaError_t launch_midpoint<double>(const Params&, const double*, const double*, int, double*, cudaStream_t);

}  // namespace discos
