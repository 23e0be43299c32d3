// Position updates of Sec. II.D.
//  * dry part of Eq. ions3 over one step (Euler-Maruyama):
//      dt (D^dry Gamma F / kT + div D^dry) + sqrt(2 dt D^dry Gamma) W,
//    with the near-wall tensor Gamma = (gamma^tot D^tot - gamma^wet D^wet) / D^dry
//    of Eqs. diff1-diff2 from the fit of Eq. fitfunction in the distance to the
//    nearest wall, and the Ito drift D^dry dGamma_perp/dy along y;
//  * plus, on the wet path, dt J(x*) v (Eq. step2);
//  * the midpoint predictor x* = x + dt/2 J(x) v of Eq. step1.
// Positions are wrapped in x, z and reflected specularly at the walls.
#include "internal.h"

namespace discos {

namespace {

template <typename T>
__device__ __forceinline__ void fit_gamma(const double* c, T yt, T& g, T& dg) {
  T a3 = T(c[2]) + yt, a5 = T(c[4]) + yt, a7 = T(c[6]) + yt;
  T i3 = T(1) / a3, i5 = T(1) / a5, i7 = T(1) / a7;
  T i5_2 = i5 * i5, i7_2 = i7 * i7;
  g = T(c[0]) + T(c[1]) * i3 + T(c[3]) * i5_2 * i5 + T(c[5]) * i7_2 * i7_2 * i7;
  dg = -T(c[1]) * i3 * i3 - T(3) * T(c[3]) * i5_2 * i5_2 - T(5) * T(c[5]) * i7_2 * i7_2 * i7_2;
}

template <typename T>
__global__ void k_dry_update(T* __restrict__ x, const int* __restrict__ species, const T* __restrict__ F,
                             const T* __restrict__ V, int N, Params P, long long step) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int sp = species ? species[i] : 0;
  T p[3] = {x[i], x[N + i], x[2 * N + i]};
  const T Ny = T(P.Ny);
  const T y = p[1];
  const T yt = y <= Ny - y ? y : Ny - y;
  const T side = y <= Ny - y ? T(1) : T(-1);
  const T Dt = T(P.D_tot[sp]), Dw = T(P.D_wet[sp]), Dd = T(P.D_dry[sp]);
  T Gam[2], dGam[2];
  for (int dir = 0; dir < 2; ++dir) {
    T gt, dgt, gw, dgw;
    fit_gamma(P.gamma[sp][dir][0], yt, gt, dgt);
    fit_gamma(P.gamma[sp][dir][1], yt, gw, dgw);
    Gam[dir] = (gt * Dt - gw * Dw) / Dd;
    dGam[dir] = (dgt * Dt - dgw * Dw) / Dd * side;
  }
  T W[4];
  normals4(u32x4{(uint32_t)i, (uint32_t)step, 0u, (uint32_t)TAG_DRY}, P.seed, W);
  const T dt = T(P.dt), kT = T(P.kT);
  const int L[3] = {P.Nx, P.Ny, P.Nz};
  for (int d = 0; d < 3; ++d) {
    T G = d == 1 ? Gam[1] : Gam[0];
    T inc = dt * (Dd * G * F[(size_t)d * N + i] / kT);
    if (d == 1 && P.drift) inc += dt * Dd * dGam[1];
    inc += sqrt(T(2) * dt * Dd * (G > T(0) ? G : T(0))) * W[d];
    if (V) inc = dt * V[(size_t)d * N + i] + inc;
    T v = p[d] + inc;
    if (d == 1) {
      v = v < T(0) ? -v : (v > Ny ? T(2) * Ny - v : v);
    } else {
      T Ld = T(L[d]);
      v = v < T(0) ? v + Ld : (v >= Ld ? v - Ld : v);
    }
    x[(size_t)d * N + i] = v;
  }
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
