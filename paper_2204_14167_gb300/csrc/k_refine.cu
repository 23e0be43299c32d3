// Double-precision reductions: the residual refinement of the mixed-precision
// Poisson solve, and the run diagnostics (charge, neutrality, momentum).
//
// Residual refinement of the mixed-precision Poisson solve.  The residual of
// Eq. poisson with the ghost-cell rows of Eqs. esbc1 / esbc3,
//     r = 4 pi lB rho + lap_h phi,
// is formed in double from the single-precision rho and phi (one rounding of
// phi's neighbours at most per term), written back in the working precision
// for the correction solve, and its squared norm, with that of the right-hand
// side b = 4 pi lB rho + ghost terms, summed in double.
#include "internal.h"

namespace discos {

namespace {

template <typename T>
__global__ void k_poisson_residual(Params P, const T* __restrict__ rho, const T* __restrict__ phi, T* __restrict__ res,
                                   double* __restrict__ norms) {
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const size_t G = (size_t)Nx * Ny * Nz;
  const double c = 4.0 * M_PI * P.lB;
  double rr = 0.0, bb = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < G; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Nx);
    const int y = (int)((i / Nx) % Ny);
    const int z = (int)(i / ((size_t)Nx * Ny));
    const double p = (double)phi[i];
    const size_t row = i - x;
    double lap = (double)phi[row + ((x + 1) & (Nx - 1))] + (double)phi[row + ((x - 1) & (Nx - 1))];
    const size_t plane = (size_t)Nx * Ny;
    const size_t zp = ((size_t)((z + 1) & (Nz - 1))) * plane, zm = ((size_t)((z - 1) & (Nz - 1))) * plane;
    const size_t off = i - (size_t)z * plane;
    lap += (double)phi[zp + off] + (double)phi[zm + off];
    double b = c * (double)rho[i];
    double ym, yp;
    if (y > 0) {
      ym = (double)phi[i - Nx];
    } else if (P.bc[0] == DISCOS_BC_DIRICHLET) {
      ym = 2.0 * P.phi_b[0] - p;
      b += 2.0 * P.phi_b[0];
    } else {
      ym = p - P.slope[0];
      b -= P.slope[0];
    }
    if (y < Ny - 1) {
      yp = (double)phi[i + Nx];
    } else if (P.bc[1] == DISCOS_BC_DIRICHLET) {
      yp = 2.0 * P.phi_b[1] - p;
      b += 2.0 * P.phi_b[1];
    } else {
      yp = p + P.slope[1];
      b += P.slope[1];
    }
    lap += ym + yp - 6.0 * p;
    const double r = c * (double)rho[i] + lap;
    if (res) res[i] = (T)r;
    rr += r * r;
    bb += b * b;
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    bb += __shfl_xor_sync(0xffffffffu, bb, o);
  }
  __shared__ double red[2][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][wid] = rr; red[1][wid] = bb; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    rr = lane < nw ? red[0][lane] : 0.0;
    bb = lane < nw ? red[1][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      rr += __shfl_xor_sync(0xffffffffu, rr, o);
      bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if (lane == 0) {
      atomicAdd(&norms[0], rr);
      atomicAdd(&norms[1], bb);
    }
  }
}

// out[0] += sum q, out[2..4] += sum F, out[5] += non-finite positions,
// out[6] += ions outside the channel; out[1] += sum rho (grid part, rho != 0).
template <typename T>
__global__ void k_diagnostics(Params P, const T* __restrict__ x, const T* __restrict__ q, const T* __restrict__ F,
                              int N, const T* __restrict__ rho, double* __restrict__ out) {
  double a[7] = {0, 0, 0, 0, 0, 0, 0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)N; i += stride) {
    const T px = x[i], py = x[N + i], pz = x[2 * N + i];
    a[0] += (double)q[i];
    if (F) {
      a[2] += (double)F[i];
      a[3] += (double)F[N + i];
      a[4] += (double)F[2 * N + i];
    }
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) a[5] += 1.0;
    else if (px < T(0) || px >= T(P.Nx) || py < T(0) || py > T(P.Ny) || pz < T(0) || pz >= T(P.Nz)) a[6] += 1.0;
  }
  if (rho) {
    const size_t G = (size_t)P.Nx * P.Ny * P.Nz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < G; i += stride) a[1] += (double)rho[i];
  }
  __shared__ double red[7][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
    if (lane == 0) red[k][wid] = a[k];
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      double v = lane < nw ? red[k][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && v != 0.0) atomicAdd(&out[k], v);
    }
  }
}

template <typename T>
__global__ void k_add_inplace(T* __restrict__ a, const T* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] += b[i];
}

}  // namespace

template <typename T>
cudaError_t launch_poisson_residual(const Params& P, const T* rho, const T* phi, T* res, double* norms,
                                    cudaStream_t s) {
  k_poisson_residual<T><<<152 * 8, 256, 0, s>>>(P, rho, phi, res, norms);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_inplace(T* a, const T* b, size_t n, cudaStream_t s) {
  k_add_inplace<T><<<152 * 8, 256, 0, s>>>(a, b, n);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diagnostics(const Params& P, const T* x, const T* q, const T* F, int N, const T* rho, double* out,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, 8 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_diagnostics<T><<<152 * 2, 256, 0, s>>>(P, x, q, F, N, rho, out);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_diagnostics<float>(const Params&, const float*, const float*, const float*, int, const float*, double*, cudaStream_t);
template cudaError_t launch_diagnostics<double>(const Params&, const double*, const double*, const double*, int, const double*, double*, cudaStream_t);
template cudaError_t launch_poisson_residual<float>(const Params&, const float*, const float*, float*, double*, cudaStream_t);
template cudaError_t launch_poisson_residual<double>(const Params&, const double*, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_add_inplace<float>(float*, const float*, size_t, cudaStream_t);
template cudaError_t launch_add_inplace<double>(double*, const double*, size_t, cudaStream_t);

}  // namespace discos
