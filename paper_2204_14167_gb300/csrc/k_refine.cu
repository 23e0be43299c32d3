// Double-precision reductions: the residual refinement of the mixed-precision
// Poisson and Stokes solves, and the run diagnostics (charge, neutrality,
// momentum).
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

template <typename T, typename TP>
__global__ void k_poisson_residual(Params P, const T* __restrict__ rho, const TP* __restrict__ phi, T* __restrict__ res,
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

// out[0] += sum v, out[1] += sum |v| in double (v: charges, or a charge
// density on the cells).
template <typename T>
__global__ void k_charge_sums(const T* __restrict__ v, size_t n, double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double t = (double)v[i];
    a += t;
    b += fabs(t);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __shared__ double red[2][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][wid] = a; red[1][wid] = b; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    a = lane < nw ? red[0][lane] : 0.0;
    b = lane < nw ? red[1][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      atomicAdd(&out[0], a);
      atomicAdd(&out[1], b);
    }
  }
}

// Neutrality of a channel between two Neumann walls (Sec. II.B.1): sets bit 2
// of the fault word when |sum q + surface| > tol (sum |q| + |surface|).
__global__ void k_neutral_flag(const double* __restrict__ sums, double surface, double surface_abs, double tol,
                               unsigned* __restrict__ fault) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && fault) {
    if (!(fabs(sums[0] + surface) <= tol * (sums[1] + surface_abs) + 1e-12)) atomicOr(fault, 4u);
  }
}

// Residual of the staggered Stokes system of Eq. disc_stokes with the
// no-slip walls of Eq. fluidbc, in double, for a velocity and pressure held
// in double:  r = f - (eta L v + G p)  on every face (the wall rows of v take
// none), L = -lap_h with the tangential ghost -u(0) below a no-slip wall,
// +u(0) below a slip wall, and v = 0 on the wall faces.  res receives r in the working precision; norms gets
// (sum r^2, sum f^2).
template <typename T>
__global__ void k_stokes_residual(Params P, const T* __restrict__ f, const double* __restrict__ v,
                                  const double* __restrict__ p, T* __restrict__ res, double* __restrict__ norms) {
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const size_t G = (size_t)Nx * Ny * Nz, Gv = (size_t)Nx * (Ny + 1) * Nz;
  const size_t n = 2 * G + Gv;
  const double eta = P.eta;
  double rr = 0.0, bb = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i < G ? 0 : (i < G + Gv ? 1 : 2);
    const size_t off = c == 0 ? 0 : (c == 1 ? G : G + Gv);
    const size_t k = i - off;
    const int Nyg = c == 1 ? Ny + 1 : Ny;
    const int x = (int)(k % Nx), y = (int)((k / Nx) % Nyg), z = (int)(k / ((size_t)Nx * Nyg));
    const double* a = v + off;
    const size_t row = k - x, plane = (size_t)Nx * Nyg;
    const size_t zo = k - (size_t)z * plane;
    const double fa = (double)f[i];
    double r = 0.0;
    const double ac = a[k];
    double lap = 6.0 * ac - a[row + ((x + 1) & (Nx - 1))] - a[row + ((x - 1) & (Nx - 1))] -
                 a[(size_t)((z + 1) & (Nz - 1)) * plane + zo] - a[(size_t)((z - 1) & (Nz - 1)) * plane + zo];
    if (c == 1) {
      if (y >= 1 && y < Ny) {
        lap -= a[k - Nx] + a[k + Nx];     // the wall faces hold v = 0
        const size_t pc = ((size_t)z * Ny + y) * Nx + x;
        r = fa - (eta * lap + (p[pc] - p[pc - Nx]));
      }
    } else {
      lap -= y > 0 ? a[k - Nx] : (P.slip[0] ? ac : -ac);           // ghost -+u(0): no slip / slip
      lap -= y < Ny - 1 ? a[k + Nx] : (P.slip[1] ? ac : -ac);
      const size_t pc = ((size_t)z * Ny + y) * Nx + x;
      const double gp = c == 0 ? p[pc] - p[row + ((x - 1) & (Nx - 1))]
                               : p[pc] - p[(size_t)((z - 1) & (Nz - 1)) * ((size_t)Nx * Ny) + (size_t)y * Nx + x];
      r = fa - (eta * lap + gp);
    }
    if (res) res[i] = (T)r;
    rr += r * r;
    bb += fa * fa;
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

// acc += d (accumulator in double), and dst = src converted.
template <typename T>
__global__ void k_accumulate(double* __restrict__ acc, const T* __restrict__ d, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc[i] += (double)d[i];
}
template <typename TD, typename TS>
__global__ void k_convert(TD* __restrict__ dst, const TS* __restrict__ src, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (TD)src[i];
}

template <typename T>
__global__ void k_add_inplace(T* __restrict__ a, const T* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] += b[i];
}

}  // namespace

template <typename T, typename TP>
cudaError_t launch_poisson_residual(const Params& P, const T* rho, const TP* phi, T* res, double* norms,
                                    cudaStream_t s) {
  k_poisson_residual<T, TP><<<152 * 8, 256, 0, s>>>(P, rho, phi, res, norms);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stokes_residual(const Params& P, const T* f, const double* v, const double* p, T* res,
                                   double* norms, cudaStream_t s) {
  k_stokes_residual<T><<<152 * 8, 256, 0, s>>>(P, f, v, p, res, norms);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_accumulate(double* acc, const T* d, size_t n, cudaStream_t s) {
  k_accumulate<T><<<152 * 8, 256, 0, s>>>(acc, d, n);
  count_launches(1);
  return cudaGetLastError();
}

template <typename TD, typename TS>
cudaError_t launch_convert(TD* dst, const TS* src, size_t n, cudaStream_t s) {
  k_convert<TD, TS><<<152 * 8, 256, 0, s>>>(dst, src, n);
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

template <typename T>
cudaError_t launch_charge_sums(const T* v, size_t n, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess || n == 0) return e;
  size_t nb = (n + 255) / 256;
  k_charge_sums<T><<<(unsigned)(nb < 152 * 4 ? nb : 152 * 4), 256, 0, s>>>(v, n, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_neutral_flag(const double* sums, double surface, double surface_abs, double tol, unsigned* fault,
                                cudaStream_t s) {
  k_neutral_flag<<<1, 32, 0, s>>>(sums, surface, surface_abs, tol, fault);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_charge_sums<float>(const float*, size_t, double*, cudaStream_t);
template cudaError_t launch_charge_sums<double>(const double*, size_t, double*, cudaStream_t);
template cudaError_t launch_diagnostics<float>(const Params&, const float*, const float*, const float*, int, const float*, double*, cudaStream_t);
template cudaError_t launch_diagnostics<double>(const Params&, const double*, const double*, const double*, int, const double*, double*, cudaStream_t);
template cudaError_t launch_poisson_residual<float, float>(const Params&, const float*, const float*, float*, double*, cudaStream_t);
template cudaError_t launch_poisson_residual<float, double>(const Params&, const float*, const double*, float*, double*, cudaStream_t);
template cudaError_t launch_poisson_residual<double, double>(const Params&, const double*, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_stokes_residual<float>(const Params&, const float*, const double*, const double*, float*, double*, cudaStream_t);
template cudaError_t launch_stokes_residual<double>(const Params&, const double*, const double*, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_accumulate<float>(double*, const float*, size_t, cudaStream_t);
template cudaError_t launch_accumulate<double>(double*, const double*, size_t, cudaStream_t);
template cudaError_t launch_convert<double, float>(double*, const float*, size_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(float*, const double*, size_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(double*, const double*, size_t, cudaStream_t);
template cudaError_t launch_add_inplace<float>(float*, const float*, size_t, cudaStream_t);
template cudaError_t launch_add_inplace<double>(double*, const double*, size_t, cudaStream_t);

}  // namespace discos
