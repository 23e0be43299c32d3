// Discrete electrostatic energy of the particle-mesh problem and its
// hand-written adjoint.
//
// With rho = S^es q (wall images included), phi the solution of Eq. poisson
// with the wall data, and phi^b the discrete lift of the wall data (the
// solution for rho = 0, a profile in y only),
//     U = (1/2) dV sum_j rho_j (phi_j + phi^b_j).
// The Poisson operator is self-adjoint, so dU/drho = phi and
//     dU/dq_i   = sum_j phi_j w_ij              (interpolation: adjoint of spreading)
//     dU/dx_i   = q_i sum_j phi_j grad_x w_ij    (gradient-kernel interpolation)
//     dU/dphi_b = sum_j rho_j e_b(y_j)           (e_b: lift of a unit wall potential)
// where w_ij are the spreading weights with the image fold.  The backward
// recomputes rho and phi instead of storing them.
#include "internal.h"

namespace discos {

namespace {

// sums[0] += U, sums[1] += sum rho e0, sums[2] += sum rho e1 (double)
template <typename T>
__global__ void k_energy_sums(const T* __restrict__ rho, const T* __restrict__ phi, const double* __restrict__ lift,
                              int Nx, int Ny, int Nz, double* __restrict__ sums) {
  // lift: [3][Ny] = (phi^b of the current wall data, e0, e1)
  __shared__ double red[3][32];
  const size_t G = (size_t)Nx * Ny * Nz;
  double u = 0.0, g0 = 0.0, g1 = 0.0;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < G; c += (size_t)gridDim.x * blockDim.x) {
    int j = (int)((c / Nx) % Ny);
    double r = (double)rho[c];
    u += r * ((double)phi[c] + lift[j]);
    g0 += r * lift[Ny + j];
    g1 += r * lift[2 * Ny + j];
  }
  for (int o = 16; o > 0; o >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, o);
    g0 += __shfl_xor_sync(0xffffffffu, g0, o);
    g1 += __shfl_xor_sync(0xffffffffu, g1, o);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][wid] = u; red[1][wid] = g0; red[2][wid] = g1; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    u = lane < nw ? red[0][lane] : 0.0;
    g0 = lane < nw ? red[1][lane] : 0.0;
    g1 = lane < nw ? red[2][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      u += __shfl_xor_sync(0xffffffffu, u, o);
      g0 += __shfl_xor_sync(0xffffffffu, g0, o);
      g1 += __shfl_xor_sync(0xffffffffu, g1, o);
    }
    if (lane == 0) {
      atomicAdd(&sums[0], 0.5 * u);
      atomicAdd(&sums[1], g0);
      atomicAdd(&sums[2], g1);
    }
  }
}

// dq_i = dU sum_p s_p w_p phi[mirror p];  dx_i = dU q_i sum_p s_p grad w_p phi[mirror p]
template <typename T>
__global__ void k_energy_grad(const T* __restrict__ x, const T* __restrict__ q, int N, Params P,
                              const T* __restrict__ phi, const double* __restrict__ dU, T* __restrict__ dx,
                              T* __restrict__ dq) {
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const KernelParams kp = P.kes;
  const int w = kp.w;
  int ion = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  int l = threadIdx.x & 7;
  int gbase = (threadIdx.x & 31) & ~7;
  bool valid = ion < N;
  T p[3] = {T(0.5), T(0.5), T(0.5)};
  if (valid) { p[0] = x[ion]; p[1] = x[N + ion]; p[2] = x[2 * N + ion]; }
  int st[3];
  T wv[3], wd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T s = p[d] - T(0.5);
    st[d] = stencil_start(s, w);
    T z = s - T(st[d] + l);
    wv[d] = l < w ? kval(z, kp) : T(0);
    wd[d] = l < w ? kder(z, kp) : T(0);
  }
  const T s0 = P.bc[0] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
  const T s1 = P.bc[1] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
  const int ix = (st[0] + l) & (Nx - 1);
  T a = T(0), gx = T(0), gy = T(0), gz = T(0);
  for (int jz = 0; jz < w; ++jz) {
    T wz = __shfl_sync(0xffffffffu, wv[2], gbase + jz);
    T dz = __shfl_sync(0xffffffffu, wd[2], gbase + jz);
    int iz = (st[2] + jz) & (Nz - 1);
    for (int jy = 0; jy < w; ++jy) {
      T wy = __shfl_sync(0xffffffffu, wv[1], gbase + jy);
      T dy = __shfl_sync(0xffffffffu, wd[1], gbase + jy);
      int iy = st[1] + jy;
      T sg = T(1);
      if (iy < 0) { iy = -1 - iy; sg = s0; }
      else if (iy >= Ny) { iy = 2 * Ny - 1 - iy; sg = s1; }
      if (valid && l < w && iy >= 0 && iy < Ny) {
        T v = sg * phi[((size_t)iz * Ny + iy) * Nx + ix];
        a += v * wv[0] * wy * wz;
        gx += v * wd[0] * wy * wz;
        gy += v * wv[0] * dy * wz;
        gz += v * wv[0] * wy * dz;
      }
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    gx += __shfl_xor_sync(0xffffffffu, gx, o);
    gy += __shfl_xor_sync(0xffffffffu, gy, o);
    gz += __shfl_xor_sync(0xffffffffu, gz, o);
  }
  if (valid && l == 0) {
    const T up = T(*dU);
    if (dq) dq[ion] = up * a;
    if (dx) {
      const T qq = q[ion];
      dx[ion] = up * qq * gx;
      dx[N + ion] = up * qq * gy;
      dx[2 * N + ion] = up * qq * gz;
    }
  }
}

__global__ void k_scale2(const double* __restrict__ sums, const double* __restrict__ dU, double* __restrict__ out) {
  if (threadIdx.x < 2) out[threadIdx.x] = (*dU) * sums[1 + threadIdx.x];
}

// The discrete lift phi^b and its derivatives by the two wall potentials,
// lift[3][Ny].  With the wall data uniform in x and z the lift is a
// function of y alone, and a linear profile satisfies both the 7-point
// Laplacian and the ghost-cell wall rows of Eqs. esbc1 / esbc3 exactly:
//   Dirichlet-Dirichlet  phi^b = phi_0 + (phi_1 - phi_0) y / Ny
//   Dirichlet-Neumann    phi^b = phi_0 + g_1 y
//   Neumann-Dirichlet    phi^b = phi_1 + g_0 (y - Ny)
// at cell centres y = j + 1/2 (g = dphi/dy on a Neumann wall).
__global__ void k_lift(Params P, double* __restrict__ lift) {
  const int Ny = P.Ny;
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) {
    const double y = j + 0.5, L = (double)Ny;
    double v, e0, e1;
    if (P.bc[0] == DISCOS_BC_DIRICHLET && P.bc[1] == DISCOS_BC_DIRICHLET) {
      e1 = y / L;
      e0 = 1.0 - e1;
      v = P.phi_b[0] * e0 + P.phi_b[1] * e1;
    } else if (P.bc[0] == DISCOS_BC_DIRICHLET) {
      e0 = 1.0; e1 = 0.0;
      v = P.phi_b[0] + P.slope[1] * y;
    } else {
      e0 = 0.0; e1 = 1.0;
      v = P.phi_b[1] + P.slope[0] * (y - L);
    }
    lift[j] = v;
    lift[Ny + j] = e0;
    lift[2 * Ny + j] = e1;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_energy_sums(const Params& P, const T* rho, const T* phi, const double* lift, double* sums,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sums, 0, 3 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_energy_sums<T><<<152 * 4, 256, 0, s>>>(rho, phi, lift, P.Nx, P.Ny, P.Nz, sums);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_energy_grad(const Params& P, const T* x, const T* q, int N, const T* phi, const double* dU, T* dx,
                               T* dq, cudaStream_t s) {
  if (N <= 0 || (!dx && !dq)) return cudaSuccess;
  int bs = 256;
  int nb = (int)(((size_t)N * 8 + bs - 1) / bs);
  k_energy_grad<T><<<nb, bs, 0, s>>>(x, q, N, P, phi, dU, dx, dq);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_lift(const Params& P, double* lift, cudaStream_t s) {
  k_lift<<<1, 256, 0, s>>>(P, lift);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale2(const double* sums, const double* dU, double* out, cudaStream_t s) {
  k_scale2<<<1, 32, 0, s>>>(sums, dU, out);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_energy_sums<float>(const Params&, const float*, const float*, const double*, double*, cudaStream_t);
template cudaError_t launch_energy_sums<double>(const Params&, const double*, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_energy_grad<float>(const Params&, const float*, const float*, int, const float*, const double*, float*, float*, cudaStream_t);
template cudaError_t launch_energy_grad<double>(const Params&, const double*, const double*, int, const double*, const double*, double*, double*, cudaStream_t);

}  // namespace discos
