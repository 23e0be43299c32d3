// Poisson solve with a metal strip in the dielectric bottom wall (Sec. IV.B,
// Fig. EOgeometry): a Dirichlet patch, phi_m(x) on the strip's cells, inside
// a Neumann wall (mixed conditions on one wall, Sec. II.B.1).
//
// The patch breaks the per-mode separability of the transform solver, but
// only along x: the strip spans the channel in z.  With B the separable
// operator of an all-dielectric bottom wall and U the strip's bottom cells,
// the true operator is A = B + 2 U U^T (a Dirichlet ghost row has diagonal
// +1 where the Neumann one has -1).  Capacitance (Woodbury) form, per z mode
// kz of the strip values:
//     phi = B^+ b - B^+ U sigma,   (I/2 + C_kz) sigma_kz = U^T (B^+ b)_kz,
// with C_kz = U^T B_kz^-1 U the response of the strip cells to unit sources
// on the strip cells, a small symmetric matrix per kz fixed by the grid and
// factored once on the host (discos.cu).  When the top wall is dielectric
// too, B is singular (constants): B^+ is the mean-zero solution (the
// transform solver projects the singular mode's right-hand side), and the
// kz = 0 system is bordered by the constant c of the potential and by the
// solvability condition sum sigma = sum b:
//     [I/2 + C_0   -1] [sigma_0]   [U^T (B^+ b)_0]
//     [ 1^T         0] [   c   ] = [    sum b    ]
// so phi = B^+ b - B^+ U sigma + c / Nz.  Two transform solves per Poisson
// solve, plus small per-kz matrix-vector products.
#include "internal.h"

namespace discos {

namespace {

// r[z][a] = phi[z][0][i0 + a]: the base solution on the strip cells.
template <typename T>
__global__ void k_strip_gather(const T* __restrict__ phi, Params P, double* __restrict__ r) {
  const int Ws = P.strip_i1 - P.strip_i0;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.Nz * Ws) return;
  const int z = t / Ws, a = t - z * Ws;
  r[t] = (double)phi[(size_t)z * P.Ny * P.Nx + P.strip_i0 + a];
}

// One block per kz: rhat = sum_z r[z] e^{-2 pi i kz z / Nz}, then
// sigma_hat = M_kz rhat (M stored [kz][Ws + 1][Ws + 1]); for the bordered
// kz = 0 system the extra entry of rhat is sum b = 4 pi lB sum rho + walls
// and the extra row of the product is the constant c.
__global__ void k_strip_solve(const double* __restrict__ r, const double* __restrict__ M, Params P,
                              const double* __restrict__ rho_sum, double walls, double2* __restrict__ shat,
                              double* __restrict__ cval) {
  extern __shared__ double2 rh[];
  const int Ws = P.strip_i1 - P.strip_i0, S = Ws + 1;
  const int Nz = P.Nz, kz = blockIdx.x;
  const bool border = P.strip_singular && kz == 0;
  for (int a = threadIdx.x; a < Ws; a += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int z = 0; z < Nz; ++z) {
      double sn, cs;
      sincospi(2.0 * (double)((kz * z) % Nz) / (double)Nz, &sn, &cs);
      const double v = r[(size_t)z * Ws + a];
      re += v * cs;
      im -= v * sn;
    }
    rh[a] = make_double2(re, im);
  }
  if (threadIdx.x == 0) rh[Ws] = make_double2(border ? 4.0 * M_PI * P.lB * rho_sum[0] + walls : 0.0, 0.0);
  __syncthreads();
  const double* Mk = M + (size_t)kz * S * S;
  const int rows = border ? S : Ws;
  for (int a = threadIdx.x; a < rows; a += blockDim.x) {
    double re = 0.0, im = 0.0;
    const int cols = border ? S : Ws;
    for (int b = 0; b < cols; ++b) {
      const double m = Mk[(size_t)a * S + b];
      re += m * rh[b].x;
      im += m * rh[b].y;
    }
    if (a < Ws) shat[(size_t)kz * Ws + a] = make_double2(re, im);
    else cval[0] = re;
  }
  if (kz == 0 && !border && threadIdx.x == 0) cval[0] = 0.0;
}

// The strip sources sigma(a, z) = (1/Nz) sum_kz sigma_hat e^{+2 pi i kz z / Nz}
// on the bottom row of the (zeroed) grid g.
template <typename T>
__global__ void k_strip_sources(const double2* __restrict__ shat, Params P, T* __restrict__ g) {
  const int Ws = P.strip_i1 - P.strip_i0;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.Nz * Ws) return;
  const int z = t / Ws, a = t - z * Ws, Nz = P.Nz;
  double acc = 0.0;
  for (int kz = 0; kz < Nz; ++kz) {
    double sn, cs;
    sincospi(2.0 * (double)((kz * z) % Nz) / (double)Nz, &sn, &cs);
    const double2 v = shat[(size_t)kz * Ws + a];
    acc += v.x * cs - v.y * sn;
  }
  g[(size_t)z * P.Ny * P.Nx + P.strip_i0 + a] = (T)(acc / (double)Nz);
}

// phi = phi_B - dphi + c / Nz
template <typename T>
__global__ void k_strip_combine(T* __restrict__ phi, const T* __restrict__ dphi, const double* __restrict__ cval,
                                size_t n, double inv_nz) {
  const double c = cval[0] * inv_nz;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    phi[i] = (T)((double)phi[i] - (double)dphi[i] + c);
}

}  // namespace

template <typename T>
cudaError_t poisson_pass(const Params& P, Workspace& W, const T* rho, T* phi, T scale, T add0, T add1,
                         cudaStream_t s, const T* add0x);

// Poisson solve with the strip (rho and phi may alias).
template <typename T>
cudaError_t launch_poisson_strip(const Params& P, Workspace& W, const T* rho, T* phi, T fourpi_lB, T add1,
                                 cudaStream_t s) {
  const size_t G = (size_t)P.Nx * P.Ny * P.Nz;
  const int Ws = P.strip_i1 - P.strip_i0;
  T* g = reinterpret_cast<T*>(W.strip_g);
  const T* add0x = reinterpret_cast<const T*>(W.strip_add0);
  cudaError_t e = cudaSuccess;
  if (P.strip_singular) e = launch_charge_sums<T>(rho, G, W.nsum, s);
  // base solve B^+ b, b with the strip's Dirichlet terms on its bottom cells
  if (e == cudaSuccess) e = poisson_pass<T>(P, W, rho, phi, fourpi_lB, T(0), add1, s, add0x);
  const int nt = P.Nz * Ws;
  if (e == cudaSuccess) {
    k_strip_gather<T><<<(nt + 255) / 256, 256, 0, s>>>(phi, P, W.strip_r);
    k_strip_solve<<<P.Nz, 128, (Ws + 1) * sizeof(double2), s>>>(W.strip_r, W.strip_M, P, W.nsum, P.strip_walls,
                                                                reinterpret_cast<double2*>(W.strip_shat),
                                                                W.strip_c);
    count_launches(2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_fill_zero<T>(g, G, s);
  if (e == cudaSuccess) {
    k_strip_sources<T><<<(nt + 255) / 256, 256, 0, s>>>(reinterpret_cast<const double2*>(W.strip_shat), P, g);
    count_launches(1);
    e = cudaGetLastError();
  }
  // B^+ U sigma: homogeneous wall data
  if (e == cudaSuccess) e = poisson_pass<T>(P, W, g, g, T(1), T(0), T(0), s, static_cast<const T*>(nullptr));
  if (e == cudaSuccess) {
    k_strip_combine<T><<<152 * 8, 256, 0, s>>>(phi, g, W.strip_c, G, 1.0 / (double)P.Nz);
    count_launches(1);
    e = cudaGetLastError();
  }
  return e;
}

template cudaError_t launch_poisson_strip<float>(const Params&, Workspace&, const float*, float*, float, float, cudaStream_t);
template cudaError_t launch_poisson_strip<double>(const Params&, Workspace&, const double*, double*, double, double, cudaStream_t);

}  // namespace discos
