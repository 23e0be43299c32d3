// Hand-written transforms along x and z and the Poisson solve of Eq. poisson
// with the wall conditions of Eqs. esbc1 / esbc3.
//
// x: real rows -> half spectra (Nx/2 + 1 modes, row pitch Px), two real rows
//    packed into one complex radix-2 transform held in shared memory.
// z: complex transforms down the columns of the half spectrum, a tile of 16
//    consecutive x-modes per block so that every load is a 16-element run.
// y: one thread per (kx, kz) mode solves the tridiagonal wall-normal system
//    in double precision with pre-factored pivots (Thomas algorithm).
#include "internal.h"

namespace discos {

namespace {

constexpr int kTileZ = 16;

__device__ __forceinline__ int bitrev(int v, int logN) {
  return logN == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - logN));
}

// In-place radix-2 decimation in time over `nvec` vectors of length N stored
// back to back in shared memory, input in bit-reversed order.  All threads of
// the block take part; ends with the block synchronised.
template <typename T>
__device__ void fft_smem(cplx<T>* buf, int N, int logN, int nvec, const cplx<T>* __restrict__ tw,
                         bool inverse) {
  const int hN = N >> 1;
  const int total = nvec * hN;
  for (int s = 1; s <= logN; ++s) {
    const int half = 1 << (s - 1);
    const int twstep = N >> s;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
      int v = b >> (logN - 1);
      int bb = b & (hN - 1);
      int grp = bb >> (s - 1);
      int pos = bb & (half - 1);
      int i0 = v * N + grp * 2 * half + pos;
      int i1 = i0 + half;
      cplx<T> wv = tw[pos * twstep];
      if (inverse) wv.im = -wv.im;
      cplx<T> u = buf[i0];
      cplx<T> t = cmul(wv, buf[i1]);
      buf[i0] = cadd(u, t);
      buf[i1] = csub(u, t);
    }
    __syncthreads();
  }
}

// Forward real transform of R rows of length N (two rows per complex FFT).
// Input value = scale * in + (row's y == 0 ? add0) + (row's y == Nyr-1 ? add1).
template <typename T>
__global__ void k_rfft_x(const T* __restrict__ in, int R, int N, int logN, int Px, cplx<T>* __restrict__ out,
                         T scale, int Nyr, T add0, T add1, const cplx<T>* __restrict__ tw, int pairs_per_block) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int PP = pairs_per_block;
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    int v = idx / N, n = idx - v * N;
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    T a = T(0), b = T(0);
    if (ra < R) {
      int y = ra % Nyr;
      a = scale * in[(size_t)ra * N + n] + (y == 0 ? add0 : T(0)) + (y == Nyr - 1 ? add1 : T(0));
    }
    if (rb < R) {
      int y = rb % Nyr;
      b = scale * in[(size_t)rb * N + n] + (y == 0 ? add0 : T(0)) + (y == Nyr - 1 ? add1 : T(0));
    }
    buf[v * N + bitrev(n, logN)] = cplx<T>{a, b};
  }
  __syncthreads();
  fft_smem(buf, N, logN, PP, tw, false);
  const int M = N / 2 + 1;
  for (int idx = threadIdx.x; idx < PP * M; idx += blockDim.x) {
    int v = idx / M, k = idx - v * M;
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    cplx<T> Zk = buf[v * N + (k & (N - 1))];
    cplx<T> Zn = buf[v * N + ((N - k) & (N - 1))];
    // A = (Z_k + conj Z_{N-k}) / 2,  B = (Z_k - conj Z_{N-k}) / (2i)
    cplx<T> A{T(0.5) * (Zk.re + Zn.re), T(0.5) * (Zk.im - Zn.im)};
    cplx<T> B{T(0.5) * (Zk.im + Zn.im), T(-0.5) * (Zk.re - Zn.re)};
    if (ra < R) out[(size_t)ra * Px + k] = A;
    if (rb < R) out[(size_t)rb * Px + k] = B;
  }
}

// Inverse of k_rfft_x (unnormalised): half spectra -> real rows times scale.
template <typename T>
__global__ void k_irfft_x(const cplx<T>* __restrict__ in, int R, int N, int logN, int Px, T* __restrict__ out,
                          T scale, const cplx<T>* __restrict__ tw, int pairs_per_block) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int PP = pairs_per_block;
  const int hN = N / 2;
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    int v = idx / N, k = idx - v * N;
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    int kk = k <= hN ? k : N - k;
    cplx<T> A{T(0), T(0)}, B{T(0), T(0)};
    if (ra < R) A = in[(size_t)ra * Px + kk];
    if (rb < R) B = in[(size_t)rb * Px + kk];
    if (k > hN) { A.im = -A.im; B.im = -B.im; }
    // Z = A + i B
    buf[v * N + bitrev(k, logN)] = cplx<T>{A.re - B.im, A.im + B.re};
  }
  __syncthreads();
  fft_smem(buf, N, logN, PP, tw, true);
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    int v = idx / N, n = idx - v * N;
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    cplx<T> z = buf[v * N + n];
    if (ra < R) out[(size_t)ra * N + n] = scale * z.re;
    if (rb < R) out[(size_t)rb * N + n] = scale * z.im;
  }
}

// Complex transform along z of the half spectra [Nz][Nyr][Px] (field f =
// blockIdx.z at offset f * field_stride), 16 x-modes per block.
// mac != 0: the three MAC fields u | v | w stored back to back with Ny, Ny+1
// and Ny rows per z-plane (Nyr = Ny is passed; grid.y = Ny + 1).
template <typename T>
__global__ void k_fft_z(cplx<T>* __restrict__ data, int Nz, int logNz, int Nyr, int Px, int Nxh, int inverse,
                        const cplx<T>* __restrict__ tw, size_t field_stride, int mac) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* base = data + blockIdx.z * field_stride;
  if (mac) {
    const int Ny = Nyr;
    if (blockIdx.z == 1) { base = data + (size_t)Nz * Ny * Px; Nyr = Ny + 1; }
    else if (blockIdx.z == 2) { base = data + (size_t)Nz * (2 * Ny + 1) * Px; }
    else { base = data; }
  }
  const int y = blockIdx.y;
  if (y >= Nyr) return;
  const int kx0 = blockIdx.x * kTileZ;
  for (int idx = threadIdx.x; idx < kTileZ * Nz; idx += blockDim.x) {
    int z = idx / kTileZ, c = idx - z * kTileZ;
    int kx = kx0 + c;
    cplx<T> v{T(0), T(0)};
    if (kx < Nxh) v = base[((size_t)z * Nyr + y) * Px + kx];
    buf[c * Nz + bitrev(z, logNz)] = v;
  }
  __syncthreads();
  fft_smem(buf, Nz, logNz, kTileZ, tw, inverse != 0);
  for (int idx = threadIdx.x; idx < kTileZ * Nz; idx += blockDim.x) {
    int z = idx / kTileZ, c = idx - z * kTileZ;
    int kx = kx0 + c;
    if (kx < Nxh) base[((size_t)z * Nyr + y) * Px + kx] = buf[c * Nz + z];
  }
}

// Wall-normal tridiagonal solve per (kx, kz) mode, double precision.
// Rows: (2 + lambda) phi_j - phi_{j-1} - phi_{j+1} = b_j with the wall rows
// modified by the ghost cells (+1 on the diagonal at a Dirichlet wall, -1 at a
// Neumann wall); inv_m [Ny][M] holds the reciprocal Thomas pivots.  One
// thread per (mode, part): the matrix is real, so the real and imaginary
// parts are independent systems.  Forward values go to a private slot of the
// double scratch Y [Ny][threads].  The (0, 0) mode of a channel with two
// Neumann walls is singular: there phi_0 = 0, the last equation (redundant
// for a neutral system) is dropped, and the mean is removed afterwards.
template <typename T>
__global__ void k_poisson_y(cplx<T>* __restrict__ S, const double* __restrict__ inv_m, int Ny, int Nz, int Nxh,
                            int Px, int singular, double norm, double* __restrict__ Y) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int M = Nxh * Nz;
  const int mode = tid >> 1, part = tid & 1;
  if (mode >= M) return;
  const int kz = mode / Nxh, kx = mode - kz * Nxh;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  T* Sr = reinterpret_cast<T*>(S);
  const size_t col = 2 * ((size_t)kz * Ny * Px + kx) + part;
  const size_t rstep = 2 * (size_t)Px;
  if (singular && mode == 0) {
    double pm = 0.0, pc = 0.0, sum = 0.0;
    Y[tid] = 0.0;
    for (int j = 0; j < Ny - 1; ++j) {
      double b = (double)Sr[col + (size_t)j * rstep];
      double nx = (j == 0) ? pc - b : 2.0 * pc - pm - b;
      pm = pc; pc = nx;
      Y[(size_t)(j + 1) * stride + tid] = nx;
    }
    for (int j = 0; j < Ny; ++j) sum += Y[(size_t)j * stride + tid];
    const double mean = sum / Ny;
    for (int j = 0; j < Ny; ++j) Sr[col + (size_t)j * rstep] = T((Y[(size_t)j * stride + tid] - mean) * norm);
    return;
  }
  double prev = 0.0;
#pragma unroll 4
  for (int j = 0; j < Ny; ++j) {
    double im = inv_m[(size_t)j * M + mode];
    double b = (double)Sr[col + (size_t)j * rstep];
    prev = fma(prev, im, b * im);
    Y[(size_t)j * stride + tid] = prev;
  }
  double xn = prev;
  Sr[col + (size_t)(Ny - 1) * rstep] = T(xn * norm);
#pragma unroll 4
  for (int j = Ny - 2; j >= 0; --j) {
    double im = inv_m[(size_t)j * M + mode];
    xn = fma(im, xn, Y[(size_t)j * stride + tid]);
    Sr[col + (size_t)j * rstep] = T(xn * norm);
  }
}

template <typename T>
int pairs_per_block(int N) {
  int pp = 1024 / N;
  return pp < 1 ? 1 : pp;
}

}  // namespace

template <typename T>
void ensure_fft_z_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_fft_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    done = true;
  }
}

// Shared by the Poisson and Stokes paths.
template <typename T>
cudaError_t fft_x_forward(const Params& P, const T* in, int R, cplx<T>* out, T scale, int Nyr, T add0, T add1,
                          const cplx<T>* tw, cudaStream_t s) {
  int N = P.Nx, logN = 31 - __builtin_clz((unsigned)N);
  int pp = pairs_per_block<T>(N);
  int pairs = (R + 1) / 2;
  int nb = (pairs + pp - 1) / pp;
  size_t sm = (size_t)pp * N * sizeof(cplx<T>);
  k_rfft_x<T><<<nb, 256, sm, s>>>(in, R, N, logN, P.Px, out, scale, Nyr, add0, add1, tw, pp);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_x_inverse(const Params& P, const cplx<T>* in, int R, T* out, T scale, const cplx<T>* tw,
                          cudaStream_t s) {
  int N = P.Nx, logN = 31 - __builtin_clz((unsigned)N);
  int pp = pairs_per_block<T>(N);
  int pairs = (R + 1) / 2;
  int nb = (pairs + pp - 1) / pp;
  size_t sm = (size_t)pp * N * sizeof(cplx<T>);
  k_irfft_x<T><<<nb, 256, sm, s>>>(in, R, N, logN, P.Px, out, scale, tw, pp);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_z(const Params& P, cplx<T>* data, int Nyr, int nfields, size_t field_stride, bool inverse,
                  const cplx<T>* tw, cudaStream_t s) {
  int Nz = P.Nz, logNz = 31 - __builtin_clz((unsigned)Nz);
  size_t sm = (size_t)kTileZ * Nz * sizeof(cplx<T>);
  ensure_fft_z_attr<T>();
  dim3 grid((P.Nxh + kTileZ - 1) / kTileZ, Nyr, nfields);
  k_fft_z<T><<<grid, 256, sm, s>>>(data, Nz, logNz, Nyr, P.Px, P.Nxh, inverse ? 1 : 0, tw, field_stride, 0);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_z_mac(const Params& P, cplx<T>* data, bool inverse, const cplx<T>* tw, cudaStream_t s) {
  int Nz = P.Nz, logNz = 31 - __builtin_clz((unsigned)Nz);
  size_t sm = (size_t)kTileZ * Nz * sizeof(cplx<T>);
  ensure_fft_z_attr<T>();
  dim3 grid((P.Nxh + kTileZ - 1) / kTileZ, P.Ny + 1, 3);
  k_fft_z<T><<<grid, 256, sm, s>>>(data, Nz, logNz, P.Ny, P.Px, P.Nxh, inverse ? 1 : 0, tw, 0, 1);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_poisson(const Params& P, Workspace& W, const T* rho, T* phi, cudaStream_t s) {
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  cplx<T>* S = reinterpret_cast<cplx<T>*>(W.spec);
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(W.tw_x);
  const cplx<T>* twz = reinterpret_cast<const cplx<T>*>(W.tw_z);
  const double fourpi_lB = 4.0 * M_PI * P.lB;
  // ghost-cell terms of the wall rows (Eqs. esbc1, esbc3)
  T add0 = P.bc[0] == DISCOS_BC_DIRICHLET ? T(2.0 * P.phi_b[0]) : T(-P.slope[0]);
  T add1 = P.bc[1] == DISCOS_BC_DIRICHLET ? T(2.0 * P.phi_b[1]) : T(P.slope[1]);
  cudaError_t e = fft_x_forward<T>(P, rho, Nz * Ny, S, T(fourpi_lB), Ny, add0, add1, twx, s);
  if (e != cudaSuccess) return e;
  e = fft_z<T>(P, S, Ny, 1, 0, false, twz, s);
  if (e != cudaSuccess) return e;
  int singular = (P.bc[0] == DISCOS_BC_NEUMANN && P.bc[1] == DISCOS_BC_NEUMANN) ? 1 : 0;
  const int threads = 2 * P.Nxh * Nz;
  const int nb = (threads + 127) / 128;
  k_poisson_y<T><<<nb, 128, 0, s>>>(S, W.inv_m, Ny, Nz, P.Nxh, P.Px, singular, 1.0 / ((double)Nx * Nz),
                                    W.ps_scratch);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = fft_z<T>(P, S, Ny, 1, 0, true, twz, s);
  if (e != cudaSuccess) return e;
  return fft_x_inverse<T>(P, S, Nz * Ny, phi, T(1), twx, s);
}

template cudaError_t launch_poisson<float>(const Params&, Workspace&, const float*, float*, cudaStream_t);
template cudaError_t launch_poisson<double>(const Params&, Workspace&, const double*, double*, cudaStream_t);
template cudaError_t fft_x_forward<float>(const Params&, const float*, int, cplx<float>*, float, int, float, float, const cplx<float>*, cudaStream_t);
template cudaError_t fft_x_forward<double>(const Params&, const double*, int, cplx<double>*, double, int, double, double, const cplx<double>*, cudaStream_t);
template cudaError_t fft_x_inverse<float>(const Params&, const cplx<float>*, int, float*, float, const cplx<float>*, cudaStream_t);
template cudaError_t fft_x_inverse<double>(const Params&, const cplx<double>*, int, double*, double, const cplx<double>*, cudaStream_t);
template cudaError_t fft_z<float>(const Params&, cplx<float>*, int, int, size_t, bool, const cplx<float>*, cudaStream_t);
template cudaError_t fft_z<double>(const Params&, cplx<double>*, int, int, size_t, bool, const cplx<double>*, cudaStream_t);
template cudaError_t fft_z_mac<float>(const Params&, cplx<float>*, bool, const cplx<float>*, cudaStream_t);
template cudaError_t fft_z_mac<double>(const Params&, cplx<double>*, bool, const cplx<double>*, cudaStream_t);

}  // namespace discos
