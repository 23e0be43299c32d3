// Hand-written transforms along x and z and the Poisson solve of Eq. poisson
// with the wall conditions of Eqs. esbc1 / esbc3.
//
// x: real rows -> half spectra (Nx/2 + 1 modes, row pitch Px), two real rows
//    packed into one complex radix-2 transform held in shared memory.
// z: complex transforms down the columns of the half spectrum, a tile of 16
//    consecutive x-modes per block so that every load is a 16-element run.
// Both use a radix-2 Stockham transform (natural order, no bit reversal).
// y: the tridiagonal wall-normal system of every (kx, kz) mode, solved by
//    warp-parallel scans over pre-factored pivots (k_ysolve.cu).
#include <atomic>
#include <type_traits>
#include "internal.h"

namespace discos {

namespace {


// Stockham auto-sort FFT over `nvec` vectors of length N = 2^logN in shared
// memory (vector v at in[v * vs .. v * vs + N)), natural order in and out, no
// bit reversal.  Radix-4 stages while they fit, then one radix-2 stage.  A
// stage with sub-transform size Ns takes butterfly j (< N/R) with
// k = j mod Ns, inputs in[j + m N/R] (m < R) twiddled by exp(-+2 pi i m k /
// (R Ns)), and writes the R-point DFT to out[R j - (R-1) k + m Ns].  Reads
// are unit-stride; the two buffers alternate.  Returns the buffer holding the
// result.  All threads take part; ends with the block synchronised.
template <typename T>
__device__ cplx<T>* fft_stockham(cplx<T>* in, cplx<T>* out, int N, int logN, int nvec, int vs,
                                 const cplx<T>* __restrict__ tw, bool inverse) {
  int Ns = 1;
  while (Ns < N) {
    if (4 * Ns <= N) {
      const int q = N >> 2;
      const int total = nvec * q;
      const int twstep = N / (4 * Ns);
      for (int b = threadIdx.x; b < total; b += blockDim.x) {
        const int v = b >> (logN - 2);
        const int j = b & (q - 1);
        const int k = j & (Ns - 1);
        cplx<T> w1 = tw[k * twstep], w2 = tw[2 * k * twstep];
        if (inverse) { w1.im = -w1.im; w2.im = -w2.im; }
        const cplx<T> w3 = cmul(w1, w2);
        const cplx<T>* iv = in + (size_t)v * vs;
        cplx<T>* ov = out + (size_t)v * vs;
        const cplx<T> a0 = iv[j];
        const cplx<T> a1 = cmul(w1, iv[j + q]);
        const cplx<T> a2 = cmul(w2, iv[j + 2 * q]);
        const cplx<T> a3 = cmul(w3, iv[j + 3 * q]);
        const cplx<T> b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3);
        const cplx<T> d = csub(a1, a3);
        // (a1 - a3) times -i (forward) or +i (inverse)
        const cplx<T> b3 = inverse ? cplx<T>{-d.im, d.re} : cplx<T>{d.im, -d.re};
        const int o = 4 * j - 3 * k;
        ov[o] = cadd(b0, b2);
        ov[o + Ns] = cadd(b1, b3);
        ov[o + 2 * Ns] = csub(b0, b2);
        ov[o + 3 * Ns] = csub(b1, b3);
      }
      Ns <<= 2;
    } else {
      const int hN = N >> 1;
      const int total = nvec * hN;
      const int twstep = N / (2 * Ns);
      for (int b = threadIdx.x; b < total; b += blockDim.x) {
        const int v = b >> (logN - 1);
        const int j = b & (hN - 1);
        const int k = j & (Ns - 1);
        cplx<T> wv = tw[k * twstep];
        if (inverse) wv.im = -wv.im;
        const cplx<T>* iv = in + (size_t)v * vs;
        cplx<T>* ov = out + (size_t)v * vs;
        cplx<T> u = iv[j];
        cplx<T> t = cmul(wv, iv[j + hN]);
        const int o = 2 * j - k;
        ov[o] = cadd(u, t);
        ov[o + Ns] = csub(u, t);
      }
      Ns <<= 1;
    }
    __syncthreads();
    cplx<T>* tmp = in; in = out; out = tmp;
  }
  return in;
}

// Forward real transform of R rows of length N (two rows per complex FFT).
// Input value = scale * in + (row's y == 0 ? add0) + (row's y == Nyr-1 ? add1).
template <typename T>
__global__ void k_rfft_x(const T* __restrict__ in, int R, int N, int logN, int Px, cplx<T>* __restrict__ out,
                         T scale, int Nyr, T add0, T add1, const cplx<T>* __restrict__ tw, int pairs_per_block) {
  extern __shared__ unsigned char smem_raw[];
  const int PP = pairs_per_block;
  cplx<T>* bufa = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufb = bufa + (size_t)PP * N;
  cplx<T>* stw = bufb + (size_t)PP * N;                        // twiddles, staged once per block
  T* rowadd = reinterpret_cast<T*>(stw + N / 2);               // [2 PP] wall terms of each row
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) stw[t] = tw[t];
  for (int t = threadIdx.x; t < 2 * PP; t += blockDim.x) {
    const int row = 2 * blockIdx.x * PP + t;
    const int y = row % Nyr;
    rowadd[t] = (y == 0 ? add0 : T(0)) + (y == Nyr - 1 ? add1 : T(0));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    const int v = idx >> logN, n = idx & (N - 1);
    const int ra = 2 * (blockIdx.x * PP + v), rb = ra + 1;
    T a = T(0), b = T(0);
    if (ra < R) a = scale * in[(size_t)ra * N + n] + rowadd[2 * v];
    if (rb < R) b = scale * in[(size_t)rb * N + n] + rowadd[2 * v + 1];
    bufa[idx] = cplx<T>{a, b};
  }
  __syncthreads();
  cplx<T>* r = fft_stockham(bufa, bufb, N, logN, PP, N, stw, false);
  const int M = N / 2 + 1;
  // idx / M by a float reciprocal: idx < 2^16, so (idx + 1/2) / M stays at
  // least 1/(2M) away from an integer, far beyond the rounding of the product
  const float invM = 1.0f / (float)M;
  for (int idx = threadIdx.x; idx < PP * M; idx += blockDim.x) {
    const int v = (int)(((float)idx + 0.5f) * invM), k = idx - v * M;
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    cplx<T> Zk = r[v * N + (k & (N - 1))];
    cplx<T> Zn = r[v * N + ((N - k) & (N - 1))];
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
  const int PP = pairs_per_block;
  cplx<T>* bufa = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufb = bufa + (size_t)PP * N;
  cplx<T>* stw = bufb + (size_t)PP * N;                        // twiddles, staged once per block
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) stw[t] = tw[t];
  const int hN = N / 2;
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    const int v = idx >> logN, k = idx & (N - 1);
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    int kk = k <= hN ? k : N - k;
    cplx<T> A{T(0), T(0)}, B{T(0), T(0)};
    if (ra < R) A = in[(size_t)ra * Px + kk];
    if (rb < R) B = in[(size_t)rb * Px + kk];
    if (k > hN) { A.im = -A.im; B.im = -B.im; }
    bufa[idx] = cplx<T>{A.re - B.im, A.im + B.re};   // Z = A + i B
  }
  __syncthreads();
  cplx<T>* r = fft_stockham(bufa, bufb, N, logN, PP, N, stw, true);
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    const int v = idx >> logN, n = idx & (N - 1);
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    cplx<T> z = r[idx];
    if (ra < R) out[(size_t)ra * N + n] = scale * z.re;
    if (rb < R) out[(size_t)rb * N + n] = scale * z.im;
  }
}

// Complex transform along z of the half spectra [Nz][Nyr][Px] (field f =
// blockIdx.z at offset f * field_stride), TK consecutive x-modes per block.
// Shared layout [column][Nz + 1] (padded so that the column-interleaved
// loads and stores do not collide in a bank).
// mac != 0: the three MAC fields u | v | w stored back to back with Ny, Ny+1
// and Ny rows per z-plane (Nyr = Ny is passed; grid.y = Ny + 1).
template <typename T>
__global__ void k_fft_z(cplx<T>* __restrict__ data, int Nz, int logNz, int Nyr, int Px, int Nxh, int inverse,
                        const cplx<T>* __restrict__ tw, size_t field_stride, int mac, int TK) {
  extern __shared__ unsigned char smem_raw[];
  const int vs = Nz + 1;
  cplx<T>* bufa = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufb = bufa + (size_t)TK * vs;
  cplx<T>* stw = bufb + (size_t)TK * vs;                       // twiddles, staged once per block
  cplx<T>* base = data + blockIdx.z * field_stride;
  if (mac) {
    const int Ny = Nyr;
    if (blockIdx.z == 1) { base = data + (size_t)Nz * Ny * Px; Nyr = Ny + 1; }
    else if (blockIdx.z == 2) { base = data + (size_t)Nz * (2 * Ny + 1) * Px; }
    else { base = data; }
  }
  const int y = blockIdx.y;
  if (y >= Nyr) return;
  for (int t = threadIdx.x; t < Nz / 2; t += blockDim.x) stw[t] = tw[t];
  const int kx0 = blockIdx.x * TK;
  const int logTK = 31 - __clz(TK);
  for (int idx = threadIdx.x; idx < TK * Nz; idx += blockDim.x) {
    const int z = idx >> logTK, c = idx & (TK - 1);
    int kx = kx0 + c;
    cplx<T> v{T(0), T(0)};
    if (kx < Nxh) v = base[((size_t)z * Nyr + y) * Px + kx];
    bufa[c * vs + z] = v;
  }
  __syncthreads();
  const int nv = Nxh - kx0 < TK ? Nxh - kx0 : TK;   // the last tile holds fewer columns
  cplx<T>* r = fft_stockham(bufa, bufb, Nz, logNz, nv, vs, stw, inverse != 0);
  for (int idx = threadIdx.x; idx < TK * Nz; idx += blockDim.x) {
    const int z = idx >> logTK, c = idx & (TK - 1);
    int kx = kx0 + c;
    if (kx < Nxh) base[((size_t)z * Nyr + y) * Px + kx] = r[c * vs + z];
  }
}

}  // namespace

// Default launch shapes of the transforms (discos_tune_transforms may replace
// them): 1024 / Nx row pairs per x-block on 256 threads; 8 columns per
// z-block (small blocks keep the launch within one wave at typical sizes),
// halved while the two buffers exceed 140 KB.
int default_fx_pairs(int Nx) {
  int pp = 1024 / Nx;
  return pp < 1 ? 1 : pp;
}
int max_tile_z(int Nz, size_t elem) {
  int tk = 16;
  while (tk > 1 && 2 * (size_t)tk * (Nz + 1) * elem > 140 * 1024) tk >>= 1;
  return tk;
}
// one radix-4 butterfly per thread: TK Nz / 4 threads, 64..256
int fz_threads(int TK, int Nz) {
  int t = TK * Nz / 4;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}
int default_tile_z(int Nz, size_t elem) {
  int tk = max_tile_z(Nz, elem);
  return tk > 8 ? 8 : tk;
}

template <typename T>
void ensure_fft_z_attr() {
  // the attribute belongs to the current device: set it once per device
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  const unsigned long long bit = 1ull << dev;
  if (done.load() & bit) return;
  if (cudaFuncSetAttribute(k_fft_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) == cudaSuccess)
    done.fetch_or(bit);
}

// Shared by the Poisson and Stokes paths.
template <typename T>
cudaError_t fft_x_forward(const Params& P, const T* in, int R, cplx<T>* out, T scale, int Nyr, T add0, T add1,
                          const cplx<T>* tw, cudaStream_t s) {
  int N = P.Nx, logN = 31 - __builtin_clz((unsigned)N);
  int pp = P.fx_pp;
  int pairs = (R + 1) / 2;
  int nb = (pairs + pp - 1) / pp;
  size_t sm = (2 * (size_t)pp * N + N / 2) * sizeof(cplx<T>) + 2 * (size_t)pp * sizeof(T);
  probe_begin(PROBE_FFT_X, s);
  k_rfft_x<T><<<nb, P.fx_threads, sm, s>>>(in, R, N, logN, P.Px, out, scale, Nyr, add0, add1, tw, pp);
  count_launches(1);
  probe_end(PROBE_FFT_X, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_x_inverse(const Params& P, const cplx<T>* in, int R, T* out, T scale, const cplx<T>* tw,
                          cudaStream_t s) {
  int N = P.Nx, logN = 31 - __builtin_clz((unsigned)N);
  int pp = P.fx_pp;
  int pairs = (R + 1) / 2;
  int nb = (pairs + pp - 1) / pp;
  size_t sm = (2 * (size_t)pp * N + N / 2) * sizeof(cplx<T>);
  probe_begin(PROBE_FFT_X, s);
  k_irfft_x<T><<<nb, P.fx_threads, sm, s>>>(in, R, N, logN, P.Px, out, scale, tw, pp);
  count_launches(1);
  probe_end(PROBE_FFT_X, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_z(const Params& P, cplx<T>* data, int Nyr, int nfields, size_t field_stride, bool inverse,
                  const cplx<T>* tw, cudaStream_t s) {
  int Nz = P.Nz, logNz = 31 - __builtin_clz((unsigned)Nz);
  const int TK = P.fz_tk;
  size_t sm = (2 * (size_t)TK * (Nz + 1) + Nz / 2) * sizeof(cplx<T>);
  ensure_fft_z_attr<T>();
  dim3 grid((P.Nxh + TK - 1) / TK, Nyr, nfields);
  probe_begin(PROBE_FFT_Z, s);
  k_fft_z<T><<<grid, fz_threads(TK, Nz), sm, s>>>(data, Nz, logNz, Nyr, P.Px, P.Nxh, inverse ? 1 : 0, tw,
                                                   field_stride, 0, TK);
  count_launches(1);
  probe_end(PROBE_FFT_Z, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_z_mac(const Params& P, cplx<T>* data, bool inverse, const cplx<T>* tw, cudaStream_t s) {
  int Nz = P.Nz, logNz = 31 - __builtin_clz((unsigned)Nz);
  const int TK = P.fz_tk;
  size_t sm = (2 * (size_t)TK * (Nz + 1) + Nz / 2) * sizeof(cplx<T>);
  ensure_fft_z_attr<T>();
  dim3 grid((P.Nxh + TK - 1) / TK, P.Ny + 1, 3);
  probe_begin(PROBE_FFT_Z, s);
  k_fft_z<T><<<grid, fz_threads(TK, Nz), sm, s>>>(data, Nz, logNz, P.Ny, P.Px, P.Nxh, inverse ? 1 : 0, tw, 0,
                                                   1, TK);
  count_launches(1);
  probe_end(PROBE_FFT_Z, s);
  return cudaGetLastError();
}

// One transform-solve-transform pass: phi = A^-1 (scale rho + wall terms)
// with the ghost-cell terms add0 / add1 on the wall rows.
template <typename T>
cudaError_t poisson_pass(const Params& P, Workspace& W, const T* rho, T* phi, T scale, T add0, T add1,
                         cudaStream_t s) {
  const int Ny = P.Ny, Nz = P.Nz;
  cplx<T>* S = reinterpret_cast<cplx<T>*>(W.spec);
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(W.tw_x);
  const cplx<T>* twz = reinterpret_cast<const cplx<T>*>(W.tw_z);
  cudaError_t e = fft_x_forward<T>(P, rho, Nz * Ny, S, scale, Ny, add0, add1, twx, s);
  if (e != cudaSuccess) return e;
  e = fft_z<T>(P, S, Ny, 1, 0, false, twz, s);
  if (e != cudaSuccess) return e;
  e = launch_poisson_y<T>(P, W, S, s);
  if (e != cudaSuccess) return e;
  e = fft_z<T>(P, S, Ny, 1, 0, true, twz, s);
  if (e != cudaSuccess) return e;
  return fft_x_inverse<T>(P, S, Nz * Ny, phi, T(1), twx, s);
}

template <typename T>
cudaError_t launch_poisson(const Params& P, Workspace& W, const T* rho, T* phi, cudaStream_t s) {
  const double fourpi_lB = 4.0 * M_PI * P.lB;
  // ghost-cell terms of the wall rows (Eqs. esbc1, esbc3)
  const T add0 = P.bc[0] == DISCOS_BC_DIRICHLET ? T(2.0 * P.phi_b[0]) : T(-P.slope[0]);
  const T add1 = P.bc[1] == DISCOS_BC_DIRICHLET ? T(2.0 * P.phi_b[1]) : T(P.slope[1]);
  const int sweeps = (sizeof(T) == sizeof(float) && W.rref) ? P.max_refine : 0;
  if (sweeps == 0) return poisson_pass<T>(P, W, rho, phi, T(fourpi_lB), add0, add1, s);
  // mixed precision with residual refinement: keep rho (phi may alias it),
  // solve, then correct with the double-precision residual (k_refine.cu)
  const size_t G = (size_t)P.Nx * P.Ny * P.Nz;
  T* rho_keep = reinterpret_cast<T*>(W.rref);
  T* res = reinterpret_cast<T*>(W.rres);
  cudaError_t e = cudaMemcpyAsync(rho_keep, rho, sizeof(T) * G, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_fill_zero<double>(W.rnorm, 2 * (DISCOS_MAX_REFINE + 1), s);
  if (e == cudaSuccess) e = poisson_pass<T>(P, W, rho_keep, phi, T(fourpi_lB), add0, add1, s);
  for (int it = 0; it < sweeps && e == cudaSuccess; ++it) {
    e = launch_poisson_residual<T>(P, rho_keep, phi, res, W.rnorm + 2 * it, s);
    if (e == cudaSuccess) e = poisson_pass<T>(P, W, res, res, T(1), T(0), T(0), s);
    if (e == cudaSuccess) e = launch_add_inplace<T>(phi, res, G, s);
  }
  if (e == cudaSuccess) e = launch_poisson_residual<T>(P, rho_keep, phi, nullptr, W.rnorm + 2 * sweeps, s);
  return e;
}

// Launch-shape autotuner of the transforms: times each candidate shape of the
// x transform (row pairs per block, threads) and of the z transform (columns
// per block) on the handle's own potential and spectrum buffers at the
// Poisson sizes, and keeps the fastest in P.  Blocks until done.
template <typename T>
cudaError_t tune_transforms_t(Params& P, Workspace& W, cudaStream_t s, float* best_ms) {
  const int N = P.Nx, R = P.Nz * P.Ny;
  T* grid = reinterpret_cast<T*>(W.phi);
  cplx<T>* S = reinterpret_cast<cplx<T>*>(W.spec);
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(W.tw_x);
  const cplx<T>* twz = reinterpret_cast<const cplx<T>*>(W.tw_z);
  cudaError_t e = launch_fill_zero<T>(grid, (size_t)P.Nx * P.Ny * P.Nz, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto time_it = [&](auto&& launch) -> float {
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 1e30f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    return ms / 10.0f;
  };
  Params Q = P;
  float bx = 1e30f, bz = 1e30f;
  int best_pp = P.fx_pp, best_th = P.fx_threads, best_tk = P.fz_tk;
  int last_pp = 0;
  for (int vals = 128; vals <= 2048 && e == cudaSuccess; vals *= 2) {
    const int pp = vals / N < 1 ? 1 : vals / N;
    if (pp == last_pp) continue;
    if ((2 * (size_t)pp * N + N / 2) * sizeof(cplx<T>) + 2 * (size_t)pp * sizeof(T) > 48 * 1024) break;
    last_pp = pp;
    int th = pp * N / 4;
    th = th < 32 ? 32 : (th > 256 ? 256 : th);
    Q.fx_pp = pp;
    Q.fx_threads = th;
    const float ms = time_it([&] { return fft_x_forward<T>(Q, grid, R, S, T(1), P.Ny, T(0), T(0), twx, s); });
    if (ms < bx) { bx = ms; best_pp = pp; best_th = th; }
  }
  Q = P;
  for (int tk = 1; tk <= max_tile_z(P.Nz, sizeof(cplx<T>)) && e == cudaSuccess; tk *= 2) {
    Q.fz_tk = tk;
    const float ms = time_it([&] { return fft_z<T>(Q, S, P.Ny, 1, 0, false, twz, s); });
    if (ms < bz) { bz = ms; best_tk = tk; }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  P.fx_pp = best_pp;
  P.fx_threads = best_th;
  P.fz_tk = best_tk;
  best_ms[0] = bx;
  best_ms[1] = bz;
  return cudaSuccess;
}

cudaError_t tune_transforms(Params& P, Workspace& W, bool mixed, cudaStream_t s, float* best_ms) {
  return mixed ? tune_transforms_t<float>(P, W, s, best_ms) : tune_transforms_t<double>(P, W, s, best_ms);
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
