// Staggered (MAC) Stokes solve of Eq. disc_stokes with no-slip walls
// (Eq. fluidbc), periodic in x and z.
//
// After transforms along x and z every (kx, kz) mode decouples.  With the
// forward-difference symbols g_x = e^{i theta_x} - 1, g_z likewise, and
// K^2 = |g_x|^2 + |g_z|^2, let A_c = K^2 - D_yy on cell rows (no-slip ghost
// u(-1) = -u(0)), A_f = K^2 - D_yy on the interior y-faces (v = 0 on the
// walls), D_y the face-to-cell difference.  Eliminating the pressure gives a
// real symmetric positive definite pentadiagonal system for v,
//   eta (K^2 A_f + D_y^T A_c D_y) v = K^2 f_y - D_y^T (g_x f_x + g_z f_z),
// then p = -(g_x f_x + g_z f_z + eta A_c D_y v) / K^2 and
//   eta A_c u = f_x + conj(g_x) p,   eta A_c w = f_z + conj(g_z) p.
// The K = 0 mode has v = 0, eta A_c u = f_x, eta A_c w = f_z, and p from
// p_j - p_{j-1} = f_y,j with zero mean.  All banded solves are in double
// precision (LDL^T for the pentadiagonal, Thomas for the tridiagonals) with
// the factors of every mode computed once when the handle is created.
#include "internal.h"

namespace discos {

template <typename T>
cudaError_t fft_x_forward(const Params& P, const T* in, int R, cplx<T>* out, T scale, int Nyr, T add0, T add1,
                          const cplx<T>* tw, cudaStream_t s);
template <typename T>
cudaError_t fft_x_inverse(const Params& P, const cplx<T>* in, int R, T* out, T scale, const cplx<T>* tw,
                          cudaStream_t s);
template <typename T>
cudaError_t fft_z(const Params& P, cplx<T>* data, int Nyr, int nfields, size_t field_stride, bool inverse,
                  const cplx<T>* tw, cudaStream_t s);
template <typename T>
cudaError_t fft_z_mac(const Params& P, cplx<T>* data, bool inverse, const cplx<T>* tw, cudaStream_t s);

namespace {

// One thread per (mode, part): lanes 2m and 2m+1 hold the real and the
// imaginary part of mode m (all band matrices are real, so the two parts
// are independent except where conj(g) p mixes them: there the partner's
// value comes by shuffle).  Factors are pre-computed per mode in double:
//   PL1, PL2, PDI [Ny-1][M]: L D L^T of the pentadiagonal (l1, l2, 1/D),
//   CI [Ny][M]: reciprocal Thomas pivots of A_c,
//   MC [M][5]: (g_x re, g_x im, g_z re, g_z im, -1/K^2; 0 for K = 0).
// Scratch SG, SY [Ny][threads] (double, one private slot per thread): g then
// u-forward values; y then v then w-forward values.
template <typename T>
__global__ void k_stokes_y(cplx<T>* __restrict__ S, cplx<T>* __restrict__ Sp, Params P,
                           const double* __restrict__ PL1, const double* __restrict__ PL2,
                           const double* __restrict__ PDI, const double* __restrict__ CI,
                           const double* __restrict__ MC, double* __restrict__ SG, double* __restrict__ SY) {
  const int Ny = P.Ny, Nz = P.Nz, Px = P.Px, Nxh = P.Nxh;
  const int M = Nxh * Nz;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int mode_raw = tid >> 1;
  const int part = tid & 1;
  const bool active = mode_raw < M;
  const int mode = active ? mode_raw : M - 1;      // idle lanes shadow the last mode, write nothing
  const int kz = mode / Nxh, kx = mode - kz * Nxh;
  const size_t M2 = (size_t)gridDim.x * blockDim.x;   // scratch row stride: one slot per thread
  const size_t me = (size_t)tid;
  const double eta = P.eta, ieta = 1.0 / P.eta;
  const double norm = 1.0 / ((double)P.Nx * P.Nz);
  const double gxr = MC[5 * (size_t)mode + 0], gxi = MC[5 * (size_t)mode + 1];
  const double gzr = MC[5 * (size_t)mode + 2], gzi = MC[5 * (size_t)mode + 3];
  const double mik2 = MC[5 * (size_t)mode + 4];   // -1/K^2
  const double K2 = mik2 != 0.0 ? -1.0 / mik2 : 0.0;
  T* Su = reinterpret_cast<T*>(S);
  T* Sv = reinterpret_cast<T*>(S + (size_t)Nz * Ny * Px);
  T* Sw = reinterpret_cast<T*>(S + (size_t)Nz * (2 * Ny + 1) * Px);
  const size_t cu = (size_t)kz * Ny * Px + kx;
  const size_t cv = (size_t)kz * (Ny + 1) * Px + kx;
  auto cpx = [&](const T* a, size_t e) { return make_double2((double)a[2 * e], (double)a[2 * e + 1]); };

  // pass A: g_j (this part) and the forward sweep of the pentadiagonal
  double gprev = 0.0, y1 = 0.0, y2 = 0.0;
  for (int j = 0; j < Ny; ++j) {
    double2 fx = cpx(Su, cu + (size_t)j * Px), fz = cpx(Sw, cu + (size_t)j * Px);
    double g = part == 0 ? (gxr * fx.x - gxi * fx.y + gzr * fz.x - gzi * fz.y)
                         : (gxr * fx.y + gxi * fx.x + gzr * fz.y + gzi * fz.x);
    SG[(size_t)j * M2 + me] = g;
    if (j >= 1) {
      const int i = j - 1;
      double fy = (double)Sv[2 * (cv + (size_t)j * Px) + part];
      double b = (K2 * fy + (g - gprev)) * ieta;
      double y = b - PL1[(size_t)i * M + mode] * y1 - PL2[(size_t)i * M + mode] * y2;
      SY[(size_t)i * M2 + me] = y;
      y2 = y1; y1 = y;
    }
    gprev = g;
  }
  // pass B: back substitution -> v on faces 1..Ny-1 (SY[i] = v at face i+1)
  {
    double x1 = 0.0, x2 = 0.0;
    for (int i = Ny - 2; i >= 0; --i) {
      double a1 = i + 1 < Ny - 1 ? PL1[(size_t)(i + 1) * M + mode] : 0.0;
      double a2 = i + 2 < Ny - 1 ? PL2[(size_t)(i + 2) * M + mode] : 0.0;
      double xi = SY[(size_t)i * M2 + me] * PDI[(size_t)i * M + mode] - a1 * x1 - a2 * x2;
      SY[(size_t)i * M2 + me] = xi;
      if (active) Sv[2 * (cv + (size_t)(i + 1) * Px) + part] = T(xi * norm);
      x2 = x1; x1 = xi;
    }
    if (active) {
      Sv[2 * cv + part] = T(0);
      Sv[2 * (cv + (size_t)Ny * Px) + part] = T(0);
    }
  }
  // pass C: p_j = -(g_j + eta (A_c D_y v)_j) / K^2 and the forward sweeps of
  // eta A_c u = f_x + conj(g_x) p, eta A_c w = f_z + conj(g_z) p
  {
    auto vf = [&](int f) { return (f >= 1 && f <= Ny - 1) ? SY[(size_t)(f - 1) * M2 + me] : 0.0; };
    double vm1 = 0.0, v0 = 0.0, v1 = vf(1), v2 = vf(2);   // faces j-1, j, j+1, j+2 at j = 0
    double yu = 0.0, yw = 0.0;
    for (int j = 0; j < Ny; ++j) {
      double em = v0 - vm1, e0 = v1 - v0, ep = v2 - v1;
      double a = K2 + 2.0 + (j == 0 ? 1.0 : 0.0) + (j == Ny - 1 ? 1.0 : 0.0);
      double acd = a * e0 - (j >= 1 ? em : 0.0) - (j <= Ny - 2 ? ep : 0.0);
      double g = SG[(size_t)j * M2 + me];
      double p = (g + eta * acd) * mik2;
      double pq = __shfl_xor_sync(0xffffffffu, p, 1);      // partner part of p
      double pre = part == 0 ? p : pq, pim = part == 0 ? pq : p;
      double2 fx = cpx(Su, cu + (size_t)j * Px), fz = cpx(Sw, cu + (size_t)j * Px);
      // conj(g) p = (gr pr + gi pi) + i (gr pi - gi pr)
      double bu = part == 0 ? fx.x + (gxr * pre + gxi * pim) : fx.y + (gxr * pim - gxi * pre);
      double bw = part == 0 ? fz.x + (gzr * pre + gzi * pim) : fz.y + (gzr * pim - gzi * pre);
      double ci = CI[(size_t)j * M + mode];
      yu = (bu * ieta + yu) * ci;
      yw = (bw * ieta + yw) * ci;
      if (Sp && active) reinterpret_cast<T*>(Sp)[2 * (cu + (size_t)j * Px) + part] = T(p * norm);
      SG[(size_t)j * M2 + me] = yu;
      // slide the v window before SY[j] (= v at face j+1, already held) is reused
      vm1 = v0; v0 = v1; v1 = v2; v2 = vf(j + 3);
      SY[(size_t)j * M2 + me] = yw;
    }
  }
  // pass D: back substitution of the two tridiagonal systems
  {
    double xu = 0.0, xw = 0.0;
    for (int j = Ny - 1; j >= 0; --j) {
      double ci = CI[(size_t)j * M + mode];
      xu = SG[(size_t)j * M2 + me] + (j < Ny - 1 ? ci * xu : 0.0);
      xw = SY[(size_t)j * M2 + me] + (j < Ny - 1 ? ci * xw : 0.0);
      if (active) {
        Su[2 * (cu + (size_t)j * Px) + part] = T(xu * norm);
        Sw[2 * (cu + (size_t)j * Px) + part] = T(xw * norm);
      }
    }
  }
}

// The pressure of the K = 0 mode (kx = kz = 0) from the saved f_y column.
template <typename T>
__global__ void k_stokes_p0(cplx<T>* __restrict__ Sp, const double* __restrict__ fy0, Params P) {
  const int part = threadIdx.x;
  if (part > 1) return;
  const int Ny = P.Ny;
  const double norm = 1.0 / ((double)P.Nx * P.Nz);
  double p = 0.0, sum = 0.0;
  for (int j = 1; j < Ny; ++j) { p += fy0[2 * j + part]; sum += p; }
  double mean = sum / Ny;
  p = 0.0;
  T* sp = reinterpret_cast<T*>(Sp);
  sp[part] = T((0.0 - mean) * norm);
  for (int j = 1; j < Ny; ++j) {
    p += fy0[2 * j + part];
    sp[2 * ((size_t)j * P.Px) + part] = T((p - mean) * norm);
  }
}

template <typename T>
__global__ void k_save_fy0(const cplx<T>* __restrict__ S, double* __restrict__ fy0, Params P) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > P.Ny) return;
  const cplx<T>* Sv = S + (size_t)P.Nz * P.Ny * P.Px;
  cplx<T> v = Sv[(size_t)j * P.Px];
  fy0[2 * j] = (double)v.re;
  fy0[2 * j + 1] = (double)v.im;
}

}  // namespace

template <typename T>
cudaError_t launch_stokes(const Params& P, Workspace& W, const T* f, T* v, T* p, cudaStream_t s) {
  const int Ny = P.Ny, Nz = P.Nz;
  cplx<T>* S = reinterpret_cast<cplx<T>*>(W.spec);
  const size_t fieldsz = (size_t)Nz * (Ny + 1) * P.Px;     // capacity of one spectrum slot
  cplx<T>* Sp = p ? S + 3 * fieldsz : nullptr;
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(W.tw_x);
  const cplx<T>* twz = reinterpret_cast<const cplx<T>*>(W.tw_z);
  const int R = Nz * (3 * Ny + 1);
  const size_t M = (size_t)P.Nxh * Nz;
  cudaError_t e = fft_x_forward<T>(P, f, R, S, T(1), 1 << 30, T(0), T(0), twx, s);
  if (e != cudaSuccess) return e;
  e = fft_z_mac<T>(P, S, false, twz, s);
  if (e != cudaSuccess) return e;
  const size_t S2 = (2 * M + 127) / 128 * 128;               // threads launched = scratch row stride
  double* fy0 = W.st_scratch + 2 * (size_t)Ny * S2;         // K = 0 column of f_y, 2 (Ny + 1) doubles
  if (p) {
    k_save_fy0<T><<<(Ny + 1 + 127) / 128, 128, 0, s>>>(S, fy0, P);
    count_launches(1);
  }
  k_stokes_y<T><<<(unsigned)(S2 / 128), 128, 0, s>>>(S, Sp, P, W.st_l1, W.st_l2, W.st_di, W.st_ci, W.st_mc,
                                                     W.st_scratch, W.st_scratch + (size_t)Ny * S2);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (p) {
    k_stokes_p0<T><<<1, 32, 0, s>>>(Sp, fy0, P);
    count_launches(1);
  }
  e = fft_z_mac<T>(P, S, true, twz, s);
  if (e != cudaSuccess) return e;
  e = fft_x_inverse<T>(P, S, R, v, T(1), twx, s);
  if (e != cudaSuccess) return e;
  if (p) {
    e = fft_z<T>(P, Sp, Ny, 1, 0, true, twz, s);
    if (e != cudaSuccess) return e;
    e = fft_x_inverse<T>(P, Sp, Nz * Ny, p, T(1), twx, s);
  }
  return e;
}

template cudaError_t launch_stokes<float>(const Params&, Workspace&, const float*, float*, float*, cudaStream_t);
template cudaError_t launch_stokes<double>(const Params&, Workspace&, const double*, double*, double*, cudaStream_t);

}  // namespace discos
