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
// precision (LDL^T for the pentadiagonal, Thomas for the tridiagonals), one
// thread per mode, work arrays in shared memory laid out [row][thread].
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

__device__ __forceinline__ double2 cd(double a, double b) { return make_double2(a, b); }

template <typename T>
__global__ void k_stokes_y(cplx<T>* __restrict__ S, cplx<T>* __restrict__ Sp, Params P) {
  extern __shared__ unsigned char smem_raw[];
  const int B = blockDim.x, t = threadIdx.x;
  const int Ny = P.Ny, Nz = P.Nz, Px = P.Px;
  double2* G = reinterpret_cast<double2*>(smem_raw);       // [Ny][B]
  double2* R = G + (size_t)Ny * B;                         // [Ny][B]
  double* L1 = reinterpret_cast<double*>(R + (size_t)Ny * B);  // [Ny][B]
  double* L2 = L1 + (size_t)Ny * B;
  double* DI = L2 + (size_t)Ny * B;
#define AT(arr, j) arr[(size_t)(j) * B + t]
  const int kx = blockIdx.x * B + t;
  const int kz = blockIdx.y;
  if (kx >= P.Nxh) return;
  const double eta = P.eta;
  const double norm = 1.0 / ((double)P.Nx * P.Nz);
  cplx<T>* Su = S;
  cplx<T>* Sv = S + (size_t)Nz * Ny * Px;
  cplx<T>* Sw = S + (size_t)Nz * (2 * Ny + 1) * Px;
  const size_t cu = (size_t)kz * Ny * Px + kx;          // column in u / w / p spectra
  const size_t cv = (size_t)kz * (Ny + 1) * Px + kx;    // column in the v spectrum
  double sx, cxv, sz, czv;
  sincospi(2.0 * kx / P.Nx, &sx, &cxv);
  sincospi(2.0 * kz / P.Nz, &sz, &czv);
  const double2 gx = cd(cxv - 1.0, sx), gz = cd(czv - 1.0, sz);
  const double K2 = (2.0 - 2.0 * cxv) + (2.0 - 2.0 * czv);
  auto ld = [&](const cplx<T>* a, size_t i) { cplx<T> v = a[i]; return cd((double)v.re, (double)v.im); };
  auto st = [&](cplx<T>* a, size_t i, double2 v) { a[i] = cplx<T>{T(v.x * norm), T(v.y * norm)}; };

  // Thomas pivots of A_c (diag K^2 + 2, +1 on the two wall rows; off-diagonals -1)
  auto ac_diag = [&](int j) { return K2 + 2.0 + (j == 0 ? 1.0 : 0.0) + (j == Ny - 1 ? 1.0 : 0.0); };
  auto tridiag_ac = [&](const cplx<T>* f, double2 gc, bool with_p, cplx<T>* out) {
    // eta A_c x = f + conj(gc) p ;  p in G
    double2 prev = cd(0, 0);
    for (int j = 0; j < Ny; ++j) {
      double2 b = ld(f, cu + (size_t)j * Px);
      if (with_p) {
        double2 p = AT(G, j);
        b.x += gc.x * p.x + gc.y * p.y;   // conj(gc) * p
        b.y += gc.x * p.y - gc.y * p.x;
      }
      b.x /= eta; b.y /= eta;
      double im = AT(L1, j);
      prev.x = (b.x + prev.x) * im;
      prev.y = (b.y + prev.y) * im;
      AT(R, j) = prev;
    }
    double2 xn = prev;
    st(out, cu + (size_t)(Ny - 1) * Px, xn);
    for (int j = Ny - 2; j >= 0; --j) {
      double im = AT(L1, j);
      double2 v = AT(R, j);
      xn.x = v.x + im * xn.x;
      xn.y = v.y + im * xn.y;
      st(out, cu + (size_t)j * Px, xn);
    }
  };
  {
    double m = ac_diag(0);
    AT(L1, 0) = 1.0 / m;
    for (int j = 1; j < Ny; ++j) {
      m = ac_diag(j) - 1.0 / m;
      AT(L1, j) = 1.0 / m;
    }
  }

  if (kx == 0 && kz == 0) {
    // K = 0: pressure from p_j - p_{j-1} = f_y,j (zero mean), v = 0
    double2 p = cd(0, 0), sum = cd(0, 0);
    AT(G, 0) = p;
    for (int j = 1; j < Ny; ++j) {
      double2 fy = ld(Sv, cv + (size_t)j * Px);
      p.x += fy.x; p.y += fy.y;
      AT(G, j) = p;
      sum.x += p.x; sum.y += p.y;
    }
    sum.x /= Ny; sum.y /= Ny;
    for (int j = 0; j < Ny; ++j) { AT(G, j).x -= sum.x; AT(G, j).y -= sum.y; }
    tridiag_ac(Su, gx, false, Su);
    tridiag_ac(Sw, gz, false, Sw);
    for (int j = 0; j <= Ny; ++j) Sv[cv + (size_t)j * Px] = cplx<T>{T(0), T(0)};
    if (Sp)
      for (int j = 0; j < Ny; ++j) st(Sp, cu + (size_t)j * Px, AT(G, j));
    return;
  }

  // g = g_x f_x + g_z f_z on cell rows
  for (int j = 0; j < Ny; ++j) {
    double2 fx = ld(Su, cu + (size_t)j * Px), fz = ld(Sw, cu + (size_t)j * Px);
    AT(G, j) = cd(gx.x * fx.x - gx.y * fx.y + gz.x * fz.x - gz.y * fz.y,
                  gx.x * fx.y + gx.y * fx.x + gz.x * fz.y + gz.y * fz.x);
  }
  // pentadiagonal P = K^2 A_f + D_y^T A_c D_y on faces 1..Ny-1 (unknown i = face - 1):
  // diag K^4 + 4K^2 + 6 (+1 on the first and last rows), off-1 -2K^2 - 4, off-2 +1
  const int n = Ny - 1;
  const double dbase = K2 * K2 + 4.0 * K2 + 6.0, e = -2.0 * K2 - 4.0, fo = 1.0;
  double Dm1 = 0.0, Dm2 = 0.0, l1m1 = 0.0;   // D_{i-1}, D_{i-2}, l1_{i-1}
  double2 ym1 = cd(0, 0), ym2 = cd(0, 0);
  for (int i = 0; i < n; ++i) {
    const int face = i + 1;
    double2 fy = ld(Sv, cv + (size_t)face * Px);
    double2 g1 = AT(G, face), g0 = AT(G, face - 1);
    // rhs = (K^2 f_y + (g_f - g_{f-1})) / eta
    double2 b = cd((K2 * fy.x + (g1.x - g0.x)) / eta, (K2 * fy.y + (g1.y - g0.y)) / eta);
    double l2 = i >= 2 ? fo / Dm2 : 0.0;
    double l1 = i >= 1 ? (e - (i >= 2 ? l2 * l1m1 * Dm2 : 0.0)) / Dm1 : 0.0;
    double d = dbase + (i == 0 ? 1.0 : 0.0) + (i == n - 1 ? 1.0 : 0.0);
    double D = d - l1 * l1 * Dm1 - l2 * l2 * Dm2;
    double2 y = cd(b.x - l1 * ym1.x - l2 * ym2.x, b.y - l1 * ym1.y - l2 * ym2.y);
    AT(L1, i) = l1;  // reused below only after the A_c pivots are rebuilt
    AT(L2, i) = l2;
    AT(DI, i) = 1.0 / D;
    AT(R, i) = y;
    ym2 = ym1; ym1 = y;
    Dm2 = Dm1; Dm1 = D; l1m1 = l1;
  }
  // back substitution: x_i = y_i / D_i - l1_{i+1} x_{i+1} - l2_{i+2} x_{i+2}
  {
    double2 x1 = cd(0, 0), x2 = cd(0, 0);
    for (int i = n - 1; i >= 0; --i) {
      double2 y = AT(R, i);
      double di = AT(DI, i);
      double a1 = i + 1 < n ? AT(L1, i + 1) : 0.0;
      double a2 = i + 2 < n ? AT(L2, i + 2) : 0.0;
      double2 xi = cd(y.x * di - a1 * x1.x - a2 * x2.x, y.y * di - a1 * x1.y - a2 * x2.y);
      AT(R, i) = xi;
      x2 = x1; x1 = xi;
    }
  }
  // v on the faces (walls zero)
  Sv[cv] = cplx<T>{T(0), T(0)};
  Sv[cv + (size_t)Ny * Px] = cplx<T>{T(0), T(0)};
  for (int f = 1; f < Ny; ++f) st(Sv, cv + (size_t)f * Px, AT(R, f - 1));
  // p_j = -(g_j + eta (A_c D_y v)_j) / K^2,  (D_y v)_j = v_{j+1} - v_j
  auto vface = [&](int f) { return (f >= 1 && f <= Ny - 1) ? AT(R, f - 1) : cd(0, 0); };
  auto dyv = [&](int j) { double2 a = vface(j + 1), b = vface(j); return cd(a.x - b.x, a.y - b.y); };
  for (int j = 0; j < Ny; ++j) {
    double a = ac_diag(j);
    double2 c = dyv(j);
    double2 acd = cd(a * c.x, a * c.y);
    if (j >= 1) { double2 m = dyv(j - 1); acd.x -= m.x; acd.y -= m.y; }
    if (j <= Ny - 2) { double2 m = dyv(j + 1); acd.x -= m.x; acd.y -= m.y; }
    double2 g = AT(G, j);
    AT(G, j) = cd(-(g.x + eta * acd.x) / K2, -(g.y + eta * acd.y) / K2);
  }
  // rebuild the A_c pivots (L1 was used by the pentadiagonal factors)
  {
    double m = ac_diag(0);
    AT(L1, 0) = 1.0 / m;
    for (int j = 1; j < Ny; ++j) {
      m = ac_diag(j) - 1.0 / m;
      AT(L1, j) = 1.0 / m;
    }
  }
  tridiag_ac(Su, gx, true, Su);
  tridiag_ac(Sw, gz, true, Sw);
  if (Sp)
    for (int j = 0; j < Ny; ++j) st(Sp, cu + (size_t)j * Px, AT(G, j));
#undef AT
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
  cudaError_t e = fft_x_forward<T>(P, f, R, S, T(1), 1 << 30, T(0), T(0), twx, s);
  if (e != cudaSuccess) return e;
  e = fft_z_mac<T>(P, S, false, twz, s);
  if (e != cudaSuccess) return e;
  int B = 32;
  while (B > 1 && (size_t)B * Ny * 56 > 150 * 1024) B >>= 1;
  size_t sm = (size_t)B * Ny * 56;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_stokes_y<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    cudaFuncSetAttribute(k_stokes_y<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr = true;
  }
  dim3 grid((P.Nxh + B - 1) / B, Nz);
  k_stokes_y<T><<<grid, B, sm, s>>>(S, Sp, P);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
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
