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
// p_j - p_{j-1} = f_y,j with zero mean.  The factors of every mode (L D L^T
// of the pentadiagonal, Thomas pivots of A_c) are computed once in double
// when the handle is created; the substitution sweeps run as warp-parallel
// scans (k_ysolve.cu).  The mixed path can refine the solution against the
// double-precision residual of the full MAC operator (launch_stokes below).
#include <type_traits>
#include "internal.h"

namespace discos {

template <typename T>
cudaError_t fft_x_forward(const Params& P, const T* in, int R, cplx<T>* out, T scale, int Nyr, T add0, T add1,
                          const cplx<T>* tw, cudaStream_t s, const T* add0x);
template <typename T>
cudaError_t fft_x_inverse(const Params& P, const cplx<T>* in, int R, T* out, T scale, const cplx<T>* tw,
                          cudaStream_t s);
template <typename T>
cudaError_t fft_z(const Params& P, cplx<T>* data, int Nyr, int nfields, size_t field_stride, bool inverse,
                  const cplx<T>* tw, cudaStream_t s);
template <typename T>
cudaError_t fft_z_mac(const Params& P, cplx<T>* data, bool inverse, const cplx<T>* tw, cudaStream_t s);

template <typename T>
cudaError_t stokes_once(const Params& P, Workspace& W, const T* f, T* v, T* p, cudaStream_t s) {
  const int Ny = P.Ny, Nz = P.Nz;
  cplx<T>* S = reinterpret_cast<cplx<T>*>(W.spec);
  const size_t fieldsz = (size_t)Nz * (Ny + 1) * P.Px;     // capacity of one spectrum slot
  cplx<T>* Sp = p ? S + 3 * fieldsz : nullptr;
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(W.tw_x);
  const cplx<T>* twz = reinterpret_cast<const cplx<T>*>(W.tw_z);
  const int R = Nz * (3 * Ny + 1);
  cudaError_t e = fft_x_forward<T>(P, f, R, S, T(1), 1 << 30, T(0), T(0), twx, s, static_cast<const T*>(nullptr));
  if (e != cudaSuccess) return e;
  e = fft_z_mac<T>(P, S, false, twz, s);
  if (e != cudaSuccess) return e;
  e = launch_stokes_y<T>(P, W, S, Sp, s);
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

// With residual refinement (mixed precision, max_refine > 0): the forcing is
// kept (f and v may alias), the single-precision solve gives v and p, both
// are carried in double, and each sweep solves for the correction from the
// double-precision residual of the MAC operator (k_refine.cu).  The
// corrections accumulate in double; v and p are the rounded results.
template <typename T>
cudaError_t launch_stokes(const Params& P, Workspace& W, const T* f, T* v, T* p, cudaStream_t s) {
  const int sweeps = (sizeof(T) == sizeof(float) && W.sref) ? P.max_refine : 0;
  if (sweeps == 0) return stokes_once<T>(P, W, f, v, p, s);
  const size_t G = (size_t)P.Nx * P.Ny * P.Nz;
  const size_t Gf = (size_t)P.Nx * P.Nz * (3 * P.Ny + 1);
  T* fk = reinterpret_cast<T*>(W.sref);
  T* res = reinterpret_cast<T*>(W.sres);
  T* pw = reinterpret_cast<T*>(W.pres);
  cudaError_t e = cudaMemcpyAsync(fk, f, sizeof(T) * Gf, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_fill_zero<double>(W.snorm, 2 * (DISCOS_MAX_REFINE + 1), s);
  if (e == cudaSuccess) e = stokes_once<T>(P, W, fk, v, pw, s);
  if (e == cudaSuccess) e = launch_convert<double, T>(W.v64, v, Gf, s);
  if (e == cudaSuccess) e = launch_convert<double, T>(W.p64, pw, G, s);
  for (int it = 0; it < sweeps && e == cudaSuccess; ++it) {
    e = launch_stokes_residual<T>(P, fk, W.v64, W.p64, res, W.snorm + 2 * it, s);
    if (e == cudaSuccess) e = stokes_once<T>(P, W, res, res, pw, s);
    if (e == cudaSuccess) e = launch_accumulate<T>(W.v64, res, Gf, s);
    if (e == cudaSuccess) e = launch_accumulate<T>(W.p64, pw, G, s);
  }
  if (e == cudaSuccess) e = launch_stokes_residual<T>(P, fk, W.v64, W.p64, (T*)nullptr, W.snorm + 2 * sweeps, s);
  if (e == cudaSuccess) e = launch_convert<T, double>(v, W.v64, Gf, s);
  if (e == cudaSuccess && p) e = launch_convert<T, double>(p, W.p64, G, s);
  return e;
}

template cudaError_t launch_stokes<float>(const Params&, Workspace&, const float*, float*, float*, cudaStream_t);
template cudaError_t launch_stokes<double>(const Params&, Workspace&, const double*, double*, double*, cudaStream_t);

}  // namespace discos
