// Device functions of the particle physics shared by the single-channel
// kernels and the batched step: list-cell coordinates, the minimum image,
// the F^P table lookup, the near-field pair terms (Eqs. fullElectro, LC,
// closerange), the wall force (Sec. II.B.2) and the near-wall mobility fit
// (Eq. fitfunction).
#pragma once
#include "internal.h"

namespace discos {

template <typename T>
__device__ __forceinline__ int cell_coord(T v, int k, int nc) {
  int c = (int)floor(v);
  c = c < 0 ? 0 : c / k;
  return c < nc ? c : nc - 1;
}

// A periodic coordinate (x or z) moved into [0, L): one shift by L for the
// positions a step can produce, a floor-based wrap (then a clamp against the
// rounding of v - L floor(v / L)) for anything further out.  Positions
// already inside are returned unchanged.
template <typename T>
__device__ __forceinline__ T wrap_coord(T v, int Li) {
  const T L = T(Li);
  if (v >= T(0) && v < L) return v;
  T w = v < T(0) ? v + L : v - L;
  if (!(w >= T(0) && w < L)) w = v - L * floor(v / L);
  return (w >= T(0) && w < L) ? w : T(0);
}

// Packed (x, y, z, q) of one ion, one vector load in the pair loop.
struct alignas(32) double4a { double x, y, z, w; };
template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4a type; };
__device__ __forceinline__ float4 make_vec4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ double4a make_vec4(double a, double b, double c, double d) { return double4a{a, b, c, d}; }
__device__ __forceinline__ void load_vec4(const float4& v, float& a, float& b, float& c, float& d) {
  a = v.x; b = v.y; c = v.z; d = v.w;
}
__device__ __forceinline__ void load_vec4(const double4a& v, double& a, double& b, double& c, double& d) {
  a = v.x; b = v.y; c = v.z; d = v.w;
}

template <typename T>
__device__ __forceinline__ T min_image(T d, T L, T half) {
  if (d > half) return sub_rn(d, L);
  if (d < -half) return add_rn(d, L);
  return d;
}

template <typename T>
__device__ __forceinline__ T fp_lookup(const T* __restrict__ tab, int n_tab, T scale, T r) {
  T t = r * scale;
  int k = (int)t;
  if (k > n_tab - 1) k = n_tab - 1;
  T fr = t - T(k);
  T a = tab[k], b = tab[k + 1];
  return a + fr * (b - a);
}

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <typename T>
__device__ __forceinline__ void pair_terms(const T xi, const T yi, const T zi, const T qi, const int si,
                                           const T xj, const T yj, const T zj, const T qj, const int sj,
                                           bool real, const Params& P, const T* __restrict__ tab, T Lx, T hx,
                                           T Lz, T hz, T psi2, T lB, T scale, T& fx, T& fy, T& fz, int& cnt) {
  const auto& Q = phys(P, T());
  T ddx = min_image(sub_rn(xi, xj), Lx, hx);
  T ddy = sub_rn(yi, yj);
  T ddz = min_image(sub_rn(zi, zj), Lz, hz);
  T r2 = add_rn(add_rn(mul_rn(ddx, ddx), mul_rn(ddy, ddy)), mul_rn(ddz, ddz));
  bool in_psi = r2 < psi2;
  bool in_lj = false;
  T rcl = T(0);
  if (real) {
    rcl = T(Q.lj_rc[si][sj]);
    in_lj = r2 < mul_rn(rcl, rcl);
  }
  if (!(in_psi || in_lj)) return;
  const T r = sqrt(r2);
  const T ir = recip(r);
  const T ir2 = ir * ir;
  T coef = T(0);
  if (in_psi) {
    coef += lB * qi * qj * (ir2 - fp_lookup(tab, P.n_tab, scale, r));
    ++cnt;
  }
  if (in_lj) {
    T sg = T(Q.lj_sigma[si][sj]);
    T sr2 = sg * sg * ir2;
    T sr6 = sr2 * sr2 * sr2;
    coef += T(24) * T(Q.lj_xi[si][sj]) * ir * (T(2) * sr6 * sr6 - sr6);
  }
  T cr = coef * ir;
  fx += cr * ddx; fy += cr * ddy; fz += cr * ddz;
}

// Short-range wall force on an ion of species si at height y (Sec. II.B.2):
// 12-6 repulsion or the 9-3 form of Eq. LJ93, from each wall within its cutoff.
template <typename T>
__device__ __forceinline__ T wall_force_y(const Params& P, int si, T yi) {
  const auto& Q = phys(P, T());
  T fy = T(0);
  const T rc = T(Q.wall_rc[si]), sg = T(Q.wall_sigma[si]), xiw = T(Q.wall_xi[si]);
  for (int wall = 0; wall < 2; ++wall) {
    T d = wall == 0 ? yi : sub_rn(T(P.Ny), yi);
    if (!(d < rc)) continue;
    T f;
    if (P.wall_type == DISCOS_WALL_WCA) {
      T sr2 = sg * sg / (d * d);
      T sr6 = sr2 * sr2 * sr2;
      f = T(24) * xiw / d * (T(2) * sr6 * sr6 - sr6);
    } else {
      T s3 = sg * sg * sg;
      T d2 = d * d, d4 = d2 * d2;
      f = T(1.5) * sqrt(T(3)) * xiw * (T(9) * s3 * s3 * s3 / (d4 * d4 * d2) - T(3) * s3 / d4);
    }
    fy += wall == 0 ? f : -f;
  }
  return fy;
}

// gamma(yt) and dgamma/dyt of the fit of Eq. fitfunction at distance yt from the wall.
template <typename T, typename C>
__device__ __forceinline__ void fit_gamma(const C* c, T yt, T& g, T& dg) {
  T a3 = T(c[2]) + yt, a5 = T(c[4]) + yt, a7 = T(c[6]) + yt;
  T i3 = recip(a3), i5 = recip(a5), i7 = recip(a7);
  T i5_2 = i5 * i5, i7_2 = i7 * i7;
  g = T(c[0]) + T(c[1]) * i3 + T(c[3]) * i5_2 * i5 + T(c[5]) * i7_2 * i7_2 * i7;
  dg = -T(c[1]) * i3 * i3 - T(3) * T(c[3]) * i5_2 * i5_2 - T(5) * T(c[5]) * i7_2 * i7_2 * i7_2;
}

// Flags an updated position in the device fault word: non-finite (bit 0) or
// outside the channel after the wall reflection (bit 1, a displacement larger
// than the channel).  The position is left as it is.
template <typename T>
__device__ __forceinline__ void check_position(const Params& P, const T p[3]) {
  if (!P.fault) return;
  if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) atomicOr(P.fault, 1u);
  else if (p[1] < T(0) || p[1] > T(P.Ny)) atomicOr(P.fault, 2u);
}

// One Euler-Maruyama step of the dry part of Eq. ions3 for one ion of species
// sp: dt (D^dry Gamma F / kT + div D^dry) + sqrt(2 dt D^dry Gamma) W, with
// Gamma = (gamma^tot D^tot - gamma^wet D^wet) / D^dry (Eqs. diff1-diff2) from
// the fit in the distance to the nearest wall and the Ito drift along y; plus
// dt V when V is given (Eq. step2).  p is wrapped in x, z and reflected at
// the walls in place.
template <typename T>
__device__ __forceinline__ void dry_move(const Params& P, int sp, T p[3], const T F[3], const T* V, const T W[3]) {
  const T Ny = T(P.Ny);
  const T y = p[1];
  const T yt = y <= Ny - y ? y : Ny - y;
  const T side = y <= Ny - y ? T(1) : T(-1);
  const auto& Q = phys(P, T());
  const T Dt = T(Q.D_tot[sp]), Dw = T(Q.D_wet[sp]), Dd = T(Q.D_dry[sp]), iDd = T(Q.inv_D_dry[sp]);
  T Gam[2], dGam[2];
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    T gt, dgt, gw, dgw;
    fit_gamma(Q.gamma[sp][dir][0], yt, gt, dgt);
    fit_gamma(Q.gamma[sp][dir][1], yt, gw, dgw);
    Gam[dir] = (gt * Dt - gw * Dw) * iDd;
    dGam[dir] = (dgt * Dt - dgw * Dw) * iDd * side;
  }
  const T dt = T(Q.dt), ikT = T(Q.inv_kT);
  const int L[3] = {P.Nx, P.Ny, P.Nz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T G = d == 1 ? Gam[1] : Gam[0];
    T inc = dt * (Dd * G * F[d] * ikT);
    if (d == 1 && P.drift) inc += dt * Dd * dGam[1];
    inc += sqrt(T(2) * dt * Dd * (G > T(0) ? G : T(0))) * W[d];
    if (V) inc = dt * V[d] + inc;
    T v = p[d] + inc;
    if (d == 1) {
      v = v < T(0) ? -v : (v > Ny ? T(2) * Ny - v : v);
    } else {
      T Ld = T(L[d]);
      v = v < T(0) ? v + Ld : (v >= Ld ? v - Ld : v);
    }
    p[d] = v;
  }
}

}  // namespace discos
