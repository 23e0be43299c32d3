// Internal device helpers of libdiscos: types, rounding-explicit arithmetic,
// the IB kernels of App. B, the Philox4x32-10 generator and the near-wall
// mobility fit of Eq. fitfunction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

namespace discos {

enum { KP4 = 0, KP6 = 1, KES = 2 };

// ----------------------------------------------------------------- complex
template <typename T> struct cplx { T re, im; };
template <typename T> __host__ __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) {
  return {a.re - b.re, a.im - b.im};
}

// ------------------------------------------- arithmetic rounded once per op
// (no contraction into FMA): the pair and cell decisions must be taken by the
// same sequence of roundings on every platform.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// ----------------------------------------------------------------- kernels
struct KernelParams {
  int kind;      // KP4, KP6, KES
  int w;         // support width in grid points
  double alpha;  // ES: w / 2
  double beta;   // ES: beta
  double inv_norm;  // ES: 1 / int exp(beta (sqrt(1 - (z/alpha)^2) - 1)) dz
  double inv_alpha;
  // single-precision copies, so that float kernels convert nothing at run time
  float alpha_f, beta_f, inv_norm_f, inv_alpha_f;
};
__host__ __device__ __forceinline__ double kp_beta(const KernelParams& kp, double) { return kp.beta; }
__host__ __device__ __forceinline__ float kp_beta(const KernelParams& kp, float) { return kp.beta_f; }
__host__ __device__ __forceinline__ double kp_inv_norm(const KernelParams& kp, double) { return kp.inv_norm; }
__host__ __device__ __forceinline__ float kp_inv_norm(const KernelParams& kp, float) { return kp.inv_norm_f; }
__host__ __device__ __forceinline__ double kp_inv_alpha(const KernelParams& kp, double) { return kp.inv_alpha; }
__host__ __device__ __forceinline__ float kp_inv_alpha(const KernelParams& kp, float) { return kp.inv_alpha_f; }

// Second moment of the 6-point kernel, 59/60 - sqrt(29)/20.
#define PESKIN6_K (59.0 / 60.0 - 5.385164807134504 / 20.0)

// 4-point Peskin kernel, App. B Eq. peskin1d (grid spacing 1).
template <typename T> __host__ __device__ __forceinline__ T peskin4(T z) {
  T a = fabs(z);
  if (a <= T(1)) return (T(3) - T(2) * a + sqrt(T(1) + T(4) * a - T(4) * a * a)) * T(0.125);
  if (a <= T(2)) {
    T s = -T(7) + T(12) * a - T(4) * a * a;
    return (T(5) - T(2) * a - sqrt(s > T(0) ? s : T(0))) * T(0.125);
  }
  return T(0);
}

// 6-point Peskin kernel.  For z = r - m (r in [0,1), m in -2..3) the value is
// the m-th of the six weights fixed by the kernel's moment conditions (even
// and odd sums 1/2, first and third moments 0, second moment K, sum of squares
// constant, continuity at the support edge): a closed form in r and
// p = phi(r), with p the root of the quadratic sum-of-squares condition.
template <typename T> __host__ __device__ __forceinline__ T peskin6_p(T r, T K) {
  T r2 = r * r, r3 = r2 * r, r4 = r2 * r2, r5 = r4 * r, r6 = r3 * r3;
  T B = -(T(84) * K * r - T(66) * K + T(28) * r3 - T(66) * r2 - T(88) * r + T(183)) * T(1.0 / 24.0);
  T disc = -(T(1008) * K * K * r2 - T(1008) * K * K * r - T(108) * K * K + T(672) * K * r4 -
             T(1344) * K * r3 - T(1896) * K * r2 + T(2568) * K * r + T(324) * K + T(112) * r6 -
             T(336) * r5 - T(500) * r4 + T(1560) * r3 + T(748) * r2 - T(1584) * r - T(243)) * T(1.0 / 192.0);
  return (-B + sqrt(disc > T(0) ? disc : T(0))) * T(1.0 / 14.0);
}
template <typename T> __host__ __device__ __forceinline__ T peskin6(T z) {
  if (!(fabs(z) < T(3))) return T(0);
  const T K = T(PESKIN6_K);
  T fl = floor(z);
  T r = z - fl;
  int m = -(int)fl;
  T p = peskin6_p(r, K);
  T r2 = r * r, r3 = r2 * r;
  switch (m) {
    case -2: return -K * r * T(0.25) + K * T(0.25) + p * T(0.5) - r3 * T(1.0 / 12.0) + r2 * T(0.25) + r * T(1.0 / 12.0) - T(0.375);
    case -1: return K * r * T(0.5) - T(0.375) * K - T(1.5) * p + r3 * T(1.0 / 6.0) - T(0.375) * r2 - r * T(2.0 / 3.0) + T(19.0 / 16.0);
    case 0: return p;
    case 1: return -K * r * T(0.5) + K * T(0.25) + p - r3 * T(1.0 / 6.0) + r2 * T(0.25) + r * T(2.0 / 3.0) - T(0.375);
    case 2: return K * r * T(0.25) - K * T(0.25) - T(1.5) * p + r3 * T(1.0 / 12.0) - r2 * T(0.25) - r * T(1.0 / 12.0) + T(0.875);
    case 3: return K * T(0.125) + p * T(0.5) + r2 * T(0.125) - T(5.0 / 16.0);
  }
  return T(0);
}

// ES kernel, App. B Eq. eskernel.
template <typename T> __host__ __device__ __forceinline__ T eskernel(T z, const KernelParams& kp) {
  const T za = z * kp_inv_alpha(kp, T());
  T t = T(1) - za * za;
  if (t < T(0)) return T(0);
  return exp(kp_beta(kp, T()) * (sqrt(t) - T(1))) * kp_inv_norm(kp, T());
}

template <typename T> __host__ __device__ __forceinline__ T kval(T z, const KernelParams& kp) {
  if (kp.kind == KP4) return peskin4(z);
  if (kp.kind == KP6) return peskin6(z);
  return eskernel(z, kp);
}

// Single precision: the square root of Eq. peskin1d through the hardware
// reciprocal square root (about 2 ulp), x * rsqrt(x); its argument lies in
// [1, 2] inside the support.
__host__ __device__ __forceinline__ float sqrt_pos(float x) {
#ifdef __CUDA_ARCH__
  return x > 0.f ? x * rsqrtf(x) : 0.f;
#else
  return x > 0.f ? sqrtf(x) : 0.f;
#endif
}
__host__ __device__ __forceinline__ float peskin4(float z) {
  const float a = fabsf(z);
  if (a <= 1.f) return (3.f - 2.f * a + sqrt_pos(1.f + 4.f * a - 4.f * a * a)) * 0.125f;
  if (a <= 2.f) return (5.f - 2.f * a - sqrt_pos(-7.f + 12.f * a - 4.f * a * a)) * 0.125f;
  return 0.f;
}

// Derivatives d phi / dz of the three kernels (used by the thermal forcing,
// whose random finite difference is evaluated in its delta -> 0 form).
template <typename T> __device__ __forceinline__ T peskin4_d(T z) {
  T a = fabs(z), sg = z < T(0) ? T(-1) : T(1);
  if (a <= T(1)) {
    T s = sqrt(T(1) + T(4) * a - T(4) * a * a);
    return sg * (T(-2) + (T(2) - T(4) * a) / s) * T(0.125);
  }
  if (a < T(2)) {
    T s = -T(7) + T(12) * a - T(4) * a * a;
    s = sqrt(s > T(0) ? s : T(0));
    return sg * (T(-2) - (T(6) - T(4) * a) / s) * T(0.125);
  }
  return T(0);
}
// single precision: 1 / sqrt through the hardware reciprocal square root
__device__ __forceinline__ float peskin4_d(float z) {
  const float a = fabsf(z), sg = z < 0.f ? -1.f : 1.f;
  if (a <= 1.f) return sg * (-2.f + (2.f - 4.f * a) * rsqrtf(1.f + 4.f * a - 4.f * a * a)) * 0.125f;
  if (a < 2.f) {
    const float s = -7.f + 12.f * a - 4.f * a * a;
    return s > 0.f ? sg * (-2.f - (6.f - 4.f * a) * rsqrtf(s)) * 0.125f : 0.f;
  }
  return 0.f;
}
template <typename T> __device__ __forceinline__ T peskin6_d(T z) {
  if (!(fabs(z) < T(3))) return T(0);
  const T K = T(PESKIN6_K);
  T fl = floor(z);
  T r = z - fl;
  int m = -(int)fl;
  T r2 = r * r, r3 = r2 * r, r4 = r2 * r2, r5 = r4 * r, r6 = r3 * r3;
  T disc = -(T(1008) * K * K * r2 - T(1008) * K * K * r - T(108) * K * K + T(672) * K * r4 -
             T(1344) * K * r3 - T(1896) * K * r2 + T(2568) * K * r + T(324) * K + T(112) * r6 -
             T(336) * r5 - T(500) * r4 + T(1560) * r3 + T(748) * r2 - T(1584) * r - T(243)) * T(1.0 / 192.0);
  T Bp = -(T(84) * K + T(84) * r2 - T(132) * r - T(88)) * T(1.0 / 24.0);
  T dd = -(T(2016) * K * K * r - T(1008) * K * K + T(2688) * K * r3 - T(4032) * K * r2 -
           T(3792) * K * r + T(2568) * K + T(672) * r5 - T(1680) * r4 - T(2000) * r3 +
           T(4680) * r2 + T(1496) * r - T(1584)) * T(1.0 / 192.0);
  T sq = sqrt(disc > T(0) ? disc : T(0));
  T pp = (-Bp + dd / (T(2) * sq)) * T(1.0 / 14.0);
  switch (m) {
    case -2: return (-K * T(0.25) - r2 * T(0.25) + r * T(0.5) + T(1.0 / 12.0)) + T(0.5) * pp;
    case -1: return (K * T(0.5) + r2 * T(0.5) - T(0.75) * r - T(2.0 / 3.0)) - T(1.5) * pp;
    case 0: return pp;
    case 1: return (-K * T(0.5) - r2 * T(0.5) + r * T(0.5) + T(2.0 / 3.0)) + pp;
    case 2: return (K * T(0.25) + r2 * T(0.25) - r * T(0.5) - T(1.0 / 12.0)) - T(1.5) * pp;
    case 3: return r * T(0.25) + T(0.5) * pp;
  }
  return T(0);
}
template <typename T> __device__ __forceinline__ T eskernel_d(T z, const KernelParams& kp) {
  const T ia = kp_inv_alpha(kp, T()), be = kp_beta(kp, T());
  const T za = z * ia;
  T t = T(1) - za * za;
  if (t <= T(0)) return T(0);
  T s = sqrt(t);
  return exp(be * (s - T(1))) * kp_inv_norm(kp, T()) * be * (-za * ia) / s;
}
template <typename T> __device__ __forceinline__ T kder(T z, const KernelParams& kp) {
  if (kp.kind == KP4) return peskin4_d(z);
  if (kp.kind == KP6) return peskin6_d(z);
  return eskernel_d(z, kp);
}

// Stencil start along one axis: grid points at integers, coordinate s,
// w points floor(s - w/2) + 1 .. floor(s - w/2) + w.
template <typename T> __host__ __device__ __forceinline__ int stencil_start(T s, int w) {
  return (int)floor(s - T(0.5) * T(w)) + 1;
}

// ----------------------------------------------------------------- Philox
struct u32x4 { uint32_t x, y, z, w; };
__host__ __device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
#else
    uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

// Four standard normals from one counter: uniforms (u + 1/2) 2^-32, then two
// Box-Muller pairs.
__device__ __forceinline__ void normals4(u32x4 c, uint64_t seed, double out[4]) {
  u32x4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double s = 2.3283064365386963e-10;  // 2^-32
  double u0 = ((double)r.x + 0.5) * s, u1 = ((double)r.y + 0.5) * s;
  double u2 = ((double)r.z + 0.5) * s, u3 = ((double)r.w + 0.5) * s;
  double a = sqrt(-2.0 * log(u0)), b = sqrt(-2.0 * log(u2));
  double s1, c1, s3, c3;
  sincospi(2.0 * u1, &s1, &c1);
  sincospi(2.0 * u3, &s3, &c3);
  out[0] = a * c1; out[1] = a * s1; out[2] = b * c3; out[3] = b * s3;
}
// Single precision: the hardware approximations of log and sin/cos (absolute
// error near 2^-21 on these arguments, far below the mixed path's
// tolerances) keep the Box-Muller transform off the slow library paths.
__device__ __forceinline__ void normals4(u32x4 c, uint64_t seed, float out[4]) {
  u32x4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float s = 2.3283064365386963e-10f, h = 1.1641532182693481e-10f;  // 2^-32, 2^-33
  const float twopi = 6.283185307179586f;
  float u0 = fmaf((float)r.x, s, h), u1 = fmaf((float)r.y, s, h);
  float u2 = fmaf((float)r.z, s, h), u3 = fmaf((float)r.w, s, h);
  float a = sqrtf(-2.0f * __logf(u0)), b = sqrtf(-2.0f * __logf(u2));
  float s1, c1, s3, c3;
  __sincosf(twopi * u1, &s1, &c1);
  __sincosf(twopi * u3, &s3, &c3);
  out[0] = a * c1; out[1] = a * s1; out[2] = b * c3; out[3] = b * s3;
}

// The first two of the four normals of normals4 (one Box-Muller pair), for
// draws that use only those.
__device__ __forceinline__ void normals2(u32x4 c, uint64_t seed, double out[2]) {
  u32x4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double s = 2.3283064365386963e-10;
  double u0 = ((double)r.x + 0.5) * s, u1 = ((double)r.y + 0.5) * s;
  double a = sqrt(-2.0 * log(u0));
  double s1, c1;
  sincospi(2.0 * u1, &s1, &c1);
  out[0] = a * c1; out[1] = a * s1;
}
__device__ __forceinline__ void normals2(u32x4 c, uint64_t seed, float out[2]) {
  u32x4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float s = 2.3283064365386963e-10f, h = 1.1641532182693481e-10f;
  float u0 = fmaf((float)r.x, s, h), u1 = fmaf((float)r.y, s, h);
  float a = sqrtf(-2.0f * __logf(u0));
  float s1, c1;
  __sincosf(6.283185307179586f * u1, &s1, &c1);
  out[0] = a * c1; out[1] = a * s1;
}

enum { TAG_DRY = 1, TAG_RFD = 2, TAG_STRESS_A = 3, TAG_STRESS_B = 4 };

// ------------------------------------------------------------ warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

}  // namespace discos
