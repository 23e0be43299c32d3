// Spreading (Eq. kernel2) of charges onto cell centres and of forces onto the
// MAC faces, with the wall image construction of Sec. II.A (Fig. folded) and
// Sec. II.B.1 applied as an index fold: a stencil point outside the channel
// is mapped to its mirror inside with the image sign.  Also the fill kernels.
//
// Thread layout: a group of 8 lanes per ion (4 ions per warp); lane l owns
// x-offset l of the stencil, so each warp-wide atomic touches 4 short runs of
// consecutive addresses.  The y and z weights are computed by the lanes of
// the group and broadcast with shuffles.
#include <cstdint>
#include <type_traits>
#include "internal.h"

namespace discos {

namespace {

// Ions in cell order put the stencils of neighbouring lanes on the same grid
// points, and their atomics then serialise.  Spreading visits the ions in
// the order ion(g) = g * stride mod N (stride coprime with N, so the map is
// a bijection; see spread_stride), which scatters each warp's ions over the
// channel; stride 0 keeps the given order.
__device__ __forceinline__ int spread_ion(int g, int N, unsigned long long stride) {
  if (!stride || g >= N) return g;
  return (int)(((unsigned long long)g * stride) % (unsigned long long)N);
}

template <typename T>
__global__ void k_spread_charge(const T* __restrict__ x, const T* __restrict__ q, int N, Params P,
                                T* __restrict__ rho, unsigned long long stride) {
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const KernelParams kp = P.kes;
  const int w = kp.w;
  int ion = spread_ion((blockIdx.x * blockDim.x + threadIdx.x) >> 3, N, stride);
  int l = threadIdx.x & 7;
  int gbase = (threadIdx.x & 31) & ~7;
  bool valid = ion < N;
  T px = T(0.5), py = T(0.5), pz = T(0.5), qq = T(0);
  if (valid) {
    px = x[ion]; py = x[N + ion]; pz = x[2 * N + ion]; qq = q[ion];
  }
  T sx = px - T(0.5), sy = py - T(0.5), sz = pz - T(0.5);
  int x0 = stencil_start(sx, w), y0 = stencil_start(sy, w), z0 = stencil_start(sz, w);
  T wx = l < w ? kval(sx - T(x0 + l), kp) : T(0);
  T wy = l < w ? kval(sy - T(y0 + l), kp) : T(0);
  T wz = l < w ? kval(sz - T(z0 + l), kp) : T(0);
  int ix = (x0 + l) & (Nx - 1);
  const T s0 = P.bc[0] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
  const T s1 = P.bc[1] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
  for (int jz = 0; jz < w; ++jz) {
    T wzj = __shfl_sync(0xffffffffu, wz, gbase + jz);
    int iz = (z0 + jz) & (Nz - 1);
    for (int jy = 0; jy < w; ++jy) {
      T wyj = __shfl_sync(0xffffffffu, wy, gbase + jy);
      int iy = y0 + jy;
      T sg = T(1);
      if (iy < 0) { iy = -1 - iy; sg = s0; }
      else if (iy >= Ny) { iy = 2 * Ny - 1 - iy; sg = s1; }
      if (P.strip && y0 + jy < 0) sg = on_strip(P, ix) ? T(-1) : T(1);
      if (valid && l < w && iy >= 0 && iy < Ny)
        atomicAdd(&rho[((size_t)iz * Ny + iy) * Nx + ix], qq * sg * wzj * wyj * wx);
    }
  }
}

// Force spreading for one MAC component c (blockIdx.y), with images of sign
// -1 for the normal component and for the tangential ones at a no-slip wall,
// +1 for the tangential ones at a slip wall.  With rfd, adds the thermal forcing of
// Eq. thermforce: the random finite difference
//   (kT/delta) [S(x + delta W/2) W - S(x - delta W/2) W]
// in its delta -> 0 form kT W_c (W . grad_x) S, which equals the finite
// difference to O(delta^2) and has no cancellation in single precision.
template <typename T>
__global__ void k_spread_force(const T* __restrict__ x, const T* __restrict__ F, int N, Params P,
                               T* __restrict__ f, long long step, int rfd, const int* __restrict__ noise_index,
                               unsigned long long stride, const int* __restrict__ sp) {
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const KernelParams kp = P.khy;
  const int w = kp.w;
  const int c = blockIdx.y;
  int ion = spread_ion((blockIdx.x * blockDim.x + threadIdx.x) >> 3, N, stride);
  int l = threadIdx.x & 7;
  int gbase = (threadIdx.x & 31) & ~7;
  bool valid = ion < N && (P.hy_filter < 0 || sp[ion] == P.hy_filter);
  T p[3] = {T(0.5), T(0.5), T(0.5)};
  T Fc = T(0);
  T Wr[3] = {T(0), T(0), T(0)};
  if (valid) {
    p[0] = x[ion]; p[1] = x[N + ion]; p[2] = x[2 * N + ion];
    Fc = F[(size_t)c * N + ion];
    if (rfd) {
      T g[4];
      const int key = noise_index ? noise_index[ion] : ion;
      normals4(u32x4{(uint32_t)key, (uint32_t)step, 0u, (uint32_t)TAG_RFD}, P.seed, g);
      Wr[0] = g[0]; Wr[1] = g[1]; Wr[2] = g[2];
    }
  }
  // grid point 0 sits at offset 0 along axis c (faces) and 1/2 otherwise
  T s[3];
  int st[3];
  T wv[3], wd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    s[d] = p[d] - (d == c ? T(0) : T(0.5));
    st[d] = stencil_start(s[d], w);
    T z = s[d] - T(st[d] + l);
    wv[d] = l < w ? kval(z, kp) : T(0);
    wd[d] = (l < w && rfd) ? kder(z, kp) : T(0);
  }
  const T a = T(P.kT) * Wr[c];
  const int Nyg = (c == 1) ? Ny + 1 : Ny;
  size_t off = 0;
  if (c >= 1) off += (size_t)Nz * Ny * Nx;
  if (c == 2) off += (size_t)Nz * (Ny + 1) * Nx;
  T* g = f + off;
  int ix = (st[0] + l) & (Nx - 1);
  for (int jz = 0; jz < w; ++jz) {
    T wzj = __shfl_sync(0xffffffffu, wv[2], gbase + jz);
    T dzj = __shfl_sync(0xffffffffu, wd[2], gbase + jz);
    int iz = (st[2] + jz) & (Nz - 1);
    for (int jy = 0; jy < w; ++jy) {
      T wyj = __shfl_sync(0xffffffffu, wv[1], gbase + jy);
      T dyj = __shfl_sync(0xffffffffu, wd[1], gbase + jy);
      int iy = st[1] + jy;
      T sg = T(1);
      bool ok = true;
      if (c == 1) {             // y-faces 0..Ny; wall faces receive real + image = 0
        if (iy < 0) { iy = -iy; sg = T(-1); }
        else if (iy > Ny) { iy = 2 * Ny - iy; sg = T(-1); }
        ok = iy > 0 && iy < Ny;
      } else {                  // cell-centred in y: tangential, like image at a slip wall
        if (iy < 0) { iy = -1 - iy; sg = P.slip[0] ? T(1) : T(-1); }
        else if (iy >= Ny) { iy = 2 * Ny - 1 - iy; sg = P.slip[1] ? T(1) : T(-1); }
        ok = iy >= 0 && iy < Ny;
      }
      T val = Fc * wv[0] * wyj * wzj;
      if (rfd) val += a * (Wr[0] * wd[0] * wyj * wzj + Wr[1] * wv[0] * dyj * wzj + Wr[2] * wv[0] * wyj * dzj);
      if (valid && l < w && ok) atomicAdd(&g[((size_t)iz * Nyg + iy) * Nx + ix], sg * val);
    }
  }
}

// The charge spread with the stencil width W fixed at compile time (4 and 6
// points): the y and z weights of the group are fetched once, the image fold
// of the W rows is resolved once per ion, and the stencil loops unroll into
// independent atomics.
template <typename T, int W>
__global__ void k_spread_charge_w(const T* __restrict__ x, const T* __restrict__ q, int N, Params P,
                                  T* __restrict__ rho, unsigned long long stride) {
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const KernelParams kp = P.kes;
  int ion = spread_ion((blockIdx.x * blockDim.x + threadIdx.x) >> 3, N, stride);
  int l = threadIdx.x & 7;
  int gbase = (threadIdx.x & 31) & ~7;
  bool valid = ion < N;
  T px = T(0.5), py = T(0.5), pz = T(0.5), qq = T(0);
  if (valid) { px = x[ion]; py = x[N + ion]; pz = x[2 * N + ion]; qq = q[ion]; }
  const T sx = px - T(0.5), sy = py - T(0.5), sz = pz - T(0.5);
  const int x0 = stencil_start(sx, W), y0 = stencil_start(sy, W), z0 = stencil_start(sz, W);
  const T wx = l < W ? kval(sx - T(x0 + l), kp) : T(0);
  const T wyl = l < W ? kval(sy - T(y0 + l), kp) : T(0);
  const T wzl = l < W ? kval(sz - T(z0 + l), kp) : T(0);
  const T s0 = P.bc[0] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
  const T s1 = P.bc[1] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
  T wy[W], wz[W];
  int roff[W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    wy[j] = __shfl_sync(0xffffffffu, wyl, gbase + j);
    wz[j] = __shfl_sync(0xffffffffu, wzl, gbase + j);
    int iy = y0 + j;
    T sg = T(1);
    if (iy < 0) { iy = -1 - iy; sg = s0; }
    else if (iy >= Ny) { iy = 2 * Ny - 1 - iy; sg = s1; }
    const bool in = iy >= 0 && iy < Ny;
    roff[j] = in ? iy * Nx : 0;
    wy[j] = in ? sg * wy[j] : T(0);
  }
  if (valid && l < W) {
    const int ix = (x0 + l) & (Nx - 1);
    const T qx = qq * wx;
    // a metal strip in the (dielectric) bottom wall: rows below the wall take
    // the conducting wall's sign in the strip's columns
    const T cs = on_strip(P, ix) ? T(-1) : T(1);
#pragma unroll
    for (int jz = 0; jz < W; ++jz) {
      const size_t zoff = (size_t)((z0 + jz) & (Nz - 1)) * Ny * Nx + ix;
      const T qz = qx * wz[jz];
#pragma unroll
      for (int jy = 0; jy < W; ++jy)
        if (wy[jy] != T(0)) atomicAdd(&rho[zoff + roff[jy]], qz * (y0 + jy < 0 ? cs : T(1)) * wy[jy]);
    }
  }
}

// LPI = lanes per ion: 4 for 4-point stencils (no idle lanes), else 8.
// One MAC component per blockIdx.y: the blocks of one component run before
// those of the next, so the grid that the atomics hit at any time is one
// component (a third of the forcing), which stays in L2.  (Spreading all
// three components from each thread shares the ion's loads and thermal draw
// but keeps the whole forcing hot at once; on the 256 x 128 x 256 channel
// that tripled the DRAM write-back and was slower.)
template <typename T, int W, int LPI>
__global__ void k_spread_force_w(const T* __restrict__ x, const T* __restrict__ F, int N, Params P,
                                 T* __restrict__ f, long long step, int rfd, const int* __restrict__ noise_index,
                                 unsigned long long stride, const int* __restrict__ sp) {
  constexpr int LOG = LPI == 4 ? 2 : 3;
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const KernelParams kp = P.khy;
  const int c = blockIdx.y;
  int ion = spread_ion((blockIdx.x * blockDim.x + threadIdx.x) >> LOG, N, stride);
  int l = threadIdx.x & (LPI - 1);
  int gbase = (threadIdx.x & 31) & ~(LPI - 1);
  bool valid = ion < N && (P.hy_filter < 0 || sp[ion] == P.hy_filter);
  T p[3] = {T(0.5), T(0.5), T(0.5)};
  T Fc = T(0);
  T Wr[3] = {T(0), T(0), T(0)};
  if (valid) {
    p[0] = x[ion]; p[1] = x[N + ion]; p[2] = x[2 * N + ion];
    Fc = F[(size_t)c * N + ion];
    if (rfd) {
      T g[4];
      const int key = noise_index ? noise_index[ion] : ion;
      normals4(u32x4{(uint32_t)key, (uint32_t)step, 0u, (uint32_t)TAG_RFD}, P.seed, g);
      Wr[0] = g[0]; Wr[1] = g[1]; Wr[2] = g[2];
    }
  }
  int st[3];
  T wv[3], wd[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T sd = p[d] - (d == c ? T(0) : T(0.5));
    st[d] = stencil_start(sd, W);
    const T z = sd - T(st[d] + l);
    wv[d] = l < W ? kval(z, kp) : T(0);
    wd[d] = (l < W && rfd) ? kder(z, kp) : T(0);
  }
  const T a = T(phys(P, T()).kT) * (c == 0 ? Wr[0] : (c == 1 ? Wr[1] : Wr[2]));
  const int Nyg = (c == 1) ? Ny + 1 : Ny;
  size_t off = 0;
  if (c >= 1) off += (size_t)Nz * Ny * Nx;
  if (c == 2) off += (size_t)Nz * (Ny + 1) * Nx;
  T* g = f + off;
  T wy[W], dy[W], wz[W], dz[W];
  int roff[W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    wy[j] = __shfl_sync(0xffffffffu, wv[1], gbase + j);
    dy[j] = __shfl_sync(0xffffffffu, wd[1], gbase + j);
    wz[j] = __shfl_sync(0xffffffffu, wv[2], gbase + j);
    dz[j] = __shfl_sync(0xffffffffu, wd[2], gbase + j);
    int iy = st[1] + j;
    T sg = T(1);
    bool ok;
    if (c == 1) {             // y-faces 0..Ny; wall faces receive real + image = 0
      if (iy < 0) { iy = -iy; sg = T(-1); }
      else if (iy > Ny) { iy = 2 * Ny - iy; sg = T(-1); }
      ok = iy > 0 && iy < Ny;
    } else {                  // cell-centred in y: tangential, like image at a slip wall
      if (iy < 0) { iy = -1 - iy; sg = P.slip[0] ? T(1) : T(-1); }
      else if (iy >= Ny) { iy = 2 * Ny - 1 - iy; sg = P.slip[1] ? T(1) : T(-1); }
      ok = iy >= 0 && iy < Ny;
    }
    roff[j] = ok ? iy * Nx : 0;
    const T keep = ok ? sg : T(0);
    wy[j] *= keep;
    dy[j] *= keep;
  }
  if (valid && l < W) {
    const int ix = (st[0] + l) & (Nx - 1);
    // value at (jy, jz) = ay[jy] wz[jz] + cy[jy] dz[jz]: the force term
    // Fc wx wy wz and the three RFD terms a W_d (d/dd of the kernel product)
    // grouped by their z factor, so a point costs one multiply-add pair
    const T fx0 = Fc * wv[0];
    const T r0 = a * Wr[0] * wd[0], r1 = a * Wr[1] * wv[0], r2 = a * Wr[2] * wv[0];
    T ay[W], cy[W];
#pragma unroll
    for (int jy = 0; jy < W; ++jy) {
      ay[jy] = rfd ? (fx0 + r0) * wy[jy] + r1 * dy[jy] : fx0 * wy[jy];
      cy[jy] = rfd ? r2 * wy[jy] : T(0);
    }
#pragma unroll
    for (int jz = 0; jz < W; ++jz) {
      T* gz = g + (size_t)((st[2] + jz) & (Nz - 1)) * Nyg * Nx + ix;
#pragma unroll
      for (int jy = 0; jy < W; ++jy) {
        if (wy[jy] == T(0) && dy[jy] == T(0)) continue;
        atomicAdd(gz + roff[jy], ay[jy] * wz[jz] + cy[jy] * dz[jz]);
      }
    }
  }
}

// Single-precision charge spreading for 4-point stencils, one thread per
// ion.  The thread evaluates the 4 weights per axis once, walks the 16
// x-rows (jy, jz) of the 4 x 4 x 4 stencil, and adds each row's four values
// with 16-byte vector reductions (atomicAdd on float4, red.global.add.v4.f32)
// on the aligned quads of x that the row covers: one quad when the row
// starts on a multiple of 4, else two, the other slots adding zero.  Images
// and signs as in k_spread_charge_w.  Needs a 16-byte aligned grid and Nx a
// multiple of 4 (quads never straddle the periodic wrap).  (For the MAC
// forcing, a grid three times larger, the same scheme lost to the lane
// groups: its scattered vector reductions thrash the L2.)
__device__ __forceinline__ void red_row4(float* row, int ix0, int Nx, float v0, float v1, float v2, float v3) {
  const int o = ix0 & 3;
  const int q0 = ix0 - o;
  float4* a = reinterpret_cast<float4*>(row + q0);
  if (o == 0) {
    atomicAdd(a, make_float4(v0, v1, v2, v3));
    return;
  }
  float4* b = reinterpret_cast<float4*>(row + ((q0 + 4) & (Nx - 1)));
  if (o == 1) {
    atomicAdd(a, make_float4(0.f, v0, v1, v2));
    atomicAdd(b, make_float4(v3, 0.f, 0.f, 0.f));
  } else if (o == 2) {
    atomicAdd(a, make_float4(0.f, 0.f, v0, v1));
    atomicAdd(b, make_float4(v2, v3, 0.f, 0.f));
  } else {
    atomicAdd(a, make_float4(0.f, 0.f, 0.f, v0));
    atomicAdd(b, make_float4(v1, v2, v3, 0.f));
  }
}

__global__ void k_spread_charge_t4(const float* __restrict__ x, const float* __restrict__ q, int N, Params P,
                                   float* __restrict__ rho, unsigned long long stride) {
  const int ion = spread_ion(blockIdx.x * blockDim.x + threadIdx.x, N, stride);
  if (ion >= N) return;
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const KernelParams kp = P.kes;
  const float sx = x[ion] - 0.5f, sy = x[N + ion] - 0.5f, sz = x[2 * N + ion] - 0.5f, qq = q[ion];
  const int x0 = stencil_start(sx, 4), y0 = stencil_start(sy, 4), z0 = stencil_start(sz, 4);
  float wx[4], wy[4], wz[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    wx[j] = kval(sx - float(x0 + j), kp);
    wy[j] = kval(sy - float(y0 + j), kp);
    wz[j] = kval(sz - float(z0 + j), kp);
  }
  const int ix0 = x0 & (Nx - 1);
  // a metal strip in the (dielectric) bottom wall: rows below the wall take
  // the conducting wall's sign in the strip's columns
  float cs[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) cs[i] = on_strip(P, (ix0 + i) & (Nx - 1)) ? -1.f : 1.f;
  const float s0 = P.bc[0] == DISCOS_BC_DIRICHLET ? -1.f : 1.f;
  const float s1 = P.bc[1] == DISCOS_BC_DIRICHLET ? -1.f : 1.f;
#pragma unroll
  for (int jy = 0; jy < 4; ++jy) {
    int iy = y0 + jy;
    float sg = 1.f;
    const bool below = iy < 0;
    if (below) { iy = -1 - iy; sg = s0; }
    else if (iy >= Ny) { iy = 2 * Ny - 1 - iy; sg = s1; }
    if (iy < 0 || iy >= Ny) continue;
    const float a = qq * sg * wy[jy];
    const float c0 = below ? cs[0] : 1.f, c1 = below ? cs[1] : 1.f, c2 = below ? cs[2] : 1.f,
                c3 = below ? cs[3] : 1.f;
#pragma unroll
    for (int jz = 0; jz < 4; ++jz) {
      const float b = a * wz[jz];
      float* row = rho + ((size_t)((z0 + jz) & (Nz - 1)) * Ny + iy) * Nx;
      red_row4(row, ix0, Nx, b * c0 * wx[0], b * c1 * wx[1], b * c2 * wx[2], b * c3 * wx[3]);
    }
  }
}

template <typename T>
__global__ void k_fill(T* __restrict__ p, size_t n, T value) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) p[i] = value;
}

}  // namespace

template <typename T>
cudaError_t launch_fill_value(T* p, size_t n, T value, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int bs = 256;
  size_t nb = (n + bs - 1) / bs;
  if (nb > 152 * 16) nb = 152 * 16;
  k_fill<T><<<(unsigned)nb, bs, 0, s>>>(p, n, value);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill_zero(T* p, size_t n, cudaStream_t s) {
  return launch_fill_value<T>(p, n, T(0), s);
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// A prime near 0.618 N that does not divide N: g * stride mod N is then a
// bijection that sends consecutive g about 0.618 N apart (Fibonacci
// hashing).  0 (the given order) for N < 3.
static unsigned long long spread_stride(int N) {
  if (N < 3) return 0ull;
  auto prime = [](unsigned long long v) {
    if (v < 2) return false;
    for (unsigned long long d = 2; d * d <= v; ++d)
      if (v % d == 0) return false;
    return true;
  };
  unsigned long long p = (unsigned long long)(0.6180339887498949 * N);
  if (p < 2) p = 2;
  while (!prime(p) || (unsigned long long)N % p == 0) ++p;
  return p;
}

template <typename T>
cudaError_t launch_spread_charge(const Params& P, const T* x, const T* q, int N, T* rho, cudaStream_t s,
                                 bool decorrelate) {
  probe_begin(PROBE_SPREAD_CHARGE, s);
  cudaError_t e = launch_fill_zero(rho, (size_t)P.Nx * P.Ny * P.Nz, s);
  if (e != cudaSuccess || N <= 0) {
    probe_end(PROBE_SPREAD_CHARGE, s);
    return e;
  }
  int bs = 256;
  int nb = (int)(((size_t)N * 8 + bs - 1) / bs);
  const unsigned long long st = decorrelate ? spread_stride(N) : 0ull;
  if (std::is_same<T, float>::value && P.kes.w == 4 && aligned16(rho))
    k_spread_charge_t4<<<(unsigned)(((size_t)N + bs - 1) / bs), bs, 0, s>>>(
        reinterpret_cast<const float*>(x), reinterpret_cast<const float*>(q), N, P, reinterpret_cast<float*>(rho), st);
  else if (P.kes.w == 4) k_spread_charge_w<T, 4><<<nb, bs, 0, s>>>(x, q, N, P, rho, st);
  else if (P.kes.w == 6) k_spread_charge_w<T, 6><<<nb, bs, 0, s>>>(x, q, N, P, rho, st);
  else k_spread_charge<T><<<nb, bs, 0, s>>>(x, q, N, P, rho, st);
  count_launches(1);
  probe_end(PROBE_SPREAD_CHARGE, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread_force(const Params& P, const T* x, const T* F, int N, T* f, int64_t step, bool rfd,
                                cudaStream_t s, bool accumulate, const int* noise_index, bool decorrelate,
                                const int* species) {
  size_t n = (size_t)P.Nx * P.Nz * (3 * P.Ny + 1);
  probe_begin(PROBE_SPREAD_FORCE, s);
  cudaError_t e = accumulate ? cudaSuccess : launch_fill_zero(f, n, s);
  if (e != cudaSuccess || N <= 0) {
    probe_end(PROBE_SPREAD_FORCE, s);
    return e;
  }
  int bs = 256;
  dim3 grid((unsigned)(((size_t)N * 8 + bs - 1) / bs), 3);
  const unsigned long long st = decorrelate ? spread_stride(N) : 0ull;
  const dim3 grid4((unsigned)(((size_t)N * 4 + bs - 1) / bs), 3);
  const dim3 grid8((unsigned)(((size_t)N * 8 + bs - 1) / bs), 3);
  auto one = [&](const Params& Q) {
    if (Q.khy.w == 4) k_spread_force_w<T, 4, 4><<<grid4, bs, 0, s>>>(x, F, N, Q, f, (long long)step, rfd ? 1 : 0, noise_index, st, species);
    else if (Q.khy.w == 6) k_spread_force_w<T, 6, 8><<<grid8, bs, 0, s>>>(x, F, N, Q, f, (long long)step, rfd ? 1 : 0, noise_index, st, species);
    else k_spread_force<T><<<grid, bs, 0, s>>>(x, F, N, Q, f, (long long)step, rfd ? 1 : 0, noise_index, st, species);
    count_launches(1);
  };
  for_each_hy_kernel(P, species, one);
  probe_end(PROBE_SPREAD_FORCE, s);
  return cudaGetLastError();
}

template cudaError_t launch_fill_value<float>(float*, size_t, float, cudaStream_t);
template cudaError_t launch_fill_value<double>(double*, size_t, double, cudaStream_t);
template cudaError_t launch_fill_zero<float>(float*, size_t, cudaStream_t);
template cudaError_t launch_fill_zero<double>(double*, size_t, cudaStream_t);
template cudaError_t launch_spread_charge<float>(const Params&, const float*, const float*, int, float*, cudaStream_t, bool);
template cudaError_t launch_spread_charge<double>(const Params&, const double*, const double*, int, double*, cudaStream_t, bool);
template cudaError_t launch_spread_force<float>(const Params&, const float*, const float*, int, float*, int64_t, bool, cudaStream_t, bool, const int*, bool, const int*);
template cudaError_t launch_spread_force<double>(const Params&, const double*, const double*, int, double*, int64_t, bool, cudaStream_t, bool, const int*, bool, const int*);

}  // namespace discos
