// Interpolation (Eq. kernel1) with ghost cells filled from the boundary
// conditions (Sec. II.A, Sec. II.B.1):
//  * the field E^P = J^es(-grad_h phi) of Eq. efieldop, E on the cell faces.
//    The face differences are folded into the weights, so each ion reads one
//    (w+1)^3 block of phi: E_x = sum_c phi_c (d_face(c+1) - d_face(c)) d_y d_z
//    and likewise for y and z;
//  * the fluid velocity J^hy v on the three face grids.
// Thread layout: 8 lanes per ion (4 for the 4-point velocity stencil), lane
// l owning x-offset l of the block, so every warp-wide load is a few runs of
// consecutive addresses; the partial sums are reduced with shuffles inside
// the group.  The step hands the ions over in cell order, so the ions of a
// warp read neighbouring grid lines (L1 reuse); out_index maps each result
// back to the caller's order.
#include <cstdint>
#include <type_traits>
#include "internal.h"

namespace discos {

namespace {

template <typename T>
__device__ __forceinline__ T group_sum8(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// phi at cell-centre row iy (possibly a ghost row), Eqs. esbc1 / esbc3:
// Dirichlet ghost -1-m = 2 phi_b - phi(m); Neumann ghost -1-m = phi(m) - g (2m+1)
// (top: Ny+m = phi(Ny-1-m) + g (2m+1)).
template <typename T>
__device__ __forceinline__ T phi_ghost(const T* __restrict__ phi, const Params& P, int iz, int iy, int ix) {
  const int Nx = P.Nx, Ny = P.Ny;
  if (iy >= 0 && iy < Ny) return phi[((size_t)iz * Ny + iy) * Nx + ix];
  if (iy < 0) {
    int m = -1 - iy;
    m = m < Ny ? m : Ny - 1;   // only reached by ions far outside the channel
    T v = phi[((size_t)iz * Ny + m) * Nx + ix];
    if (on_strip(P, ix)) return T(2) * strip_phi_m(P, ix, T()) - v;
    if (P.bc[0] == DISCOS_BC_DIRICHLET) return T(2) * T(phys(P, T()).phi_b[0]) - v;
    return v - T(phys(P, T()).slope[0]) * T(2 * m + 1);
  }
  int m = iy - Ny;
  m = m < Ny ? m : Ny - 1;
  T v = phi[((size_t)iz * Ny + (Ny - 1 - m)) * Nx + ix];
  if (P.bc[1] == DISCOS_BC_DIRICHLET) return T(2) * T(phys(P, T()).phi_b[1]) - v;
  return v + T(phys(P, T()).slope[1]) * T(2 * m + 1);
}

template <typename T>
__global__ void k_interp_efield(const T* __restrict__ x, const T* __restrict__ q, int N, Params P,
                                const T* __restrict__ phi, T* __restrict__ out, int as_force,
                                const T* __restrict__ F_add, const int* __restrict__ out_index) {
  const KernelParams kp = P.kes;
  const int w = kp.w;
  int ion = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  int l = threadIdx.x & 7;
  int gbase = (threadIdx.x & 31) & ~7;
  bool valid = ion < N;
  T p[3] = {T(0.5), T(0.5), T(0.5)};
  if (valid) { p[0] = x[ion]; p[1] = x[N + ion]; p[2] = x[2 * N + ion]; }
  // block of cells [fs - 1, fs + w - 1] per axis, fs = first face of the face stencil
  int c0[3];
  T cw[3], ew[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int fs = stencil_start(p[d], w);
    c0[d] = fs - 1;
    int c = c0[d] + l;
    bool in = l <= w;
    cw[d] = in ? kval(p[d] - (T(c) + T(0.5)), kp) : T(0);
    ew[d] = in ? (kval(p[d] - T(c + 1), kp) - kval(p[d] - T(c), kp)) : T(0);
  }
  const int ix = (c0[0] + l) & (P.Nx - 1);
  T Ex = T(0), Ey = T(0), Ez = T(0);
  for (int jz = 0; jz <= w; ++jz) {
    T cz = __shfl_sync(0xffffffffu, cw[2], gbase + jz);
    T ez = __shfl_sync(0xffffffffu, ew[2], gbase + jz);
    int iz = (c0[2] + jz) & (P.Nz - 1);
    for (int jy = 0; jy <= w; ++jy) {
      T cy = __shfl_sync(0xffffffffu, cw[1], gbase + jy);
      T ey = __shfl_sync(0xffffffffu, ew[1], gbase + jy);
      if (valid && l <= w) {
        T v = phi_ghost(phi, P, iz, c0[1] + jy, ix);
        Ex += v * ew[0] * cy * cz;
        Ey += v * cw[0] * ey * cz;
        Ez += v * cw[0] * cy * ez;
      }
    }
  }
  Ex = group_sum8(Ex);
  Ey = group_sum8(Ey);
  Ez = group_sum8(Ez);
  if (valid && l == 0) {
    const int o = out_index ? out_index[ion] : ion;
    if (as_force) {
      T qq = q[ion];
      T a0 = F_add ? F_add[ion] : T(0), a1 = F_add ? F_add[N + ion] : T(0), a2 = F_add ? F_add[2 * N + ion] : T(0);
      const auto& Q = phys(P, T());
      out[o] = qq * (Ex + T(Q.E_ext[0])) + a0;
      out[N + o] = qq * (Ey + T(Q.E_ext[1])) + a1;
      out[2 * N + o] = qq * (Ez + T(Q.E_ext[2])) + a2;
    } else {
      out[o] = Ex; out[N + o] = Ey; out[2 * N + o] = Ez;
    }
  }
}

template <typename T>
__global__ void k_interp_velocity(const T* __restrict__ x, int N, Params P, const T* __restrict__ v,
                                  T* __restrict__ out, const int* __restrict__ out_index,
                                  const int* __restrict__ sp) {
  const KernelParams kp = P.khy;
  const int w = kp.w;
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  int ion = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  int l = threadIdx.x & 7;
  int gbase = (threadIdx.x & 31) & ~7;
  bool valid = ion < N && (P.hy_filter < 0 || sp[ion] == P.hy_filter);
  T p[3] = {T(0.5), T(0.5), T(0.5)};
  if (valid) { p[0] = x[ion]; p[1] = x[N + ion]; p[2] = x[2 * N + ion]; }
  const size_t G = (size_t)Nx * Ny * Nz;
  for (int c = 0; c < 3; ++c) {
    const T* g = v + (c >= 1 ? G : 0) + (c == 2 ? (size_t)Nx * (Ny + 1) * Nz : 0);
    const int Nyg = c == 1 ? Ny + 1 : Ny;
    T s[3];
    int st[3];
    T wv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      s[d] = p[d] - (d == c ? T(0) : T(0.5));
      st[d] = stencil_start(s[d], w);
      wv[d] = l < w ? kval(s[d] - T(st[d] + l), kp) : T(0);
    }
    const int ix = (st[0] + l) & (Nx - 1);
    T acc = T(0);
    for (int jz = 0; jz < w; ++jz) {
      T wz = __shfl_sync(0xffffffffu, wv[2], gbase + jz);
      int iz = (st[2] + jz) & (Nz - 1);
      for (int jy = 0; jy < w; ++jy) {
        T wy = __shfl_sync(0xffffffffu, wv[1], gbase + jy);
        if (valid && l < w) {
          int iy = st[1] + jy;
          T sg = T(1);
          if (c == 1) {           // normal component: ghost face -m = -v(m)
            if (iy < 0) { iy = -iy; sg = T(-1); }
            else if (iy > Ny) { iy = 2 * Ny - iy; sg = T(-1); }
          } else {                // tangential: ghost -1-m = -u(m) (no slip) or +u(m) (slip)
            if (iy < 0) { iy = -1 - iy; sg = P.slip[0] ? T(1) : T(-1); }
            else if (iy >= Ny) { iy = 2 * Ny - 1 - iy; sg = P.slip[1] ? T(1) : T(-1); }
          }
          iy = iy < 0 ? 0 : (iy >= Nyg ? Nyg - 1 : iy);   // ions far outside only
          acc += sg * g[((size_t)iz * Nyg + iy) * Nx + ix] * wv[0] * wy * wz;
        }
      }
    }
    acc = group_sum8(acc);
    if (valid && l == 0) out[(size_t)c * N + (out_index ? out_index[ion] : ion)] = acc;
  }
}

// The same two gathers with the stencil width W fixed at compile time (4 and
// 6 points): each lane fetches the y and z weights of its group once, the
// wall rules of the W (+1) rows are resolved once per ion, and the stencil
// loops unroll into independent loads.
template <typename T, int W>
__global__ void k_interp_efield_w(const T* __restrict__ x, const T* __restrict__ q, int N, Params P,
                                  const T* __restrict__ phi, T* __restrict__ out, int as_force,
                                  const T* __restrict__ F_add, const int* __restrict__ out_index) {
  const KernelParams kp = P.kes;
  const int Nx = P.Nx, Ny = P.Ny;
  const auto& Q = phys(P, T());
  int ion = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  int l = threadIdx.x & 7;
  int gbase = (threadIdx.x & 31) & ~7;
  bool valid = ion < N;
  T p[3] = {T(0.5), T(0.5), T(0.5)};
  if (valid) { p[0] = x[ion]; p[1] = x[N + ion]; p[2] = x[2 * N + ion]; }
  int c0[3];
  T cw[3], ew[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    c0[d] = stencil_start(p[d], W) - 1;
    const int c = c0[d] + l;
    const bool in = l <= W;
    cw[d] = in ? kval(p[d] - (T(c) + T(0.5)), kp) : T(0);
    ew[d] = in ? (kval(p[d] - T(c + 1), kp) - kval(p[d] - T(c), kp)) : T(0);
  }
  T cy[W + 1], ey[W + 1], cz[W + 1], ez[W + 1], rs[W + 1], ra[W + 1];
  int roff[W + 1];
#pragma unroll
  for (int j = 0; j <= W; ++j) {
    cy[j] = __shfl_sync(0xffffffffu, cw[1], gbase + j);
    ey[j] = __shfl_sync(0xffffffffu, ew[1], gbase + j);
    cz[j] = __shfl_sync(0xffffffffu, cw[2], gbase + j);
    ez[j] = __shfl_sync(0xffffffffu, ew[2], gbase + j);
    // phi at row iy = rs * phi[row] + ra (ghost rows of Eqs. esbc1 / esbc3)
    const int iy = c0[1] + j;
    int row = iy;
    T sg = T(1), ad = T(0);
    if (iy < 0) {
      int m = -1 - iy;
      m = m < Ny ? m : Ny - 1;
      row = m;
      if (P.bc[0] == DISCOS_BC_DIRICHLET) { sg = T(-1); ad = T(2) * T(Q.phi_b[0]); }
      else ad = -T(Q.slope[0]) * T(2 * m + 1);
    } else if (iy >= Ny) {
      int m = iy - Ny;
      m = m < Ny ? m : Ny - 1;
      row = Ny - 1 - m;
      if (P.bc[1] == DISCOS_BC_DIRICHLET) { sg = T(-1); ad = T(2) * T(Q.phi_b[1]); }
      else ad = T(Q.slope[1]) * T(2 * m + 1);
    }
    roff[j] = row * Nx;
    rs[j] = sg;
    ra[j] = ad;
  }
  T Ex = T(0), Ey = T(0), Ez = T(0);
  if (valid && l <= W) {
    const int ix = (c0[0] + l) & (Nx - 1);
    // a metal strip in the bottom wall: the rows below it take the Dirichlet
    // rule with the strip potential of this column
    const bool strip_col = on_strip(P, ix);
    const T pm2 = strip_col ? T(2) * strip_phi_m(P, ix, T()) : T(0);
#pragma unroll
    for (int jz = 0; jz <= W; ++jz) {
      const size_t zoff = (size_t)((c0[2] + jz) & (P.Nz - 1)) * Ny * Nx + ix;
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int jy = 0; jy <= W; ++jy) {
        const bool sb = strip_col && c0[1] + jy < 0;
        const T v = sb ? pm2 - phi[zoff + roff[jy]] : rs[jy] * phi[zoff + roff[jy]] + ra[jy];
        a1 += v * cy[jy];
        a2 += v * ey[jy];
      }
      Ex += a1 * cz[jz];
      Ey += a2 * cz[jz];
      Ez += a1 * ez[jz];
    }
    Ex *= ew[0];
    Ey *= cw[0];
    Ez *= cw[0];
  }
  Ex = group_sum8(Ex);
  Ey = group_sum8(Ey);
  Ez = group_sum8(Ez);
  if (valid && l == 0) {
    const int o = out_index ? out_index[ion] : ion;
    if (as_force) {
      T qq = q[ion];
      T a0 = F_add ? F_add[ion] : T(0), a1 = F_add ? F_add[N + ion] : T(0), a2 = F_add ? F_add[2 * N + ion] : T(0);
      out[o] = qq * (Ex + T(Q.E_ext[0])) + a0;
      out[N + o] = qq * (Ey + T(Q.E_ext[1])) + a1;
      out[2 * N + o] = qq * (Ez + T(Q.E_ext[2])) + a2;
    } else {
      out[o] = Ex; out[N + o] = Ey; out[2 * N + o] = Ez;
    }
  }
}

// LPI = lanes per ion, the stencil width rounded up to 4 or 8.
template <typename T, int W, int LPI>
__global__ void k_interp_velocity_w(const T* __restrict__ x, int N, Params P, const T* __restrict__ v,
                                    T* __restrict__ out, const int* __restrict__ out_index,
                                    const int* __restrict__ sp) {
  constexpr int LOG = LPI == 4 ? 2 : 3;
  const KernelParams kp = P.khy;
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  int ion = (blockIdx.x * blockDim.x + threadIdx.x) >> LOG;
  int l = threadIdx.x & (LPI - 1);
  int gbase = (threadIdx.x & 31) & ~(LPI - 1);
  bool valid = ion < N && (P.hy_filter < 0 || sp[ion] == P.hy_filter);
  T p[3] = {T(0.5), T(0.5), T(0.5)};
  if (valid) { p[0] = x[ion]; p[1] = x[N + ion]; p[2] = x[2 * N + ion]; }
  const size_t G = (size_t)Nx * Ny * Nz;
  // one velocity component per blockIdx.y: the blocks of a component run
  // together, so the gathers of that time hit one component's grid, which
  // stays in L2 (the three together do not at 256 x 128 x 256)
  {
    const int c = blockIdx.y;
    const T* g = v + (c >= 1 ? G : 0) + (c == 2 ? (size_t)Nx * (Ny + 1) * Nz : 0);
    const int Nyg = c == 1 ? Ny + 1 : Ny;
    int st[3];
    T wv[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T sd = p[d] - (d == c ? T(0) : T(0.5));
      st[d] = stencil_start(sd, W);
      wv[d] = l < W ? kval(sd - T(st[d] + l), kp) : T(0);
    }
    T wy[W], wz[W];
    int roff[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
      wy[j] = __shfl_sync(0xffffffffu, wv[1], gbase + j);
      wz[j] = __shfl_sync(0xffffffffu, wv[2], gbase + j);
      int iy = st[1] + j;
      T sg = T(1);
      if (c == 1) {           // normal component: ghost face -m = -v(m)
        if (iy < 0) { iy = -iy; sg = T(-1); }
        else if (iy > Ny) { iy = 2 * Ny - iy; sg = T(-1); }
      } else {                // tangential: ghost -1-m = -u(m) (no slip) or +u(m) (slip)
        if (iy < 0) { iy = -1 - iy; sg = P.slip[0] ? T(1) : T(-1); }
        else if (iy >= Ny) { iy = 2 * Ny - 1 - iy; sg = P.slip[1] ? T(1) : T(-1); }
      }
      iy = iy < 0 ? 0 : (iy >= Nyg ? Nyg - 1 : iy);   // ions far outside only
      roff[j] = iy * Nx;
      wy[j] *= sg;
    }
    T acc = T(0);
    if (valid && l < W) {
      const int ix = (st[0] + l) & (Nx - 1);
#pragma unroll
      for (int jz = 0; jz < W; ++jz) {
        const T* gz = g + (size_t)((st[2] + jz) & (Nz - 1)) * Nyg * Nx + ix;
        T a = T(0);
#pragma unroll
        for (int jy = 0; jy < W; ++jy) a += wy[jy] * gz[roff[jy]];
        acc += a * wz[jz];
      }
      acc *= wv[0];
    }
#pragma unroll
    for (int o = LPI / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (valid && l == 0) out[(size_t)c * N + (out_index ? out_index[ion] : ion)] = acc;
  }
}

// Single precision, 4-point kernels: the field E = -grad_h phi on the
// faces, interpolated (Eq. efieldop), one thread per ion.  The thread
// evaluates its weights once per axis; each of the 5 x 5 rows (y, z) of the
// 5 x 5 x 5 block of cell values around the ion is read as the two aligned
// quads of x that cover it (16-byte loads, 2 per row instead of 5 scalar
// ones), and per row the x-weights of the centre (cw) and of the face
// difference (ew) give the two partial sums that the three components need.
// Ghost rows as in k_interp_efield_w.  Needs a 16-byte aligned potential and
// Nx a multiple of 4.
__device__ __forceinline__ void row5(const float* __restrict__ row, int ix0, int Nx, float (&v)[5]) {
  const int o = ix0 & 3, q0 = ix0 - o;
  const float4 a = __ldg(reinterpret_cast<const float4*>(row + q0));
  const float4 b = __ldg(reinterpret_cast<const float4*>(row + ((q0 + 4) & (Nx - 1))));
  if (o == 0) { v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; }
  else if (o == 1) { v[0] = a.y; v[1] = a.z; v[2] = a.w; v[3] = b.x; v[4] = b.y; }
  else if (o == 2) { v[0] = a.z; v[1] = a.w; v[2] = b.x; v[3] = b.y; v[4] = b.z; }
  else { v[0] = a.w; v[1] = b.x; v[2] = b.y; v[3] = b.z; v[4] = b.w; }
}

__global__ void k_interp_efield_t4(const float* __restrict__ x, const float* __restrict__ q, int N, Params P,
                                   const float* __restrict__ phi, float* __restrict__ out, int as_force,
                                   const float* __restrict__ F_add, const int* __restrict__ out_index) {
  const int ion = blockIdx.x * blockDim.x + threadIdx.x;
  if (ion >= N) return;
  const KernelParams kp = P.kes;
  const int Nx = P.Nx, Ny = P.Ny;
  const PhysF& Q = P.f;
  const float p[3] = {x[ion], x[N + ion], x[2 * N + ion]};
  int c0[3];
  float cw[3][5], ew[3][5];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    c0[d] = stencil_start(p[d], 4) - 1;
    float kprev = kval(p[d] - float(c0[d]), kp);
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      const int c = c0[d] + l;
      cw[d][l] = kval(p[d] - (float(c) + 0.5f), kp);
      const float knext = kval(p[d] - float(c + 1), kp);
      ew[d][l] = knext - kprev;
      kprev = knext;
    }
  }
  const int ix0 = c0[0] & (Nx - 1);
  // a metal strip in the bottom wall: the rows below it take the Dirichlet
  // rule with the strip potential of each column
  bool sc[5];
  float pm2[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int col = (ix0 + i) & (Nx - 1);
    sc[i] = on_strip(P, col);
    pm2[i] = sc[i] ? 2.f * strip_phi_m(P, col, 0.f) : 0.f;
  }
  float Ex = 0.f, Ey = 0.f, Ez = 0.f;
#pragma unroll
  for (int jy = 0; jy < 5; ++jy) {
    // phi at row iy = rs * phi[row] + ra (ghost rows of Eqs. esbc1 / esbc3)
    const int iy = c0[1] + jy;
    int row = iy;
    float rs = 1.f, ra = 0.f;
    const bool below = iy < 0;
    if (below) {
      int m = -1 - iy;
      m = m < Ny ? m : Ny - 1;
      row = m;
      if (P.bc[0] == DISCOS_BC_DIRICHLET) { rs = -1.f; ra = 2.f * Q.phi_b[0]; }
      else ra = -Q.slope[0] * float(2 * m + 1);
    } else if (iy >= Ny) {
      int m = iy - Ny;
      m = m < Ny ? m : Ny - 1;
      row = Ny - 1 - m;
      if (P.bc[1] == DISCOS_BC_DIRICHLET) { rs = -1.f; ra = 2.f * Q.phi_b[1]; }
      else ra = Q.slope[1] * float(2 * m + 1);
    }
    float a1 = 0.f, a2 = 0.f, a3 = 0.f;     // sums over z: centre-x centre-z, centre-x edge-z, edge-x centre-z
#pragma unroll
    for (int jz = 0; jz < 5; ++jz) {
      float vals[5];
      row5(phi + ((size_t)((c0[2] + jz) & (P.Nz - 1)) * Ny + row) * Nx, ix0, Nx, vals);
      float sc_c = 0.f, sc_e = 0.f;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        const float vv = (below && sc[i]) ? pm2[i] - vals[i] : rs * vals[i] + ra;
        sc_c += vv * cw[0][i];
        sc_e += vv * ew[0][i];
      }
      a1 += sc_c * cw[2][jz];
      a2 += sc_c * ew[2][jz];
      a3 += sc_e * cw[2][jz];
    }
    Ex += a3 * cw[1][jy];
    Ey += a1 * ew[1][jy];
    Ez += a2 * cw[1][jy];
  }
  const int o = out_index ? out_index[ion] : ion;
  if (as_force) {
    const float qq = q[ion];
    const float f0 = F_add ? F_add[ion] : 0.f, f1 = F_add ? F_add[N + ion] : 0.f, f2 = F_add ? F_add[2 * N + ion] : 0.f;
    out[o] = qq * (Ex + Q.E_ext[0]) + f0;
    out[N + o] = qq * (Ey + Q.E_ext[1]) + f1;
    out[2 * N + o] = qq * (Ez + Q.E_ext[2]) + f2;
  } else {
    out[o] = Ex; out[N + o] = Ey; out[2 * N + o] = Ez;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_interp_efield(const Params& P, const T* x, const T* q, int N, const T* phi, T* out,
                                 bool as_force, cudaStream_t s, const T* F_add, const int* out_index) {
  if (N <= 0) return cudaSuccess;
  int bs = 256;
  int nb = (int)(((size_t)N * 8 + bs - 1) / bs);
  probe_begin(PROBE_INTERP_E, s);
  if (std::is_same<T, float>::value && P.kes.w == 4 && ((uintptr_t)phi & 15u) == 0)
    k_interp_efield_t4<<<(int)(((size_t)N + bs - 1) / bs), bs, 0, s>>>(
        reinterpret_cast<const float*>(x), reinterpret_cast<const float*>(q), N, P, reinterpret_cast<const float*>(phi),
        reinterpret_cast<float*>(out), as_force ? 1 : 0, reinterpret_cast<const float*>(F_add), out_index);
  else if (P.kes.w == 4) k_interp_efield_w<T, 4><<<nb, bs, 0, s>>>(x, q, N, P, phi, out, as_force ? 1 : 0, F_add, out_index);
  else if (P.kes.w == 6) k_interp_efield_w<T, 6><<<nb, bs, 0, s>>>(x, q, N, P, phi, out, as_force ? 1 : 0, F_add, out_index);
  else k_interp_efield<T><<<nb, bs, 0, s>>>(x, q, N, P, phi, out, as_force ? 1 : 0, F_add, out_index);
  count_launches(1);
  probe_end(PROBE_INTERP_E, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interp_velocity(const Params& P, const T* x, int N, const T* v, T* out, cudaStream_t s,
                                   const int* out_index, const int* species) {
  if (N <= 0) return cudaSuccess;
  int bs = 256;
  int nb = (int)(((size_t)N * 8 + bs - 1) / bs);
  probe_begin(PROBE_INTERP_V, s);
  auto one = [&](const Params& Q) {
    if (Q.khy.w == 4)
      k_interp_velocity_w<T, 4, 4><<<dim3((unsigned)(((size_t)N * 4 + bs - 1) / bs), 3), bs, 0, s>>>(x, N, Q, v, out,
                                                                                             out_index, species);
    else if (Q.khy.w == 6)
      k_interp_velocity_w<T, 6, 8><<<dim3((unsigned)nb, 3), bs, 0, s>>>(x, N, Q, v, out, out_index, species);
    else k_interp_velocity<T><<<nb, bs, 0, s>>>(x, N, Q, v, out, out_index, species);
    count_launches(1);
  };
  for_each_hy_kernel(P, species, one);
  probe_end(PROBE_INTERP_V, s);
  return cudaGetLastError();
}

template cudaError_t launch_interp_efield<float>(const Params&, const float*, const float*, int, const float*, float*, bool, cudaStream_t, const float*, const int*);
template cudaError_t launch_interp_efield<double>(const Params&, const double*, const double*, int, const double*, double*, bool, cudaStream_t, const double*, const int*);
template cudaError_t launch_interp_velocity<float>(const Params&, const float*, int, const float*, float*, cudaStream_t, const int*, const int*);
template cudaError_t launch_interp_velocity<double>(const Params&, const double*, int, const double*, double*, cudaStream_t, const int*, const int*);

}  // namespace discos
