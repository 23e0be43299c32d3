// Batched replicas: many independent small channels (Nx = Nz = 32, Ny = 16
// or 32, up to 512 ions each) advanced by the dry-diffusion step of
// Sec. II.D in one persistent launch.
//
// One CTA per SM pulls replicas from a work queue ordered by descending ion
// count (longest first, so uneven replicas balance across SMs) and keeps the
// whole replica in shared memory for the step:
//   * the cell-centred grid, [Ny] planes of [32 z][33] floats (padded rows: a
//     warp reading a row or a column of a plane hits 32 distinct banks);
//   * the ions (positions, charges, species, forces) and their cell list.
// A step is, entirely on chip:
//   1. stable counting sort of the ions into list cells (warp 0), beside
//   2. charge spreading with the wall images (Eq. kernel2, Sec. II.B.1), 8
//      lanes per ion, fire-and-forget shared-memory atomics;
//   3. the Poisson solve of Eq. poisson: a separable discrete Hartley
//      transform in x and z (real to real; cas(kx x) cas(kz z) are
//      eigenvectors of the periodic second differences with the same
//      eigenvalues as the Fourier modes), 32-point transforms held in the
//      registers of one lane each, then one tridiagonal solve in y per mode
//      (FP32 Thomas with pre-factored pivots; the modes with K^2 < 0.5, whose
//      systems are ill conditioned, in FP64 on their own warps), then the
//      same transform back;
//   4. E^P = J^es(-grad_h phi) at the ions (Eq. efieldop), ghost rows from
//      Eqs. esbc1 / esbc3, 8 lanes per ion;
//   5. the near field (Eqs. fullElectro, LC, closerange) with wall images and
//      the wall force (Sec. II.B.2), one warp per ion over the cell list;
//   6. the Euler-Maruyama update of Eq. ions3 with the near-wall mobility and
//      drift, Philox counters (ion, step, replica, 1);
//   7. the y histogram of the new positions, and on the last step the FP64
//      sums of charge and force.
// The stencil width W and Ny are template parameters, so the stencil loops
// unroll and the wall-normal systems live in registers.  The last CTA to
// finish resets the queue and advances the device step counter, so the
// launch can be replayed from a CUDA graph.
#pragma once
#include "physics.cuh"

namespace discos {
namespace batched {

constexpr int BP = 33;            // padded row pitch of a plane
constexpr int PLANE = 32 * BP;    // floats per y-plane
constexpr int MAXN = 512;         // ions per replica
constexpr int NT = 512;           // threads per CTA
constexpr int LO_THREADS = 64;    // threads that solve the low modes in double

// cos(2 pi k / 32) from the quarter wave (a switch, so that a constant k
// folds to an immediate); sin(2 pi k / 32) = cos(2 pi (k - 8) / 32)
__host__ __device__ constexpr float cos_quarter(int k) {
  switch (k) {
    case 0: return 1.000000000e+00f;
    case 1: return 9.807852804e-01f;
    case 2: return 9.238795325e-01f;
    case 3: return 8.314696123e-01f;
    case 4: return 7.071067812e-01f;
    case 5: return 5.555702330e-01f;
    case 6: return 3.826834324e-01f;
    case 7: return 1.950903220e-01f;
    case 8: return 0.0f;
    default: return 0.0f;
  }
}
__host__ __device__ constexpr float cos32(int k) {
  k &= 31;
  return k <= 8 ? cos_quarter(k) : k <= 16 ? -cos_quarter(16 - k) : k <= 24 ? -cos_quarter(k - 16) : cos_quarter(32 - k);
}
__host__ __device__ constexpr float sin32(int k) { return cos32(k + 24); }

constexpr int brev4(int i) { return ((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3); }

// In-register radix-2 FFT of length 16, exp(-2 pi i n k / 16), natural order.
__device__ __forceinline__ void fft16(float (&re)[16], float (&im)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int j = brev4(i);
    if (j > i) {
      float t = re[i]; re[i] = re[j]; re[j] = t;
      t = im[i]; im[i] = im[j]; im[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= 16; len <<= 1) {
    const int half = len >> 1;
#pragma unroll
    for (int i = 0; i < 16; i += len) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float wr = cos32(k * (32 / len)), wi = -sin32(k * (32 / len));
        const int a = i + k, b = i + k + half;
        const float xr = re[b] * wr - im[b] * wi;
        const float xi = re[b] * wi + im[b] * wr;
        re[b] = re[a] - xr; im[b] = im[a] - xi;
        re[a] += xr; im[a] += xi;
      }
    }
  }
}

// Discrete Hartley transform of length 32, H(k) = sum_n a(n) cas(2 pi n k / 32),
// from the 16-point FFT of z(n) = a(2n) + i a(2n+1): with E, O the transforms of
// the even and odd samples, X(k) = E(k) + w^k O(k), X(k+16) = E(k) - w^k O(k)
// and H = Re X - Im X.  Applied twice it gives 32 times the input.
__device__ __forceinline__ void dht32(float (&a)[32]) {
  float zr[16], zi[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) { zr[n] = a[2 * n]; zi[n] = a[2 * n + 1]; }
  fft16(zr, zi);
  a[0] = zr[0] + zi[0];
  a[16] = zr[0] - zi[0];
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    const int kc = 16 - k;
    const float Er = 0.5f * (zr[k] + zr[kc]), Ei = 0.5f * (zi[k] - zi[kc]);
    const float Or = 0.5f * (zi[k] + zi[kc]), Oi = -0.5f * (zr[k] - zr[kc]);
    const float c = cos32(k), s = sin32(k);
    const float Tr = c * Or + s * Oi, Ti = c * Oi - s * Or;
    a[k] = (Er + Tr) - (Ei + Ti);
    a[k + 16] = (Er - Tr) - (Ei - Ti);
  }
}

// Separable Hartley transform of the planes owned by this warp: x along each
// row (lane = z), then z along each column (lane = x).
template <int NY>
__device__ __forceinline__ void planes_dht(float* __restrict__ G) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int y = warp; y < NY; y += NT / 32) {
    float* pl = G + y * PLANE;
    float a[32];
#pragma unroll
    for (int x = 0; x < 32; ++x) a[x] = pl[lane * BP + x];
    dht32(a);
#pragma unroll
    for (int x = 0; x < 32; ++x) pl[lane * BP + x] = a[x];
    __syncwarp();
#pragma unroll
    for (int z = 0; z < 32; ++z) a[z] = pl[z * BP + lane];
    dht32(a);
#pragma unroll
    for (int z = 0; z < 32; ++z) pl[z * BP + lane] = a[z];
    __syncwarp();
  }
}

// Thomas solve of one wall-normal system in place (column `col` of G):
// rows -phi_{j-1} + d_j phi_j - phi_{j+1} = b_j, reciprocal pivots piv[j];
// b = scale * G + the wall terms of mode (0, 0).  R is the arithmetic type;
// with preload the pivots are fetched into registers up front.
template <typename R, bool preload, int NY>
__device__ __forceinline__ void ysolve_column(float* __restrict__ G, int col, const R* __restrict__ piv, R scale,
                                              R w0, R w1, bool mode0) {
  R b[NY];
  R p[preload ? NY : 1];
#pragma unroll
  for (int j = 0; j < NY; ++j) {
    b[j] = scale * (R)G[j * PLANE + col];
    if (preload) p[preload ? j : 0] = piv[j];
  }
  if (mode0) {
    b[0] += w0;
    b[NY - 1] += w1;
  }
#pragma unroll
  for (int j = 1; j < NY; ++j) b[j] += b[j - 1] * (preload ? p[preload ? j - 1 : 0] : piv[j - 1]);
  R xn = R(0);
#pragma unroll
  for (int j = NY - 1; j >= 0; --j) {
    xn = (b[j] + xn) * (preload ? p[preload ? j : 0] : piv[j]);
    G[j * PLANE + col] = (float)xn;
  }
}

template <int W, int NY>
__global__ void __launch_bounds__(NT, 1) k_batched_step(Params P, BatchArgs B) {
  extern __shared__ float4 smem4[];
  float* G = reinterpret_cast<float*>(smem4);
  float* sx = G + NY * PLANE;
  float* sy = sx + MAXN;
  float* sz = sy + MAXN;
  float* sq = sz + MAXN;
  float* sF = sq + MAXN;                       // [3][MAXN]
  int* ssp = reinterpret_cast<int*>(sF + 3 * MAXN);
  int* scell = ssp + MAXN;                     // list cell, then (cell, rank inside it)
  int* slist = scell + MAXN;                   // ions in cell order
  int* cstart = slist + MAXN;                  // [n_cells + 1]
  float* stab = reinterpret_cast<float*>(cstart + B.n_cells + 1);
  __shared__ int s_slot;
  __shared__ double s_red[NT / 32][4];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n_cells = B.n_cells;
  for (int i = tid; i <= P.n_tab; i += NT) stab[i] = B.fptab[i];
  const long long step_base = *reinterpret_cast<volatile long long*>(B.dstep);
  const float scale_poisson = (float)(4.0 * M_PI * P.lB / (32.0 * 32.0));
  const double scale_poisson64 = 4.0 * M_PI * P.lB / (32.0 * 32.0);
  const KernelParams kp = P.kes;
  const float Lx = 32.0f, Lz = 32.0f, hx = 16.0f, hz = 16.0f;
  const float psi = P.f.psi;
  const float psi2 = mul_rn(psi, psi);
  const float lB = P.f.lB, tscale = P.f.tab_scale;
  const bool dir0 = P.bc[0] == DISCOS_BC_DIRICHLET, dir1 = P.bc[1] == DISCOS_BC_DIRICHLET;
  const float s0 = dir0 ? -1.0f : 1.0f, s1 = dir1 ? -1.0f : 1.0f;
  const float slope0 = P.f.slope[0], slope1 = P.f.slope[1];

  for (;;) {
    if (tid == 0) s_slot = atomicAdd(&B.queue[0], 1);
    __syncthreads();
    const int slot = s_slot;
    __syncthreads();
    if (slot >= B.R) break;
    const int r = B.order[slot];
    const int base = B.offsets[r];
    int N = B.offsets[r + 1] - base;
    // the host checked its copy of the offsets; a device copy that disagrees
    // is not trusted beyond the arrays' bounds
    if (N < 0 || N > MAXN || base < 0 || base + N > B.Ntot) N = 0;
    if (N == 0) continue;
    const double pb0d = B.phi_b ? B.phi_b[2 * r] : P.phi_b[0];
    const double pb1d = B.phi_b ? B.phi_b[2 * r + 1] : P.phi_b[1];
    const float pb0 = (float)pb0d, pb1 = (float)pb1d;
    // wall terms of the (0, 0) mode (Eqs. esbc1 / esbc3); the transform of a
    // constant over the 32 x 32 plane is 1024 times it, the scale divides by 1024
    const double w0 = dir0 ? 2.0 * pb0d : -P.slope[0];
    const double w1 = dir1 ? 2.0 * pb1d : P.slope[1];
    for (int i = tid; i < N; i += NT) {
      sx[i] = B.x[base + i];
      sy[i] = B.x[B.Ntot + base + i];
      sz[i] = B.x[2 * B.Ntot + base + i];
      sq[i] = B.q[base + i];
      const int spi = B.species ? B.species[base + i] : 0;
      ssp[i] = spi < 0 ? 0 : (spi >= P.nspecies ? P.nspecies - 1 : spi);   // indexes tables and the histogram
    }
    __syncthreads();

    for (int st = 0; st < B.steps; ++st) {
      const long long step = step_base + st;
      const bool last = st == B.steps - 1;
      // -- zero the grid and the cell counts; cell of every ion
      {
        float4* g4 = reinterpret_cast<float4*>(G);
        for (int i = tid; i < NY * PLANE / 4; i += NT) g4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = tid; c <= n_cells; c += NT) cstart[c] = 0;
        for (int i = tid; i < N; i += NT) {
          const int cx = cell_coord(sx[i], P.k_cell, P.ncx);
          const int cy = cell_coord(sy[i], P.k_cell, P.ncy);
          const int cz = cell_coord(sz[i], P.k_cell, P.ncz);
          scell[i] = (cz * P.ncy + cy) * P.ncx + cx;
        }
      }
      __syncthreads();
      if (warp == 0) {
        // -- stable counting sort: ranks by match_any within 32-ion chunks, in order
        for (int c0 = 0; c0 < N; c0 += 32) {
          const int i = c0 + lane;
          const bool v = i < N;
          const int c = v ? scell[i] : -1 - lane;
          const unsigned act = __ballot_sync(0xffffffffu, v);
          const unsigned grp = __match_any_sync(0xffffffffu, c);
          const int before = __popc(grp & act & ((1u << lane) - 1u));
          int rank = 0;
          if (v) rank = cstart[c + 1] + before;
          __syncwarp();
          if (v && before == 0) cstart[c + 1] += __popc(grp & act);
          __syncwarp();
          if (v) scell[i] = (c << 10) | rank;
        }
        __syncwarp();
        int run = 0;                           // inclusive scan of cstart[1..n_cells]
        for (int c0 = 1; c0 <= n_cells; c0 += 32) {
          const int c = c0 + lane;
          int v = c <= n_cells ? cstart[c] : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
          }
          if (c <= n_cells) cstart[c] = v + run;
          run += __shfl_sync(0xffffffffu, v, 31);
        }
        __syncwarp();
        for (int i = lane; i < N; i += 32) {
          const int cr = scell[i];
          slist[cstart[cr >> 10] + (cr & 1023)] = i;
        }
      } else {
        // -- charge spreading, 8 lanes per ion on warps 1..
        const int t = tid - 32;
        const int l = t & 7;
        const int gbase = lane & ~7;
        for (int i0 = 0; i0 < N; i0 += (NT - 32) / 8) {
          const int ion = i0 + (t >> 3);
          const bool valid = ion < N;
          float px = 0.5f, py = 0.5f, pz = 0.5f, qq = 0.f;
          if (valid) { px = sx[ion]; py = sy[ion]; pz = sz[ion]; qq = sq[ion]; }
          const float ax = px - 0.5f, ay = py - 0.5f, az = pz - 0.5f;
          const int x0 = stencil_start(ax, W), y0 = stencil_start(ay, W), z0 = stencil_start(az, W);
          const float wx = l < W ? kval(ax - (float)(x0 + l), kp) : 0.f;
          const float wyl = l < W ? kval(ay - (float)(y0 + l), kp) : 0.f;
          const float wzl = l < W ? kval(az - (float)(z0 + l), kp) : 0.f;
          float wy[W], wz[W];
          int roff[W];
#pragma unroll
          for (int j = 0; j < W; ++j) {
            wy[j] = __shfl_sync(0xffffffffu, wyl, gbase + j);
            wz[j] = __shfl_sync(0xffffffffu, wzl, gbase + j);
            int iy = y0 + j;
            float sg = 1.f;
            if (iy < 0) { iy = -1 - iy; sg = s0; }
            else if (iy >= NY) { iy = 2 * NY - 1 - iy; sg = s1; }
            const bool in = iy >= 0 && iy < NY;
            roff[j] = in ? iy * PLANE : 0;
            wy[j] = in ? sg * wy[j] : 0.f;
          }
          if (valid && l < W) {
            const int ix = (x0 + l) & 31;
            const float qx = qq * wx;
#pragma unroll
            for (int jz = 0; jz < W; ++jz) {
              const int zoff = ((z0 + jz) & 31) * BP + ix;
              const float qz = qx * wz[jz];
#pragma unroll
              for (int jy = 0; jy < W; ++jy) atomicAdd(&G[roff[jy] + zoff], qz * wy[jy]);
            }
          }
        }
      }
      __syncthreads();
      // -- Poisson: transform, wall-normal solves, transform back
      planes_dht<NY>(G);
      __syncthreads();
      if (tid < NT - LO_THREADS) {
        for (int t = tid; t < B.n_hi; t += NT - LO_THREADS) {
          const int m = B.modes[B.n_lo + t];
          const int kz = m >> 5, kx = m & 31;
          const int kxm = kx <= 16 ? kx : 32 - kx;
          ysolve_column<float, true, NY>(G, kz * BP + kx, B.piv32 + (size_t)(kz * 17 + kxm) * NY, scale_poisson,
                                         (float)w0, (float)w1, m == 0);
        }
      } else {
        for (int t = tid - (NT - LO_THREADS); t < B.n_lo; t += LO_THREADS) {
          const int m = B.modes[t];
          const int kz = m >> 5, kx = m & 31;
          const int kxm = kx <= 16 ? kx : 32 - kx;
          ysolve_column<double, false, NY>(G, kz * BP + kx, B.piv64 + (size_t)(kz * 17 + kxm) * NY,
                                           scale_poisson64, w0, w1, m == 0);
        }
      }
      __syncthreads();
      planes_dht<NY>(G);
      __syncthreads();
      // -- E^P at the ions: 8 lanes per ion, lane l owns x cell c0 + l of the
      //    (W+1)^3 block; the face differences are folded into the weights
      {
        const int l = tid & 7;
        const int gbase = lane & ~7;
        for (int i0 = 0; i0 < N; i0 += NT / 8) {
          const int ion = i0 + (tid >> 3);
          const bool valid = ion < N;
          float p[3] = {0.5f, 0.5f, 0.5f};
          if (valid) { p[0] = sx[ion]; p[1] = sy[ion]; p[2] = sz[ion]; }
          int c0[3];
          float cw[3], ew[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            c0[d] = stencil_start(p[d], W) - 1;
            const int c = c0[d] + l;
            const bool in = l <= W;
            cw[d] = in ? kval(p[d] - ((float)c + 0.5f), kp) : 0.f;
            ew[d] = in ? (kval(p[d] - (float)(c + 1), kp) - kval(p[d] - (float)c, kp)) : 0.f;
          }
          float cy[W + 1], ey[W + 1], cz[W + 1], ez[W + 1], rs[W + 1], ra[W + 1];
          int roff[W + 1];
#pragma unroll
          for (int j = 0; j <= W; ++j) {
            cy[j] = __shfl_sync(0xffffffffu, cw[1], gbase + j);
            ey[j] = __shfl_sync(0xffffffffu, ew[1], gbase + j);
            cz[j] = __shfl_sync(0xffffffffu, cw[2], gbase + j);
            ez[j] = __shfl_sync(0xffffffffu, ew[2], gbase + j);
            // row of cell iy and its ghost rule: phi = rs * G[row] + ra
            const int iy = c0[1] + j;
            int row = iy;
            float sg = 1.f, ad = 0.f;
            if (iy < 0) {
              int m = -1 - iy;
              m = m < NY ? m : NY - 1;
              row = m;
              if (dir0) { sg = -1.f; ad = 2.0f * pb0; } else { ad = -slope0 * (float)(2 * m + 1); }
            } else if (iy >= NY) {
              int m = iy - NY;
              m = m < NY ? m : NY - 1;
              row = NY - 1 - m;
              if (dir1) { sg = -1.f; ad = 2.0f * pb1; } else { ad = slope1 * (float)(2 * m + 1); }
            }
            roff[j] = row * PLANE;
            rs[j] = sg;
            ra[j] = ad;
          }
          float Ex = 0.f, Ey = 0.f, Ez = 0.f;
          if (valid && l <= W) {
            const int ix = (c0[0] + l) & 31;
#pragma unroll
            for (int jz = 0; jz <= W; ++jz) {
              const int zoff = ((c0[2] + jz) & 31) * BP + ix;
              float a1 = 0.f, a2 = 0.f;
#pragma unroll
              for (int jy = 0; jy <= W; ++jy) {
                const float v = fmaf(rs[jy], G[roff[jy] + zoff], ra[jy]);
                a1 = fmaf(v, cy[jy], a1);
                a2 = fmaf(v, ey[jy], a2);
              }
              Ex = fmaf(a1, cz[jz], Ex);
              Ey = fmaf(a2, cz[jz], Ey);
              Ez = fmaf(a1, ez[jz], Ez);
            }
            Ex *= ew[0];
            Ey *= cw[0];
            Ez *= cw[0];
          }
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) {
            Ex += __shfl_xor_sync(0xffffffffu, Ex, o);
            Ey += __shfl_xor_sync(0xffffffffu, Ey, o);
            Ez += __shfl_xor_sync(0xffffffffu, Ez, o);
          }
          if (valid && l == 0) {
            const float qq = sq[ion];
            sF[ion] = qq * (Ex + P.f.E_ext[0]);
            sF[MAXN + ion] = qq * (Ey + P.f.E_ext[1]);
            sF[2 * MAXN + ion] = qq * (Ez + P.f.E_ext[2]);
          }
        }
      }
      __syncthreads();
      // -- near field and wall force: one warp per ion, lanes 0..26 over the
      //    27 neighbour cells, then lanes 0..8 / 9..17 over the wall-row cells
      //    for the image partners; fixed shuffle reduction
      for (int i = warp; i < N; i += NT / 32) {
        const float xi = sx[i], yi = sy[i], zi = sz[i], qi = sq[i];
        const int si = ssp[i];
        const int cx = cell_coord(xi, P.k_cell, P.ncx);
        const int cy = cell_coord(yi, P.k_cell, P.ncy);
        const int cz = cell_coord(zi, P.k_cell, P.ncz);
        float fx = 0.f, fy = 0.f, fz = 0.f;
        int cnt = 0;
        if (lane < 27) {
          const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
          const int cyy = cy + dy;
          if (cyy >= 0 && cyy < P.ncy) {
            int czz = cz + dz;
            czz = czz < 0 ? czz + P.ncz : (czz >= P.ncz ? czz - P.ncz : czz);
            int cxx = cx + dx;
            cxx = cxx < 0 ? cxx + P.ncx : (cxx >= P.ncx ? cxx - P.ncx : cxx);
            const int c = (czz * P.ncy + cyy) * P.ncx + cxx;
            for (int k = cstart[c]; k < cstart[c + 1]; ++k) {
              const int j = slist[k];
              if (j == i) continue;
              pair_terms(xi, yi, zi, qi, si, sx[j], sy[j], sz[j], sq[j], ssp[j], true, P, stab, Lx, hx, Lz, hz,
                         psi2, lB, tscale, fx, fy, fz, cnt);
            }
          }
        }
        const bool near0 = yi < psi, near1 = sub_rn((float)NY, yi) < psi;
        if ((near0 && lane < 9) || (near1 && lane >= 9 && lane < 18)) {
          const int wall = lane < 9 ? 0 : 1;
          const int l9 = lane - 9 * wall;
          const int dx = l9 % 3 - 1, dz = l9 / 3 - 1;
          int czz = cz + dz;
          czz = czz < 0 ? czz + P.ncz : (czz >= P.ncz ? czz - P.ncz : czz);
          int cxx = cx + dx;
          cxx = cxx < 0 ? cxx + P.ncx : (cxx >= P.ncx ? cxx - P.ncx : cxx);
          const int cyy = wall == 0 ? 0 : P.ncy - 1;
          const float sgn = (wall == 0 ? dir0 : dir1) ? -1.f : 1.f;
          const int c = (czz * P.ncy + cyy) * P.ncx + cxx;
          for (int k = cstart[c]; k < cstart[c + 1]; ++k) {
            const int j = slist[k];
            const float yj = sy[j];
            const float yimg = wall == 0 ? -yj : sub_rn((float)(2 * NY), yj);
            pair_terms(xi, yi, zi, qi, si, sx[j], yimg, sz[j], sgn * sq[j], 0, false, P, stab, Lx, hx, Lz, hz,
                       psi2, lB, tscale, fx, fy, fz, cnt);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fx += __shfl_xor_sync(0xffffffffu, fx, o);
          fy += __shfl_xor_sync(0xffffffffu, fy, o);
          fz += __shfl_xor_sync(0xffffffffu, fz, o);
          cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        }
        if (lane == 0) {
          fy += wall_force_y(P, si, yi);
          sF[i] += fx;
          sF[MAXN + i] += fy;
          sF[2 * MAXN + i] += fz;
          if (last && B.nbr) B.nbr[base + i] = cnt;
        }
      }
      __syncthreads();
      // -- update, histogram, outputs of the last step
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = tid; i < N; i += NT) {
        const int sp = ssp[i];
        float p[3] = {sx[i], sy[i], sz[i]};
        const float f[3] = {sF[i], sF[MAXN + i], sF[2 * MAXN + i]};
        float Wn[4];
        normals4(u32x4{(uint32_t)i, (uint32_t)step, (uint32_t)r, (uint32_t)TAG_DRY}, P.seed, Wn);
        dry_move(P, sp, p, f, (const float*)nullptr, Wn);
        check_position(P, p);
        sx[i] = p[0]; sy[i] = p[1]; sz[i] = p[2];
        if (B.hist) {
          int bin = (int)floorf(p[1]);
          bin = bin < 0 ? 0 : (bin >= NY ? NY - 1 : bin);
          atomicAdd(&B.hist[((size_t)r * P.nspecies + sp) * NY + bin], 1u);
        }
        if (last) {
          if (B.F_out) {
            B.F_out[base + i] = f[0];
            B.F_out[B.Ntot + base + i] = f[1];
            B.F_out[2 * B.Ntot + base + i] = f[2];
          }
          acc[0] += (double)sq[i];
          acc[1] += (double)f[0];
          acc[2] += (double)f[1];
          acc[3] += (double)f[2];
        }
      }
      if (last && B.sums) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 4; ++k) s_red[warp][k] = acc[k];
        }
      }
      __syncthreads();
      if (last && B.sums && tid < 4) {
        double s = 0.0;
        for (int wi = 0; wi < NT / 32; ++wi) s += s_red[wi][tid];
        B.sums[4 * r + tid] = s;
      }
    }
    // positions back to global memory
    for (int i = tid; i < N; i += NT) {
      B.x[base + i] = sx[i];
      B.x[B.Ntot + base + i] = sy[i];
      B.x[2 * B.Ntot + base + i] = sz[i];
    }
  }
  // the last CTA out resets the queue and advances the step counter
  if (tid == 0) {
    __threadfence();
    const int done = atomicAdd(&B.queue[1], 1);
    if (done == (int)gridDim.x - 1) {
      B.queue[0] = 0;
      B.queue[1] = 0;
      *B.dstep = step_base + B.steps;
      __threadfence();
    }
  }
}

// Launch (or, with launch = false, set the shared-memory attribute of) the
// kernel for stencil width W; Ny selects the instantiation.
template <int W>
cudaError_t launch_w(const Params& P, const BatchArgs& B, int grid, size_t smem, cudaStream_t s, bool launch) {
  if (P.Ny == 32) {
    if (!launch)
      return cudaFuncSetAttribute(k_batched_step<W, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batched_step<W, 32><<<grid, NT, smem, s>>>(P, B);
  } else {
    if (!launch)
      return cudaFuncSetAttribute(k_batched_step<W, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batched_step<W, 16><<<grid, NT, smem, s>>>(P, B);
  }
  return cudaGetLastError();
}

}  // namespace batched
}  // namespace discos
