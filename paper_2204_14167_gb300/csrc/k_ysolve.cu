// Wall-normal banded solves as warp-parallel scans.
//
// After the x and z transforms every (kx, kz) mode is an independent banded
// system in y: the Poisson tridiagonal (2 + K^2) phi_j - phi_{j-1} - phi_{j+1}
// = b_j with the wall rows of Eqs. esbc1 / esbc3, and the Stokes
// pentadiagonal / tridiagonal pair of Eq. disc_stokes (algebra in
// k_stokes.cu).  Their factors are pre-computed per mode; what remains per
// step are linear recurrences along y (forward and backward substitutions),
// first order for a tridiagonal, second order for the pentadiagonal.
//
// One warp solves one mode.  Lane l owns R consecutive rows; a recurrence
// s_j = A_j s_{j-1} + c_j is solved by composing each lane's affine maps, an
// inclusive scan of the composed maps across the warp (shuffles, log2 32
// levels), and a final local pass from the state entering the lane.  The
// critical path is ~R + 5 map compositions instead of Ny dependent steps.
//
// Precision follows conditioning.  K^2 = lambda_x + lambda_z sets the
// condition numbers: for K^2 >= 0.5 the tridiagonal has kappa <= 9 and the
// pentadiagonal kappa <= 81, so the mixed path solves those modes in single
// precision (error well below 1e-5); the modes with K^2 < 0.5 (a few percent,
// the ill-conditioned ones and the singular K = 0 mode) are solved in double.
// The FP64 path solves every mode in double.
#include <atomic>
#include <type_traits>
#include "internal.h"

namespace discos {

namespace {

template <typename T> struct C { T r, i; };
template <typename T> __device__ __forceinline__ C<T> cz() { return C<T>{T(0), T(0)}; }
template <typename T> __device__ __forceinline__ C<T> cadd2(C<T> a, C<T> b) { return C<T>{a.r + b.r, a.i + b.i}; }
template <typename T> __device__ __forceinline__ C<T> csub2(C<T> a, C<T> b) { return C<T>{a.r - b.r, a.i - b.i}; }
template <typename T> __device__ __forceinline__ C<T> cscale(T s, C<T> a) { return C<T>{s * a.r, s * a.i}; }
template <typename T> __device__ __forceinline__ C<T> cfma(T s, C<T> a, C<T> b) {
  return C<T>{fma(s, a.r, b.r), fma(s, a.i, b.i)};
}
template <typename T> __device__ __forceinline__ T shup(T v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
template <typename T> __device__ __forceinline__ T shdn(T v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }

// first order, two complex offsets sharing the multiplier: s -> a s + b
template <typename T> struct M1 { T a; C<T> b0, b1; };
template <typename T> __device__ __forceinline__ M1<T> m1_id() { return M1<T>{T(1), cz<T>(), cz<T>()}; }
// apply `in` first, then `out`
template <typename T> __device__ __forceinline__ M1<T> m1_comp(const M1<T>& out, const M1<T>& in) {
  return M1<T>{out.a * in.a, cfma(out.a, in.b0, out.b0), cfma(out.a, in.b1, out.b1)};
}
template <typename T> __device__ __forceinline__ M1<T> m1_sh(const M1<T>& m, int o, bool up) {
  M1<T> r;
  r.a = up ? shup(m.a, o) : shdn(m.a, o);
  r.b0.r = up ? shup(m.b0.r, o) : shdn(m.b0.r, o);
  r.b0.i = up ? shup(m.b0.i, o) : shdn(m.b0.i, o);
  r.b1.r = up ? shup(m.b1.r, o) : shdn(m.b1.r, o);
  r.b1.i = up ? shup(m.b1.i, o) : shdn(m.b1.i, o);
  return r;
}
// Exclusive scan: forward (lane order) gives m_{l-1} o ... o m_0 on lane l;
// backward gives m_{l+1} o ... o m_31.
template <typename T> __device__ __forceinline__ M1<T> m1_exscan(M1<T> m, int lane, bool forward) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    M1<T> q = m1_sh(m, o, forward);
    bool take = forward ? lane >= o : lane + o < 32;
    if (take) m = m1_comp(m, q);
  }
  M1<T> e = m1_sh(m, 1, forward);
  bool first = forward ? lane == 0 : lane == 31;
  return first ? m1_id<T>() : e;
}

// second order on a complex state (s0, s1): s -> A s + c, A real 2 x 2
template <typename T> struct M2 { T a00, a01, a10, a11; C<T> c0, c1; };
template <typename T> __device__ __forceinline__ M2<T> m2_id() {
  return M2<T>{T(1), T(0), T(0), T(1), cz<T>(), cz<T>()};
}
template <typename T> __device__ __forceinline__ M2<T> m2_comp(const M2<T>& o, const M2<T>& n) {
  M2<T> r;
  r.a00 = o.a00 * n.a00 + o.a01 * n.a10;
  r.a01 = o.a00 * n.a01 + o.a01 * n.a11;
  r.a10 = o.a10 * n.a00 + o.a11 * n.a10;
  r.a11 = o.a10 * n.a01 + o.a11 * n.a11;
  r.c0 = cadd2(cadd2(cscale(o.a00, n.c0), cscale(o.a01, n.c1)), o.c0);
  r.c1 = cadd2(cadd2(cscale(o.a10, n.c0), cscale(o.a11, n.c1)), o.c1);
  return r;
}
template <typename T> __device__ __forceinline__ M2<T> m2_sh(const M2<T>& m, int o, bool up) {
  M2<T> r;
#define SH(x) (up ? shup(x, o) : shdn(x, o))
  r.a00 = SH(m.a00); r.a01 = SH(m.a01); r.a10 = SH(m.a10); r.a11 = SH(m.a11);
  r.c0.r = SH(m.c0.r); r.c0.i = SH(m.c0.i); r.c1.r = SH(m.c1.r); r.c1.i = SH(m.c1.i);
#undef SH
  return r;
}
template <typename T> __device__ __forceinline__ M2<T> m2_exscan(M2<T> m, int lane, bool forward) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    M2<T> q = m2_sh(m, o, forward);
    bool take = forward ? lane >= o : lane + o < 32;
    if (take) m = m2_comp(m, q);
  }
  M2<T> e = m2_sh(m, 1, forward);
  bool first = forward ? lane == 0 : lane == 31;
  return first ? m2_id<T>() : e;
}

template <typename TS> __device__ __forceinline__ C<double> ldc(const cplx<TS>* p) {
  cplx<TS> v = *p;
  return C<double>{(double)v.re, (double)v.im};
}

// ------------------------------------------------------------------ Poisson
// piv [M][Ny]: reciprocal Thomas pivots.  Forward y_j = piv_j (b_j + y_{j-1}),
// backward x_j = y_j + piv_j x_{j+1}.  The singular K = 0 mode of two
// Neumann walls: the right-hand side's mean is removed (so the last equation
// is redundant), phi_0 = 0, phi_{j+1} = 2 phi_j - phi_{j-1} - b_j, then the
// mean of phi is removed.
// One mode's solve; col points at its column (rows cs apart).
template <typename TS, typename TC, int R>
__device__ __forceinline__ void poisson_mode(cplx<TS>* __restrict__ col, size_t cs, const TC* __restrict__ piv,
                                             int mode, int Ny, int singular, TC norm) {
  const int lane = threadIdx.x & 31;
  const TC* pv = piv + (size_t)mode * Ny;
  const int j0 = lane * R;
  C<TC> b[R];
  TC m[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int j = j0 + r;
    if (j < Ny) {
      cplx<TS> v = col[(size_t)j * cs];
      b[r] = C<TC>{(TC)v.re, (TC)v.im};
      m[r] = pv[j];
    } else {
      b[r] = cz<TC>();
      m[r] = TC(1);
    }
  }
  C<TC> x[R];
  if (singular && mode == 0) {
    // the right-hand side projected onto the operator's range (mean over y
    // removed): the result is the mean-zero (minimum-norm) solution, also
    // for a non-neutral right-hand side
    C<TC> bs = cz<TC>();
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (j0 + r < Ny) bs = cadd2(bs, b[r]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bs.r += __shfl_xor_sync(0xffffffffu, bs.r, o);
      bs.i += __shfl_xor_sync(0xffffffffu, bs.i, o);
    }
    const C<TC> bm = cscale(TC(1) / TC(Ny), bs);
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (j0 + r < Ny) b[r] = csub2(b[r], bm);
    // state (phi_j, phi_{j-1}); row j maps it to (phi_{j+1}, phi_j)
    M2<TC> loc = m2_id<TC>();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int j = j0 + r;
      M2<TC> mj = m2_id<TC>();
      if (j == 0) mj = M2<TC>{TC(1), TC(0), TC(1), TC(0), C<TC>{-b[r].r, -b[r].i}, cz<TC>()};
      else if (j < Ny - 1) mj = M2<TC>{TC(2), TC(-1), TC(1), TC(0), C<TC>{-b[r].r, -b[r].i}, cz<TC>()};
      loc = m2_comp(mj, loc);
    }
    M2<TC> pre = m2_exscan(loc, lane, true);
    C<TC> s0 = pre.c0, s1 = pre.c1;     // state entering the lane, from (0, 0)
    C<TC> sum = cz<TC>();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int j = j0 + r;
      x[r] = s0;
      if (j < Ny) sum = cadd2(sum, s0);
      C<TC> n0 = s0, n1 = s1;
      if (j == 0) { n0 = csub2(s0, b[r]); n1 = s0; }
      else if (j < Ny - 1) { n0 = csub2(csub2(cscale(TC(2), s0), s1), b[r]); n1 = s0; }
      s0 = n0; s1 = n1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sum.r += __shfl_xor_sync(0xffffffffu, sum.r, o);
      sum.i += __shfl_xor_sync(0xffffffffu, sum.i, o);
    }
    C<TC> mean = cscale(TC(1) / TC(Ny), sum);
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = csub2(x[r], mean);
  } else {
    // forward: y_j = m_j y_{j-1} + m_j b_j
    M1<TC> loc = m1_id<TC>();
#pragma unroll
    for (int r = 0; r < R; ++r) loc = m1_comp(M1<TC>{m[r], cscale(m[r], b[r]), cz<TC>()}, loc);
    M1<TC> pre = m1_exscan(loc, lane, true);
    C<TC> y = pre.b0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      y = cscale(m[r], cadd2(b[r], y));
      x[r] = y;          // forward values for now
    }
    // backward: x_j = y_j + m_j x_{j+1}, x_{Ny-1} = y_{Ny-1}
    M1<TC> locb = m1_id<TC>();
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      int j = j0 + r;
      TC a = (j < Ny - 1) ? m[r] : TC(0);
      if (j >= Ny) a = TC(1);
      C<TC> c = (j < Ny) ? x[r] : cz<TC>();
      locb = m1_comp(M1<TC>{a, c, cz<TC>()}, locb);
    }
    M1<TC> preb = m1_exscan(locb, lane, false);
    C<TC> xn = preb.b0;
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      int j = j0 + r;
      if (j < Ny) {
        TC a = (j < Ny - 1) ? m[r] : TC(0);
        xn = cfma(a, xn, x[r]);
        x[r] = xn;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int j = j0 + r;
    if (j < Ny) col[(size_t)j * cs] = cplx<TS>{(TS)(x[r].r * norm), (TS)(x[r].i * norm)};
  }
}


template <typename TS, typename TC, int R>
__global__ void k_poisson_scan(cplx<TS>* __restrict__ S, const TC* __restrict__ piv, const int* __restrict__ list,
                               int n_list, const unsigned char* __restrict__ skip, int Ny, int Nz, int Nxh, int Px,
                               int singular, TC norm) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n_list) return;
  const int mode = list ? list[w] : w;
  if (skip && skip[mode]) return;
  const int kz = mode / Nxh, kx = mode - kz * Nxh;
  poisson_mode<TS, TC, R>(S + (size_t)kz * Ny * Px + kx, (size_t)Px, piv, mode, Ny, singular, norm);
}

// The same over tiles of TM consecutive x-modes at one kz staged in shared
// memory (coalesced row loads and stores; modes in `skip` are left alone).
template <typename TS, typename TC, int R, int TM>
__global__ void k_poisson_scan_staged(cplx<TS>* __restrict__ S, const TC* __restrict__ piv,
                                      const unsigned char* __restrict__ skip, int Ny, int Nxh, int Px, int singular,
                                      TC norm) {
  extern __shared__ unsigned char smem_raw[];
  cplx<TS>* tile = reinterpret_cast<cplx<TS>*>(smem_raw);     // [TM][Ny + 1]
  const int PR = Ny + 1;
  const int ntx = (Nxh + TM - 1) / TM;
  const int kz = blockIdx.x / ntx, kx0 = (blockIdx.x - kz * ntx) * TM;
  cplx<TS>* base = S + (size_t)kz * Ny * Px;
  for (int idx = threadIdx.x; idx < TM * Ny; idx += blockDim.x) {
    const int c = idx % TM, row = idx / TM;
    tile[c * PR + row] = kx0 + c < Nxh ? base[(size_t)row * Px + kx0 + c] : cplx<TS>{TS(0), TS(0)};
  }
  __syncthreads();
  const int wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wib; c < TM; c += nw) {
    const int kx = kx0 + c;
    if (kx >= Nxh) break;
    const int mode = kz * Nxh + kx;
    if (skip && skip[mode]) continue;
    poisson_mode<TS, TC, R>(tile + c * PR, 1, piv, mode, Ny, singular, norm);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < TM * Ny; idx += blockDim.x) {
    const int c = idx % TM, row = idx / TM;
    const int kx = kx0 + c;
    if (kx < Nxh && !(skip && skip[kz * Nxh + kx])) base[(size_t)row * Px + kx] = tile[c * PR + row];
  }
}

// ------------------------------------------------------------------- Stokes
// Per mode (K > 0), with g = g_x f_x + g_z f_z on cell rows:
//  A  forward L D L^T substitution over the faces f = 1..Ny-1:
//       y_f = rhs_f - l1_f y_{f-1} - l2_f y_{f-2},  rhs_f = (K^2 f_y,f + g_f - g_{f-1}) / eta
//  B  backward: v_f = y_f d_f - l1_{f+1} v_{f+1} - l2_{f+2} v_{f+2}
//  C  p_j = -(g_j + eta (A_c D_y v)_j) / K^2 (row-local), then the forward
//     Thomas sweeps of eta A_c u = f_x + conj(g_x) p and eta A_c w = f_z + conj(g_z) p
//  D  their backward sweeps.
// Tables [M][Ny] indexed by face (L1, L2, DI; entry 0 unused) or cell row (CI);
// MC [M][5] = (g_x, g_z, -1/K^2; 0 for K = 0).  The K = 0 mode (all-zero
// pentadiagonal factors) gives v = 0 and p = 0 here; its pressure, needed only
// for output, is p_j = sum_{f=1..j} f_y,f with the mean removed.
// The four sweeps of one mode.  Su, Sv, Sw point at the mode's column of
// the u, v, w spectra, rows cs apart (the spectrum itself, or a staged copy
// in shared memory); Sp (rows P.Px apart, the spectrum's layout) may be NULL.
// sg, sv: the warp's shared-memory rows of g and v.
template <typename TS, typename TC, int R>
__device__ __forceinline__ void stokes_mode(cplx<TS>* __restrict__ Su, cplx<TS>* __restrict__ Sv,
                                            cplx<TS>* __restrict__ Sw, size_t cs, cplx<TS>* __restrict__ Sp,
                                            int mode, const Params& P, const TC* __restrict__ L1,
                                            const TC* __restrict__ L2, const TC* __restrict__ DI,
                                            const TC* __restrict__ CI, const TC* __restrict__ MC, C<TC>* sg,
                                            C<TC>* sv) {
  const int Ny = P.Ny, Px = P.Px, Nxh = P.Nxh;
  const int lane = threadIdx.x & 31;
  const int kz = mode / Nxh, kx = mode - kz * Nxh;
  const TC* l1 = L1 + (size_t)mode * Ny;
  const TC* l2 = L2 + (size_t)mode * Ny;
  const TC* di = DI + (size_t)mode * Ny;
  const TC* ci = CI + (size_t)mode * Ny;
  const TC gxr = MC[5 * (size_t)mode], gxi = MC[5 * (size_t)mode + 1];
  const TC gzr = MC[5 * (size_t)mode + 2], gzi = MC[5 * (size_t)mode + 3];
  const TC mik2 = MC[5 * (size_t)mode + 4];
  const TC K2 = mik2 != TC(0) ? TC(-1) / mik2 : TC(0);
  const auto& Q = phys(P, TC());      // constants in the arithmetic type, no conversions
  const TC eta = Q.eta, ieta = Q.inv_eta;
  const TC norm = Q.inv_nxnz;
  const int j0 = lane * R;
  C<TC> fx[R], fz[R], fy[R], g[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int j = j0 + r;
    if (j < Ny) {
      cplx<TS> a = Su[(size_t)j * cs], b = Sw[(size_t)j * cs], c = Sv[(size_t)j * cs];
      fx[r] = C<TC>{(TC)a.re, (TC)a.im};
      fz[r] = C<TC>{(TC)b.re, (TC)b.im};
      fy[r] = C<TC>{(TC)c.re, (TC)c.im};
      g[r] = C<TC>{gxr * fx[r].r - gxi * fx[r].i + gzr * fz[r].r - gzi * fz[r].i,
                   gxr * fx[r].i + gxi * fx[r].r + gzr * fz[r].i + gzi * fz[r].r};
      sg[j] = g[r];
    } else {
      fx[r] = fz[r] = fy[r] = g[r] = cz<TC>();
    }
  }
  // K = 0 pressure (output only): p_j = sum_{f=1..j} f_y,f, mean removed
  if (mode == 0 && Sp) {
    M1<TC> loc = m1_id<TC>();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int j = j0 + r;
      C<TC> add = (j >= 1 && j < Ny) ? fy[r] : cz<TC>();
      loc = m1_comp(M1<TC>{TC(1), add, cz<TC>()}, loc);
    }
    M1<TC> pre = m1_exscan(loc, lane, true);
    C<TC> p = pre.b0, sum = cz<TC>(), pv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int j = j0 + r;
      if (j >= 1 && j < Ny) p = cadd2(p, fy[r]);
      pv[r] = p;
      if (j < Ny) sum = cadd2(sum, p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sum.r += __shfl_xor_sync(0xffffffffu, sum.r, o);
      sum.i += __shfl_xor_sync(0xffffffffu, sum.i, o);
    }
    C<TC> mean = cscale(TC(1) / TC(Ny), sum);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int j = j0 + r;
      if (j < Ny) {
        C<TC> q = csub2(pv[r], mean);
        Sp[(size_t)kz * Ny * Px + kx + (size_t)j * Px] = cplx<TS>{(TS)(q.r * norm), (TS)(q.i * norm)};
      }
    }
  }
  __syncwarp();
  // ---- A: forward, state (y_f, y_{f-1})
  C<TC> y[R];
  {
    M2<TC> loc = m2_id<TC>();
    C<TC> rhs[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int f = j0 + r;
      rhs[r] = cz<TC>();
      if (f >= 1 && f < Ny) {
        C<TC> gm = sg[f - 1];
        rhs[r] = cscale(ieta, C<TC>{K2 * fy[r].r + (g[r].r - gm.r), K2 * fy[r].i + (g[r].i - gm.i)});
        M2<TC> mf{-l1[f], -l2[f], TC(1), TC(0), rhs[r], cz<TC>()};
        loc = m2_comp(mf, loc);
      }
    }
    M2<TC> pre = m2_exscan(loc, lane, true);
    C<TC> s0 = pre.c0, s1 = pre.c1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int f = j0 + r;
      if (f >= 1 && f < Ny) {
        C<TC> n0 = csub2(csub2(rhs[r], cscale(l1[f], s0)), cscale(l2[f], s1));
        s1 = s0; s0 = n0;
      }
      y[r] = s0;
    }
  }
  // ---- B: backward, state (v_f, v_{f+1})
  C<TC> v[R];
  {
    M2<TC> loc = m2_id<TC>();
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      int f = j0 + r;
      if (f >= 1 && f < Ny) {
        TC a1 = f + 1 < Ny ? l1[f + 1] : TC(0);
        TC a2 = f + 2 < Ny ? l2[f + 2] : TC(0);
        M2<TC> mf{-a1, -a2, TC(1), TC(0), cscale(di[f], y[r]), cz<TC>()};
        loc = m2_comp(mf, loc);
      }
    }
    M2<TC> pre = m2_exscan(loc, lane, false);
    C<TC> s0 = pre.c0, s1 = pre.c1;
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      int f = j0 + r;
      if (f >= 1 && f < Ny) {
        TC a1 = f + 1 < Ny ? l1[f + 1] : TC(0);
        TC a2 = f + 2 < Ny ? l2[f + 2] : TC(0);
        C<TC> n0 = csub2(csub2(cscale(di[f], y[r]), cscale(a1, s0)), cscale(a2, s1));
        s1 = s0; s0 = n0;
        v[r] = n0;
      } else {
        v[r] = cz<TC>();
      }
      if (f <= Ny) sv[f] = v[r];
    }
    if (lane == 0) sv[Ny] = cz<TC>();
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int f = j0 + r;
    if (f < Ny + 1) {
      C<TC> vv = (f >= 1 && f < Ny) ? v[r] : cz<TC>();
      Sv[(size_t)f * cs] = cplx<TS>{(TS)(vv.r * norm), (TS)(vv.i * norm)};
    }
  }
  if (lane == 0) Sv[(size_t)Ny * cs] = cplx<TS>{TS(0), TS(0)};
  // ---- C: pressure (row-local) and the forward sweeps for u and w
  C<TC> bu[R], bw[R];
  TC cm[R];
  {
    M1<TC> loc = m1_id<TC>();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int j = j0 + r;
      bu[r] = bw[r] = cz<TC>();
      cm[r] = TC(1);
      if (j < Ny) {
        C<TC> e0 = csub2(sv[j + 1], sv[j]);
        // A_c's diagonal: the tangential ghost adds +1 at a no-slip wall, -1 at a slip wall
        TC a = K2 + TC(2) + (j == 0 ? (P.slip[0] ? TC(-1) : TC(1)) : TC(0)) +
               (j == Ny - 1 ? (P.slip[1] ? TC(-1) : TC(1)) : TC(0));
        C<TC> acd = cscale(a, e0);
        if (j >= 1) acd = csub2(acd, csub2(sv[j], sv[j - 1]));
        if (j <= Ny - 2) acd = csub2(acd, csub2(sv[j + 2], sv[j + 1]));
        C<TC> p = cscale(mik2, cfma(eta, acd, g[r]));
        if (Sp && mode != 0)
          Sp[(size_t)kz * Ny * Px + kx + (size_t)j * Px] = cplx<TS>{(TS)(p.r * norm), (TS)(p.i * norm)};
        // conj(g) p = (gr pr + gi pi) + i (gr pi - gi pr)
        bu[r] = cscale(ieta, C<TC>{fx[r].r + gxr * p.r + gxi * p.i, fx[r].i + gxr * p.i - gxi * p.r});
        bw[r] = cscale(ieta, C<TC>{fz[r].r + gzr * p.r + gzi * p.i, fz[r].i + gzr * p.i - gzi * p.r});
        cm[r] = ci[j];
        loc = m1_comp(M1<TC>{cm[r], cscale(cm[r], bu[r]), cscale(cm[r], bw[r])}, loc);
      }
    }
    M1<TC> pre = m1_exscan(loc, lane, true);
    C<TC> yu = pre.b0, yw = pre.b1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int j = j0 + r;
      if (j < Ny) {
        yu = cscale(cm[r], cadd2(bu[r], yu));
        yw = cscale(cm[r], cadd2(bw[r], yw));
      }
      bu[r] = yu;
      bw[r] = yw;
    }
  }
  // ---- D: backward sweeps x_j = y_j + c_j x_{j+1}
  {
    M1<TC> loc = m1_id<TC>();
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      int j = j0 + r;
      if (j < Ny) {
        TC a = j < Ny - 1 ? cm[r] : TC(0);
        loc = m1_comp(M1<TC>{a, bu[r], bw[r]}, loc);
      }
    }
    M1<TC> pre = m1_exscan(loc, lane, false);
    C<TC> xu = pre.b0, xw = pre.b1;
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      int j = j0 + r;
      if (j < Ny) {
        TC a = j < Ny - 1 ? cm[r] : TC(0);
        xu = cfma(a, xu, bu[r]);
        xw = cfma(a, xw, bw[r]);
        Su[(size_t)j * cs] = cplx<TS>{(TS)(xu.r * norm), (TS)(xu.i * norm)};
        Sw[(size_t)j * cs] = cplx<TS>{(TS)(xw.r * norm), (TS)(xw.i * norm)};
      }
    }
  }
}


template <typename TS, typename TC, int R>
__global__ void k_stokes_scan(cplx<TS>* __restrict__ S, cplx<TS>* __restrict__ Sp, Params P,
                              const TC* __restrict__ L1, const TC* __restrict__ L2, const TC* __restrict__ DI,
                              const TC* __restrict__ CI, const TC* __restrict__ MC, const int* __restrict__ list,
                              int n_list, const unsigned char* __restrict__ skip) {
  extern __shared__ unsigned char smem_raw[];
  const int Ny = P.Ny, Nz = P.Nz, Px = P.Px, Nxh = P.Nxh;
  const int wib = threadIdx.x >> 5;
  const int w = blockIdx.x * (blockDim.x >> 5) + wib;
  if (w >= n_list) return;
  const int mode = list ? list[w] : w;
  if (skip && skip[mode]) return;
  C<TC>* sg = reinterpret_cast<C<TC>*>(smem_raw) + (size_t)wib * (2 * Ny + 1);   // g [Ny]
  C<TC>* sv = sg + Ny;                                                              // v [Ny + 1]
  const int kz = mode / Nxh, kx = mode - kz * Nxh;
  cplx<TS>* Su = S + (size_t)kz * Ny * Px + kx;
  cplx<TS>* Sv = S + (size_t)Nz * Ny * Px + (size_t)kz * (Ny + 1) * Px + kx;
  cplx<TS>* Sw = S + (size_t)Nz * (2 * Ny + 1) * Px + (size_t)kz * Ny * Px + kx;
  stokes_mode<TS, TC, R>(Su, Sv, Sw, (size_t)Px, Sp, mode, P, L1, L2, DI, CI, MC, sg, sv);
}

// The same solve over a tile of TM consecutive x-modes at one kz, staged in
// shared memory: the block reads the tile's rows of the three spectra with
// coalesced loads (TM consecutive modes of a row are contiguous), each warp
// solves its modes from the staged columns, and the block writes the tile
// back, leaving the modes in `skip` (solved by the double-precision launch
// on the side stream) untouched.  Pressure is not produced.
template <typename TS, typename TC, int R, int TM>
__global__ void k_stokes_scan_staged(cplx<TS>* __restrict__ S, Params P, const TC* __restrict__ L1,
                                     const TC* __restrict__ L2, const TC* __restrict__ DI,
                                     const TC* __restrict__ CI, const TC* __restrict__ MC,
                                     const unsigned char* __restrict__ skip) {
  extern __shared__ unsigned char smem_raw[];
  const int Ny = P.Ny, Nz = P.Nz, Px = P.Px, Nxh = P.Nxh;
  const int PR = Ny + 1;                                 // staged column pitch (rows)
  cplx<TS>* tile = reinterpret_cast<cplx<TS>*>(smem_raw);                 // [3][TM][PR]
  C<TC>* wbuf = reinterpret_cast<C<TC>*>(tile + 3 * TM * PR);              // per warp: g [Ny], v [Ny + 1]
  const int ntx = (Nxh + TM - 1) / TM;
  const int kz = blockIdx.x / ntx, kx0 = (blockIdx.x - kz * ntx) * TM;
  const int wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  cplx<TS>* const b0 = S + (size_t)kz * Ny * Px;
  cplx<TS>* const b1 = S + (size_t)Nz * Ny * Px + (size_t)kz * (Ny + 1) * Px;
  cplx<TS>* const b2 = S + (size_t)Nz * (2 * Ny + 1) * Px + (size_t)kz * Ny * Px;
  const int total = 3 * TM * PR;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = idx % TM, row = (idx / TM) % PR, f = idx / (TM * PR);
    const int nrow = f == 1 ? Ny + 1 : Ny;
    cplx<TS> v{TS(0), TS(0)};
    if (row < nrow && kx0 + c < Nxh) v = (f == 0 ? b0 : (f == 1 ? b1 : b2))[(size_t)row * Px + kx0 + c];
    tile[(f * TM + c) * PR + row] = v;
  }
  __syncthreads();
  C<TC>* sg = wbuf + (size_t)wib * (2 * Ny + 1);
  C<TC>* sv = sg + Ny;
  for (int c = wib; c < TM; c += nw) {
    const int kx = kx0 + c;
    if (kx >= Nxh) break;
    const int mode = kz * Nxh + kx;
    if (skip && skip[mode]) continue;
    stokes_mode<TS, TC, R>(tile + (0 * TM + c) * PR, tile + (1 * TM + c) * PR, tile + (2 * TM + c) * PR, 1,
                           nullptr, mode, P, L1, L2, DI, CI, MC, sg, sv);
    __syncwarp();
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = idx % TM, row = (idx / TM) % PR, f = idx / (TM * PR);
    const int nrow = f == 1 ? Ny + 1 : Ny;
    const int kx = kx0 + c;
    if (row < nrow && kx < Nxh && !(skip && skip[kz * Nxh + kx]))
      (f == 0 ? b0 : (f == 1 ? b1 : b2))[(size_t)row * Px + kx] = tile[(f * TM + c) * PR + row];
  }
}


// ------------------------------------------------------------------ sweeps
// The single-precision bulk of the mixed path (every mode but the low ones,
// which are solved in double on the side stream): one thread per mode, the
// same recurrences as the scans above run sequentially along y, in place in
// the spectra.  A warp takes 32 consecutive x-modes of one kz, so each of
// its row accesses is one contiguous run of 256 bytes, and the factor tables
// are stored [row][mode] for the same reason.  Per row and mode this is a
// few dozen instructions, where a warp-wide scan spends log2(32) levels of
// map compositions per mode; the modes run in parallel instead of the rows.
// Threads are laid out over (kz, kx) with kx padded to a multiple of 32.
__device__ __forceinline__ C<float> ldcf(const cplx<float>* p) {
  const cplx<float> v = *p;
  return C<float>{v.re, v.im};
}
__device__ __forceinline__ void stcf(cplx<float>* p, C<float> v, float s) { *p = cplx<float>{v.r * s, v.i * s}; }

// Rows are handled in blocks of SB: the block's loads (spectra and factor
// rows) are issued together before its sequential recurrence, so one memory
// latency covers SB rows (the stores of a block may alias later loads only
// through the in-place spectra, which is why the prefetch is explicit).
// 16 rows for the Poisson sweep; 8 for the Stokes sweep, which holds three
// fields per row (16 there needs all 255 registers and runs slower).
constexpr int SB_POISSON = 16, SB_STOKES = 8;

__global__ void k_poisson_sweep(cplx<float>* __restrict__ S, const float* __restrict__ piv,
                                const unsigned char* __restrict__ skip, int Ny, int Nz, int Nxh, int Px,
                                float norm) {
  const int NxhP = (Nxh + 31) & ~31;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int kz = t / NxhP, kx = t - kz * NxhP;
  if (kz >= Nz || kx >= Nxh) return;
  const int mode = kz * Nxh + kx;
  if (skip && skip[mode]) return;
  const size_t M = (size_t)Nz * Nxh;
  cplx<float>* col = S + (size_t)kz * Ny * Px + kx;
  // forward y_j = piv_j (b_j + y_{j-1}), in place
  C<float> y = cz<float>();
  for (int jb = 0; jb < Ny; jb += SB_POISSON) {
    C<float> b[SB_POISSON];
    float m[SB_POISSON];
#pragma unroll
    for (int r = 0; r < SB_POISSON; ++r) {
      const int j = jb + r;
      b[r] = j < Ny ? ldcf(col + (size_t)j * Px) : cz<float>();
      m[r] = j < Ny ? piv[(size_t)j * M + mode] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < SB_POISSON; ++r) {
      const int j = jb + r;
      if (j < Ny) {
        y = cscale(m[r], cadd2(b[r], y));
        stcf(col + (size_t)j * Px, y, 1.f);
      }
    }
  }
  // backward x_j = y_j + piv_j x_{j+1}, x_{Ny-1} = y_{Ny-1}
  C<float> xn = cz<float>();
  for (int jt = Ny - 1; jt >= 0; jt -= SB_POISSON) {
    C<float> b[SB_POISSON];
    float a[SB_POISSON];
#pragma unroll
    for (int r = 0; r < SB_POISSON; ++r) {
      const int j = jt - r;
      b[r] = j >= 0 ? ldcf(col + (size_t)j * Px) : cz<float>();
      a[r] = (j >= 0 && j < Ny - 1) ? piv[(size_t)j * M + mode] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < SB_POISSON; ++r) {
      const int j = jt - r;
      if (j >= 0) {
        xn = cfma(a[r], xn, b[r]);
        stcf(col + (size_t)j * Px, xn, norm);
      }
    }
  }
}

__global__ void k_stokes_sweep(cplx<float>* __restrict__ S, cplx<float>* __restrict__ Sp, Params P,
                               const float* __restrict__ L1, const float* __restrict__ L2,
                               const float* __restrict__ DI, const float* __restrict__ CI,
                               const float* __restrict__ MC, const unsigned char* __restrict__ skip) {
  const int Ny = P.Ny, Nz = P.Nz, Px = P.Px, Nxh = P.Nxh;
  const int NxhP = (Nxh + 31) & ~31;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int kz = t / NxhP, kx = t - kz * NxhP;
  if (kz >= Nz || kx >= Nxh) return;
  const int mode = kz * Nxh + kx;
  if (skip && skip[mode]) return;
  const size_t M = (size_t)Nz * Nxh;
  cplx<float>* Su = S + (size_t)kz * Ny * Px + kx;
  cplx<float>* Sv = S + (size_t)Nz * Ny * Px + (size_t)kz * (Ny + 1) * Px + kx;
  cplx<float>* Sw = S + (size_t)Nz * (2 * Ny + 1) * Px + (size_t)kz * Ny * Px + kx;
  const float gxr = MC[5 * (size_t)mode], gxi = MC[5 * (size_t)mode + 1];
  const float gzr = MC[5 * (size_t)mode + 2], gzi = MC[5 * (size_t)mode + 3];
  const float mik2 = MC[5 * (size_t)mode + 4];
  const float K2 = mik2 != 0.f ? -1.f / mik2 : 0.f;
  const float eta = P.f.eta, ieta = P.f.inv_eta, norm = P.f.inv_nxnz;
  const float wb = P.slip[0] ? -1.f : 1.f, wt = P.slip[1] ? -1.f : 1.f;
  auto gsum = [&](C<float> fx, C<float> fz) {
    return C<float>{gxr * fx.r - gxi * fx.i + gzr * fz.r - gzi * fz.i,
                    gxr * fx.i + gxi * fx.r + gzr * fz.i + gzi * fz.r};
  };
  // A: y_f = ieta (K^2 fy_f + g_f - g_{f-1}) - l1_f y_{f-1} - l2_f y_{f-2}, f = 1..Ny-1 (over fy)
  {
    C<float> gprev = gsum(ldcf(Su), ldcf(Sw));
    C<float> y1 = cz<float>(), y2 = cz<float>();
    for (int fb = 1; fb < Ny; fb += SB_STOKES) {
      // raw loads first (nothing computed from them until all are issued)
      C<float> ux[SB_STOKES], uz[SB_STOKES], fy[SB_STOKES];
      float l1[SB_STOKES], l2[SB_STOKES];
#pragma unroll
      for (int r = 0; r < SB_STOKES; ++r) {
        const int f = fb + r;
        const bool in = f < Ny;
        ux[r] = in ? ldcf(Su + (size_t)f * Px) : cz<float>();
        uz[r] = in ? ldcf(Sw + (size_t)f * Px) : cz<float>();
        fy[r] = in ? ldcf(Sv + (size_t)f * Px) : cz<float>();
        l1[r] = in ? L1[(size_t)f * M + mode] : 0.f;
        l2[r] = in ? L2[(size_t)f * M + mode] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < SB_STOKES; ++r) {
        const int f = fb + r;
        if (f < Ny) {
          const C<float> g = gsum(ux[r], uz[r]);
          const C<float> rhs =
              cscale(ieta, C<float>{K2 * fy[r].r + (g.r - gprev.r), K2 * fy[r].i + (g.i - gprev.i)});
          const C<float> y = csub2(csub2(rhs, cscale(l1[r], y1)), cscale(l2[r], y2));
          stcf(Sv + (size_t)f * Px, y, 1.f);
          y2 = y1; y1 = y; gprev = g;
        }
      }
    }
  }
  // B: v_f = di_f y_f - l1_{f+1} v_{f+1} - l2_{f+2} v_{f+2}, f = Ny-1..1 (over y, unscaled)
  {
    C<float> v1 = cz<float>(), v2 = cz<float>();
    for (int ft = Ny - 1; ft >= 1; ft -= SB_STOKES) {
      C<float> yv[SB_STOKES];
      float d[SB_STOKES], a1[SB_STOKES], a2[SB_STOKES];
#pragma unroll
      for (int r = 0; r < SB_STOKES; ++r) {
        const int f = ft - r;
        const bool in = f >= 1;
        yv[r] = in ? ldcf(Sv + (size_t)f * Px) : cz<float>();
        d[r] = in ? DI[(size_t)f * M + mode] : 0.f;
        a1[r] = (in && f + 1 < Ny) ? L1[(size_t)(f + 1) * M + mode] : 0.f;
        a2[r] = (in && f + 2 < Ny) ? L2[(size_t)(f + 2) * M + mode] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < SB_STOKES; ++r) {
        const int f = ft - r;
        if (f >= 1) {
          const C<float> v = csub2(csub2(cscale(d[r], yv[r]), cscale(a1[r], v1)), cscale(a2[r], v2));
          stcf(Sv + (size_t)f * Px, v, 1.f);
          v2 = v1; v1 = v;
        }
      }
    }
  }
  // C: the pressure row by row from a window (v_{j-1}, v_j, v_{j+1}, v_{j+2})
  // (wall faces 0 and Ny carry v = 0), then the forward sweeps of the u and
  // w tridiagonals, in place; face j of v is final (scaled) once row j is
  // done.  A block loads the v faces it will need (jb + 2 .. jb + SB_STOKES + 1)
  // before it overwrites faces jb .. jb + SB_STOKES - 1.
  {
    C<float> vm1 = cz<float>(), v0 = cz<float>();
    C<float> vp1 = Ny >= 2 ? ldcf(Sv + (size_t)Px) : cz<float>();
    C<float> yu = cz<float>(), yw = cz<float>();
    for (int jb = 0; jb < Ny; jb += SB_STOKES) {
      C<float> fx[SB_STOKES], fz[SB_STOKES], vn[SB_STOKES];
      float c[SB_STOKES];
#pragma unroll
      for (int r = 0; r < SB_STOKES; ++r) {
        const int j = jb + r;
        const bool in = j < Ny;
        fx[r] = in ? ldcf(Su + (size_t)j * Px) : cz<float>();
        fz[r] = in ? ldcf(Sw + (size_t)j * Px) : cz<float>();
        c[r] = in ? CI[(size_t)j * M + mode] : 0.f;
        vn[r] = (j + 2 <= Ny - 1) ? ldcf(Sv + (size_t)(j + 2) * Px) : cz<float>();   // v_{j+2}
      }
#pragma unroll
      for (int r = 0; r < SB_STOKES; ++r) {
        const int j = jb + r;
        if (j < Ny) {
          const C<float> vp2 = vn[r];
          // A_c's diagonal: the tangential ghost adds +1 at a no-slip wall, -1 at a slip wall
          const float a = K2 + 2.f + (j == 0 ? wb : 0.f) + (j == Ny - 1 ? wt : 0.f);
          C<float> acd = cscale(a, csub2(vp1, v0));
          if (j >= 1) acd = csub2(acd, csub2(v0, vm1));
          if (j <= Ny - 2) acd = csub2(acd, csub2(vp2, vp1));
          const C<float> p = cscale(mik2, cfma(eta, acd, gsum(fx[r], fz[r])));
          if (Sp) Sp[(size_t)kz * Ny * Px + kx + (size_t)j * Px] = cplx<float>{p.r * norm, p.i * norm};
          const C<float> bu =
              cscale(ieta, C<float>{fx[r].r + gxr * p.r + gxi * p.i, fx[r].i + gxr * p.i - gxi * p.r});
          const C<float> bw =
              cscale(ieta, C<float>{fz[r].r + gzr * p.r + gzi * p.i, fz[r].i + gzr * p.i - gzi * p.r});
          yu = cscale(c[r], cadd2(bu, yu));
          yw = cscale(c[r], cadd2(bw, yw));
          stcf(Su + (size_t)j * Px, yu, 1.f);
          stcf(Sw + (size_t)j * Px, yw, 1.f);
          stcf(Sv + (size_t)j * Px, v0, norm);
          vm1 = v0; v0 = vp1; vp1 = vp2;
        }
      }
    }
    Sv[(size_t)Ny * Px] = cplx<float>{0.f, 0.f};
  }
  // D: backward x_j = y_j + ci_j x_{j+1}, x_{Ny-1} = y_{Ny-1}
  {
    C<float> xu = cz<float>(), xw = cz<float>();
    for (int jt = Ny - 1; jt >= 0; jt -= SB_STOKES) {
      C<float> bu[SB_STOKES], bw[SB_STOKES];
      float a[SB_STOKES];
#pragma unroll
      for (int r = 0; r < SB_STOKES; ++r) {
        const int j = jt - r;
        bu[r] = j >= 0 ? ldcf(Su + (size_t)j * Px) : cz<float>();
        bw[r] = j >= 0 ? ldcf(Sw + (size_t)j * Px) : cz<float>();
        a[r] = (j >= 0 && j < Ny - 1) ? CI[(size_t)j * M + mode] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < SB_STOKES; ++r) {
        const int j = jt - r;
        if (j >= 0) {
          xu = cfma(a[r], xu, bu[r]);
          xw = cfma(a[r], xw, bw[r]);
          stcf(Su + (size_t)j * Px, xu, norm);
          stcf(Sw + (size_t)j * Px, xw, norm);
        }
      }
    }
  }
}

template <typename TS, typename TC>
cudaError_t poisson_scan_launch(const Params& P, cplx<TS>* S, const TC* piv, const int* list, int n,
                                const unsigned char* skip, cudaStream_t s) {
  const int Ny = P.Ny;
  const int singular = (P.bc[0] == DISCOS_BC_NEUMANN && P.bc[1] == DISCOS_BC_NEUMANN) ? 1 : 0;
  const TC norm = (TC)P.inv_nxnz;
  const int bs = list ? 64 : 256;          // a list: 2 warps per block (as in stokes_scan_launch)
  const int nb = (n * 32 + bs - 1) / bs;
  if (n <= 0) return cudaSuccess;
  if (!list) {
    // every mode in order: the shared-memory staged kernel, 32 modes per block
    constexpr int TM = 32;
    const int nbs = P.Nz * ((P.Nxh + TM - 1) / TM);
    const size_t sm = (size_t)TM * (Ny + 1) * sizeof(cplx<TS>);
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    if (sm > 48 * 1024 && cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !(done.load() & (1ull << dev))) {
      cudaError_t e = cudaSuccess;
      e = Ny <= 32 ? cudaFuncSetAttribute(k_poisson_scan_staged<TS, TC, 1, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
        : Ny <= 64 ? cudaFuncSetAttribute(k_poisson_scan_staged<TS, TC, 2, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
        : Ny <= 128 ? cudaFuncSetAttribute(k_poisson_scan_staged<TS, TC, 4, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
        : cudaFuncSetAttribute(k_poisson_scan_staged<TS, TC, 8, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) return e;
      done.fetch_or(1ull << dev);
    }
    if (Ny <= 32) k_poisson_scan_staged<TS, TC, 1, TM><<<nbs, bs, sm, s>>>(S, piv, skip, Ny, P.Nxh, P.Px, singular, norm);
    else if (Ny <= 64) k_poisson_scan_staged<TS, TC, 2, TM><<<nbs, bs, sm, s>>>(S, piv, skip, Ny, P.Nxh, P.Px, singular, norm);
    else if (Ny <= 128) k_poisson_scan_staged<TS, TC, 4, TM><<<nbs, bs, sm, s>>>(S, piv, skip, Ny, P.Nxh, P.Px, singular, norm);
    else k_poisson_scan_staged<TS, TC, 8, TM><<<nbs, bs, sm, s>>>(S, piv, skip, Ny, P.Nxh, P.Px, singular, norm);
    count_launches(1);
    return cudaGetLastError();
  }
  if (Ny <= 32) k_poisson_scan<TS, TC, 1><<<nb, bs, 0, s>>>(S, piv, list, n, skip, Ny, P.Nz, P.Nxh, P.Px, singular, norm);
  else if (Ny <= 64) k_poisson_scan<TS, TC, 2><<<nb, bs, 0, s>>>(S, piv, list, n, skip, Ny, P.Nz, P.Nxh, P.Px, singular, norm);
  else if (Ny <= 128) k_poisson_scan<TS, TC, 4><<<nb, bs, 0, s>>>(S, piv, list, n, skip, Ny, P.Nz, P.Nxh, P.Px, singular, norm);
  else k_poisson_scan<TS, TC, 8><<<nb, bs, 0, s>>>(S, piv, list, n, skip, Ny, P.Nz, P.Nxh, P.Px, singular, norm);
  count_launches(1);
  return cudaGetLastError();
}

template <typename TS, typename TC, int R, int TM>
cudaError_t stokes_staged_launch(const Params& P, cplx<TS>* S, const TC* L1, const TC* L2, const TC* DI,
                                 const TC* CI, const TC* MC, const unsigned char* skip, cudaStream_t s) {
  const int warps = 8;
  const size_t sm = 3 * (size_t)TM * (P.Ny + 1) * sizeof(cplx<TS>) + warps * (size_t)(2 * P.Ny + 1) * sizeof(C<TC>);
  // the attribute belongs to the current device: set it once per device
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !(done.load() & (1ull << dev))) {
    cudaError_t e = cudaFuncSetAttribute(k_stokes_scan_staged<TS, TC, R, TM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    done.fetch_or(1ull << dev);
  }
  const int nb = P.Nz * ((P.Nxh + TM - 1) / TM);
  k_stokes_scan_staged<TS, TC, R, TM><<<nb, 32 * warps, sm, s>>>(S, P, L1, L2, DI, CI, MC, skip);
  count_launches(1);
  return cudaGetLastError();
}

template <typename TS, typename TC>
cudaError_t stokes_scan_launch(const Params& P, cplx<TS>* S, cplx<TS>* Sp, const TC* L1, const TC* L2,
                               const TC* DI, const TC* CI, const TC* MC, const int* list, int n,
                               const unsigned char* skip, cudaStream_t s) {
  const int Ny = P.Ny;
  if (n <= 0) return cudaSuccess;
  // every mode in order and no pressure wanted: the shared-memory staged kernel
  if (!list && !Sp) {
    constexpr int TM = sizeof(TS) == 4 ? 16 : 8;
    if (Ny <= 32) return stokes_staged_launch<TS, TC, 1, TM>(P, S, L1, L2, DI, CI, MC, skip, s);
    if (Ny <= 64) return stokes_staged_launch<TS, TC, 2, TM>(P, S, L1, L2, DI, CI, MC, skip, s);
    if (Ny <= 128) return stokes_staged_launch<TS, TC, 4, TM>(P, S, L1, L2, DI, CI, MC, skip, s);
    return stokes_staged_launch<TS, TC, 8, TM>(P, S, L1, L2, DI, CI, MC, skip, s);
  }
  const size_t per_warp = (size_t)(2 * Ny + 1) * sizeof(C<TC>);
  // a list (the double-precision low modes, a few percent of all) runs 2
  // warps per block, so that its FP64-bound warps spread over all SMs
  int warps = list ? 2 : 8;
  while (warps > 1 && warps * per_warp > 48 * 1024) --warps;   // stay within the default shared-memory limit
  const size_t sm = (size_t)warps * per_warp;
  const int nb = (n + warps - 1) / warps;
  const int bs = 32 * warps;
  if (Ny <= 32) k_stokes_scan<TS, TC, 1><<<nb, bs, sm, s>>>(S, Sp, P, L1, L2, DI, CI, MC, list, n, skip);
  else if (Ny <= 64) k_stokes_scan<TS, TC, 2><<<nb, bs, sm, s>>>(S, Sp, P, L1, L2, DI, CI, MC, list, n, skip);
  else if (Ny <= 128) k_stokes_scan<TS, TC, 4><<<nb, bs, sm, s>>>(S, Sp, P, L1, L2, DI, CI, MC, list, n, skip);
  else k_stokes_scan<TS, TC, 8><<<nb, bs, sm, s>>>(S, Sp, P, L1, L2, DI, CI, MC, list, n, skip);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_poisson_y_impl(const Params& P, Workspace& W, cplx<T>* S, cudaStream_t s) {
  const int M = P.Nxh * P.Nz;
  if constexpr (std::is_same<T, float>::value) {
    // low modes (double) on the side stream, the rest (single) on s
    cudaError_t e = cudaEventRecord(W.yev0, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(W.ystream, W.yev0, 0);
    if (e == cudaSuccess) e = poisson_scan_launch<float, double>(P, S, W.piv64, W.lo_modes, W.n_lo, nullptr, W.ystream);
    if (e == cudaSuccess) e = cudaEventRecord(W.yev1, W.ystream);
    if (e == cudaSuccess) {
      const int nt = P.Nz * ((P.Nxh + 31) & ~31);
      k_poisson_sweep<<<(nt + 127) / 128, 128, 0, s>>>(S, W.piv32t, W.is_lo, P.Ny, P.Nz, P.Nxh, P.Px,
                                                      (float)P.inv_nxnz);
      count_launches(1);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, W.yev1, 0);
    return e;
  } else {
    return poisson_scan_launch<double, double>(P, S, W.piv64, nullptr, M, nullptr, s);
  }
}

template <typename T>
cudaError_t launch_poisson_y(const Params& P, Workspace& W, cplx<T>* S, cudaStream_t s) {
  probe_begin(PROBE_POISSON_Y, s);
  cudaError_t e = launch_poisson_y_impl<T>(P, W, S, s);
  probe_end(PROBE_POISSON_Y, s);
  return e;
}

template <typename T>
cudaError_t launch_stokes_y_impl(const Params& P, Workspace& W, cplx<T>* S, cplx<T>* Sp, cudaStream_t s) {
  const int M = P.Nxh * P.Nz;
  if constexpr (std::is_same<T, float>::value) {
    cudaError_t e = cudaEventRecord(W.yev0, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(W.ystream, W.yev0, 0);
    if (e == cudaSuccess)
      e = stokes_scan_launch<float, double>(P, S, Sp, W.st_l1, W.st_l2, W.st_di, W.st_ci, W.st_mc, W.lo_modes,
                                            W.n_lo, nullptr, W.ystream);
    if (e == cudaSuccess) e = cudaEventRecord(W.yev1, W.ystream);
    if (e == cudaSuccess) {
      const int nt = P.Nz * ((P.Nxh + 31) & ~31);
      k_stokes_sweep<<<(nt + 127) / 128, 128, 0, s>>>(S, Sp, P, W.st_l1f, W.st_l2f, W.st_dif, W.st_cif, W.st_mcf,
                                                     W.is_lo);
      count_launches(1);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, W.yev1, 0);
    return e;
  } else {
    return stokes_scan_launch<double, double>(P, S, Sp, W.st_l1, W.st_l2, W.st_di, W.st_ci, W.st_mc, nullptr, M,
                                              nullptr, s);
  }
}

template <typename T>
cudaError_t launch_stokes_y(const Params& P, Workspace& W, cplx<T>* S, cplx<T>* Sp, cudaStream_t s) {
  probe_begin(PROBE_STOKES_Y, s);
  cudaError_t e = launch_stokes_y_impl<T>(P, W, S, Sp, s);
  probe_end(PROBE_STOKES_Y, s);
  return e;
}

template cudaError_t launch_poisson_y<float>(const Params&, Workspace&, cplx<float>*, cudaStream_t);
template cudaError_t launch_poisson_y<double>(const Params&, Workspace&, cplx<double>*, cudaStream_t);
template cudaError_t launch_stokes_y<float>(const Params&, Workspace&, cplx<float>*, cplx<float>*, cudaStream_t);
template cudaError_t launch_stokes_y<double>(const Params&, Workspace&, cplx<double>*, cplx<double>*, cudaStream_t);

}  // namespace discos
