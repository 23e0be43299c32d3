// Stochastic stress forcing sqrt(2 kT eta / (dV dt)) div_h Z of
// Eq. stokes_temporal on the MAC faces.  Z is symmetric: diagonal entries
// sqrt(2) N(0,1) at cell centres, off-diagonal entries N(0,1) on the edges
// (xy at (x=i, y=j), xz at (x=i, z=k), yz at (y=j, z=k), j = 0..Ny), the
// off-diagonal entries on the wall edges scaled by sqrt(2) at a no-slip wall
// and by 0 at a slip wall, so that the noise covariance matches the viscous
// operator with those walls (discrete fluctuation-dissipation balance).  Normals come from Philox counters
// (cell of an Nx x (Ny+1) x Nz lattice, step, 0, tag 3 / tag 4).
//
// Each block generates Z for a 32 x 8 x 8 tile of cells plus the six faces of
// its one-cell halo in shared memory and then forms the three face
// divergences of its cells, adding them to the force grids with atomics: the
// step runs this kernel on its side stream while the force spreading adds
// into the same (zeroed) grids on the main stream.  A tile cell takes two
// Philox draws (A: xx, yy | zz, xy; B: xz, yz); a halo face takes only the
// draws whose entries the divergences read there (the low x and y faces the
// first normal pair of A, the low z face all of A, the high x and y faces
// the second pair of A and B, the high z face B).  The halo's edges and
// corners are never read.  Every entry keeps the value of its own counter,
// whichever draws a cell takes.
#include <atomic>
#include "internal.h"

namespace discos {

namespace {

constexpr int TX = 32, TY = 8, TZ = 8;
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HN = HX * HY * HZ;

constexpr int N_TILE = TX * TY * TZ;
constexpr int N_XF = TY * TZ, N_YF = TX * TZ, N_ZF = TX * TY;   // cells of one halo face
constexpr int N_HALO_ITEMS = N_TILE + 2 * (N_XF + N_YF + N_ZF);
// draws a halo item takes: bit 0 the first normal pair of A, bit 1 its
// second pair, bit 2 draw B
constexpr unsigned DRAW_A01 = 1u, DRAW_A23 = 2u, DRAW_B = 4u;

// Item t of a block's halo fill: the tile's cells first, then the low and
// high x faces, the y faces and the z faces.  Every segment is a multiple of
// 32 items long, so the draws a warp takes are the same for all its lanes.
__device__ __forceinline__ void halo_item(int t, int& hx, int& hy, int& hz, unsigned& need) {
  if (t < N_TILE) {
    hx = 1 + t % TX; hy = 1 + (t / TX) % TY; hz = 1 + t / (TX * TY);
    need = DRAW_A01 | DRAW_A23 | DRAW_B;
    return;
  }
  t -= N_TILE;
  if (t < 2 * N_XF) {
    const int hi = t / N_XF, r = t - hi * N_XF;
    hx = hi ? TX + 1 : 0; hy = 1 + r % TY; hz = 1 + r / TY;
    need = hi ? (DRAW_A23 | DRAW_B) : DRAW_A01;
    return;
  }
  t -= 2 * N_XF;
  if (t < 2 * N_YF) {
    const int hi = t / N_YF, r = t - hi * N_YF;
    hy = hi ? TY + 1 : 0; hx = 1 + r % TX; hz = 1 + r / TX;
    need = hi ? (DRAW_A23 | DRAW_B) : DRAW_A01;
    return;
  }
  t -= 2 * N_YF;
  const int hi = t / N_ZF, r = t - hi * N_ZF;
  hz = hi ? TZ + 1 : 0; hx = 1 + r % TX; hy = 1 + r / TX;
  need = hi ? DRAW_B : (DRAW_A01 | DRAW_A23);
}

template <typename T>
__global__ void k_stress_noise(T* __restrict__ f, Params P, long long step, T amp) {
  static_assert(N_TILE % 32 == 0 && N_XF % 32 == 0 && N_YF % 32 == 0 && N_ZF % 32 == 0,
                "halo segments must be whole warps");
  extern __shared__ unsigned char smem_raw[];
  T (*Zd)[HN] = reinterpret_cast<T (*)[HN]>(smem_raw);            // xx, yy, zz
  T (*Ze)[HN] = reinterpret_cast<T (*)[HN]>(smem_raw) + 3;        // xy, xz, yz
  const int Nx = P.Nx, Ny = P.Ny, Nz = P.Nz;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * TZ;
  const int tid = threadIdx.x;
  const T r2 = T(1.4142135623730951);
  for (int t = tid; t < N_HALO_ITEMS; t += blockDim.x) {
    int hx, hy, hz;
    unsigned need;
    halo_item(t, hx, hy, hz, need);
    const int h = (hz * HY + hy) * HX + hx;
    int i = (i0 + hx - 1) & (Nx - 1);
    int j = j0 + hy - 1;
    int k = (k0 + hz - 1) & (Nz - 1);
    T a[4] = {T(0), T(0), T(0), T(0)}, b[2] = {T(0), T(0)};
    const bool edge_row = j >= 0 && j <= Ny;      // xy and yz live on j = 0..Ny
    if (edge_row) {
      uint32_t cell = (uint32_t)(((size_t)k * (Ny + 1) + j) * Nx + i);
      if (need & DRAW_A23) normals4(u32x4{cell, (uint32_t)step, 0u, (uint32_t)TAG_STRESS_A}, P.seed, a);
      else if (need & DRAW_A01) normals2(u32x4{cell, (uint32_t)step, 0u, (uint32_t)TAG_STRESS_A}, P.seed, a);
      if (need & DRAW_B) normals2(u32x4{cell, (uint32_t)step, 0u, (uint32_t)TAG_STRESS_B}, P.seed, b);
    }
    const bool centre = j >= 0 && j < Ny;
    // wall edges: sqrt 2 at a no-slip wall, no shear stress at a slip wall
    const T wall = j == 0 ? (P.slip[0] ? T(0) : r2) : (j == Ny ? (P.slip[1] ? T(0) : r2) : T(1));
    if (need & DRAW_A01) {
      Zd[0][h] = centre ? r2 * a[0] : T(0);
      Zd[1][h] = centre ? r2 * a[1] : T(0);
    }
    if (need & DRAW_A23) {
      Zd[2][h] = centre ? r2 * a[2] : T(0);
      Ze[0][h] = edge_row ? wall * a[3] : T(0);                // xy
    }
    if (need & DRAW_B) {
      Ze[1][h] = centre ? b[0] : T(0);                         // xz
      Ze[2][h] = edge_row ? wall * b[1] : T(0);                // yz
    }
  }
  __syncthreads();
  const size_t G = (size_t)Nx * Ny * Nz;
  T* fx = f;
  T* fy = f + G;
  T* fz = f + G + (size_t)Nx * (Ny + 1) * Nz;
  for (int c = tid; c < TX * TY * TZ; c += blockDim.x) {
    int lx = c % TX, ly = (c / TX) % TY, lz = c / (TX * TY);
    int i = i0 + lx, j = j0 + ly, k = k0 + lz;
    if (i >= Nx || j >= Ny || k >= Nz) continue;
    int h = ((lz + 1) * HY + (ly + 1)) * HX + (lx + 1);
    const int sx = 1, sy = HX, sz = HX * HY;
    // x-face (i, j+1/2, k+1/2)
    T dx = (Zd[0][h] - Zd[0][h - sx]) + (Ze[0][h + sy] - Ze[0][h]) + (Ze[1][h + sz] - Ze[1][h]);
    // z-face (i+1/2, j+1/2, k)
    T dz = (Ze[1][h + sx] - Ze[1][h]) + (Ze[2][h + sy] - Ze[2][h]) + (Zd[2][h] - Zd[2][h - sz]);
    atomicAdd(&fx[((size_t)k * Ny + j) * Nx + i], amp * dx);
    atomicAdd(&fz[((size_t)k * Ny + j) * Nx + i], amp * dz);
    if (j >= 1) {
      // y-face (i+1/2, j, k+1/2)
      T dy = (Ze[0][h + sx] - Ze[0][h]) + (Zd[1][h] - Zd[1][h - sy]) + (Ze[2][h + sz] - Ze[2][h]);
      atomicAdd(&fy[((size_t)k * (Ny + 1) + j) * Nx + i], amp * dy);
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_stress_noise(const Params& P, T* f, int64_t step, cudaStream_t s) {
  dim3 grid((P.Nx + TX - 1) / TX, (P.Ny + TY - 1) / TY, (P.Nz + TZ - 1) / TZ);
  T amp = T(sqrt(2.0 * P.kT * P.eta / P.dt));
  const size_t sm = 6 * (size_t)HN * sizeof(T);
  // the attribute belongs to the current device: set it once per device
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !(done.load() & (1ull << dev))) {
    cudaError_t e = cudaFuncSetAttribute(k_stress_noise<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    done.fetch_or(1ull << dev);
  }
  probe_begin(PROBE_NOISE, s);
  k_stress_noise<T><<<grid, 256, sm, s>>>(f, P, (long long)step, amp);
  count_launches(1);
  probe_end(PROBE_NOISE, s);
  return cudaGetLastError();
}

template cudaError_t launch_stress_noise<float>(const Params&, float*, int64_t, cudaStream_t);
template cudaError_t launch_stress_noise<double>(const Params&, double*, int64_t, cudaStream_t);

}  // namespace discos
