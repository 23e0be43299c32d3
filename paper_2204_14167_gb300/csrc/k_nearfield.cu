// Near-field forces over the cell list: the P3M local correction of
// Eqs. fullElectro and LC, F^LC = l_B q_i q_j (1/r^2 - f^P(r)) rhat for every
// partner within psi, including the mirror images of the ions across each
// wall (charge -q at a Dirichlet wall, +q at a Neumann wall, Sec. II.B.1); the
// ion-ion LJ force of Eq. closerange; and the wall force of Sec. II.B.2.
//
// One warp per ion in cell order (neighbouring warps share cells, so the
// partner loads hit the same lines).  Each ion sums over its own partners
// (full neighbour loop, no atomics, fixed reduction order).  Whether a pair is
// inside a cutoff is decided with one rounding per operation in the order
// dx = x_i - x_j, minimum image by +-L, r2 = (dx^2 + dy^2) + dz^2, so the
// neighbour counts are reproducible bit for bit.  Image partners of ion i
// can only sit in the list-cell row next to the wall, because a list cell is
// at least psi wide.
#include "physics.cuh"

namespace discos {

namespace {

template <typename T>
__global__ void k_gather(const T* __restrict__ x, const T* __restrict__ q, const int* __restrict__ species, int N,
                         const int* __restrict__ perm, T* __restrict__ xs, T* __restrict__ qs, int* __restrict__ sps) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  int i = perm[s];
  xs[s] = x[i];
  xs[N + s] = x[N + i];
  xs[2 * N + s] = x[2 * N + i];
  qs[s] = q[i];
  sps[s] = species ? species[i] : 0;
}

// One warp per ion (cell order).  Lanes 0..26 take the 27 neighbour cells;
// for an ion within psi of a wall, lanes 0..8 (bottom) and 9..17 (top) then
// take the 9 wall-row cells around it for the image partners.  The partial
// sums are reduced with a fixed shuffle tree (deterministic).
template <typename T>
__global__ void k_near_field(const T* __restrict__ xs, const T* __restrict__ qs, const int* __restrict__ sps,
                             const int* __restrict__ perm, const int* __restrict__ start, int N, Params P,
                             const T* __restrict__ tab, T* __restrict__ F, int* __restrict__ nbr, int accumulate) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= N) return;                       // whole warps exit together
  // once the fault word is set the positions are garbage and may share one
  // cell; skip the pair loops (the host reports the fault at the next step)
  if (P.fault && *reinterpret_cast<const volatile unsigned*>(P.fault)) return;
  const T xi = xs[s], yi = xs[N + s], zi = xs[2 * N + s], qi = qs[s];
  const int si = sps[s];
  const int cx = cell_coord(xi, P.k_cell, P.ncx);
  const int cy = cell_coord(yi, P.k_cell, P.ncy);
  const int cz = cell_coord(zi, P.k_cell, P.ncz);
  const T Lx = T(P.Nx), Lz = T(P.Nz), hx = mul_rn(T(0.5), Lx), hz = mul_rn(T(0.5), Lz);
  const T psi = T(P.psi);
  const T psi2 = mul_rn(psi, psi);
  const T lB = T(P.lB), scale = T(P.tab_scale);
  T fx = T(0), fy = T(0), fz = T(0);
  int cnt = 0;
  if (lane < 27) {
    int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
    int cyy = cy + dy;
    if (cyy >= 0 && cyy < P.ncy) {
      int czz = cz + dz;
      czz = czz < 0 ? czz + P.ncz : (czz >= P.ncz ? czz - P.ncz : czz);
      int cxx = cx + dx;
      cxx = cxx < 0 ? cxx + P.ncx : (cxx >= P.ncx ? cxx - P.ncx : cxx);
      int c = (czz * P.ncy + cyy) * P.ncx + cxx;
      int b = start[c], e = start[c + 1];
      for (int j = b; j < e; ++j) {
        if (j == s) continue;
        pair_terms(xi, yi, zi, qi, si, xs[j], xs[N + j], xs[2 * N + j], qs[j], sps[j], true, P, tab, Lx, hx, Lz,
                   hz, psi2, lB, scale, fx, fy, fz, cnt);
      }
    }
  }
  // wall images: bottom (y -> -y) on lanes 0..8, top (y -> 2 Ny - y) on lanes 9..17
  const bool near0 = yi < psi, near1 = sub_rn(T(P.Ny), yi) < psi;
  if ((near0 && lane < 9) || (near1 && lane >= 9 && lane < 18)) {
    const int wall = lane < 9 ? 0 : 1;
    const int l9 = lane - 9 * wall;
    int dx = l9 % 3 - 1, dz = l9 / 3 - 1;
    int czz = cz + dz;
    czz = czz < 0 ? czz + P.ncz : (czz >= P.ncz ? czz - P.ncz : czz);
    int cxx = cx + dx;
    cxx = cxx < 0 ? cxx + P.ncx : (cxx >= P.ncx ? cxx - P.ncx : cxx);
    const int cyy = wall == 0 ? 0 : P.ncy - 1;
    const T sgn = P.bc[wall] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
    const T twoNy = T(2 * P.Ny);
    int c = (czz * P.ncy + cyy) * P.ncx + cxx;
    int b = start[c], e = start[c + 1];
    for (int j = b; j < e; ++j) {
      T yj = xs[N + j];
      T yimg = wall == 0 ? -yj : sub_rn(twoNy, yj);
      pair_terms(xi, yi, zi, qi, si, xs[j], yimg, xs[2 * N + j], sgn * qs[j], 0, false, P, tab, Lx, hx, Lz, hz,
                 psi2, lB, scale, fx, fy, fz, cnt);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if (lane != 0) return;
  fy += wall_force_y(P, si, yi);
  const int i = perm[s];
  if (accumulate) {
    F[i] += fx;
    F[N + i] += fy;
    F[2 * N + i] += fz;
  } else {
    F[i] = fx;
    F[N + i] = fy;
    F[2 * N + i] = fz;
  }
  if (nbr) nbr[i] = cnt;
}

}  // namespace

template <typename T>
cudaError_t launch_near_field(const Params& P, Workspace& W, const T* x, const T* q, const int* species, int N,
                              T* F, int* nbr, cudaStream_t s, bool accumulate) {
  if (N <= 0) return cudaSuccess;
  cudaError_t e = launch_cell_list<T>(P, W, x, N, s);
  if (e != cudaSuccess) return e;
  T* xs = reinterpret_cast<T*>(W.xs);
  T* qs = reinterpret_cast<T*>(W.qs);
  int bs = 256;
  int nb = (N + bs - 1) / bs;
  probe_begin(PROBE_NEAR_FIELD, s);
  k_gather<T><<<nb, bs, 0, s>>>(x, q, species, N, W.perm, xs, qs, W.sps);
  count_launches(1);
  k_near_field<T><<<(N + 7) / 8, 256, 0, s>>>(xs, qs, W.sps, W.perm, W.cell_start, N, P,
                                                  reinterpret_cast<const T*>(W.fptab), F, nbr, accumulate ? 1 : 0);
  count_launches(1);
  probe_end(PROBE_NEAR_FIELD, s);
  return cudaGetLastError();
}

template cudaError_t launch_near_field<float>(const Params&, Workspace&, const float*, const float*, const int*, int, float*, int*, cudaStream_t, bool);
template cudaError_t launch_near_field<double>(const Params&, Workspace&, const double*, const double*, const int*, int, double*, int*, cudaStream_t, bool);

}  // namespace discos
