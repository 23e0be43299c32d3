// Near-field forces over the cell list: the P3M local correction of
// Eqs. fullElectro and LC, F^LC = l_B q_i q_j (1/r^2 - f^P(r)) rhat for every
// partner within psi, including the mirror images of the ions across each
// wall (charge -q at a Dirichlet wall, +q at a Neumann wall, Sec. II.B.1); the
// ion-ion LJ force of Eq. closerange; and the wall force of Sec. II.B.2.
//
// One thread per ion, ions in cell order: the threads of a warp are
// neighbours along a row of list cells, so they walk nearly the same partner
// ranges and the partner loads hit the same L1 lines.  The three list cells
// of a (dy, dz) row are consecutive in cell order, so each row is one
// contiguous partner range (two where the row wraps in x).  Each ion sums its
// own partners in a fixed order (no atomics: deterministic).  Whether a pair
// is inside a cutoff is decided with one rounding per operation in the order
// dx = x_i - x_j, minimum image by +-L, r2 = (dx^2 + dy^2) + dz^2, so the
// neighbour counts are reproducible bit for bit.  An ion within psi of a wall
// sits in the wall row of list cells (a list cell is at least psi wide), and
// so do the ions whose images can reach it: the image partners are visited
// in the same (dy = 0) rows.  With a metal strip in the dielectric bottom
// wall, a partner's bottom image takes the sign of the wall under it.
#include "physics.cuh"

namespace discos {

namespace {

// Sorted copies of the ions (cell order), x and z wrapped into the periodic
// box, plus a packed (x, y, z, q) copy for the pair loop.
template <typename T>
__global__ void k_gather(const T* __restrict__ x, const T* __restrict__ q, const int* __restrict__ species, int N,
                         const int* __restrict__ perm, int Nx, int Nz, T* __restrict__ xs, T* __restrict__ qs,
                         int* __restrict__ sps, typename Vec4<T>::type* __restrict__ xq) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  int i = perm[s];
  const T px = wrap_coord(x[i], Nx), py = x[N + i], pz = wrap_coord(x[2 * N + i], Nz), qq = q ? q[i] : T(0);
  xs[s] = px;
  xs[N + s] = py;
  xs[2 * N + s] = pz;
  qs[s] = qq;
  sps[s] = species ? species[i] : 0;
  xq[s] = make_vec4(px, py, pz, qq);
}

template <typename T>
__device__ __forceinline__ void row_ranges(const int* __restrict__ start, int base, int cx, int ncx, int& a0,
                                           int& b0, int& a1, int& b1) {
  if (cx >= 1 && cx + 1 < ncx) {
    a0 = start[base + cx - 1]; b0 = start[base + cx + 2]; a1 = b1 = 0;
  } else if (cx == 0) {
    a0 = start[base]; b0 = start[base + 2];
    a1 = start[base + ncx - 1]; b1 = start[base + ncx];
  } else {
    a0 = start[base + cx - 1]; b0 = start[base + ncx];
    a1 = start[base]; b1 = start[base + 1];
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_near_field(const typename Vec4<T>::type* __restrict__ xq,
                                                    const int* __restrict__ sps, const int* __restrict__ start,
                                                    int N, Params P, const T* __restrict__ tab, T* __restrict__ F,
                                                    int* __restrict__ nbr, const int* __restrict__ f_index,
                                                    const int* __restrict__ n_index, int accumulate) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  // once the fault word is set the positions are garbage and may share one
  // cell; skip the pair loops (the host reports the fault at the next step)
  if (P.fault && *reinterpret_cast<const volatile unsigned*>(P.fault)) return;
  T xi, yi, zi, qi;
  load_vec4(xq[s], xi, yi, zi, qi);
  const int si = sps[s];
  const int cx = cell_coord(xi, P.k_cell, P.ncx);
  const int cy = cell_coord(yi, P.k_cell, P.ncy);
  const int cz = cell_coord(zi, P.k_cell, P.ncz);
  const T Lx = T(P.Nx), Lz = T(P.Nz), hx = mul_rn(T(0.5), Lx), hz = mul_rn(T(0.5), Lz);
  const T psi = T(P.psi);
  const T psi2 = mul_rn(psi, psi);
  const T lB = T(P.lB), scale = T(P.tab_scale);
  const bool near0 = yi < psi && cy == 0, near1 = sub_rn(T(P.Ny), yi) < psi && cy == P.ncy - 1;
  const T sg0 = P.bc[0] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
  const T sg1 = P.bc[1] == DISCOS_BC_DIRICHLET ? T(-1) : T(1);
  const T twoNy = T(2 * P.Ny);
  T fx = T(0), fy = T(0), fz = T(0);
  int cnt = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    int czz = cz + dz;
    czz = czz < 0 ? czz + P.ncz : (czz >= P.ncz ? czz - P.ncz : czz);
    for (int dy = -1; dy <= 1; ++dy) {
      const int cyy = cy + dy;
      if (cyy < 0 || cyy >= P.ncy) continue;
      int a0, b0, a1, b1;
      row_ranges<T>(start, (czz * P.ncy + cyy) * P.ncx, cx, P.ncx, a0, b0, a1, b1);
      const bool img = dy == 0 && (near0 || near1);
      for (int part = 0; part < 2; ++part) {
        const int a = part ? a1 : a0, b = part ? b1 : b0;
        for (int j = a; j < b; ++j) {
          T xj, yj, zj, qj;
          load_vec4(xq[j], xj, yj, zj, qj);
          const int sj = sps[j];
          if (j != s)
            pair_terms(xi, yi, zi, qi, si, xj, yj, zj, qj, sj, true, P, tab, Lx, hx, Lz, hz, psi2, lB, scale, fx,
                       fy, fz, cnt);
          if (img) {
            // a metal strip in the bottom wall: the partner's image is the
            // conducting wall's (opposite sign) above the strip's columns
            const T sgj = P.strip ? (on_strip(P, (int)floor(xj)) ? T(-1) : T(1)) : sg0;
            if (near0)
              pair_terms(xi, yi, zi, qi, si, xj, -yj, zj, sgj * qj, 0, false, P, tab, Lx, hx, Lz, hz, psi2, lB,
                         scale, fx, fy, fz, cnt);
            if (near1)
              pair_terms(xi, yi, zi, qi, si, xj, sub_rn(twoNy, yj), zj, sg1 * qj, 0, false, P, tab, Lx, hx, Lz,
                         hz, psi2, lB, scale, fx, fy, fz, cnt);
          }
        }
      }
    }
  }
  fy += wall_force_y(P, si, yi);
  const int i = f_index ? f_index[s] : s;
  if (accumulate) {
    F[i] += fx;
    F[N + i] += fy;
    F[2 * N + i] += fz;
  } else {
    F[i] = fx;
    F[N + i] = fy;
    F[2 * N + i] = fz;
  }
  if (nbr) nbr[n_index ? n_index[s] : s] = cnt;
}

}  // namespace

template <typename T>
cudaError_t launch_sort_ions(const Params& P, Workspace& W, const T* x, const T* q, const int* species, int N,
                             cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  cudaError_t e = launch_cell_list<T>(P, W, x, N, s);
  if (e != cudaSuccess) return e;
  const int bs = 256;
  k_gather<T><<<(N + bs - 1) / bs, bs, 0, s>>>(x, q, species, N, W.perm, P.Nx, P.Nz, reinterpret_cast<T*>(W.xs),
                                              reinterpret_cast<T*>(W.qs), W.sps,
                                              reinterpret_cast<typename Vec4<T>::type*>(W.xq));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_near_field_sorted(const Params& P, Workspace& W, int N, T* F, int* nbr, const int* f_index,
                                     const int* n_index, cudaStream_t s, bool accumulate) {
  if (N <= 0) return cudaSuccess;
  probe_begin(PROBE_NEAR_FIELD, s);
  k_near_field<T><<<(N + 127) / 128, 128, 0, s>>>(reinterpret_cast<const typename Vec4<T>::type*>(W.xq), W.sps,
                                                  W.cell_start, N, P, reinterpret_cast<const T*>(W.fptab), F, nbr,
                                                  f_index, n_index, accumulate ? 1 : 0);
  count_launches(1);
  probe_end(PROBE_NEAR_FIELD, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_near_field(const Params& P, Workspace& W, const T* x, const T* q, const int* species, int N,
                              T* F, int* nbr, cudaStream_t s, bool accumulate) {
  if (N <= 0) return cudaSuccess;
  cudaError_t e = launch_sort_ions<T>(P, W, x, q, species, N, s);
  if (e != cudaSuccess) return e;
  return launch_near_field_sorted<T>(P, W, N, F, nbr, W.perm, W.perm, s, accumulate);
}

template cudaError_t launch_sort_ions<float>(const Params&, Workspace&, const float*, const float*, const int*, int, cudaStream_t);
template cudaError_t launch_sort_ions<double>(const Params&, Workspace&, const double*, const double*, const int*, int, cudaStream_t);
template cudaError_t launch_near_field_sorted<float>(const Params&, Workspace&, int, float*, int*, const int*, const int*, cudaStream_t, bool);
template cudaError_t launch_near_field_sorted<double>(const Params&, Workspace&, int, double*, int*, const int*, const int*, cudaStream_t, bool);
template cudaError_t launch_near_field<float>(const Params&, Workspace&, const float*, const float*, const int*, int, float*, int*, cudaStream_t, bool);
template cudaError_t launch_near_field<double>(const Params&, Workspace&, const double*, const double*, const int*, int, double*, int*, cudaStream_t, bool);

}  // namespace discos
