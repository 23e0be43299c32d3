// The C ABI of libdiscos: handle creation (validation, workspace, constant
// tables) and the entry points that enqueue the hot-path kernels.  The
// four-stage time step follows Sec. II.D of the paper.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>
#include "internal.h"

namespace discos {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }

// The probe of the handle whose entry point is running on this thread.
static thread_local Probe* g_cur_probe = nullptr;

void probe_begin(int family, cudaStream_t s) {
  Probe* p = g_cur_probe;
  if (p && p->family == family && p->n < Probe::kMax) cudaEventRecord(p->ev[2 * p->n], s);
}

void probe_end(int family, cudaStream_t s) {
  Probe* p = g_cur_probe;
  if (p && p->family == family && p->n < Probe::kMax) {
    cudaEventRecord(p->ev[2 * p->n + 1], s);
    ++p->n;
  }
}

struct ProbeScope {
  explicit ProbeScope(discos_handle* h) { g_cur_probe = h ? &h->probe : nullptr; }
  ~ProbeScope() { g_cur_probe = nullptr; }
};
void count_launches(long long n) { g_launches += n; }

discos_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return DISCOS_OK;
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return DISCOS_ERR_CUDA;
}

discos_status invalid(const std::string& m) {
  set_error(m);
  return DISCOS_ERR_INVALID_ARG;
}

void* dalloc(discos_handle* h, size_t bytes, bool* ok) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (h->alloc_fn) {
    p = h->alloc_fn(bytes, h->alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (!p) *ok = false;
  return p;
}

void dfree(discos_handle* h, void* p) {
  if (!p) return;
  if (h->free_fn) h->free_fn(p, h->alloc_ctx);
  else cudaFree(p);
}

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int kernel_width(int kind, int es_w) {
  if (kind == DISCOS_KERNEL_PESKIN4) return 4;
  if (kind == DISCOS_KERNEL_PESKIN6) return 6;
  if (kind == DISCOS_KERNEL_ES) return es_w;
  return -1;
}

KernelParams make_kernel(int kind, int es_w, double es_beta) {
  KernelParams kp{};
  kp.kind = kind;
  kp.w = kernel_width(kind, es_w);
  if (kind == DISCOS_KERNEL_ES) {
    kp.alpha = 0.5 * es_w;
    kp.beta = es_beta;
    kp.inv_norm = 1.0 / es_normalisation(es_w, es_beta);
    kp.inv_alpha = 1.0 / kp.alpha;
  }
  kp.alpha_f = (float)kp.alpha;
  kp.beta_f = (float)kp.beta;
  kp.inv_norm_f = (float)kp.inv_norm;
  kp.inv_alpha_f = (float)kp.inv_alpha;
  return kp;
}

// The F^P table depends only on the kernel, psi and n_tab: computed once per
// process for each combination.
std::vector<double> cached_fp_table(const KernelParams& kp, double psi, int n_tab) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, double, double, int>, std::vector<double>> cache;
  auto key = std::make_tuple(kp.kind, kp.w, kp.beta, psi, n_tab);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  std::vector<double> tab(n_tab + 1);
  std::string err;
  build_fp_table(kp, psi, n_tab, tab.data(), &err);
  cache[key] = tab;
  return tab;
}

template <typename T>
void upload_twiddles(void* dst, int N) {
  std::vector<cplx<T>> tw(N / 2);
  for (int k = 0; k < N / 2; ++k) {
    double a = -2.0 * M_PI * k / N;
    tw[k] = cplx<T>{T(std::cos(a)), T(std::sin(a))};
  }
  cudaMemcpy(dst, tw.data(), sizeof(cplx<T>) * tw.size(), cudaMemcpyHostToDevice);
}

template <typename T>
void upload_table(void* dst, const std::vector<double>& t) {
  std::vector<T> v(t.begin(), t.end());
  cudaMemcpy(dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// Per-mode factors of the Stokes wall-normal systems (see k_stokes.cu):
// the L D L^T factors of the pentadiagonal K^2 A_f + D_y^T A_c D_y
// (diagonal K^4 + 4K^2 + 6, +1 (no-slip) or -1 (slip) on the first and last
// rows; first off-diagonal -2K^2 - 4; second off-diagonal 1) and the Thomas
// pivots of A_c (diagonal K^2 + 2, +-1 on the wall rows; off-diagonals -1).
void upload_stokes_factors(discos_handle* h) {
  const discos_config& c = h->cfg;
  const int Ny = c.Ny, Nxh = h->P.Nxh, Nz = c.Nz;
  const size_t M = (size_t)Nxh * Nz;
  const int n = Ny - 1;   // unknowns: faces f = 1..Ny-1, index i = f - 1
  std::vector<double> l1((size_t)Ny * M, 0.0), l2((size_t)Ny * M, 0.0), di((size_t)Ny * M, 0.0);
  std::vector<double> ci((size_t)Ny * M), mc(5 * M);
  for (int kz = 0; kz < Nz; ++kz)
    for (int kx = 0; kx < Nxh; ++kx) {
      const size_t m = (size_t)kz * Nxh + kx;
      const double tx = 2.0 * M_PI * kx / c.Nx, tz = 2.0 * M_PI * kz / c.Nz;
      const double K2 = (2.0 - 2.0 * std::cos(tx)) + (2.0 - 2.0 * std::cos(tz));
      const bool zero = kx == 0 && kz == 0;
      mc[5 * m + 0] = std::cos(tx) - 1.0;
      mc[5 * m + 1] = std::sin(tx);
      mc[5 * m + 2] = std::cos(tz) - 1.0;
      mc[5 * m + 3] = std::sin(tz);
      mc[5 * m + 4] = zero ? 0.0 : -1.0 / K2;
      const double e = -2.0 * K2 - 4.0, f = 1.0;
      // the tangential ghost of a no-slip wall (-u(0)) adds +1 to its cell
      // row's diagonal, that of a slip wall (+u(0)) -1 (Eq. fluidbc)
      const double sb = h->P.slip[0] ? -1.0 : 1.0, st = h->P.slip[1] ? -1.0 : 1.0;
      double Dm1 = 0.0, Dm2 = 0.0, l1m1 = 0.0;
      for (int i = 0; i < n; ++i) {
        double a2 = i >= 2 ? f / Dm2 : 0.0;
        double a1 = i >= 1 ? (e - (i >= 2 ? a2 * l1m1 * Dm2 : 0.0)) / Dm1 : 0.0;
        double d = K2 * K2 + 4.0 * K2 + 6.0 + (i == 0 ? sb : 0.0) + (i == n - 1 ? st : 0.0);
        double D = d - a1 * a1 * Dm1 - a2 * a2 * Dm2;
        l1[m * Ny + i + 1] = zero ? 0.0 : a1;
        l2[m * Ny + i + 1] = zero ? 0.0 : a2;
        di[m * Ny + i + 1] = zero ? 0.0 : 1.0 / D;
        Dm2 = Dm1; Dm1 = D; l1m1 = a1;
      }
      double mm = 0.0;
      for (int j = 0; j < Ny; ++j) {
        double a = K2 + 2.0 + (j == 0 ? sb : 0.0) + (j == Ny - 1 ? st : 0.0);
        mm = j == 0 ? a : a - 1.0 / mm;
        ci[m * Ny + j] = 1.0 / mm;
      }
    }
  Workspace& W = h->W;
  cudaMemcpy(W.st_l1, l1.data(), sizeof(double) * l1.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(W.st_l2, l2.data(), sizeof(double) * l2.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(W.st_di, di.data(), sizeof(double) * di.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(W.st_ci, ci.data(), sizeof(double) * ci.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(W.st_mc, mc.data(), sizeof(double) * mc.size(), cudaMemcpyHostToDevice);
  if (h->mixed) {
    // single-precision copies for the sweeps, which read the factors row by
    // row across modes: [Ny][M] (the mode constants stay [M][5])
    auto up_t = [&](float* dst, const std::vector<double>& v) {
      std::vector<float> f(v.size());
      for (size_t m = 0; m < M; ++m)
        for (int j = 0; j < Ny; ++j) f[(size_t)j * M + m] = (float)v[m * Ny + j];
      cudaMemcpy(dst, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice);
    };
    up_t(W.st_l1f, l1); up_t(W.st_l2f, l2); up_t(W.st_dif, di); up_t(W.st_cif, ci);
    std::vector<float> mcf(mc.begin(), mc.end());
    cudaMemcpy(W.st_mcf, mcf.data(), sizeof(float) * mcf.size(), cudaMemcpyHostToDevice);
  }
}

// Inverse of a dense n x n matrix (row major) by Gauss-Jordan elimination
// with partial pivoting, in double; false if singular.
bool invert_dense(std::vector<double>& a, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
    if (!(std::fabs(a[(size_t)piv * n + col]) > 0.0)) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)piv * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    const double d = 1.0 / a[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) { a[(size_t)col * n + k] *= d; inv[(size_t)col * n + k] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

// Metal strip (k_strip.cu): the strip's cell columns, the bottom-row terms
// of the base solve, and per z mode the inverse capacitance matrix
// (I/2 + C_kz)^-1, C_kz[a][b] = (1/Nx) sum_kx g(kx, kz) cos(2 pi kx (a - b) / Nx)
// with g = [T^-1]_00 the bottom-to-bottom entry of the wall-normal
// tridiagonal inverse of mode (kx, kz) for an all-dielectric bottom wall.
// When that operator is singular (top wall dielectric as well), its (0, 0)
// mode takes the pseudo-inverse entry (DCT-II eigenbasis of the
// all-Neumann second difference) and the kz = 0 matrix is the bordered
// one of k_strip.cu.
void setup_strip(discos_handle* h, std::vector<double>& add0, std::vector<double>& Minv) {
  const discos_config& c = h->cfg;
  Params& P = h->P;
  const int Nx = c.Nx, Ny = c.Ny, Nz = c.Nz;
  const int Ws = P.strip_i1 - P.strip_i0, S = Ws + 1;
  add0.assign(Nx, 0.0);
  for (int i = 0; i < Nx; ++i)
    add0[i] = on_strip(P, i) ? 2.0 * (P.strip_phi + P.E_ext[0] * ((i + 0.5) - P.strip_xc)) : -P.slope[0];
  const double top = c.bc[1] == DISCOS_BC_DIRICHLET ? 2.0 * c.phi_b[1] : P.slope[1];
  double sum0 = 0.0;
  for (double v : add0) sum0 += v;
  P.strip_walls = (double)Nz * sum0 + (double)Nx * Nz * top;
  std::vector<double> g((size_t)Nx);
  std::vector<double> cp(Ny), dd(Ny);
  Minv.assign((size_t)Nz * S * S, 0.0);
  for (int kz = 0; kz < Nz; ++kz) {
    const double lz = 2.0 - 2.0 * std::cos(2.0 * M_PI * kz / Nz);
    for (int kx = 0; kx < Nx; ++kx) {
      const double lam = lz + 2.0 - 2.0 * std::cos(2.0 * M_PI * kx / Nx);
      if (P.strip_singular && kx == 0 && kz == 0) {
        double acc = 0.0;
        for (int m = 1; m < Ny; ++m) {
          const double v0 = std::cos(M_PI * m / (2.0 * Ny));
          acc += (2.0 / Ny) * v0 * v0 / (2.0 - 2.0 * std::cos(M_PI * m / Ny));
        }
        g[kx] = acc;
        continue;
      }
      // Thomas solve of T u = e_0, T = tridiag(-1, 2 + lam, -1) with the wall rows
      for (int j = 0; j < Ny; ++j) {
        dd[j] = 2.0 + lam + (j == 0 ? -1.0 : 0.0) +
                (j == Ny - 1 ? (c.bc[1] == DISCOS_BC_DIRICHLET ? 1.0 : -1.0) : 0.0);
      }
      std::vector<double> rhs(Ny, 0.0);
      rhs[0] = 1.0;
      double m = dd[0];
      cp[0] = -1.0 / m;
      rhs[0] /= m;
      for (int j = 1; j < Ny; ++j) {
        m = dd[j] + cp[j - 1];
        cp[j] = -1.0 / m;
        rhs[j] = (rhs[j] + rhs[j - 1]) / m;
      }
      for (int j = Ny - 2; j >= 0; --j) rhs[j] -= cp[j] * rhs[j + 1];
      g[kx] = rhs[0];
    }
    std::vector<double> cd(Ws);
    for (int d = 0; d < Ws; ++d) {
      double acc = 0.0;
      for (int kx = 0; kx < Nx; ++kx) acc += g[kx] * std::cos(2.0 * M_PI * (double)((long long)kx * d % Nx) / Nx);
      cd[d] = acc / Nx;
    }
    const bool border = P.strip_singular && kz == 0;
    const int n = border ? S : Ws;
    std::vector<double> a((size_t)n * n, 0.0);
    for (int i = 0; i < Ws; ++i)
      for (int j = 0; j < Ws; ++j) a[(size_t)i * n + j] = cd[i > j ? i - j : j - i] + (i == j ? 0.5 : 0.0);
    if (border) {
      for (int i = 0; i < Ws; ++i) {
        a[(size_t)i * n + Ws] = -1.0;
        a[(size_t)Ws * n + i] = 1.0;
      }
    }
    invert_dense(a, n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) Minv[(size_t)kz * S * S + (size_t)i * S + j] = a[(size_t)i * n + j];
  }
}

void free_workspace(discos_handle* h) {
  free_batch(h);
  Workspace& W = h->W;
  void* ptrs[] = {W.phi, W.spec, W.fgrid, W.piv64, W.piv32, W.piv32t, W.tw_x, W.tw_z, W.fptab, W.cell_of, W.counts, W.fill,
                  W.cell_start, W.perm, W.tile_sums, W.xs, W.qs, W.sps, W.xq, W.F, W.xstar, W.V,
                  W.st_l1, W.st_l2, W.st_di, W.st_ci, W.st_mc,
                  W.lo_modes, W.is_lo, W.st_l1f, W.st_l2f, W.st_dif, W.st_cif, W.st_mcf, W.Fn, W.edata, W.rref, W.rres, W.rnorm,
                  W.fault, W.diag, W.nsum, W.phi64, W.sref, W.sres, W.pres, W.v64, W.p64, W.snorm,
                  W.strip_g, W.strip_add0, W.strip_r, W.strip_shat, W.strip_M, W.strip_c};
  for (void* p : ptrs) dfree(h, p);
  W = Workspace{};
}

// Neutrality of a channel between two Neumann walls (Sec. II.B.1): the
// charge plus the walls' surface charge must vanish, else the Poisson problem
// has no solution.  Relative tolerance 1e-9 (FP64) / 1e-6 (MIXED) of the
// summed magnitudes.
bool all_neumann(const discos_handle* h) {
  return h->P.bc[0] == DISCOS_BC_NEUMANN && h->P.bc[1] == DISCOS_BC_NEUMANN && !h->P.strip;
}
double surface_total(const discos_handle* h, bool absolute) {
  const double a = h->cfg.surf_charge[0], b = h->cfg.surf_charge[1];
  return (absolute ? std::fabs(a) + std::fabs(b) : a + b) * (double)h->cfg.Nx * (double)h->cfg.Nz;
}
double neutral_tol(const discos_handle* h) { return h->mixed ? 1e-6 : 1e-9; }

// Synchronous check of n charges (or cell charges) v before a solve.
template <typename T>
discos_status check_neutral_sync(discos_handle* h, const T* v, size_t n, cudaStream_t s, const char* what) {
  if (!all_neumann(h)) return DISCOS_OK;
  double buf[2] = {0.0, 0.0};
  cudaError_t e = launch_charge_sums<T>(v, n, h->W.nsum, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf, h->W.nsum, sizeof(buf), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, what);
  const double net = buf[0] + surface_total(h, false);
  if (!(std::fabs(net) <= neutral_tol(h) * (buf[1] + surface_total(h, true)) + 1e-12)) {
    set_error(std::string(what) + ": two Neumann walls need a neutral channel (charge + surface charge = " +
              std::to_string(net) + ")");
    return DISCOS_ERR_NOT_NEUTRAL;
  }
  return DISCOS_OK;
}

// The single-operation entry points work on the ions in the caller's order.
template <typename T>
cudaError_t spread_impl(discos_handle* h, const T* x, const T* val, const int* species, int N, int which, T* grid,
                        cudaStream_t s) {
  if (which == DISCOS_SPREAD_CHARGE) return launch_spread_charge<T>(h->P, x, val, N, grid, s);
  return launch_spread_force<T>(h->P, x, val, N, grid, 0, false, s, false, nullptr, false, species);
}

template <typename T>
cudaError_t interp_impl(discos_handle* h, const T* x, const int* species, int N, int which, const T* grid, T* out,
                        cudaStream_t s) {
  if (which == DISCOS_INTERP_VELOCITY) return launch_interp_velocity<T>(h->P, x, N, grid, out, s, nullptr, species);
  return launch_interp_efield<T>(h->P, x, static_cast<const T*>(nullptr), N, grid, out, false, s,
                                 static_cast<const T*>(nullptr), nullptr);
}

// Stages 1 and 2 of Sec. II.D.  The ions are first binned and copied into
// cell order (W.xs, W.qs, W.sps, W.xq; W.perm maps a sorted index to the
// caller's), so that every particle kernel after it walks space in order and
// its grid accesses stay local.  The near field does not depend on the
// potential, so it runs on the handle's side stream while the main stream
// spreads the charge and solves the Poisson problem; the field interpolation
// then adds the near-field forces (F = q (E + E_ext) + F_near).  `side_extra`
// enqueues further independent work on the side stream before it rejoins
// (the step uses it for the stochastic stress).  With sorted_out the forces
// stay in cell order (the step's own use), else they are written in the
// caller's order; nbr is always in the caller's order.
template <typename T, typename Extra>
discos_status forces_impl(discos_handle* h, const T* x, const T* q, const int* species, int N, T* F, int* nbr,
                          cudaStream_t s, Extra side_extra, bool sorted_out) {
  const Params& P = h->P;
  Workspace& W = h->W;
  T* phi = reinterpret_cast<T*>(W.phi);
  T* Fn = reinterpret_cast<T*>(W.Fn);
  cudaError_t e = launch_sort_ions<T>(P, W, x, q, species, N, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
  if (e == cudaSuccess) e = launch_near_field_sorted<T>(P, W, N, Fn, nbr, nullptr, W.perm, h->side, false);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->side);
  // the extra side work (the step's stochastic stress) runs on past the
  // field interpolation; the caller waits for ev_extra before using it
  if (e == cudaSuccess) e = side_extra(h->side);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_extra, h->side);
  const T* xs = reinterpret_cast<const T*>(W.xs);
  const T* qs = reinterpret_cast<const T*>(W.qs);
  if (e == cudaSuccess) e = launch_spread_charge<T>(P, xs, qs, N, phi, s, true);
  if (e == cudaSuccess) e = launch_poisson<T>(P, W, phi, phi, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_join, 0);
  if (e == cudaSuccess) e = launch_interp_efield<T>(P, xs, qs, N, phi, F, true, s, Fn, sorted_out ? nullptr : W.perm);
  return cuda_status(e, "discos_forces");
}

template <typename T>
discos_status forces_impl(discos_handle* h, const T* x, const T* q, const int* species, int N, T* F, int* nbr,
                          cudaStream_t s) {
  return forces_impl<T>(h, x, q, species, N, F, nbr, s, [](cudaStream_t) { return cudaSuccess; }, false);
}

template <typename T>
discos_status step_impl(discos_handle* h, T* x, const T* q, const int* species, int N, int64_t step0,
                        int nsteps, T* F_out, cudaStream_t s) {
  const Params& P = h->P;
  Workspace& W = h->W;
  T* F = reinterpret_cast<T*>(W.F);
  T* fg = reinterpret_cast<T*>(W.fgrid);
  T* V = reinterpret_cast<T*>(W.V);
  T* xs = reinterpret_cast<T*>(W.xstar);
  const T* xsrt = reinterpret_cast<const T*>(W.xs);
  const bool wet = h->cfg.wet != 0;
  const bool thermal = P.kT > 0.0;
  const bool drift = P.drift != 0;
  const size_t nf = (size_t)P.Nx * P.Nz * (3 * P.Ny + 1);
  for (int n = 0; n < nsteps; ++n) {
    const int64_t step = step0 + n;
    // two Neumann walls: a non-neutral channel sets bit 2 of the fault word,
    // and the next discos_step call returns DISCOS_ERR_NOT_NEUTRAL
    if (all_neumann(h)) {
      cudaError_t e = launch_charge_sums<T>(q, (size_t)N, W.nsum, s);
      if (e == cudaSuccess)
        e = launch_neutral_flag(W.nsum, surface_total(h, false), surface_total(h, true), neutral_tol(h), W.fault, s);
      if (e != cudaSuccess) return cuda_status(e, "discos_step");
    }
    // the fluid forcing starts from zero; the stochastic stress is added on
    // the side stream while the main stream spreads the forces into the same
    // grid (both with atomics)
    if (wet) {
      cudaError_t ez = launch_fill_zero<T>(fg, nf, s);
      if (ez != cudaSuccess) return cuda_status(ez, "discos_step");
    }
    auto side = [&](cudaStream_t ss) -> cudaError_t {
      return (wet && thermal) ? launch_stress_noise<T>(P, fg, step, ss) : cudaSuccess;
    };
    // F comes back in cell order: everything below works on the sorted ions
    // and the update writes each new position back to the caller's index
    discos_status st = forces_impl<T>(h, x, q, species, N, F, nullptr, s, side, true);
    if (st != DISCOS_OK) return st;
    cudaError_t e = cudaSuccess;
    if (wet) {
      e = launch_spread_force<T>(P, xsrt, F, N, fg, step, drift && thermal, s, true, W.perm, true, W.sps);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_extra, 0);
      if (e == cudaSuccess) e = launch_stokes<T>(P, W, fg, fg, nullptr, s);
      if (e == cudaSuccess) e = launch_interp_velocity<T>(P, xsrt, N, fg, V, s, nullptr, W.sps);
      if (drift) {
        if (e == cudaSuccess) e = launch_midpoint<T>(P, xsrt, V, N, xs, s);
        if (e == cudaSuccess) e = launch_interp_velocity<T>(P, xs, N, fg, V, s, nullptr, W.sps);
      }
      if (e == cudaSuccess) e = launch_dry_update<T>(P, x, W.sps, F, V, N, step, s, xsrt, W.perm);
    } else {
      e = launch_dry_update<T>(P, x, W.sps, F, nullptr, N, step, s, xsrt, W.perm);
    }
    if (e != cudaSuccess) return cuda_status(e, "discos_step");
  }
  cudaError_t e = cudaSuccess;
  if (F_out && nsteps > 0) e = launch_scatter3<T>(F, W.perm, N, reinterpret_cast<T*>(F_out), s);
  // the fault word travels to the host behind the steps; the next call reads it
  if (e == cudaSuccess && nsteps > 0)
    e = cudaMemcpyAsync(h->fault_host, W.fault, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && nsteps > 0) e = cudaEventRecord(h->ev_fault, s);
  return cuda_status(e, "discos_step");
}

// Electrostatic energy and its adjoint (k_energy.cu).  rho goes to the
// force-grid buffer, phi to the potential buffer; both are recomputed by the
// backward rather than kept from the forward.
template <typename T>
discos_status energy_impl(discos_handle* h, const Params& P, const T* x, const T* q, int N, double* U,
                          const double* dU, T* dx, T* dq, double* dphi_b, cudaStream_t s) {
  Workspace& W = h->W;
  T* rho = reinterpret_cast<T*>(W.fgrid);
  T* phi = reinterpret_cast<T*>(W.phi);
  double* lift = W.edata;
  double* sums = W.edata + 3 * P.Ny;
  const char* where = U ? "discos_energy" : "discos_energy_backward";
  cudaError_t e = launch_spread_charge<T>(P, x, q, N, rho, s);
  if (e == cudaSuccess) e = launch_poisson<T>(P, W, rho, phi, s);
  if (e == cudaSuccess && (U || dphi_b)) e = launch_lift(P, lift, s);
  if (e == cudaSuccess && (U || dphi_b)) e = launch_energy_sums<T>(P, rho, phi, lift, sums, s);
  if (e == cudaSuccess && U) e = cudaMemcpyAsync(U, sums, sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && dphi_b) e = launch_scale2(sums, dU, dphi_b, s);
  if (e == cudaSuccess && (dx || dq)) e = launch_energy_grad<T>(P, x, q, N, phi, dU, dx, dq, s);
  return cuda_status(e, where);
}

discos_status energy_args(discos_handle* h, const double* phi_b, Params* P) {
  if (h->P.strip) return invalid("the energy is not defined with a metal strip");
  if (h->P.bc[0] == DISCOS_BC_NEUMANN && h->P.bc[1] == DISCOS_BC_NEUMANN)
    return invalid("the energy needs at least one Dirichlet wall (two Neumann walls fix no potential)");
  *P = h->P;
  if (phi_b) {
    if (!std::isfinite(phi_b[0]) || !std::isfinite(phi_b[1])) return invalid("phi_b must be finite");
    P->phi_b[0] = phi_b[0];
    P->phi_b[1] = phi_b[1];
    P->f.phi_b[0] = (float)phi_b[0];
    P->f.phi_b[1] = (float)phi_b[1];
  }
  return DISCOS_OK;
}

// The library launches on the current device; the handle's workspace lives on
// the device that was current when it was created.
discos_status check_device(discos_handle* h) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
    return invalid("the current CUDA device is not the one the handle was created on");
  return DISCOS_OK;
}

discos_status check_n(discos_handle* h, int N) {
  if (!h) return invalid("null handle");
  if (N < 0 || N > h->cfg.max_ions) return invalid("N outside [0, max_ions]");
  return check_device(h);
}


}  // namespace
}  // namespace discos

using namespace discos;

extern "C" {

const char* discos_last_error(void) { return g_err.c_str(); }

long long discos_launch_count(void) { return g_launches.load(); }

discos_status discos_probe(discos_handle* h, int family) {
  if (!h) return invalid("null handle");
  if (family < -1 || family >= PROBE_COUNT) return invalid("unknown kernel family");
  Probe& p = h->probe;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e, "discos_probe");
  if (!p.created && family >= 0) {
    for (int i = 0; i < 2 * Probe::kMax; ++i) {
      e = cudaEventCreate(&p.ev[i]);
      if (e != cudaSuccess) return cuda_status(e, "discos_probe");
    }
    p.created = true;
  }
  p.family = family;
  p.n = 0;
  return DISCOS_OK;
}

discos_status discos_probe_read(discos_handle* h, double* total_ms, int* launches) {
  if (!h || !total_ms || !launches) return invalid("null argument");
  Probe& p = h->probe;
  double tot = 0.0;
  for (int i = 0; i < p.n; ++i) {
    cudaError_t e = cudaEventSynchronize(p.ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_status(e, "discos_probe_read");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_status(e, "discos_probe_read");
    tot += ms;
  }
  *total_ms = tot;
  *launches = p.n;
  return DISCOS_OK;
}

discos_status discos_create(const discos_config* cfg, discos_alloc_fn alloc_fn, discos_free_fn free_fn,
                            void* alloc_ctx, discos_handle** out) {
  if (!cfg || !out) return invalid("null argument");
  *out = nullptr;
  const discos_config& c = *cfg;
  if (!is_pow2(c.Nx) || c.Nx < 16 || c.Nx > 512) return invalid("Nx must be a power of two in [16, 512]");
  if (!is_pow2(c.Nz) || c.Nz < 16 || c.Nz > 512) return invalid("Nz must be a power of two in [16, 512]");
  if (c.Ny < 8 || c.Ny > 256) return invalid("Ny must be in [8, 256]");
  for (int w = 0; w < 2; ++w)
    if (c.bc[w] != DISCOS_BC_DIRICHLET && c.bc[w] != DISCOS_BC_NEUMANN) return invalid("bad wall type");
  int wes = kernel_width(c.kernel_es, c.es_w[0]);
  int why = kernel_width(c.kernel_hy, c.es_w[1]);
  if (wes < 4 || wes > 7 || why < 4 || why > 7) return invalid("kernel must be PESKIN4, PESKIN6 or ES with width 4..7");
  if (wes > c.Ny - 2 || why > c.Ny - 2) return invalid("kernel wider than the channel");
  if (c.hy_species != 0 && c.hy_species != 1) return invalid("hy_species must be 0 or 1");
  if (c.hy_species) {
    if (c.nspecies < 1 || c.nspecies > DISCOS_MAX_SPECIES) return invalid("nspecies must be 1..4");
    for (int a = 0; a < c.nspecies; ++a) {
      const int wa = kernel_width(c.kernel_hy_s[a], c.hy_w_s[a]);
      if (wa < 4 || wa > 7) return invalid("per-species kernel must be PESKIN4, PESKIN6 or ES with width 4..7");
      if (wa > c.Ny - 2) return invalid("per-species kernel wider than the channel");
      if (c.kernel_hy_s[a] == DISCOS_KERNEL_ES && !(c.hy_beta_s[a] > 0.0)) return invalid("ES kernel beta must be positive");
    }
  }
  if (!(c.psi > 0.0) || c.n_tab < 2) return invalid("psi > 0 and n_tab >= 2 required");
  if (c.nspecies < 1 || c.nspecies > DISCOS_MAX_SPECIES) return invalid("nspecies must be 1..4");
  if (c.max_refine < 0 || c.max_refine > DISCOS_MAX_REFINE) return invalid("max_refine must be 0..DISCOS_MAX_REFINE");
  if (c.max_ions < 1) return invalid("max_ions must be positive");
  if (c.precision != DISCOS_FP64 && c.precision != DISCOS_MIXED) return invalid("bad precision");
  if (!(c.dt > 0.0) || c.kT < 0.0) return invalid("dt > 0 and kT >= 0 required");
  if (c.wet && !(c.eta > 0.0)) return invalid("eta > 0 required for the wet path");
  if (c.wall_type != DISCOS_WALL_WCA && c.wall_type != DISCOS_WALL_LJ93) return invalid("bad wall_type");
  double rcmax = c.psi;
  for (int a = 0; a < c.nspecies; ++a) {
    if (!(c.D_tot[a] > c.D_wet[a]) || c.D_wet[a] < 0.0) return invalid("need D_tot > D_wet >= 0");
    for (int b = 0; b < c.nspecies; ++b) rcmax = std::max(rcmax, c.lj_rc[a][b]);
  }
  int k = (int)std::ceil(rcmax - 1e-12);
  if (k < 1) k = 1;
  if (c.Nx / k < 3 || c.Nz / k < 3) return invalid("cutoff too large for the box (need 3 list cells per periodic axis)");
  if (2.0 * c.psi > std::min(c.Nx, c.Nz)) return invalid("psi must be at most half the periodic box");
  for (int w = 0; w < 2; ++w)
    if (c.bc_hy[w] != DISCOS_HY_NOSLIP && c.bc_hy[w] != DISCOS_HY_SLIP) return invalid("bad bc_hy");
  if (c.bc_hy[0] == DISCOS_HY_SLIP && c.bc_hy[1] == DISCOS_HY_SLIP)
    return invalid("at most one slip wall (two leave uniform flow along the walls undamped)");
  int strip_i0 = 0, strip_i1 = 0;
  if (c.strip) {
    if (c.bc[0] != DISCOS_BC_NEUMANN) return invalid("the metal strip sits in a dielectric (NEUMANN) bottom wall");
    if (!std::isfinite(c.strip_x[0]) || !std::isfinite(c.strip_x[1]) || !std::isfinite(c.strip_phi))
      return invalid("strip_x and strip_phi must be finite");
    strip_i0 = std::max(0, (int)std::ceil(c.strip_x[0] - 0.5));
    strip_i1 = std::min(c.Nx, (int)std::ceil(c.strip_x[1] - 0.5));
    if (strip_i1 <= strip_i0) return invalid("the metal strip covers no cell column");
    if (strip_i1 - strip_i0 > 128) return invalid("the metal strip is at most 128 cell columns wide");
    if (c.max_refine > 0) return invalid("residual refinement is not available with a metal strip");
  }

  discos_handle* h = new discos_handle();
  h->cfg = c;
  h->mixed = c.precision == DISCOS_MIXED;
  h->alloc_fn = alloc_fn;
  h->free_fn = free_fn;
  h->alloc_ctx = alloc_ctx;
  cudaGetDevice(&h->device);

  Params& P = h->P;
  std::memset(&P, 0, sizeof(P));
  P.Nx = c.Nx; P.Ny = c.Ny; P.Nz = c.Nz;
  P.Nxh = c.Nx / 2 + 1;
  P.Px = (P.Nxh + 15) / 16 * 16;
  for (int w = 0; w < 2; ++w) { P.bc[w] = c.bc[w]; P.phi_b[w] = c.phi_b[w]; }
  // dphi/dy on the walls: -eps dphi/dn = varsigma with n the inward normal
  P.slope[0] = -4.0 * M_PI * c.lB * c.surf_charge[0];
  P.slope[1] = 4.0 * M_PI * c.lB * c.surf_charge[1];
  P.kes = make_kernel(c.kernel_es, c.es_w[0], c.es_beta[0]);
  P.khy = make_kernel(c.kernel_hy, c.es_w[1], c.es_beta[1]);
  P.hy_species = c.hy_species;
  P.hy_filter = -1;
  if (c.hy_species)
    for (int a = 0; a < c.nspecies; ++a) P.khy_s[a] = make_kernel(c.kernel_hy_s[a], c.hy_w_s[a], c.hy_beta_s[a]);
  P.lB = c.lB; P.eta = c.eta; P.kT = c.kT; P.dt = c.dt; P.psi = c.psi;
  P.n_tab = c.n_tab;
  P.tab_scale = c.n_tab / c.psi;
  P.nspecies = c.nspecies;
  for (int a = 0; a < DISCOS_MAX_SPECIES; ++a) {
    P.D_tot[a] = c.D_tot[a];
    P.D_wet[a] = c.D_wet[a];
    P.D_dry[a] = c.D_tot[a] - c.D_wet[a];
    std::memcpy(P.gamma[a], c.gamma_coef[a], sizeof(P.gamma[a]));
    for (int b = 0; b < DISCOS_MAX_SPECIES; ++b) {
      P.lj_sigma[a][b] = c.lj_sigma[a][b];
      P.lj_xi[a][b] = c.lj_xi[a][b];
      P.lj_rc[a][b] = c.lj_rc[a][b];
    }
    P.wall_sigma[a] = c.wall_sigma[a];
    P.wall_xi[a] = c.wall_xi[a];
    P.wall_rc[a] = c.wall_rc[a];
  }
  P.wall_type = c.wall_type;
  for (int d = 0; d < 3; ++d) P.E_ext[d] = c.E_ext[d];
  P.inv_kT = 1.0 / c.kT;
  P.max_refine = c.precision == DISCOS_MIXED ? c.max_refine : 0;
  {
    const size_t elem = c.precision == DISCOS_MIXED ? 2 * sizeof(float) : 2 * sizeof(double);
    P.fx_pp = default_fx_pairs(c.Nx);
    P.fx_threads = 256;
    P.fx_staged = c.Nx >= 32 ? 1 : 0;
    P.fz_tma = (c.precision == DISCOS_MIXED && c.Nz <= 256) ? 1 : 0;
    P.fz_tk = default_tile_z(c.Nz, elem);
  }
  {
    PhysF& f = P.f;
    for (int a = 0; a < DISCOS_MAX_SPECIES; ++a) {
      P.inv_D_dry[a] = P.D_dry[a] != 0.0 ? 1.0 / P.D_dry[a] : 0.0;
      f.D_tot[a] = (float)P.D_tot[a];
      f.D_wet[a] = (float)P.D_wet[a];
      f.D_dry[a] = (float)P.D_dry[a];
      f.inv_D_dry[a] = (float)P.inv_D_dry[a];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int k = 0; k < 7; ++k) f.gamma[a][i][j][k] = (float)P.gamma[a][i][j][k];
      for (int b = 0; b < DISCOS_MAX_SPECIES; ++b) {
        f.lj_sigma[a][b] = (float)P.lj_sigma[a][b];
        f.lj_xi[a][b] = (float)P.lj_xi[a][b];
        f.lj_rc[a][b] = (float)P.lj_rc[a][b];
      }
      f.wall_sigma[a] = (float)P.wall_sigma[a];
      f.wall_xi[a] = (float)P.wall_xi[a];
      f.wall_rc[a] = (float)P.wall_rc[a];
    }
    for (int d = 0; d < 3; ++d) f.E_ext[d] = (float)P.E_ext[d];
    for (int w = 0; w < 2; ++w) {
      f.slope[w] = (float)P.slope[w];
      f.phi_b[w] = (float)P.phi_b[w];
    }
    f.dt = (float)P.dt;
    f.kT = (float)P.kT;
    f.inv_kT = (float)P.inv_kT;
    f.lB = (float)P.lB;
    f.psi = (float)P.psi;
    f.tab_scale = (float)P.tab_scale;
    P.inv_eta = P.eta > 0.0 ? 1.0 / P.eta : 0.0;
    P.inv_nxnz = 1.0 / ((double)c.Nx * c.Nz);
    f.eta = (float)P.eta;
    f.inv_eta = (float)P.inv_eta;
    f.inv_nxnz = (float)P.inv_nxnz;
  }
  P.k_cell = k;
  P.ncx = c.Nx / k; P.ncy = std::max(1, c.Ny / k); P.ncz = c.Nz / k;
  if (c.strip) {
    P.strip = 1;
    P.strip_i0 = strip_i0;
    P.strip_i1 = strip_i1;
    P.strip_singular = c.bc[1] == DISCOS_BC_NEUMANN ? 1 : 0;
    P.strip_phi = c.strip_phi;
    P.strip_xc = 0.5 * (c.strip_x[0] + c.strip_x[1]);
    P.f.strip_phi = (float)P.strip_phi;
    P.f.strip_xc = (float)P.strip_xc;
  }
  P.drift = c.drift;
  P.seed = c.seed;
  P.slip[0] = c.bc_hy[0] == DISCOS_HY_SLIP ? 1 : 0;
  P.slip[1] = c.bc_hy[1] == DISCOS_HY_SLIP ? 1 : 0;

  // workspace
  const size_t rs = h->mixed ? sizeof(float) : sizeof(double);
  const size_t G = (size_t)c.Nx * c.Ny * c.Nz;
  const size_t Gf = (size_t)c.Nx * c.Nz * (3 * c.Ny + 1);
  const size_t specslot = (size_t)c.Nz * (c.Ny + 1) * P.Px;
  const size_t modes = (size_t)P.Nxh * c.Nz;
  const int n_cells = P.ncx * P.ncy * P.ncz;
  const size_t M = (size_t)c.max_ions;
  Workspace& W = h->W;
  W.n_cells = n_cells;
  bool ok = true;
  W.phi = dalloc(h, rs * G, &ok);
  W.spec = dalloc(h, 2 * rs * 4 * specslot, &ok);
  W.fgrid = dalloc(h, rs * Gf, &ok);
  W.piv64 = (double*)dalloc(h, sizeof(double) * modes * c.Ny, &ok);
  W.tw_x = dalloc(h, 2 * rs * (c.Nx / 2), &ok);
  W.tw_z = dalloc(h, 2 * rs * (c.Nz / 2), &ok);
  W.fptab = dalloc(h, rs * (c.n_tab + 1), &ok);
  W.cell_of = (int*)dalloc(h, sizeof(int) * M, &ok);
  W.counts = (int*)dalloc(h, sizeof(int) * n_cells, &ok);
  W.fill = (int*)dalloc(h, sizeof(int) * n_cells, &ok);
  W.cell_start = (int*)dalloc(h, sizeof(int) * (n_cells + 1), &ok);
  W.perm = (int*)dalloc(h, sizeof(int) * M, &ok);
  W.tile_sums = (int*)dalloc(h, sizeof(int) * ((n_cells + 1023) / 1024 + 1), &ok);
  W.xs = dalloc(h, rs * 3 * M, &ok);
  W.qs = dalloc(h, rs * M, &ok);
  W.sps = (int*)dalloc(h, sizeof(int) * M, &ok);
  W.xq = dalloc(h, (h->mixed ? 16 : 32) * M, &ok);
  W.F = dalloc(h, rs * 3 * M, &ok);
  W.xstar = dalloc(h, rs * 3 * M, &ok);
  W.V = dalloc(h, rs * 3 * M, &ok);
  W.Fn = dalloc(h, rs * 3 * M, &ok);
  W.edata = (double*)dalloc(h, sizeof(double) * (3 * (size_t)c.Ny + 4), &ok);
  W.fault = (unsigned*)dalloc(h, sizeof(unsigned), &ok);
  W.diag = (double*)dalloc(h, 8 * sizeof(double), &ok);
  W.nsum = (double*)dalloc(h, 4 * sizeof(double), &ok);
  if (h->mixed && c.max_refine > 0) {
    W.rref = dalloc(h, rs * G, &ok);
    W.rres = dalloc(h, rs * G, &ok);
    W.rnorm = (double*)dalloc(h, sizeof(double) * 2 * (DISCOS_MAX_REFINE + 1), &ok);
    W.phi64 = (double*)dalloc(h, sizeof(double) * G, &ok);
    if (c.wet) {
      W.sref = dalloc(h, rs * Gf, &ok);
      W.sres = dalloc(h, rs * Gf, &ok);
      W.pres = dalloc(h, rs * G, &ok);
      W.v64 = (double*)dalloc(h, sizeof(double) * Gf, &ok);
      W.p64 = (double*)dalloc(h, sizeof(double) * G, &ok);
      W.snorm = (double*)dalloc(h, sizeof(double) * 2 * (DISCOS_MAX_REFINE + 1), &ok);
    }
  }
  if (h->mixed) {
    W.is_lo = (unsigned char*)dalloc(h, modes, &ok);
    W.lo_modes = (int*)dalloc(h, sizeof(int) * modes, &ok);
    W.piv32 = (float*)dalloc(h, sizeof(float) * modes * c.Ny, &ok);
    W.piv32t = (float*)dalloc(h, sizeof(float) * modes * c.Ny, &ok);
    if (c.wet) {
      W.st_l1f = (float*)dalloc(h, sizeof(float) * c.Ny * modes, &ok);
      W.st_l2f = (float*)dalloc(h, sizeof(float) * c.Ny * modes, &ok);
      W.st_dif = (float*)dalloc(h, sizeof(float) * c.Ny * modes, &ok);
      W.st_cif = (float*)dalloc(h, sizeof(float) * c.Ny * modes, &ok);
      W.st_mcf = (float*)dalloc(h, sizeof(float) * 5 * modes, &ok);
    }
  }
  if (c.wet) {
    W.st_l1 = (double*)dalloc(h, sizeof(double) * c.Ny * modes, &ok);
    W.st_l2 = (double*)dalloc(h, sizeof(double) * c.Ny * modes, &ok);
    W.st_di = (double*)dalloc(h, sizeof(double) * c.Ny * modes, &ok);
    W.st_ci = (double*)dalloc(h, sizeof(double) * c.Ny * modes, &ok);
    W.st_mc = (double*)dalloc(h, sizeof(double) * 5 * modes, &ok);
  }
  std::vector<double> strip_add0, strip_M;
  if (c.strip) {
    const int Ws = P.strip_i1 - P.strip_i0;
    W.strip_g = dalloc(h, rs * G, &ok);
    W.strip_add0 = dalloc(h, rs * c.Nx, &ok);
    W.strip_r = (double*)dalloc(h, sizeof(double) * c.Nz * Ws, &ok);
    W.strip_shat = (double*)dalloc(h, 2 * sizeof(double) * c.Nz * Ws, &ok);
    W.strip_M = (double*)dalloc(h, sizeof(double) * c.Nz * (Ws + 1) * (Ws + 1), &ok);
    W.strip_c = (double*)dalloc(h, sizeof(double), &ok);
  }
  if (!ok) {
    free_workspace(h);
    delete h;
    set_error("device allocation failed");
    return DISCOS_ERR_OOM;
  }
  if (c.strip) {
    setup_strip(h, strip_add0, strip_M);
    if (h->mixed) upload_table<float>(W.strip_add0, strip_add0);
    else upload_table<double>(W.strip_add0, strip_add0);
    cudaMemcpy(W.strip_M, strip_M.data(), sizeof(double) * strip_M.size(), cudaMemcpyHostToDevice);
    cudaMemset(W.strip_c, 0, sizeof(double));
  }
  // Thomas pivots of the Poisson wall-normal systems, one set per (kx, kz), [M][Ny]
  {
    std::vector<double> inv((size_t)c.Ny * modes);
    for (int kz = 0; kz < c.Nz; ++kz)
      for (int kx = 0; kx < P.Nxh; ++kx) {
        double lam = (2.0 - 2.0 * std::cos(2.0 * M_PI * kx / c.Nx)) + (2.0 - 2.0 * std::cos(2.0 * M_PI * kz / c.Nz));
        size_t mode = (size_t)kz * P.Nxh + kx;
        double m = 0.0;
        for (int j = 0; j < c.Ny; ++j) {
          double d = 2.0 + lam;
          if (j == 0) d += c.bc[0] == DISCOS_BC_DIRICHLET ? 1.0 : -1.0;
          if (j == c.Ny - 1) d += c.bc[1] == DISCOS_BC_DIRICHLET ? 1.0 : -1.0;
          m = j == 0 ? d : d - 1.0 / m;
          inv[mode * c.Ny + j] = m != 0.0 ? 1.0 / m : 0.0;
        }
      }
    cudaMemcpy(W.piv64, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice);
    if (h->mixed) {
      // modes solved in double: K^2 = lambda_x + lambda_z < 0.5 (see k_ysolve.cu)
      std::vector<unsigned char> lo(modes, 0);
      std::vector<int> list;
      for (int kz = 0; kz < c.Nz; ++kz)
        for (int kx = 0; kx < P.Nxh; ++kx) {
          double K2 = (2.0 - 2.0 * std::cos(2.0 * M_PI * kx / c.Nx)) + (2.0 - 2.0 * std::cos(2.0 * M_PI * kz / c.Nz));
          if (K2 < 0.5) {
            size_t m = (size_t)kz * P.Nxh + kx;
            lo[m] = 1;
            list.push_back((int)m);
          }
        }
      W.n_lo = (int)list.size();
      std::vector<float> inv32(inv.begin(), inv.end());
      // the single-precision sweeps read the pivots row by row across modes: [Ny][M]
      std::vector<float> inv32t(inv.size());
      for (size_t m = 0; m < modes; ++m)
        for (int j = 0; j < c.Ny; ++j) inv32t[(size_t)j * modes + m] = (float)inv[m * c.Ny + j];
      cudaMemcpy(W.piv32t, inv32t.data(), sizeof(float) * inv32t.size(), cudaMemcpyHostToDevice);
      cudaMemcpy(W.is_lo, lo.data(), lo.size(), cudaMemcpyHostToDevice);
      if (!list.empty()) cudaMemcpy(W.lo_modes, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice);
      cudaMemcpy(W.piv32, inv32.data(), sizeof(float) * inv32.size(), cudaMemcpyHostToDevice);
    }
  }
  h->P.fault = W.fault;
  cudaMemset(W.fault, 0, sizeof(unsigned));
  if (c.wet) upload_stokes_factors(h);
  cudaMemset(W.fgrid, 0, rs * Gf);   // the wall rows of f_y stay zero from here on
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&W.ystream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&W.yev0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&W.yev1, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_extra, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fault, cudaEventDisableTiming) != cudaSuccess ||
      cudaHostAlloc((void**)&h->fault_host, sizeof(unsigned), cudaHostAllocDefault) != cudaSuccess) {
    free_workspace(h);
    delete h;
    set_error("stream or event creation failed");
    return DISCOS_ERR_CUDA;
  }
  *h->fault_host = 0u;     // pinned memory comes back uninitialised
  std::vector<double> tab = cached_fp_table(P.kes, c.psi, c.n_tab);
  if (h->mixed) {
    upload_twiddles<float>(W.tw_x, c.Nx);
    upload_twiddles<float>(W.tw_z, c.Nz);
    upload_table<float>(W.fptab, tab);
  } else {
    upload_twiddles<double>(W.tw_x, c.Nx);
    upload_twiddles<double>(W.tw_z, c.Nz);
    upload_table<double>(W.fptab, tab);
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_workspace(h);
    delete h;
    return cuda_status(e, "discos_create");
  }
  *out = h;
  return DISCOS_OK;
}

discos_status discos_destroy(discos_handle* h) {
  if (!h) return invalid("null handle");
  cudaDeviceSynchronize();
  if (h->W.ystream) cudaStreamDestroy(h->W.ystream);
  if (h->W.yev0) cudaEventDestroy(h->W.yev0);
  if (h->W.yev1) cudaEventDestroy(h->W.yev1);
  free_workspace(h);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->probe.created)
    for (int i = 0; i < 2 * Probe::kMax; ++i) cudaEventDestroy(h->probe.ev[i]);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_extra) cudaEventDestroy(h->ev_extra);
  if (h->ev_fault) cudaEventDestroy(h->ev_fault);
  if (h->fault_host) cudaFreeHost(h->fault_host);
  delete h;
  return DISCOS_OK;
}

discos_status discos_spread(discos_handle* h, const void* x, const void* val, int N, int which, void* grid,
                            void* stream) {
  return discos_spread_species(h, x, val, nullptr, N, which, grid, stream);
}

discos_status discos_spread_species(discos_handle* h, const void* x, const void* val, const int* species, int N,
                                    int which, void* grid, void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (!grid || (N > 0 && (!x || !val))) return invalid("null pointer");
  if (which != DISCOS_SPREAD_CHARGE && which != DISCOS_SPREAD_FORCE)
    return invalid("which must be DISCOS_SPREAD_CHARGE or DISCOS_SPREAD_FORCE");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = h->mixed
      ? spread_impl<float>(h, (const float*)x, (const float*)val, species, N, which, (float*)grid, s)
      : spread_impl<double>(h, (const double*)x, (const double*)val, species, N, which, (double*)grid, s);
  return cuda_status(e, "discos_spread");
}

discos_status discos_solve_poisson(discos_handle* h, const void* rho, void* phi, void* stream) {
  ProbeScope probe_scope(h);
  if (!h) return invalid("null handle");
  if (!rho || !phi) return invalid("null pointer");
  discos_status st = check_device(h);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t G = (size_t)h->P.Nx * h->P.Ny * h->P.Nz;
  st = h->mixed ? check_neutral_sync<float>(h, (const float*)rho, G, s, "discos_solve_poisson")
                : check_neutral_sync<double>(h, (const double*)rho, G, s, "discos_solve_poisson");
  if (st) return st;
  cudaError_t e = h->mixed ? launch_poisson<float>(h->P, h->W, (const float*)rho, (float*)phi, s)
                           : launch_poisson<double>(h->P, h->W, (const double*)rho, (double*)phi, s);
  return cuda_status(e, "discos_solve_poisson");
}

discos_status discos_solve_stokes(discos_handle* h, const void* f, void* v, void* p, void* stream) {
  ProbeScope probe_scope(h);
  if (!h) return invalid("null handle");
  if (!f || !v) return invalid("null pointer");
  if (!(h->P.eta > 0.0)) return invalid("eta must be positive");
  if (!h->cfg.wet) return invalid("the handle was created without the hydrodynamic stage (wet = 0)");
  if (discos_status st = check_device(h)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = h->mixed ? launch_stokes<float>(h->P, h->W, (const float*)f, (float*)v, (float*)p, s)
                           : launch_stokes<double>(h->P, h->W, (const double*)f, (double*)v, (double*)p, s);
  return cuda_status(e, "discos_solve_stokes");
}

discos_status discos_interpolate(discos_handle* h, const void* x, int N, int which, const void* grid, void* out,
                                 void* stream) {
  return discos_interpolate_species(h, x, nullptr, N, which, grid, out, stream);
}

discos_status discos_interpolate_species(discos_handle* h, const void* x, const int* species, int N, int which,
                                         const void* grid, void* out, void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (!grid || (N > 0 && (!x || !out))) return invalid("null pointer");
  if (which != DISCOS_INTERP_EFIELD && which != DISCOS_INTERP_VELOCITY)
    return invalid("which must be DISCOS_INTERP_EFIELD or DISCOS_INTERP_VELOCITY");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = h->mixed
      ? interp_impl<float>(h, (const float*)x, species, N, which, (const float*)grid, (float*)out, s)
      : interp_impl<double>(h, (const double*)x, species, N, which, (const double*)grid, (double*)out, s);
  return cuda_status(e, "discos_interpolate");
}

discos_status discos_cell_list(discos_handle* h, const void* x, int N, int* cell_start, int* perm, int* n_cells_out,
                               void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (N > 0 && !x) return invalid("null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  if (n_cells_out) *n_cells_out = h->W.n_cells;
  cudaError_t e = h->mixed ? launch_cell_list<float>(h->P, h->W, (const float*)x, N, s)
                           : launch_cell_list<double>(h->P, h->W, (const double*)x, N, s);
  if (e == cudaSuccess && cell_start)
    e = cudaMemcpyAsync(cell_start, h->W.cell_start, sizeof(int) * (h->W.n_cells + 1), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && perm && N > 0)
    e = cudaMemcpyAsync(perm, h->W.perm, sizeof(int) * N, cudaMemcpyDeviceToDevice, s);
  return cuda_status(e, "discos_cell_list");
}

discos_status discos_near_field(discos_handle* h, const void* x, const void* q, const int* species, int N, void* F,
                                int* nbr_count, void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (N > 0 && (!x || !q || !F)) return invalid("null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = h->mixed
      ? launch_near_field<float>(h->P, h->W, (const float*)x, (const float*)q, species, N, (float*)F, nbr_count, s)
      : launch_near_field<double>(h->P, h->W, (const double*)x, (const double*)q, species, N, (double*)F, nbr_count, s);
  return cuda_status(e, "discos_near_field");
}

discos_status discos_forces(discos_handle* h, const void* x, const void* q, const int* species, int N, void* F,
                            int* nbr_count, void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (N > 0 && (!x || !q || !F)) return invalid("null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  st = h->mixed ? check_neutral_sync<float>(h, (const float*)q, (size_t)N, s, "discos_forces")
                : check_neutral_sync<double>(h, (const double*)q, (size_t)N, s, "discos_forces");
  if (st) return st;
  return h->mixed ? forces_impl<float>(h, (const float*)x, (const float*)q, species, N, (float*)F, nbr_count, s)
                  : forces_impl<double>(h, (const double*)x, (const double*)q, species, N, (double*)F, nbr_count, s);
}

discos_status discos_step(discos_handle* h, void* x, const void* q, const int* species, int N, int64_t step0,
                          int nsteps, void* F_out, void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (nsteps < 0) return invalid("nsteps must be >= 0");
  if (N > 0 && (!x || !q)) return invalid("null pointer");
  if (cudaEventQuery(h->ev_fault) == cudaSuccess && *h->fault_host) {
    if (*h->fault_host & 4u) {
      set_error("a previous step found the channel between two Neumann walls not neutral (fault word bit 2)");
      return DISCOS_ERR_NOT_NEUTRAL;
    }
    set_error(std::string("a previous step flagged the device fault word (") + std::to_string(*h->fault_host) +
              "): bit 0 non-finite position, bit 1 ion outside the channel; see discos_fault");
    return DISCOS_ERR_DEVICE_FAULT;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return h->mixed ? step_impl<float>(h, (float*)x, (const float*)q, species, N, step0, nsteps, (float*)F_out, s)
                  : step_impl<double>(h, (double*)x, (const double*)q, species, N, step0, nsteps, (double*)F_out, s);
}

discos_status discos_energy(discos_handle* h, const void* x, const void* q, int N, const double* phi_b, double* U,
                            void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (!U || (N > 0 && (!x || !q))) return invalid("null pointer");
  Params P;
  if ((st = energy_args(h, phi_b, &P))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return h->mixed ? energy_impl<float>(h, P, (const float*)x, (const float*)q, N, U, nullptr, nullptr, nullptr,
                                       nullptr, s)
                  : energy_impl<double>(h, P, (const double*)x, (const double*)q, N, U, nullptr, nullptr, nullptr,
                                        nullptr, s);
}

discos_status discos_energy_backward(discos_handle* h, const void* x, const void* q, int N, const double* phi_b,
                                     const double* dU, void* dx, void* dq, double* dphi_b, void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (!dU || (N > 0 && (!x || !q))) return invalid("null pointer");
  Params P;
  if ((st = energy_args(h, phi_b, &P))) return st;
  if (N == 0) { dx = nullptr; dq = nullptr; }
  cudaStream_t s = (cudaStream_t)stream;
  return h->mixed ? energy_impl<float>(h, P, (const float*)x, (const float*)q, N, nullptr, dU, (float*)dx,
                                       (float*)dq, dphi_b, s)
                  : energy_impl<double>(h, P, (const double*)x, (const double*)q, N, nullptr, dU, (double*)dx,
                                        (double*)dq, dphi_b, s);
}

static discos_status refine_history(discos_handle* h, const double* norms, double* rel, int* n, void* stream) {
  if (!h || !rel || !n) return invalid("null pointer");
  *n = 0;
  if (!norms) return DISCOS_OK;
  const int m = h->P.max_refine + 1;
  double buf[2 * (DISCOS_MAX_REFINE + 1)];
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(buf, norms, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "discos_refine_history");
  for (int i = 0; i < m; ++i) rel[i] = buf[2 * i + 1] > 0.0 ? std::sqrt(buf[2 * i] / buf[2 * i + 1]) : 0.0;
  *n = m;
  return DISCOS_OK;
}

discos_status discos_refine_history(discos_handle* h, double* rel, int* n, void* stream) {
  return refine_history(h, h ? h->W.rnorm : nullptr, rel, n, stream);
}

discos_status discos_refine_history_stokes(discos_handle* h, double* rel, int* n, void* stream) {
  return refine_history(h, h ? h->W.snorm : nullptr, rel, n, stream);
}

discos_status discos_fault(discos_handle* h, int sync, int clear, unsigned* word, void* stream) {
  if (!h || !word) return invalid("null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (sync) {
    e = cudaMemcpyAsync(h->fault_host, h->W.fault, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_fault, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(h->ev_fault);
    if (e != cudaSuccess) return cuda_status(e, "discos_fault");
  }
  *word = cudaEventQuery(h->ev_fault) == cudaSuccess ? *h->fault_host : 0u;
  if (clear) {
    e = cudaMemsetAsync(h->W.fault, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "discos_fault");
    *h->fault_host = 0u;
  }
  return DISCOS_OK;
}

discos_status discos_diagnostics(discos_handle* h, const void* x, const void* q, const void* F, int N, int with_rho,
                                 double* out, void* stream) {
  ProbeScope probe_scope(h);
  discos_status st = check_n(h, N);
  if (st) return st;
  if (!out || (N > 0 && (!x || !q))) return invalid("null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (h->mixed) {
    float* rho = with_rho ? reinterpret_cast<float*>(h->W.fgrid) : nullptr;
    if (rho) e = launch_spread_charge<float>(h->P, (const float*)x, (const float*)q, N, rho, s);
    if (e == cudaSuccess)
      e = launch_diagnostics<float>(h->P, (const float*)x, (const float*)q, (const float*)F, N, rho, out, s);
  } else {
    double* rho = with_rho ? reinterpret_cast<double*>(h->W.fgrid) : nullptr;
    if (rho) e = launch_spread_charge<double>(h->P, (const double*)x, (const double*)q, N, rho, s);
    if (e == cudaSuccess)
      e = launch_diagnostics<double>(h->P, (const double*)x, (const double*)q, (const double*)F, N, rho, out, s);
  }
  return cuda_status(e, "discos_diagnostics");
}

discos_status discos_tune_transforms(discos_handle* h, int* fx_pairs, int* fx_threads, int* fz_tile,
                                     float* ms, void* stream) {
  if (!h) return invalid("null handle");
  float best[2] = {0.f, 0.f};
  cudaError_t e = tune_transforms(h->P, h->W, h->mixed, (cudaStream_t)stream, best);
  if (e != cudaSuccess) return cuda_status(e, "discos_tune_transforms");
  if (fx_pairs) *fx_pairs = h->P.fx_staged ? 0 : h->P.fx_pp;
  if (fx_threads) *fx_threads = h->P.fx_threads;
  if (fz_tile) *fz_tile = h->P.fz_tma ? 0 : h->P.fz_tk;
  if (ms) { ms[0] = best[0]; ms[1] = best[1]; }
  return DISCOS_OK;
}

discos_status discos_set_transform_shape(discos_handle* h, int fx_pairs, int fx_threads, int fz_tile) {
  if (!h) return invalid("null handle");
  const size_t elem = h->mixed ? 2 * sizeof(float) : 2 * sizeof(double);
  const int N = h->P.Nx;
  if (fz_tile == 0) {
    if (!h->mixed || h->P.Nz > 256) return invalid("the tiled z transform (fz_tile = 0) needs MIXED and Nz <= 256");
  } else if (fz_tile < 1 || (fz_tile & (fz_tile - 1)) || fz_tile > max_tile_z(h->P.Nz, elem)) {
    return invalid("fz_tile: 0 or a power of two up to the shared-memory limit");
  }
  if (fx_pairs == 0) {
    if (N < 32) return invalid("the staged x transform (fx_pairs = 0) needs Nx >= 32");
  } else {
    if (fx_pairs < 1 || (size_t)fx_pairs * N > 2048 ||
        (2 * (size_t)fx_pairs * N + N / 2) * elem + 2 * (size_t)fx_pairs * elem > 48 * 1024)
      return invalid("fx_pairs: 0, or 1 .. 2048 / Nx row pairs within 48 KB of shared memory");
    if (fx_threads < 32 || fx_threads > 1024 || fx_threads % 32)
      return invalid("fx_threads: a multiple of 32 in 32..1024");
    h->P.fx_pp = fx_pairs;
    h->P.fx_threads = fx_threads;
  }
  h->P.fx_staged = fx_pairs == 0 ? 1 : 0;
  h->P.fz_tma = fz_tile == 0 ? 1 : 0;
  if (fz_tile > 0) h->P.fz_tk = fz_tile;
  return DISCOS_OK;
}

}  // extern "C"
