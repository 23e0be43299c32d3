// Internal declarations shared by the libdiscos translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include "../../include/discos.h"
#include "common.cuh"

namespace discos {

// Single-precision copies of the physics constants: float kernels read these
// (through phys()), so that they convert nothing from double at run time --
// on this GPU a conversion from double runs on the slow double pipe.
struct PhysF {
  float D_tot[DISCOS_MAX_SPECIES], D_wet[DISCOS_MAX_SPECIES], D_dry[DISCOS_MAX_SPECIES];
  float inv_D_dry[DISCOS_MAX_SPECIES];
  float gamma[DISCOS_MAX_SPECIES][2][2][7];
  float lj_sigma[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];
  float lj_xi[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];
  float lj_rc[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];
  float wall_sigma[DISCOS_MAX_SPECIES], wall_xi[DISCOS_MAX_SPECIES], wall_rc[DISCOS_MAX_SPECIES];
  float E_ext[3], slope[2], phi_b[2];
  float dt, kT, inv_kT, lB, psi, tab_scale;
  float eta, inv_eta, inv_nxnz;
  float strip_phi, strip_xc;
};

// Everything a kernel needs to know about the run, passed by value.
struct Params {
  int Nx, Ny, Nz;
  int Nxh, Px;                 // Nx/2 + 1 x-modes, padded row pitch of spectra
  int bc[2];
  double phi_b[2];
  double slope[2];             // dphi/dy on Neumann walls (bottom, top)
  KernelParams kes, khy;
  // hydrodynamic kernel per species (App. B): with hy_species, S^hy and J^hy run once per species s with
  // khy = khy_s[s] and hy_filter = s (ions of other species skipped); hy_filter < 0 takes every ion
  int hy_species, hy_filter;
  KernelParams khy_s[DISCOS_MAX_SPECIES];
  double lB, eta, kT, dt, psi;
  int n_tab;
  double tab_scale;            // n_tab / psi
  int nspecies;
  double D_dry[DISCOS_MAX_SPECIES], D_tot[DISCOS_MAX_SPECIES], D_wet[DISCOS_MAX_SPECIES];
  double gamma[DISCOS_MAX_SPECIES][2][2][7];
  double lj_sigma[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];
  double lj_xi[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];
  double lj_rc[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];
  int wall_type;
  double wall_sigma[DISCOS_MAX_SPECIES], wall_xi[DISCOS_MAX_SPECIES], wall_rc[DISCOS_MAX_SPECIES];
  double E_ext[3];
  int k_cell, ncx, ncy, ncz;
  int drift;
  uint64_t seed;
  int max_refine;              // residual refinement sweeps of the mixed Poisson solve
  int fx_pp, fx_threads, fz_tk;  // transform launch shapes (k_fft.cu; discos_tune_transforms)
  int fx_staged;               // 1: bulk-staged persistent x transforms (fx_pp, fx_threads unused)
  int fz_tma;                  // 1: TMA-tiled z transforms (single precision, 16 <= Nz <= 256; fz_tk unused)
  // metal strip in the bottom wall (k_strip.cu): Dirichlet on the cell columns [strip_i0, strip_i1) with
  // phi_m(x) = strip_phi + E_ext[0] (x - strip_xc); strip_singular: the all-dielectric base operator is
  // singular (top wall Neumann); strip_walls: the sum of the base solve's wall terms over the grid
  int strip, strip_i0, strip_i1, strip_singular;
  int slip[2];                 // hydrodynamic slip walls (bottom, top): tangential images and ghosts +1, else -1
  double strip_phi, strip_xc, strip_walls;
  unsigned* fault;             // device fault word: bit 0 non-finite position, bit 1 escaped ion,
                               // bit 2 a non-neutral channel between two Neumann walls,
                               // bit 3 a bounded wait on a bulk copy ran out (bulk.cuh)
  double inv_D_dry[DISCOS_MAX_SPECIES], inv_kT;
  double inv_eta, inv_nxnz;    // 1 / eta (0 without a fluid), 1 / (Nx Nz): the transforms' normalisation
  PhysF f;
};

// Whether the bottom-wall cell column ix (0 <= ix < Nx) lies on the metal strip.
__host__ __device__ __forceinline__ bool on_strip(const Params& P, int ix) {
  return P.strip && ix >= P.strip_i0 && ix < P.strip_i1;
}

// The physics constants in the arithmetic type of the caller.
__host__ __device__ __forceinline__ const Params& phys(const Params& P, double) { return P; }
__host__ __device__ __forceinline__ const PhysF& phys(const Params& P, float) { return P.f; }

// The metal strip's potential phi_m at cell column ix (centre ix + 1/2).
template <typename T>
__host__ __device__ __forceinline__ T strip_phi_m(const Params& P, int ix, T) {
  const auto& Q = phys(P, T());
  return T(Q.strip_phi) + T(Q.E_ext[0]) * (T(ix) + T(0.5) - T(Q.strip_xc));
}

// Kernel families that can be timed live (discos_probe).
enum ProbeFamily {
  PROBE_NONE = -1, PROBE_CELL_LIST = 0, PROBE_NEAR_FIELD, PROBE_NOISE, PROBE_SPREAD_CHARGE, PROBE_FFT_X,
  PROBE_FFT_Z, PROBE_POISSON_Y, PROBE_INTERP_E, PROBE_SPREAD_FORCE, PROBE_STOKES_Y, PROBE_INTERP_V,
  PROBE_UPDATE, PROBE_COUNT
};

// CUDA events recorded around every launch of one kernel family.
struct Probe {
  int family = PROBE_NONE;
  static const int kMax = 4096;
  cudaEvent_t ev[2 * kMax];
  int n = 0;
  bool created = false;
};
void probe_begin(int family, cudaStream_t s);
void probe_end(int family, cudaStream_t s);

// Device workspace owned by a handle.
struct Workspace {
  // grids
  void* phi = nullptr;         // [Nz][Ny][Nx] real: rho, then phi
  void* spec = nullptr;        // 3 spectra [Nz][Ny+1][Px] complex real
  void* fgrid = nullptr;       // fx|fy|fz real
  double* piv64 = nullptr;     // Poisson Thomas reciprocal pivots [M][Ny]
  float* piv32 = nullptr;      // single-precision copy (mixed path; the batched replicas)
  float* piv32t = nullptr;     // single-precision copy [Ny][M] (mixed path; the sweeps of k_ysolve.cu)
  void* tw_x = nullptr;        // twiddles exp(-2 pi i k / Nx), k < Nx/2
  void* tw_z = nullptr;        // twiddles exp(-2 pi i k / Nz), k < Nz/2
  void* fptab = nullptr;       // F^P table [n_tab + 1] real
  // ions
  int* cell_of = nullptr;      // [max_ions]
  int* counts = nullptr;       // [n_cells]
  int* fill = nullptr;         // [n_cells]
  int* cell_start = nullptr;   // [n_cells + 1]
  int* perm = nullptr;         // [max_ions]
  int* tile_sums = nullptr;    // scan scratch
  void* xs = nullptr;          // sorted positions [3][max_ions] real
  void* qs = nullptr;          // sorted charges [max_ions] real
  int* sps = nullptr;          // sorted species [max_ions]
  void* xq = nullptr;          // sorted (x, y, z, q) packed [max_ions] float4 / 32-byte double4
  void* F = nullptr;           // forces [3][max_ions] real
  void* xstar = nullptr;       // midpoint positions [3][max_ions] real
  void* V = nullptr;           // interpolated velocities [3][max_ions] real
  void* Fn = nullptr;          // near-field forces of the current step [3][max_ions] real
  // Stokes wall-normal factors [M][Ny] in double: L D L^T of the pentadiagonal
  // indexed by face (l1, l2, 1/D), A_c Thomas pivots by cell row; [M][5]
  // per-mode constants (g_x, g_z, -1/K^2)
  double* st_l1 = nullptr;
  double* st_l2 = nullptr;
  double* st_di = nullptr;
  double* st_ci = nullptr;
  double* st_mc = nullptr;
  // mixed precision: modes with K^2 < 0.5 are solved in double (k_ysolve.cu)
  int n_lo = 0;
  int* lo_modes = nullptr;       // [n_lo] mode indices kz * Nxh + kx
  unsigned char* is_lo = nullptr;  // [M]
  float* st_l1f = nullptr;       // single-precision copies of the Stokes factors, [Ny][M] (mc: [M][5])
  float* st_l2f = nullptr;
  float* st_dif = nullptr;
  float* st_cif = nullptr;
  float* st_mcf = nullptr;
  // the double-precision low modes run on their own stream, beside the rest
  cudaStream_t ystream = nullptr;
  cudaEvent_t yev0 = nullptr, yev1 = nullptr;
  double* edata = nullptr;      // energy: lift profiles [3][Ny], then 3 sums
  void* rref = nullptr;         // refinement (mixed, max_refine > 0): rho kept for the residual
  void* rres = nullptr;         //   residual, then correction
  double* rnorm = nullptr;      //   (|r|^2, |b|^2) before each sweep and after the last
  double* phi64 = nullptr;      //   the refined potential, accumulated in double
  // refinement of the Stokes solve (mixed, max_refine > 0, wet)
  void* sref = nullptr;         //   forcing kept for the residual (f and v may alias)
  void* sres = nullptr;         //   residual, then velocity correction
  void* pres = nullptr;         //   pressure of each solve
  double* v64 = nullptr;        //   velocity and pressure accumulated in double
  double* p64 = nullptr;
  double* snorm = nullptr;      //   (|r|^2, |f|^2) before each sweep and after the last
  // metal strip (k_strip.cu)
  void* strip_g = nullptr;      //   [Nz][Ny][Nx] real: the strip sources, then their solve
  void* strip_add0 = nullptr;   //   [Nx] real: bottom-row terms of the base solve (2 phi_m on the strip, -g off it)
  double* strip_r = nullptr;    //   [Nz][Ws] base solution on the strip cells
  double* strip_shat = nullptr; //   [Nz][Ws] complex strip sources per z mode
  double* strip_M = nullptr;    //   [Nz][Ws + 1][Ws + 1] inverse capacitance matrices
  double* strip_c = nullptr;    //   the constant of the bordered kz = 0 system
  unsigned* fault = nullptr;    // device fault word (Params::fault)
  double* diag = nullptr;       // scratch of discos_diagnostics
  double* nsum = nullptr;       // neutrality sums (sum q, sum |q|) of an all-Neumann channel
  int n_cells = 0;
};

// Arguments of the batched step kernel (k_batched.cu), passed by value.
struct BatchArgs {
  int R, Ntot, steps, n_cells, n_lo, n_hi;
  const int* offsets;          // [R + 1]
  const int* order;            // [R] replicas by descending ion count
  float* x;                    // [3][Ntot]
  const float* q;              // [Ntot]
  const int* species;          // [Ntot] or null
  const double* phi_b;         // [R][2] or null
  unsigned* hist;              // [R][nspecies][Ny] or null
  double* sums;                // [R][4] or null
  float* F_out;                // [3][Ntot] or null
  int* nbr;                    // [Ntot] or null
  int* queue;                  // work counter, finished-CTA counter
  long long* dstep;            // step index of the next launch
  const float* piv32;          // Poisson pivots [M][Ny] (complex-mode index)
  const double* piv64;
  const short* modes;          // Hartley modes kz * 32 + kx: n_lo low modes, then n_hi
  const float* fptab;
};

// State of the batched path, set up on first use.
struct BatchState {
  int* order = nullptr;
  int order_cap = 0;
  std::vector<int> offsets_seen;
  int* queue = nullptr;
  long long* dstep = nullptr;
  short* modes = nullptr;
  int n_lo = 0, n_hi = 0;
  int nsm = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> exec_key;
  int steps_per_launch = 1;     // launch shape (discos_tune_batched)
};

size_t batched_smem_bytes(int Ny, int n_cells, int n_tab);
bool batched_supported(const Params& P);
cudaError_t batched_prepare(const Params& P, int n_cells);
cudaError_t launch_batched_reset(int* queue, long long* dstep, long long step0, cudaStream_t s);
cudaError_t launch_batched_step(const Params& P, const BatchArgs& B, int grid, cudaStream_t s);

}  // namespace discos

struct discos_handle {
  discos_config cfg;
  discos::Params P;
  discos::Workspace W;
  bool mixed;
  discos_alloc_fn alloc_fn;
  discos_free_fn free_fn;
  void* alloc_ctx;
  int device;
  discos::Probe probe;
  cudaStream_t side = nullptr;       // independent work of a step runs here
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_extra = nullptr;        // the side stream's extra work (the stochastic stress) is done
  discos::BatchState* batch = nullptr;   // batched replicas (batch_api.cu)
  unsigned* fault_host = nullptr;        // pinned copy of the fault word, written after each discos_step
  cudaEvent_t ev_fault = nullptr;
};

namespace discos {

void set_error(const std::string& msg);
discos_status invalid(const std::string& m);
void* dalloc(discos_handle* h, size_t bytes, bool* ok);
void dfree(discos_handle* h, void* p);
void free_batch(discos_handle* h);
// Number of kernels this library has launched since it was loaded.
void count_launches(long long n);
discos_status cuda_status(cudaError_t e, const char* where);

// Transform launch shapes (k_fft.cu).
int default_fx_pairs(int Nx);
int max_tile_z(int Nz, size_t elem);
int default_tile_z(int Nz, size_t elem);
int fz_threads(int TK, int Nz);
cudaError_t tune_transforms(Params& P, Workspace& W, bool mixed, cudaStream_t s, float* best_ms);

// Host code that builds the F^P table (fptable.cpp).
bool build_fp_table(const KernelParams& kp, double psi, int n_tab, double* out, std::string* err);
double es_normalisation(int w, double beta);

// Launch wrappers (one per kernel family); T = float or double.
template <typename T> cudaError_t launch_cell_list(const Params& P, Workspace& W, const T* x, int N, cudaStream_t s);
template <typename T> cudaError_t launch_spread_charge(const Params& P, const T* x, const T* q, int N, T* rho, cudaStream_t s,
                                                       bool decorrelate = false);
// Adds the stochastic stress divergence into f with atomics (f prepared by the caller).
template <typename T> cudaError_t launch_stress_noise(const Params& P, T* f, int64_t step, cudaStream_t s);
template <typename T> cudaError_t launch_poisson(const Params& P, Workspace& W, const T* rho, T* phi, cudaStream_t s);
template <typename T> cudaError_t launch_poisson_strip(const Params& P, Workspace& W, const T* rho, T* phi, T fourpi_lB,
                                                       T add1, cudaStream_t s);
template <typename T> cudaError_t launch_stokes(const Params& P, Workspace& W, const T* f, T* v, T* p, cudaStream_t s);
template <typename T> cudaError_t launch_near_field(const Params& P, Workspace& W, const T* x, const T* q,
                                                    const int* species, int N, T* F, int* nbr, cudaStream_t s,
                                                    bool accumulate = true);
// Cell list of x, then sorted copies of the ions (W.xs, W.qs, W.sps, W.xq;
// W.perm maps sorted index -> caller's index).
template <typename T> cudaError_t launch_sort_ions(const Params& P, Workspace& W, const T* x, const T* q,
                                                   const int* species, int N, cudaStream_t s);
// Near field of the sorted ions; F written at f_index[s] and nbr at
// n_index[s] (NULL: at s, the sorted order).
template <typename T> cudaError_t launch_near_field_sorted(const Params& P, Workspace& W, int N, T* F, int* nbr,
                                                           const int* f_index, const int* n_index, cudaStream_t s,
                                                           bool accumulate);
template <typename T> cudaError_t launch_dry_update(const Params& P, T* x, const int* species, const T* F,
                                                   const T* V, int N, int64_t step, cudaStream_t s,
                                                   const T* xin = nullptr, const int* index = nullptr);
template <typename T> cudaError_t launch_scatter3(const T* src, const int* index, int N, T* dst, cudaStream_t s);

// Spreading and interpolation (k_spread.cu, k_interp.cu).  decorrelate:
// visit the ions in a scattered order (atomics of ions in cell order collide);
// noise_index: the caller's index of each ion (the RFD noise key); out_index:
// where each ion's result goes.
// Runs f(Q) once with the run's hydrodynamic kernel (Q.hy_filter = -1: every
// ion), or, with a kernel per species (App. B), once per species s with
// Q.khy = that species' kernel and Q.hy_filter = s when the ions' species are
// known; without them every ion counts as species 0.
template <typename Fn>
inline void for_each_hy_kernel(const Params& P, const int* species, Fn&& f) {
  Params Q = P;
  Q.hy_filter = -1;
  if (!P.hy_species) { f(Q); return; }
  if (!species) { Q.khy = P.khy_s[0]; f(Q); return; }
  for (int s = 0; s < P.nspecies; ++s) {
    Q.khy = P.khy_s[s];
    Q.hy_filter = s;
    f(Q);
  }
}

template <typename T> cudaError_t launch_spread_force(const Params& P, const T* x, const T* F, int N, T* f,
                                                      int64_t step, bool rfd, cudaStream_t s, bool accumulate,
                                                      const int* noise_index, bool decorrelate,
                                                      const int* species = nullptr);
template <typename T> cudaError_t launch_interp_efield(const Params& P, const T* x, const T* q, int N, const T* phi,
                                                       T* out, bool as_force, cudaStream_t s, const T* F_add,
                                                       const int* out_index);
template <typename T> cudaError_t launch_interp_velocity(const Params& P, const T* x, int N, const T* v, T* out,
                                                         cudaStream_t s, const int* out_index,
                                                         const int* species = nullptr);
template <typename T> cudaError_t launch_midpoint(const Params& P, const T* x, const T* V, int N, T* xstar,
                                                  cudaStream_t s);
template <typename T> cudaError_t launch_fill_zero(T* p, size_t n, cudaStream_t s);
template <typename T> cudaError_t launch_fill_value(T* p, size_t n, T value, cudaStream_t s);
template <typename T> cudaError_t launch_energy_sums(const Params& P, const T* rho, const T* phi, const double* lift,
                                                      double* sums, cudaStream_t s);
template <typename T> cudaError_t launch_energy_grad(const Params& P, const T* x, const T* q, int N, const T* phi,
                                                      const double* dU, T* dx, T* dq, cudaStream_t s);
cudaError_t launch_lift(const Params& P, double* lift, cudaStream_t s);
cudaError_t launch_scale2(const double* sums, const double* dU, double* out, cudaStream_t s);
template <typename T, typename TP> cudaError_t launch_poisson_residual(const Params& P, const T* rho, const TP* phi,
                                                                        T* res, double* norms, cudaStream_t s);
template <typename T> cudaError_t launch_stokes_residual(const Params& P, const T* f, const double* v, const double* p,
                                                          T* res, double* norms, cudaStream_t s);
template <typename T> cudaError_t launch_accumulate(double* acc, const T* d, size_t n, cudaStream_t s);
template <typename TD, typename TS> cudaError_t launch_convert(TD* dst, const TS* src, size_t n, cudaStream_t s);
template <typename T> cudaError_t launch_diagnostics(const Params& P, const T* x, const T* q, const T* F, int N,
                                                      const T* rho, double* out, cudaStream_t s);
template <typename T> cudaError_t launch_add_inplace(T* a, const T* b, size_t n, cudaStream_t s);
// out[0..1] = (sum v, sum |v|) in double.
template <typename T> cudaError_t launch_charge_sums(const T* v, size_t n, double* out, cudaStream_t s);
// Sets bit 2 of *fault when the sums of launch_charge_sums plus the surface
// charge are not neutral to tol.
cudaError_t launch_neutral_flag(const double* sums, double surface, double surface_abs, double tol, unsigned* fault,
                                cudaStream_t s);
template <typename T> cudaError_t launch_poisson_y(const Params& P, Workspace& W, cplx<T>* S, cudaStream_t s);
template <typename T> cudaError_t launch_stokes_y(const Params& P, Workspace& W, cplx<T>* S, cplx<T>* Sp,
                                                  cudaStream_t s);

}  // namespace discos
