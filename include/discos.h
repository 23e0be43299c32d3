/*
 * libdiscos: GB300 (sm_103a) implementation of the per-time-step
 * particle-grid hot path of the DISCOS method for ions in a channel with
 * walls at y = 0 and y = Ny, periodic in x and z (Ladiges et al., "Modeling
 * electrokinetic flows with the discrete ion stochastic continuum overdamped
 * solvent algorithm", arXiv 2204.14167).
 *
 * Units are reduced: grid spacing 1 (cell volume 1), kT as configured,
 * permittivity eps = 1/(4 pi lB) so the Coulomb force is lB q_i q_j / r^2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Precision. A handle is created for DISCOS_FP64 (every array is double)
 *   or DISCOS_MIXED (ion and grid arrays are float; the wall-normal banded
 *   solves, the RFD weight differences and global sums run in double).
 *   "real" below means that type.
 * - Ion arrays are structure-of-arrays and live on the device: positions
 *   x[3][N] (x row, then y row, then z row, each N reals), charges q[N],
 *   species[N] (int32, may be NULL = all species 0), forces F[3][N].
 * - Grids are [Nz][Ny][Nx] (x fastest) for cell-centred quantities and
 *   for x- and z-face quantities; y-face quantities are [Nz][Ny+1][Nx]
 *   with rows 0 and Ny on the walls.
 * - Ownership. Every pointer argument is borrowed: the caller owns it and
 *   keeps it valid until the work queued on `stream` has finished. The
 *   library owns only the workspace it allocates in discos_create.
 * - Streams. `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   Calls only enqueue work; results are ready when the stream is.
 * - Errors. Every function returns a discos_status. Arguments are checked
 *   before anything is enqueued; on failure nothing is enqueued and
 *   discos_last_error() describes the cause. A CUDA launch error returns
 *   DISCOS_ERR_CUDA.
 */
#ifndef DISCOS_H
#define DISCOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int discos_status;
enum {
  DISCOS_OK = 0,
  DISCOS_ERR_INVALID_ARG = 1,
  DISCOS_ERR_OOM = 2,
  DISCOS_ERR_NOT_NEUTRAL = 3,
  DISCOS_ERR_NOT_CONVERGED = 4,
  DISCOS_ERR_DEVICE_FAULT = 5,
  DISCOS_ERR_TIMEOUT = 6,
  DISCOS_ERR_CUDA = 7
};

enum { DISCOS_BC_DIRICHLET = 0, DISCOS_BC_NEUMANN = 1 };
enum { DISCOS_HY_NOSLIP = 0, DISCOS_HY_SLIP = 1 };
enum { DISCOS_KERNEL_PESKIN4 = 0, DISCOS_KERNEL_PESKIN6 = 1, DISCOS_KERNEL_ES = 2 };
enum { DISCOS_FP64 = 0, DISCOS_MIXED = 1 };
enum { DISCOS_WALL_WCA = 0, DISCOS_WALL_LJ93 = 1 };
enum { DISCOS_SPREAD_CHARGE = 0, DISCOS_SPREAD_FORCE = 1 };
enum { DISCOS_INTERP_EFIELD = 0, DISCOS_INTERP_VELOCITY = 1 };

#define DISCOS_MAX_SPECIES 4
#define DISCOS_MAX_REFINE 4

/* Run configuration.  Citations are to the paper's sections and equations. */
typedef struct discos_config {
  int Nx, Ny, Nz;          /* cells; Nx, Nz powers of two in [16, 512], Ny in [8, 256] */
  int bc[2];               /* electrostatic wall type, bottom and top: Eq. esbc1 / Eq. esbc3 */
  double phi_b[2];         /* wall potential of a Dirichlet wall (Eq. esbc1) */
  double surf_charge[2];   /* surface charge of a Neumann wall (Eq. esbc3; -eps dphi/dn = varsigma) */
  int kernel_es;           /* electrostatic kernel (App. B) */
  int kernel_hy;           /* hydrodynamic kernel (App. B) */
  int es_w[2];             /* ES kernel width in points (4..7) for [es, hy] kernels */
  double es_beta[2];       /* ES kernel beta for [es, hy] kernels (Eq. eskernel) */
  double lB;               /* Bjerrum length: eps = 1/(4 pi lB) */
  double eta;              /* viscosity (Eq. disc_stokes) */
  double kT;               /* thermal energy */
  double dt;               /* time step */
  double psi;              /* P3M near-field cutoff (Eq. fullElectro) */
  int n_tab;               /* entries - 1 of the F^P table on [0, psi] (Eq. LC) */
  int nspecies;            /* 1..DISCOS_MAX_SPECIES */
  double D_tot[DISCOS_MAX_SPECIES];  /* total diffusion (Eq. diffSum) */
  double D_wet[DISCOS_MAX_SPECIES];  /* wet part; D_dry = D_tot - D_wet */
  /* Eq. fitfunction coefficients c1..c7: [species][0 = parallel, 1 = perpendicular][0 = tot, 1 = wet][7] */
  double gamma_coef[DISCOS_MAX_SPECIES][2][2][7];
  double lj_sigma[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];  /* Eq. potential */
  double lj_xi[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];
  double lj_rc[DISCOS_MAX_SPECIES][DISCOS_MAX_SPECIES];
  int wall_type;           /* DISCOS_WALL_WCA (12-6) or DISCOS_WALL_LJ93 (Eq. LJ93) */
  double wall_sigma[DISCOS_MAX_SPECIES];
  double wall_xi[DISCOS_MAX_SPECIES];
  double wall_rc[DISCOS_MAX_SPECIES];
  double E_ext[3];         /* applied uniform field: F_ext = q E_ext (Eq. totalforce) */
  int precision;           /* DISCOS_FP64 or DISCOS_MIXED */
  int max_refine;          /* DISCOS_MIXED: sweeps (0..DISCOS_MAX_REFINE) of residual refinement of every
                              Poisson solve (r = 4 pi lB rho + lap_h phi in double, phi += A^-1 r) and,
                              with wet = 1, every Stokes solve (r = f - (eta L v + G p) in double,
                              (v, p) += the solve of r); the corrections accumulate in double */
  int wet;                 /* 1: hydrodynamic stage (Stokes + midpoint); 0: dry diffusion only */
  int drift;               /* 1: stochastic drift terms on (RFD + midpoint, div D^dry) */
  int max_ions;            /* capacity of the per-ion workspace */
  uint64_t seed;           /* Philox key for all noise */
  /* Metal strip (Sec. IV.B, Fig. EOgeometry; mixed conditions on one wall,
     Sec. II.B.1): strip = 1 puts a conducting strip into the bottom wall,
     which must be a dielectric (NEUMANN) wall.  The strip spans the channel
     in z and covers the bottom cells whose centre x + 1/2 lies in
     [strip_x[0], strip_x[1]); on them the wall condition is Dirichlet with
     phi_m(x) = strip_phi + E_ext[0] (x - x_c), x_c the strip's centre, so
     that the total potential phi + phi_E (phi_E = -E_ext[0] (x - x_c)) is
     strip_phi on the metal.  Wall images and ghost cells follow the cell
     column: Dirichlet rules above the strip, Neumann rules elsewhere. */
  int strip;
  double strip_x[2];
  double strip_phi;
  /* Hydrodynamic wall conditions, bottom and top (Eq. fluidbc): NOSLIP, or
     SLIP (zero normal velocity, zero shear stress: like tangential images in
     spreading, mirrored tangential ghosts in interpolation and in the
     viscous operator, no stochastic stress on the wall edges).  At most one
     slip wall: with two, uniform flow along the walls is undamped. */
  int bc_hy[2];
  /* Hydrodynamic kernel per species (App. B: on one hydrodynamic grid the
     cations spread and interpolate with the ES kernel of w = 7, beta = 7 and
     the anions with w = 4, beta = 8).  hy_species = 1: species s uses
     (kernel_hy_s[s], hy_w_s[s], hy_beta_s[s]) in S^hy, J^hy and the thermal
     forcing instead of (kernel_hy, es_w[1], es_beta[1]); force spreading and
     velocity interpolation then take the species of each ion
     (discos_spread_species, discos_interpolate_species; the calls without
     species treat every ion as species 0). */
  int hy_species;
  int kernel_hy_s[DISCOS_MAX_SPECIES];
  int hy_w_s[DISCOS_MAX_SPECIES];
  double hy_beta_s[DISCOS_MAX_SPECIES];
} discos_config;

typedef struct discos_handle discos_handle;

/* Device-memory allocator hooks; NULL uses cudaMalloc / cudaFree. */
typedef void* (*discos_alloc_fn)(size_t bytes, void* ctx);
typedef void (*discos_free_fn)(void* ptr, void* ctx);

/* Creates a handle: validates the configuration, allocates the workspace,
 * builds the F^P pair-force table of Sec. II.B.1 (Eq. LC) for the
 * electrostatic kernel and uploads all constants (with a metal strip, also
 * the strip's capacitance matrices).  The handle belongs to the CUDA device
 * that is current at creation; every later call must be made with that
 * device current (else INVALID_ARG).  Synchronous.
 * Errors: INVALID_ARG (bad sizes, kernel, cutoff, strip), OOM (alloc_fn or
 * cudaMalloc returned NULL; whatever was allocated is freed and no handle is
 * returned), CUDA. */
discos_status discos_create(const discos_config* cfg, discos_alloc_fn alloc_fn,
                            discos_free_fn free_fn, void* alloc_ctx, discos_handle** out);

/* Frees the workspace and the handle (synchronises the device first). */
discos_status discos_destroy(discos_handle* h);

/* Static description of the last error on this thread. */
const char* discos_last_error(void);

/* Number of CUDA kernels the library has enqueued since it was loaded (all
 * handles, all threads); a diagnostic for launch accounting. */
long long discos_launch_count(void);

/* Live timing of one kernel family (measurement hook).  discos_probe
 * synchronises the device, then records a CUDA event pair on the launching
 * stream around every launch of `family` made through this handle (at most
 * 4096 launches), -1 switches it off; discos_probe_read waits for the events
 * and returns the summed duration in ms and the number of launches. */
enum {
  DISCOS_PROBE_CELL_LIST = 0, DISCOS_PROBE_NEAR_FIELD, DISCOS_PROBE_NOISE, DISCOS_PROBE_SPREAD_CHARGE,
  DISCOS_PROBE_FFT_X, DISCOS_PROBE_FFT_Z, DISCOS_PROBE_POISSON_Y, DISCOS_PROBE_INTERP_E,
  DISCOS_PROBE_SPREAD_FORCE, DISCOS_PROBE_STOKES_Y, DISCOS_PROBE_INTERP_V, DISCOS_PROBE_UPDATE
};
discos_status discos_probe(discos_handle* h, int family);
discos_status discos_probe_read(discos_handle* h, double* total_ms, int* launches);

/* Spreading, Eq. kernel2 with the wall image construction of Sec. II.A
 * (Fig. folded) and Sec. II.B.1.
 * which = DISCOS_SPREAD_CHARGE: val = q[N]; grid = rho[Nz][Ny][Nx] cell
 *   centred, images of sign -1 (Dirichlet wall) / +1 (Neumann wall).
 * which = DISCOS_SPREAD_FORCE: val = F[3][N]; grid = fx[Nz][Ny][Nx] followed
 *   by fy[Nz][Ny+1][Nx] followed by fz[Nz][Ny][Nx] (one contiguous buffer),
 *   opposite normal images, tangential images opposite at a no-slip wall
 *   and like at a slip wall.
 * The grid is overwritten (not accumulated into). */
discos_status discos_spread(discos_handle* h, const void* x, const void* val, int N, int which,
                            void* grid, void* stream);

/* discos_spread with the species of each ion (int32 [N], values in
 * [0, nspecies); may be NULL = all species 0): with cfg.hy_species = 1,
 * DISCOS_SPREAD_FORCE spreads every ion with its own species' hydrodynamic
 * kernel (App. B); otherwise identical to discos_spread.  Species outside
 * [0, nspecies) are not spread (no error is raised on the device). */
discos_status discos_spread_species(discos_handle* h, const void* x, const void* val, const int* species, int N,
                                    int which, void* grid, void* stream);

/* Poisson solve -eps lap_h phi = rho (Eq. poisson) with the wall conditions
 * of Eqs. esbc1 / esbc3, periodic in x and z: DFTs in x and z and a double
 * precision tridiagonal solve per (kx, kz) mode in y (with a metal strip,
 * plus the capacitance correction on the strip's cells).  rho, phi:
 * [Nz][Ny][Nx] reals (may alias).  For two Neumann walls (no strip) the
 * potential has zero mean and the charge plus surface charge must vanish
 * (Sec. II.B.1): the call sums rho in double first (waiting for `stream`) and
 * returns NOT_NEUTRAL, with nothing launched, beyond 1e-9 (FP64) / 1e-6
 * (MIXED) of the summed magnitudes. */
discos_status discos_solve_poisson(discos_handle* h, const void* rho, void* phi, void* stream);

/* Staggered Stokes solve with no-slip or slip walls (Eqs. disc_stokes, fluidbc):
 * f = fx|fy|fz as in discos_spread(FORCE); v = u|v|w in the same layout
 * (wall rows of v are zero); p = [Nz][Ny][Nx] pressure (mean zero), may be
 * NULL.  f and v may alias. */
discos_status discos_solve_stokes(discos_handle* h, const void* f, void* v, void* p, void* stream);

/* Interpolation, Eq. kernel1 with ghost cells filled from the boundary
 * conditions.
 * which = DISCOS_INTERP_EFIELD: grid = phi; out[3][N] = E^P = J^es(-grad_h phi)
 *   (Eq. efieldop) with E on the cell faces.
 * which = DISCOS_INTERP_VELOCITY: grid = u|v|w; out[3][N] = J^hy v. */
discos_status discos_interpolate(discos_handle* h, const void* x, int N, int which,
                                 const void* grid, void* out, void* stream);

/* discos_interpolate with the species of each ion (as in
 * discos_spread_species): with cfg.hy_species = 1, DISCOS_INTERP_VELOCITY
 * interpolates every ion with its own species' hydrodynamic kernel; out
 * entries of ions with a species outside [0, nspecies) are left untouched. */
discos_status discos_interpolate_species(discos_handle* h, const void* x, const int* species, int N, int which,
                                         const void* grid, void* out, void* stream);

/* Cell list of Sec. II.B.1's neighbour sets: list cells of k grid cells per
 * axis (k = ceil(max(psi, largest LJ cutoff))), cell = min(floor(x) div k,
 * nc - 1) with x and z first moved into the periodic box [0, L) (positions
 * outside it are binned at their periodic image); counting sort, ions
 * stable by index inside a cell.
 * cell_start[n_cells + 1] and perm[N] are int32 device arrays (either may be
 * NULL); n_cells_out (host, may be NULL) receives n_cells. */
discos_status discos_cell_list(discos_handle* h, const void* x, int N, int* cell_start,
                               int* perm, int* n_cells_out, void* stream);

/* Allocation-free variant of discos_cell_list, for callers that cannot
 * allocate device memory at the point where they need a cell list: work
 * enqueued while a stream is being captured into a CUDA graph, code inside a
 * host framework whose caching allocator already owns the device memory, and
 * fixed-latency loops that must not enter the allocator.  The paper has no
 * counterpart; it builds exactly the list discos_cell_list builds, from the
 * configuration alone (no handle).
 * - It calls no allocating routine.  Its scratch is a file-scope device array
 *   of 1048576 + 2 * 262144 + 258 ints (about 6.3 MB) that every GPU loading
 *   this library holds until the process exits; hence at most 1048576 ions
 *   and 262144 list cells per call, larger requests return INVALID_ARG with
 *   nothing enqueued.
 * - Positions that are not finite, or outside [0, Ny] in y, are still binned
 *   (all of them valid list entries) but switch off the per-cell ordering of
 *   that call: such ions can all share one cell, where the ordering would
 *   take quadratic time.  The order inside a cell is then unspecified.
 * - The first call on a device (with that device current) looks up the
 *   array's device address; make that first call before any stream capture.
 * - All calls share the one array: calls that overlap on the GPU (different
 *   streams without ordering) race.  Each call clears what must start at
 *   zero, so consecutive calls on one stream are independent.
 * Arguments as in discos_cell_list; cfg supplies Nx, Ny, Nz, psi, nspecies,
 * lj_rc and precision (the type of x); cell_start must hold n_cells + 1 ints
 * (n_cells is written to n_cells_out first, -1 if over the limit). */
discos_status discos_cell_list_noalloc(const discos_config* cfg, const void* x, int N, int* cell_start,
                                       int* perm, int* n_cells_out, void* stream);

/* Near-field forces added to F[3][N] (F += ...): the P3M local correction
 * with wall images (Eqs. coulomb, fullElectro, LC), the ion-ion LJ force
 * (Eq. closerange) and the wall force (Sec. II.B.2).  nbr_count[N] (int32,
 * may be NULL) receives the number of real and image partners within psi. */
discos_status discos_near_field(discos_handle* h, const void* x, const void* q, const int* species,
                                int N, void* F, int* nbr_count, void* stream);

/* Total force, Eq. totalforce: stages 1 and 2 of Sec. II.D
 * (spread, Poisson, field interpolation, near field, wall, external field).
 * F[3][N] is overwritten; nbr_count may be NULL.  Two Neumann walls (no
 * strip): sum q plus the surface charges is checked first as in
 * discos_solve_poisson (NOT_NEUTRAL). */
discos_status discos_forces(discos_handle* h, const void* x, const void* q, const int* species,
                            int N, void* F, int* nbr_count, void* stream);

/* Advances N ions by nsteps steps of Sec. II.D: forces, then either the dry
 * Euler-Maruyama update of Eq. ions3 (cfg.wet = 0) or the fluid forcing,
 * Stokes solve and midpoint update of Eqs. step1-step2 (cfg.wet = 1).
 * x is updated in place (wrapped in x, z; specular reflection at the walls).
 * step0 is the index of the first step (it keys the Philox noise).
 * F_out[3][N] (may be NULL) receives the forces of the last step.
 * Each step bins the ions and works on copies in cell order; results go
 * back to the caller's order.  Two Neumann walls (no strip): every step sums
 * q in double on the device and sets bit 2 of the fault word when the
 * channel is not neutral (discos_solve_poisson's test); the next call then
 * returns NOT_NEUTRAL (see discos_fault). */
discos_status discos_step(discos_handle* h, void* x, const void* q, const int* species, int N,
                          int64_t step0, int nsteps, void* F_out, void* stream);

/* Batched replicas: R independent channels that share the handle's
 * configuration (grid, walls, kernels, physics) and differ in their ions and
 * wall potentials, advanced together by the dry-diffusion step of Sec. II.D
 * (forces of Eq. totalforce, update of Eq. ions3).  Each replica is worked
 * on by one thread block with its whole grid in shared memory; the blocks
 * take replicas longest first from a device work queue.
 * Limits: a DISCOS_MIXED handle with Nx = Nz = 32, Ny = 16 or 32, a 4- or
 * 6-point electrostatic kernel, cfg.wet = 0, at least one Dirichlet wall;
 * 0..512 ions per replica.
 * Ion arrays are packed replica after replica: replica r owns the ions
 * offsets[r] .. offsets[r+1]-1 of x[3][Ntot] (x row, y row, z row, each Ntot
 * floats), q[Ntot] and species[Ntot]; ion i of replica r is ion
 * i - offsets[r] of that replica for the Philox noise, keyed (i, step, r, 1).
 * All device arrays are borrowed and must stay valid until the stream has
 * finished the call's work. */
typedef struct discos_batch {
  int R;                      /* number of replicas, >= 1 */
  const int* offsets_host;    /* host int[R + 1], offsets[0] = 0, non-decreasing */
  const int* offsets;         /* device copy of offsets_host */
  void* x;                    /* device float[3][Ntot], Ntot = offsets[R]; updated in place */
  const void* q;              /* device float[Ntot] */
  const int* species;         /* device int[Ntot] or NULL (all species 0) */
  const double* phi_b;        /* device double[R][2] wall potentials, or NULL (cfg.phi_b for all) */
  unsigned int* hist;         /* device uint32[R][nspecies][Ny] or NULL: after every step, +1 in
                                 the y cell of every ion (the equilibrium density profiles) */
  double* sums;               /* device double[R][4] or NULL: sum q, sum F_x, sum F_y, sum F_z
                                 over the replica's ions at the last step, accumulated in double */
  void* F_out;                /* device float[3][Ntot] or NULL: forces of the last step */
  int* nbr_count;             /* device int[Ntot] or NULL: near-field partners of the last step */
} discos_batch;

/* Advances every replica by nsteps steps, the first with index step0.  The
 * launches (one per step, or per steps_per_launch steps, see below) are
 * replayed from a CUDA graph captured on the first call with the same
 * arguments.  A call whose offsets differ from the previous call's uploads a
 * new replica order and waits for that copy (the only host wait).
 * Errors: INVALID_ARG for the limits above and malformed offsets. */
discos_status discos_step_batched(discos_handle* h, const discos_batch* b, int64_t step0, int nsteps,
                                  void* stream);

/* Launch-shape autotuner of the batched step: times every candidate number
 * of steps per launch (1, 2, 4, 8, 16; more steps per launch keep the ions
 * in shared memory across steps, fewer give the scheduler finer work units)
 * on trial_steps steps of a scratch copy of b's positions (b is not
 * modified), keeps the fastest for later discos_step_batched calls on h and
 * returns it and its time per step (either out pointer may be NULL).
 * Blocks until the trials are done. */
discos_status discos_tune_batched(discos_handle* h, const discos_batch* b, int trial_steps,
                                  int* steps_per_launch, double* ms_per_step, void* stream);

/* Sets the number of steps per batched launch directly (1..1024). */
discos_status discos_set_batched_shape(discos_handle* h, int steps_per_launch);

/* Discrete electrostatic energy of the particle-mesh problem.  The paper
 * defines no energy; this is the grid energy of its electrostatic stage
 * (Sec. II.B.1, Eqs. poisson, esbc1, esbc3):
 *     U = sum_j rho_j (phi^rho_j / 2 + phi^b_j) = (1/2) sum_j rho_j (phi_j + phi^b_j)
 * with rho = S^es q (images included, cell volume 1), phi the solution of
 * Eq. poisson with the wall data, phi^rho its part with homogeneous wall data
 * and phi^b the discrete lift of the wall data (the solution for rho = 0).
 * The P3M near-field pair energy is not included.
 * phi_b: host double[2], the two wall potentials to use in place of
 *   cfg.phi_b (NULL = cfg.phi_b); Neumann walls ignore theirs.
 * U: device double[1], overwritten.
 * Errors: INVALID_ARG for two Neumann walls (no potential is fixed). */
discos_status discos_energy(discos_handle* h, const void* x, const void* q, int N, const double* phi_b,
                            double* U, void* stream);

/* Hand-written adjoint of discos_energy: given the upstream scalar dU
 * (device double[1]), writes
 *   dx[3][N] = dU * dU/dx_i = dU q_i sum_j phi_j grad w(x_i - r_j)   (gradient-kernel interpolation)
 *   dq[N]    = dU * dU/dq_i = dU (J^es phi)_i                        (interpolation = adjoint of spreading)
 *   dphi_b[2] (device double) = dU * sum_j rho_j dphi^b_j / dphi_b,w
 * using that the discrete Poisson operator is self-adjoint (dU/drho = phi).
 * rho and phi are recomputed, not stored.  dx, dq are reals (device) and
 * overwritten; any of dx, dq, dphi_b may be NULL.  phi_b as in discos_energy.
 * Errors: as discos_energy. */
discos_status discos_energy_backward(discos_handle* h, const void* x, const void* q, int N,
                                     const double* phi_b, const double* dU, void* dx, void* dq,
                                     double* dphi_b, void* stream);

/* The device fault word.  Kernels that move ions set bit 0 when a new
 * position is not finite and bit 1 when an ion ends outside the channel (a
 * displacement larger than the channel); the step sets bit 2 for a
 * non-neutral channel between two Neumann walls; a kernel whose bounded wait
 * on an asynchronous bulk copy ran out sets bit 3 (its results are then
 * incomplete).  None stops the other kernels, whose indexing stays in bounds
 * for any position.  discos_step copies the
 * word to the host behind its steps, and the next discos_step call returns
 * DISCOS_ERR_NOT_NEUTRAL (bit 2) or DISCOS_ERR_DEVICE_FAULT, before
 * enqueueing anything, once that copy shows a set bit.  discos_fault returns the word (sync != 0: read now, waiting for
 * `stream`; else the last copy that has arrived, 0 if none) and with
 * clear != 0 resets it. */
discos_status discos_fault(discos_handle* h, int sync, int clear, unsigned* word, void* stream);

/* Reductions in double over the ions (and the grid): out[8] (device doubles)
 * = {sum q_i, dV sum_j rho_j (with_rho != 0: the charge is spread again, wall
 * images folded in; else 0), sum F_x, sum F_y, sum F_z (F[3][N] may be NULL),
 * count of non-finite positions, count of ions outside the channel, 0}.
 * Neutrality (Sec. II.B.1) is sum q + the surface charges times Nx Nz. */
discos_status discos_diagnostics(discos_handle* h, const void* x, const void* q, const void* F, int N,
                                 int with_rho, double* out, void* stream);

/* Relative residuals ||b - A phi|| / ||b|| (double) of the most recent
 * Poisson solve of a DISCOS_MIXED handle created with max_refine > 0: rel[0]
 * after the single-precision solve, rel[k] after k refinement sweeps
 * (n = max_refine + 1 values written to the host array rel).  Waits for
 * `stream`.  Other handles return n = 0. */
discos_status discos_refine_history(discos_handle* h, double* rel, int* n, void* stream);

/* The same for the most recent Stokes solve of a DISCOS_MIXED wet handle
 * created with max_refine > 0: relative residuals ||f - (eta L v + G p)|| /
 * ||f|| of the MAC system of Eq. disc_stokes, with v and p carried in
 * double (rel[0] after the single-precision solve, rel[k] after k sweeps).
 * Other handles return n = 0. */
discos_status discos_refine_history_stokes(discos_handle* h, double* rel, int* n, void* stream);

/* Launch-shape autotuner of the x and z transforms (used by every Poisson
 * and Stokes solve of the handle): times each candidate shape (x: 128 to
 * 2048 grid values per block, i.e. 1..2048/Nx row pairs, and, for Nx >= 32,
 * the bulk-staged persistent kernel, reported as fx_pairs = 0; z: 4..16
 * columns per block in single precision, 2..16 in double, within the
 * shared-memory limit) on the handle's own
 * buffers at the Poisson sizes, keeps the fastest, and returns it (out
 * pointers may be NULL; ms[2] = the x and z times per launch).  Overwrites
 * the handle's potential and spectrum workspace; blocks until done.  A new
 * handle starts with the staged x kernel (Nx >= 32) and 8 z columns. */
discos_status discos_tune_transforms(discos_handle* h, int* fx_pairs, int* fx_threads, int* fz_tile,
                                     float* ms, void* stream);

/* Sets the transform launch shape directly: fx_pairs row pairs per x block
 * (fx_pairs * Nx <= 2048, within 48 KB of shared memory), fx_threads (a
 * multiple of 32), fz_tile columns per z block (a power of two); fx_pairs = 0
 * selects the bulk-staged persistent x kernel (Nx >= 32; fx_threads is then
 * ignored).  The staged kernel reads and writes whole rows with bulk copies
 * and needs 16-byte aligned grids: a caller's grid that is not falls back to
 * the per-row kernel.  Errors: INVALID_ARG outside those limits. */
discos_status discos_set_transform_shape(discos_handle* h, int fx_pairs, int fx_threads, int fz_tile);

/* Host-only (no GPU needed): the F^P pair-force table that discos_create
 * builds (Sec. II.B.1, Eq. LC), for kernel `kernel` (es_w, es_beta used by
 * DISCOS_KERNEL_ES), f^P(k psi / n_tab) for k = 0..n_tab with l_B = 1 and
 * unit charges, written to the host array out[n_tab + 1].
 * Errors: INVALID_ARG. */
discos_status discos_fp_table(int kernel, int es_w, double es_beta, double psi, int n_tab, double* out);

#ifdef __cplusplus
}
#endif
#endif
