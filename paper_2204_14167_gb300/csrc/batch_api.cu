// Host side of the batched replicas (discos_step_batched,
// discos_tune_batched): argument checks, the longest-first replica order,
// the CUDA graph of step launches and the launch-shape autotuner.  The
// kernel is in k_batched.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include "internal.h"

namespace discos {

namespace {

constexpr int kMaxIons = 512;     // per replica (shared-memory capacity)
constexpr int kChunk = 32;        // launches per captured graph

const int kStepsPerLaunch[] = {1, 2, 4, 8, 16};

discos_status check_batch(discos_handle* h, const discos_batch* b, int* Ntot) {
  if (!h || !b) return invalid("null handle or batch");
  const discos_config& c = h->cfg;
  if (!h->mixed) return invalid("batched replicas need a DISCOS_MIXED handle (single-precision grids on chip)");
  if (c.Nx != 32 || c.Nz != 32 || !batched_supported(h->P))
    return invalid("batched replicas need Nx = Nz = 32, Ny = 16 or 32 and a 4- or 6-point kernel");
  if (c.bc[0] == DISCOS_BC_NEUMANN && c.bc[1] == DISCOS_BC_NEUMANN)
    return invalid("batched replicas need at least one Dirichlet wall");
  if (c.wet) return invalid("batched replicas run the dry step (cfg.wet = 0)");
  if (c.strip) return invalid("batched replicas have no metal strip");
  const Params& P = h->P;
  if (P.ncx < 3 || P.ncz < 3 || P.ncx * P.ncy * P.ncz > 4096) return invalid("list cells outside the batched limits");
  if (c.n_tab > 1024) return invalid("n_tab > 1024 for the batched path");
  if (batched_smem_bytes(c.Ny, P.ncx * P.ncy * P.ncz, c.n_tab) > 226 * 1024)
    return invalid("the replica does not fit in shared memory");
  if (b->R < 1) return invalid("R must be >= 1");
  if (!b->offsets_host || !b->offsets) return invalid("offsets_host and offsets are required");
  if (b->offsets_host[0] != 0) return invalid("offsets[0] must be 0");
  for (int r = 0; r < b->R; ++r) {
    const int n = b->offsets_host[r + 1] - b->offsets_host[r];
    if (n < 0 || n > kMaxIons) return invalid("every replica needs 0..512 ions (offsets must be non-decreasing)");
  }
  *Ntot = b->offsets_host[b->R];
  if (*Ntot > 0 && (!b->x || !b->q)) return invalid("null pointer");
  return DISCOS_OK;
}

cudaError_t ensure_state(discos_handle* h) {
  if (h->batch) return cudaSuccess;
  BatchState* S = new BatchState();
  h->batch = S;
  cudaError_t e = cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) return e;
  bool ok = true;
  S->queue = (int*)dalloc(h, 2 * sizeof(int), &ok);
  S->dstep = (long long*)dalloc(h, sizeof(long long), &ok);
  S->modes = (short*)dalloc(h, 1024 * sizeof(short), &ok);
  if (!ok) return cudaErrorMemoryAllocation;
  // Hartley modes (kx, kz) share the wall-normal system of the Fourier mode
  // (min(kx, 32 - kx), kz); the ill-conditioned ones (K^2 < 0.5) go first.
  std::vector<short> lo, hi;
  for (int kz = 0; kz < 32; ++kz)
    for (int kx = 0; kx < 32; ++kx) {
      const double K2 = (2.0 - 2.0 * std::cos(2.0 * M_PI * kx / 32.0)) + (2.0 - 2.0 * std::cos(2.0 * M_PI * kz / 32.0));
      (K2 < 0.5 ? lo : hi).push_back((short)(kz * 32 + kx));
    }
  if ((int)lo.size() > 64) return cudaErrorInvalidValue;
  S->n_lo = (int)lo.size();
  S->n_hi = (int)hi.size();
  lo.insert(lo.end(), hi.begin(), hi.end());
  e = cudaMemcpy(S->modes, lo.data(), lo.size() * sizeof(short), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(S->queue, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = batched_prepare(h->P, h->P.ncx * h->P.ncy * h->P.ncz);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking);
  return e;
}

// Longest replica first; ties by index.
cudaError_t update_order(discos_handle* h, const discos_batch* b, cudaStream_t s) {
  BatchState* S = h->batch;
  std::vector<int> off(b->offsets_host, b->offsets_host + b->R + 1);
  if (off == S->offsets_seen) return cudaSuccess;
  if (b->R > S->order_cap) {
    dfree(h, S->order);
    bool ok = true;
    S->order = (int*)dalloc(h, sizeof(int) * b->R, &ok);
    if (!ok) { S->order = nullptr; S->order_cap = 0; return cudaErrorMemoryAllocation; }
    S->order_cap = b->R;
  }
  std::vector<int> ord(b->R);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return off[a + 1] - off[a] > off[c + 1] - off[c]; });
  cudaError_t e = cudaMemcpyAsync(S->order, ord.data(), sizeof(int) * b->R, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // ord is a local buffer
  if (e == cudaSuccess) S->offsets_seen = off;
  // the graph holds the order pointer, which may have moved
  if (S->exec) { cudaGraphExecDestroy(S->exec); S->exec = nullptr; S->exec_key.clear(); }
  return e;
}

BatchArgs make_args(discos_handle* h, const discos_batch* b, int Ntot, int steps) {
  BatchState* S = h->batch;
  const Params& P = h->P;
  BatchArgs A{};
  A.R = b->R;
  A.Ntot = Ntot;
  A.steps = steps;
  A.n_cells = P.ncx * P.ncy * P.ncz;
  A.n_lo = S->n_lo;
  A.n_hi = S->n_hi;
  A.offsets = b->offsets;
  A.order = S->order;
  A.x = (float*)b->x;
  A.q = (const float*)b->q;
  A.species = b->species;
  A.phi_b = b->phi_b;
  A.hist = b->hist;
  A.sums = b->sums;
  A.F_out = (float*)b->F_out;
  A.nbr = b->nbr_count;
  A.queue = S->queue;
  A.dstep = S->dstep;
  A.piv32 = h->W.piv32;
  A.piv64 = h->W.piv64;
  A.modes = S->modes;
  A.fptab = (const float*)h->W.fptab;
  return A;
}

// Runs nsteps steps from step0: launches of `steps_per_launch` steps, whole
// chunks of kChunk launches replayed from a captured graph.
discos_status run_batched(discos_handle* h, const discos_batch* b, int Ntot, int64_t step0, int nsteps, int spl,
                          bool use_graph, cudaStream_t s) {
  BatchState* S = h->batch;
  const int grid = std::max(1, std::min(b->R, S->nsm));
  cudaError_t e = launch_batched_reset(S->queue, S->dstep, (long long)step0, s);
  if (e != cudaSuccess) return cuda_status(e, "discos_step_batched");
  const BatchArgs A = make_args(h, b, Ntot, spl);
  long long launches = nsteps / spl;
  const int rem = nsteps % spl;
  if (use_graph && launches >= kChunk) {
    std::vector<unsigned char> key(sizeof(BatchArgs) + sizeof(int));
    std::memcpy(key.data(), &A, sizeof(BatchArgs));
    std::memcpy(key.data() + sizeof(BatchArgs), &grid, sizeof(int));
    if (!S->exec || key != S->exec_key) {
      if (S->exec) { cudaGraphExecDestroy(S->exec); S->exec = nullptr; }
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(S->cap_stream, cudaStreamCaptureModeThreadLocal);
      for (int i = 0; i < kChunk && e == cudaSuccess; ++i) e = launch_batched_step(h->P, A, grid, S->cap_stream);
      cudaError_t e2 = cudaStreamEndCapture(S->cap_stream, &g);
      count_launches(-kChunk);   // captured, not launched
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&S->exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) { S->exec = nullptr; return cuda_status(e, "discos_step_batched (graph)"); }
      S->exec_key = key;
    }
    for (; launches >= kChunk; launches -= kChunk) {
      e = cudaGraphLaunch(S->exec, s);
      if (e != cudaSuccess) return cuda_status(e, "discos_step_batched (graph launch)");
      count_launches(kChunk);
    }
  }
  for (; launches > 0; --launches) {
    e = launch_batched_step(h->P, A, grid, s);
    if (e != cudaSuccess) return cuda_status(e, "discos_step_batched");
  }
  if (rem > 0) {
    const BatchArgs Ar = make_args(h, b, Ntot, rem);
    e = launch_batched_step(h->P, Ar, grid, s);
    if (e != cudaSuccess) return cuda_status(e, "discos_step_batched");
  }
  return DISCOS_OK;
}

}  // namespace

void free_batch(discos_handle* h) {
  BatchState* S = h->batch;
  if (!S) return;
  if (S->exec) cudaGraphExecDestroy(S->exec);
  if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
  dfree(h, S->order);
  dfree(h, S->queue);
  dfree(h, S->dstep);
  dfree(h, S->modes);
  delete S;
  h->batch = nullptr;
}

}  // namespace discos

using namespace discos;

extern "C" {

discos_status discos_step_batched(discos_handle* h, const discos_batch* b, int64_t step0, int nsteps, void* stream) {
  int Ntot = 0;
  discos_status st = check_batch(h, b, &Ntot);
  if (st) return st;
  if (nsteps < 0) return invalid("nsteps must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = ensure_state(h);
  if (e == cudaSuccess) e = update_order(h, b, s);
  if (e != cudaSuccess) return cuda_status(e, "discos_step_batched (setup)");
  if (nsteps == 0) return DISCOS_OK;
  return run_batched(h, b, Ntot, step0, nsteps, h->batch->steps_per_launch, true, s);
}

discos_status discos_tune_batched(discos_handle* h, const discos_batch* b, int trial_steps, int* steps_per_launch_out,
                                  double* ms_per_step_out, void* stream) {
  int Ntot = 0;
  discos_status st = check_batch(h, b, &Ntot);
  if (st) return st;
  if (trial_steps < 16 || trial_steps > 4096) return invalid("trial_steps must be in [16, 4096]");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = ensure_state(h);
  if (e == cudaSuccess) e = update_order(h, b, s);
  if (e != cudaSuccess) return cuda_status(e, "discos_tune_batched (setup)");
  // trials run on a scratch copy of the positions, with no outputs
  bool ok = true;
  void* xs = dalloc(h, sizeof(float) * 3 * (size_t)std::max(Ntot, 1), &ok);
  if (!ok) return DISCOS_ERR_OOM;
  discos_batch tb = *b;
  tb.x = xs;
  tb.hist = nullptr;
  tb.sums = nullptr;
  tb.F_out = nullptr;
  tb.nbr_count = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  int pick = kStepsPerLaunch[0];
  for (int spl : kStepsPerLaunch) {
    for (int rep = 0; rep < 2 && st == DISCOS_OK; ++rep) {   // the first pass warms up
      e = cudaMemcpyAsync(xs, b->x, sizeof(float) * 3 * (size_t)Ntot, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) { st = cuda_status(e, "discos_tune_batched"); break; }
      cudaEventRecord(e0, s);
      st = run_batched(h, &tb, Ntot, 0, trial_steps, spl, false, s);
      cudaEventRecord(e1, s);
      if (st) break;
      e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { st = cuda_status(e, "discos_tune_batched"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep == 1 && ms / trial_steps < best) { best = ms / trial_steps; pick = spl; }
    }
    if (st) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  dfree(h, xs);
  if (st) return st;
  h->batch->steps_per_launch = pick;
  if (steps_per_launch_out) *steps_per_launch_out = pick;
  if (ms_per_step_out) *ms_per_step_out = best;
  return DISCOS_OK;
}

discos_status discos_set_batched_shape(discos_handle* h, int steps_per_launch) {
  if (!h) return invalid("null handle");
  if (steps_per_launch < 1 || steps_per_launch > 1024) return invalid("steps_per_launch must be in [1, 1024]");
  cudaError_t e = ensure_state(h);
  if (e != cudaSuccess) return cuda_status(e, "discos_set_batched_shape");
  h->batch->steps_per_launch = steps_per_launch;
  return DISCOS_OK;
}

}  // extern "C"
