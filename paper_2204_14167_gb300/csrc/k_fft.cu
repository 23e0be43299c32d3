// Hand-written transforms along x and z and the Poisson solve of Eq. poisson
// with the wall conditions of Eqs. esbc1 / esbc3.
//
// x: real rows -> half spectra (Nx/2 + 1 modes, row pitch Px), two real rows
//    packed into one complex transform per warp, held in registers (a
//    shared-memory Stockham transform serves Nx = 16).
// z: complex transforms down the columns of the half spectrum, in place, two
//    x-mode columns per warp held in registers.
// y: the tridiagonal wall-normal system of every (kx, kz) mode, solved by
//    warp-parallel scans over pre-factored pivots (k_ysolve.cu).
#include <atomic>
#include <type_traits>
#include <cuda.h>
#include <cudaTypedefs.h>
#include "internal.h"
#include "bulk.cuh"

namespace discos {

namespace {


// Stockham auto-sort FFT over `nvec` vectors of length N = 2^logN in shared
// memory (vector v at in[v * vs .. v * vs + N)), natural order in and out, no
// bit reversal.  Radix-4 stages while they fit, then one radix-2 stage.  A
// stage with sub-transform size Ns takes butterfly j (< N/R) with
// k = j mod Ns, inputs in[j + m N/R] (m < R) twiddled by exp(-+2 pi i m k /
// (R Ns)), and writes the R-point DFT to out[R j - (R-1) k + m Ns].  Reads
// are unit-stride; the two buffers alternate.  Returns the buffer holding the
// result.  All threads take part; ends with the block synchronised.
template <typename T>
__device__ cplx<T>* fft_stockham(cplx<T>* in, cplx<T>* out, int N, int logN, int nvec, int vs,
                                 const cplx<T>* __restrict__ tw, bool inverse) {
  int Ns = 1;
  while (Ns < N) {
    if (4 * Ns <= N) {
      const int q = N >> 2;
      const int total = nvec * q;
      const int twstep = N / (4 * Ns);
      for (int b = threadIdx.x; b < total; b += blockDim.x) {
        const int v = b >> (logN - 2);
        const int j = b & (q - 1);
        const int k = j & (Ns - 1);
        cplx<T> w1 = tw[k * twstep], w2 = tw[2 * k * twstep];
        if (inverse) { w1.im = -w1.im; w2.im = -w2.im; }
        const cplx<T> w3 = cmul(w1, w2);
        const cplx<T>* iv = in + (size_t)v * vs;
        cplx<T>* ov = out + (size_t)v * vs;
        const cplx<T> a0 = iv[j];
        const cplx<T> a1 = cmul(w1, iv[j + q]);
        const cplx<T> a2 = cmul(w2, iv[j + 2 * q]);
        const cplx<T> a3 = cmul(w3, iv[j + 3 * q]);
        const cplx<T> b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3);
        const cplx<T> d = csub(a1, a3);
        // (a1 - a3) times -i (forward) or +i (inverse)
        const cplx<T> b3 = inverse ? cplx<T>{-d.im, d.re} : cplx<T>{d.im, -d.re};
        const int o = 4 * j - 3 * k;
        ov[o] = cadd(b0, b2);
        ov[o + Ns] = cadd(b1, b3);
        ov[o + 2 * Ns] = csub(b0, b2);
        ov[o + 3 * Ns] = csub(b1, b3);
      }
      Ns <<= 2;
    } else {
      const int hN = N >> 1;
      const int total = nvec * hN;
      const int twstep = N / (2 * Ns);
      for (int b = threadIdx.x; b < total; b += blockDim.x) {
        const int v = b >> (logN - 1);
        const int j = b & (hN - 1);
        const int k = j & (Ns - 1);
        cplx<T> wv = tw[k * twstep];
        if (inverse) wv.im = -wv.im;
        const cplx<T>* iv = in + (size_t)v * vs;
        cplx<T>* ov = out + (size_t)v * vs;
        cplx<T> u = iv[j];
        cplx<T> t = cmul(wv, iv[j + hN]);
        const int o = 2 * j - k;
        ov[o] = cadd(u, t);
        ov[o + Ns] = csub(u, t);
      }
      Ns <<= 1;
    }
    __syncthreads();
    cplx<T>* tmp = in; in = out; out = tmp;
  }
  return in;
}

// Forward real transform of R rows of length N (two rows per complex FFT).
// Input value = scale * in + (row's y == 0 ? add0) + (row's y == Nyr-1 ? add1).
template <typename T>
__global__ void k_rfft_x(const T* __restrict__ in, int R, int N, int logN, int Px, cplx<T>* __restrict__ out,
                         T scale, int Nyr, T add0, T add1, const cplx<T>* __restrict__ tw, int pairs_per_block,
                         const T* __restrict__ add0x) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int PP = pairs_per_block;
  cplx<T>* bufa = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufb = bufa + (size_t)PP * N;
  cplx<T>* stw = bufb + (size_t)PP * N;                        // twiddles, staged once per block
  T* rowadd = reinterpret_cast<T*>(stw + N / 2);               // [2 PP] wall terms of each row
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) stw[t] = tw[t];
  for (int t = threadIdx.x; t < 2 * PP; t += blockDim.x) {
    const int row = 2 * blockIdx.x * PP + t;
    const int y = row % Nyr;
    rowadd[t] = (y == 0 ? add0 : T(0)) + (y == Nyr - 1 ? add1 : T(0));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    const int v = idx >> logN, n = idx & (N - 1);
    const int ra = 2 * (blockIdx.x * PP + v), rb = ra + 1;
    T a = T(0), b = T(0);
    if (ra < R) a = scale * in[(size_t)ra * N + n] + rowadd[2 * v] + ((add0x && ra % Nyr == 0) ? add0x[n] : T(0));
    if (rb < R) b = scale * in[(size_t)rb * N + n] + rowadd[2 * v + 1] + ((add0x && rb % Nyr == 0) ? add0x[n] : T(0));
    bufa[idx] = cplx<T>{a, b};
  }
  __syncthreads();
  cplx<T>* r = fft_stockham(bufa, bufb, N, logN, PP, N, stw, false);
  const int M = N / 2 + 1;
  // idx / M by a float reciprocal: idx < 2^16, so (idx + 1/2) / M stays at
  // least 1/(2M) away from an integer, far beyond the rounding of the product
  const float invM = 1.0f / (float)M;
  for (int idx = threadIdx.x; idx < PP * M; idx += blockDim.x) {
    const int v = (int)(((float)idx + 0.5f) * invM), k = idx - v * M;
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    cplx<T> Zk = r[v * N + (k & (N - 1))];
    cplx<T> Zn = r[v * N + ((N - k) & (N - 1))];
    // A = (Z_k + conj Z_{N-k}) / 2,  B = (Z_k - conj Z_{N-k}) / (2i)
    cplx<T> A{T(0.5) * (Zk.re + Zn.re), T(0.5) * (Zk.im - Zn.im)};
    cplx<T> B{T(0.5) * (Zk.im + Zn.im), T(-0.5) * (Zk.re - Zn.re)};
    if (ra < R) out[(size_t)ra * Px + k] = A;
    if (rb < R) out[(size_t)rb * Px + k] = B;
  }
}

// Inverse of k_rfft_x (unnormalised): half spectra -> real rows times scale.
template <typename T>
__global__ void k_irfft_x(const cplx<T>* __restrict__ in, int R, int N, int logN, int Px, T* __restrict__ out,
                          T scale, const cplx<T>* __restrict__ tw, int pairs_per_block) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int PP = pairs_per_block;
  cplx<T>* bufa = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufb = bufa + (size_t)PP * N;
  cplx<T>* stw = bufb + (size_t)PP * N;                        // twiddles, staged once per block
  for (int t = threadIdx.x; t < N / 2; t += blockDim.x) stw[t] = tw[t];
  const int hN = N / 2;
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    const int v = idx >> logN, k = idx & (N - 1);
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    int kk = k <= hN ? k : N - k;
    cplx<T> A{T(0), T(0)}, B{T(0), T(0)};
    if (ra < R) A = in[(size_t)ra * Px + kk];
    if (rb < R) B = in[(size_t)rb * Px + kk];
    if (k > hN) { A.im = -A.im; B.im = -B.im; }
    bufa[idx] = cplx<T>{A.re - B.im, A.im + B.re};   // Z = A + i B
  }
  __syncthreads();
  cplx<T>* r = fft_stockham(bufa, bufb, N, logN, PP, N, stw, true);
  for (int idx = threadIdx.x; idx < PP * N; idx += blockDim.x) {
    const int v = idx >> logN, n = idx & (N - 1);
    int p = blockIdx.x * PP + v;
    int ra = 2 * p, rb = 2 * p + 1;
    cplx<T> z = r[idx];
    if (ra < R) out[(size_t)ra * N + n] = scale * z.re;
    if (rb < R) out[(size_t)rb * N + n] = scale * z.im;
  }
}

// ------------------------------------------------------------------------
// Register-resident transforms (the default for Nx >= 32 and every Nz).
//
// A length N = P G transform held by a group of G lanes, P values per lane:
// lane r holds x[r + G p], p < P.  Four steps: a P-point DFT over each
// lane's registers (register p then holds k2 = bitrev(p)), the twiddles
// W_N^(r k2), then a G-point DFT across the lanes (radix-2 stages on
// __shfl_xor, decimation in frequency), after which lane r, register p holds
// X[k2 + P bitrev(r)].  Only the real-pair split of the x
// transform and the reordering of its inverse go through shared memory.

// exp(-+2 pi i m / N) for 0 <= m < N from the half table tw[m], m < N/2.
template <typename T>
__device__ __forceinline__ cplx<T> twid(const cplx<T>* __restrict__ tw, int m, int N, bool inverse) {
  const int h = N >> 1;
  cplx<T> w = tw[m & (h - 1)];
  if (m & h) { w.re = -w.re; w.im = -w.im; }
  if (inverse) w.im = -w.im;
  return w;
}

template <int P>
__host__ __device__ constexpr int brev_c(int i) {
  int r = 0;
  for (int b = 1; b < P; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
  return r;
}

// P-point DFT of the registers, radix-2 decimation in frequency: natural
// order in, register p holds output brev_c<P>(p) (every register index is a
// compile-time constant, so the values stay in registers).
template <typename T, int P>
__device__ __forceinline__ void reg_dft(cplx<T> (&v)[P], const cplx<T>* __restrict__ tw, int N, bool inverse) {
#pragma unroll
  for (int half = P / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int i = 0; i < P; i += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const cplx<T> a = v[i + j], b = v[i + j + half];
        v[i + j] = cadd(a, b);
        const cplx<T> d = csub(a, b);
        v[i + j + half] = j == 0 ? d : cmul(d, twid(tw, j * (N / (2 * half)), N, inverse));
      }
    }
  }
}

// G-point DFT across the lanes r = 0..G-1 of a group (G = 16 or 32), one per
// register: after it lane r holds output bitrev(r).
template <typename T, int P>
__device__ __forceinline__ void lane_dft(cplx<T> (&v)[P], int r, int G, const cplx<T>* __restrict__ tw, int N,
                                         bool inverse) {
  for (int s = G >> 1; s >= 1; s >>= 1) {
    const bool hi = (r & s) != 0;
    const cplx<T> w = twid(tw, (r & (s - 1)) * (N / (2 * s)), N, inverse);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const cplx<T> u{__shfl_xor_sync(0xffffffffu, v[p].re, s), __shfl_xor_sync(0xffffffffu, v[p].im, s)};
      v[p] = hi ? cmul(csub(u, v[p]), w) : cadd(v[p], u);
    }
  }
}

// Forward real transform of two rows per warp (packed as one complex
// transform of length N = 32 P), half spectra out.  Input value = scale * in
// + the row's wall term (y == 0: add0, y == Nyr - 1: add1).
template <typename T, int P>
__global__ void k_rfft_x_w(const T* __restrict__ in, int R, int Px, cplx<T>* __restrict__ out, T scale, int Nyr,
                           T add0, T add1, const cplx<T>* __restrict__ tw, const T* __restrict__ add0x) {
  constexpr int N = 32 * P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  cplx<T>* sz = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)wib * 32 * (P + 1);
  const int ra = 2 * (blockIdx.x * (blockDim.x >> 5) + wib), rb = ra + 1;
  if (ra >= R) return;                       // whole warps
  const bool hasb = rb < R;
  const int ya = ra % Nyr, yb = rb % Nyr;
  const T adda = (ya == 0 ? add0 : T(0)) + (ya == Nyr - 1 ? add1 : T(0));
  const T addb = (yb == 0 ? add0 : T(0)) + (yb == Nyr - 1 ? add1 : T(0));
  const T* pa = in + (size_t)ra * N;
  const T* pb = in + (size_t)rb * N;
  // a bottom row may carry a term per column (the metal strip's wall data)
  const bool xa = add0x && ya == 0, xb = add0x && yb == 0;
  cplx<T> v[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int n = lane + 32 * p;
    v[p] = cplx<T>{scale * pa[n] + adda + (xa ? add0x[n] : T(0)),
                   hasb ? scale * pb[n] + addb + (xb ? add0x[n] : T(0)) : T(0)};
  }
  reg_dft<T, P>(v, tw, N, false);
#pragma unroll
  for (int p = 1; p < P; ++p) v[p] = cmul(v[p], twid(tw, lane * brev_c<P>(p), N, false));
  lane_dft<T, P>(v, lane, 32, tw, N, false);
  const int k1 = (int)(__brev((unsigned)lane) >> 27);
#pragma unroll
  for (int p = 0; p < P; ++p) sz[k1 * (P + 1) + brev_c<P>(p)] = v[p];
  __syncwarp();
  // A = (Z_k + conj Z_{N-k}) / 2,  B = (Z_k - conj Z_{N-k}) / (2i)
  for (int k = lane; k <= N / 2; k += 32) {
    const int kn = (N - k) & (N - 1);
    const cplx<T> Zk = sz[(k / P) * (P + 1) + (k % P)];
    const cplx<T> Zn = sz[(kn / P) * (P + 1) + (kn % P)];
    out[(size_t)ra * Px + k] = cplx<T>{T(0.5) * (Zk.re + Zn.re), T(0.5) * (Zk.im - Zn.im)};
    if (hasb) out[(size_t)rb * Px + k] = cplx<T>{T(0.5) * (Zk.im + Zn.im), T(-0.5) * (Zk.re - Zn.re)};
  }
}

// Inverse of k_rfft_x_w (unnormalised): half spectra -> real rows times scale.
template <typename T, int P>
__global__ void k_irfft_x_w(const cplx<T>* __restrict__ in, int R, int Px, T* __restrict__ out, T scale,
                            const cplx<T>* __restrict__ tw) {
  constexpr int N = 32 * P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  cplx<T>* sz = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)wib * 32 * (P + 1);
  const int ra = 2 * (blockIdx.x * (blockDim.x >> 5) + wib), rb = ra + 1;
  if (ra >= R) return;
  const bool hasb = rb < R;
  cplx<T> v[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int k = lane + 32 * p;
    const int kk = k <= N / 2 ? k : N - k;
    cplx<T> A = in[(size_t)ra * Px + kk];
    cplx<T> B = hasb ? in[(size_t)rb * Px + kk] : cplx<T>{T(0), T(0)};
    if (k > N / 2) { A.im = -A.im; B.im = -B.im; }
    v[p] = cplx<T>{A.re - B.im, A.im + B.re};      // Z = A + i B
  }
  reg_dft<T, P>(v, tw, N, true);
#pragma unroll
  for (int p = 1; p < P; ++p) v[p] = cmul(v[p], twid(tw, lane * brev_c<P>(p), N, true));
  lane_dft<T, P>(v, lane, 32, tw, N, true);
  const int k1 = (int)(__brev((unsigned)lane) >> 27);
#pragma unroll
  for (int p = 0; p < P; ++p) sz[k1 * (P + 1) + brev_c<P>(p)] = v[p];
  __syncwarp();
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int n = lane + 32 * p;
    const cplx<T> z = sz[(n / P) * (P + 1) + (n % P)];
    out[(size_t)ra * N + n] = scale * z.re;
    if (hasb) out[(size_t)rb * N + n] = scale * z.im;
  }
}



// The twiddles that one lane of a 32 P-point row transform uses, loaded
// once per thread by the persistent staged kernels (the per-row kernels read
// them from the table each time): the register stages (W_N^(j N / 2h) in the
// loop order of reg_dft), the inter-stage twiddles W_N^(lane bitrev(p)), and
// one per lane stage of lane_dft.
template <typename T, int P>
struct LaneTwiddles {
  static constexpr int NR = P > 1 ? P - 1 : 1;
  cplx<T> r[NR], m[P], l[5];
  __device__ __forceinline__ void load(const cplx<T>* __restrict__ tw, int lane, bool inverse) {
    constexpr int N = 32 * P;
    int k = 0;
#pragma unroll
    for (int half = P / 2; half >= 1; half >>= 1)
#pragma unroll
      for (int j = 1; j < half; ++j) r[k++] = twid(tw, j * (N / (2 * half)), N, inverse);
#pragma unroll
    for (int p = 0; p < P; ++p) m[p] = twid(tw, lane * brev_c<P>(p), N, inverse);
    int st = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) l[st++] = twid(tw, (lane & (s - 1)) * (N / (2 * s)), N, inverse);
  }
};

// reg_dft, lane twiddle, lane_dft with the twiddles in registers (G = 32).
template <typename T, int P>
__device__ __forceinline__ void row_dft(cplx<T> (&v)[P], const LaneTwiddles<T, P>& t, int lane) {
  int k = 0;
#pragma unroll
  for (int half = P / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int i = 0; i < P; i += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const cplx<T> a = v[i + j], b = v[i + j + half];
        v[i + j] = cadd(a, b);
        const cplx<T> d = csub(a, b);
        v[i + j + half] = j == 0 ? d : cmul(d, t.r[k + j - 1]);
      }
    }
    k += half > 1 ? half - 1 : 0;
  }
#pragma unroll
  for (int p = 1; p < P; ++p) v[p] = cmul(v[p], t.m[p]);
  int st = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1, ++st) {
    const bool hi = (lane & s) != 0;
    const cplx<T> w = t.l[st];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const cplx<T> u{__shfl_xor_sync(0xffffffffu, v[p].re, s), __shfl_xor_sync(0xffffffffu, v[p].im, s)};
      v[p] = hi ? cmul(csub(u, v[p]), w) : cadd(v[p], u);
    }
  }
}

// ------------------------------------------------------------------------
// Bulk-staged x transforms.  The rows of one transform launch lie back to
// back in memory, so a chunk of C = 2 W rows (W warps, one row pair each) is
// a single bulk copy into shared memory (the TMA engine's untiled form).  The
// CTAs are persistent (as many as fit on the SMs) and walk the chunks with
// the grid as stride, keeping XS_NB chunks in flight: while the warps
// transform chunk i out of shared memory, the next XS_NB - 1 chunks stream
// in.  The transform of a row pair is that of k_rfft_x_w / k_irfft_x_w.
// Shared memory: XS_NB barriers (32 bytes), XS_NB chunk buffers, and the
// per-warp real-pair scratch.
constexpr int XS_NB = 3;

// On a wait that ran out: flag it, let the copies still in flight land (each
// wait again bounded), and leave.
__device__ __forceinline__ void staged_abort(uint64_t* bar, int it, int nchunks, unsigned* fault) {
  for (int j = it; j < it + XS_NB; ++j) {
    const int cj = blockIdx.x + j * gridDim.x;
    if (cj < nchunks) mbar_wait(&bar[j % XS_NB], (unsigned)((j / XS_NB) & 1));
  }
  if (threadIdx.x == 0 && fault) atomicOr(fault, FAULT_ASYNC_WAIT);
}

template <typename T, int P>
__global__ void k_rfft_x_staged(const T* __restrict__ in, int R, int Px, cplx<T>* __restrict__ out, T scale,
                                int Nyr, T add0, T add1, const cplx<T>* __restrict__ tw,
                                const T* __restrict__ add0x, unsigned* __restrict__ fault) {
  constexpr int N = 32 * P;
  const int C = 2 * (blockDim.x >> 5);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  T* buf = reinterpret_cast<T*>(smem_raw + 32);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  cplx<T>* sz = reinterpret_cast<cplx<T>*>(buf + (size_t)XS_NB * C * N) + (size_t)wib * 32 * (P + 1);
  const int nchunks = (R + C - 1) / C;
  LaneTwiddles<T, P> twl;
  twl.load(tw, lane, false);
  auto load = [&](int c, int b) {
    const int rows = min(C, R - c * C);
    bulk_load(buf + (size_t)b * C * N, in + (size_t)c * C * N, (unsigned)((size_t)rows * N * sizeof(T)), &bar[b]);
  };
  if (threadIdx.x == 0) {
    for (int b = 0; b < XS_NB; ++b) mbar_init(&bar[b], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int b = 0; b < XS_NB; ++b)
      if (blockIdx.x + b * (int)gridDim.x < nchunks) load(blockIdx.x + b * gridDim.x, b);
  int it = 0;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x, ++it) {
    const int b = it % XS_NB;
    const bool ok = mbar_wait(&bar[b], (unsigned)((it / XS_NB) & 1));
    if (!__syncthreads_and(ok)) {
      staged_abort(bar, it, nchunks, fault);
      return;
    }
    const int ra = c * C + 2 * wib, rb = ra + 1;
    if (ra < R) {
      const bool hasb = rb < R;
      const int ya = ra % Nyr, yb = rb % Nyr;
      const T adda = (ya == 0 ? add0 : T(0)) + (ya == Nyr - 1 ? add1 : T(0));
      const T addb = (yb == 0 ? add0 : T(0)) + (yb == Nyr - 1 ? add1 : T(0));
      const T* pa = buf + (size_t)b * C * N + (size_t)(2 * wib) * N;
      const T* pb = pa + N;
      const bool xa = add0x && ya == 0, xb = add0x && yb == 0;
      cplx<T> v[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int n = lane + 32 * p;
        v[p] = cplx<T>{scale * pa[n] + adda + (xa ? add0x[n] : T(0)),
                       hasb ? scale * pb[n] + addb + (xb ? add0x[n] : T(0)) : T(0)};
      }
      row_dft<T, P>(v, twl, lane);
      const int k1 = (int)(__brev((unsigned)lane) >> 27);
#pragma unroll
      for (int p = 0; p < P; ++p) sz[k1 * (P + 1) + brev_c<P>(p)] = v[p];
      __syncwarp();
      for (int k = lane; k <= N / 2; k += 32) {
        const int kn = (N - k) & (N - 1);
        const cplx<T> Zk = sz[(k / P) * (P + 1) + (k % P)];
        const cplx<T> Zn = sz[(kn / P) * (P + 1) + (kn % P)];
        out[(size_t)ra * Px + k] = cplx<T>{T(0.5) * (Zk.re + Zn.re), T(0.5) * (Zk.im - Zn.im)};
        if (hasb) out[(size_t)rb * Px + k] = cplx<T>{T(0.5) * (Zk.im + Zn.im), T(-0.5) * (Zk.re - Zn.re)};
      }
    }
    __syncthreads();   // every warp is done with buffer b (and with its scratch)
    if (threadIdx.x == 0) {
      const int cn = c + XS_NB * gridDim.x;
      if (cn < nchunks) {
        async_proxy_fence();
        load(cn, b);
      }
    }
  }
}

template <typename T, int P>
__global__ void k_irfft_x_staged(const cplx<T>* __restrict__ in, int R, int Px, T* __restrict__ out, T scale,
                                 const cplx<T>* __restrict__ tw, unsigned* __restrict__ fault) {
  constexpr int N = 32 * P;
  const int C = 2 * (blockDim.x >> 5);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw + 32);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  cplx<T>* sz = buf + (size_t)XS_NB * C * Px + (size_t)wib * 32 * (P + 1);
  const int nchunks = (R + C - 1) / C;
  LaneTwiddles<T, P> twl;
  twl.load(tw, lane, true);
  auto load = [&](int c, int b) {
    const int rows = min(C, R - c * C);
    bulk_load(buf + (size_t)b * C * Px, in + (size_t)c * C * Px, (unsigned)((size_t)rows * Px * sizeof(cplx<T>)),
              &bar[b]);
  };
  if (threadIdx.x == 0) {
    for (int b = 0; b < XS_NB; ++b) mbar_init(&bar[b], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int b = 0; b < XS_NB; ++b)
      if (blockIdx.x + b * (int)gridDim.x < nchunks) load(blockIdx.x + b * gridDim.x, b);
  int it = 0;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x, ++it) {
    const int b = it % XS_NB;
    const bool ok = mbar_wait(&bar[b], (unsigned)((it / XS_NB) & 1));
    if (!__syncthreads_and(ok)) {
      staged_abort(bar, it, nchunks, fault);
      return;
    }
    const int ra = c * C + 2 * wib, rb = ra + 1;
    if (ra < R) {
      const bool hasb = rb < R;
      const cplx<T>* ia = buf + (size_t)b * C * Px + (size_t)(2 * wib) * Px;
      const cplx<T>* ib = ia + Px;
      cplx<T> v[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int k = lane + 32 * p;
        const int kk = k <= N / 2 ? k : N - k;
        cplx<T> A = ia[kk];
        cplx<T> B = hasb ? ib[kk] : cplx<T>{T(0), T(0)};
        if (k > N / 2) { A.im = -A.im; B.im = -B.im; }
        v[p] = cplx<T>{A.re - B.im, A.im + B.re};      // Z = A + i B
      }
      row_dft<T, P>(v, twl, lane);
      const int k1 = (int)(__brev((unsigned)lane) >> 27);
#pragma unroll
      for (int p = 0; p < P; ++p) sz[k1 * (P + 1) + brev_c<P>(p)] = v[p];
      __syncwarp();
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int n = lane + 32 * p;
        const cplx<T> z = sz[(n / P) * (P + 1) + (n % P)];
        out[(size_t)ra * N + n] = scale * z.re;
        if (hasb) out[(size_t)rb * N + n] = scale * z.im;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int cn = c + XS_NB * gridDim.x;
      if (cn < nchunks) {
        async_proxy_fence();
        load(cn, b);
      }
    }
  }
}

// Complex transform along z, in place: 32 / G x-mode columns per warp, G
// lanes per column (G = 8 for float: 4 columns x 8 bytes fill a 32-byte
// sector per z row; G = 16 for double), M = Nz / G values per lane.
// blockIdx.y = y row, blockIdx.z = field (mac: the three MAC spectra
// u | v | w with Ny, Ny + 1, Ny rows).
template <typename T, int G, int M>
__global__ void k_fft_z_w(cplx<T>* __restrict__ data, int Nyr, int Px, int Nxh, int inverse,
                          const cplx<T>* __restrict__ tw, size_t field_stride, int mac) {
  constexpr int Nz = G * M;
  constexpr int LOGG = G == 8 ? 3 : (G == 16 ? 4 : 5);
  const int lane = threadIdx.x & 31, r = lane & (G - 1);
  const int kx = (32 / G) * (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) + lane / G;
  cplx<T>* base = data + blockIdx.z * field_stride;
  if (mac) {
    const int Ny = Nyr;
    if (blockIdx.z == 1) { base = data + (size_t)Nz * Ny * Px; Nyr = Ny + 1; }
    else if (blockIdx.z == 2) { base = data + (size_t)Nz * (2 * Ny + 1) * Px; }
    else { base = data; }
  }
  const int y = blockIdx.y;
  if (y >= Nyr) return;                      // whole blocks
  const bool ok = kx < Nxh;
  cplx<T>* col = base + (size_t)y * Px + kx;
  const size_t zs = (size_t)Nyr * Px;
  cplx<T> v[M];
#pragma unroll
  for (int m = 0; m < M; ++m) v[m] = ok ? col[(size_t)(r + G * m) * zs] : cplx<T>{T(0), T(0)};
  const bool inv = inverse != 0;
  reg_dft<T, M>(v, tw, Nz, inv);
#pragma unroll
  for (int p = 1; p < M; ++p) v[p] = cmul(v[p], twid(tw, r * brev_c<M>(p), Nz, inv));
  lane_dft<T, M>(v, r, G, tw, Nz, inv);
  const int k1 = (int)(__brev((unsigned)r) >> (32 - LOGG));
  if (ok) {
#pragma unroll
    for (int p = 0; p < M; ++p) col[(size_t)(brev_c<M>(p) + M * k1) * zs] = v[p];
  }
}


// ------------------------------------------------------------------------
// TMA-tiled z transform (single precision, 16 <= Nz <= 256).  One CTA per
// (32 x-modes, y row, field): a 3-D tensor map over the field's spectrum
// ([Px complex as 2 Px floats][Nyr][Nz]) lets one cp.async.bulk.tensor copy
// bring the whole [Nz][32] column tile into shared memory, completing on an
// mbarrier.  The CTA's 8 warps then run the Nz = N1 x 16 point transform as
// two passes of register DFTs with the lanes across the 32 columns, so each
// access to the tile is one conflict-free row: pass 1, for each i1, the
// 16-point DFT of x[i1 + N1 m] over m times W^(i1 k2), back into the same
// rows of the tile; pass 2, for each k2, the N1-point DFT over i1, written
// as X[k2 + 16 k1] straight to the spectrum (one coalesced 256-byte row per
// warp access; padding columns are skipped).  Several CTAs per SM keep
// their tiles in flight.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, unsigned bytes,
                                            uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

struct ZField {
  cplx<float>* base;   // the field's spectrum [Nz][Nyr][Px]
  int Nyr;
};

template <int N1>
__global__ void __launch_bounds__(256) k_fft_z_tma(const __grid_constant__ CUtensorMap m0,
                                                   const __grid_constant__ CUtensorMap m1,
                                                   const __grid_constant__ CUtensorMap m2, ZField f0, ZField f1,
                                                   ZField f2, int Px, int Nxh, int inverse,
                                                   const cplx<float>* __restrict__ tw, unsigned* __restrict__ fault) {
  constexpr int N2 = 16, Nz = N1 * N2;
  const int field = blockIdx.z;
  const ZField F = field == 0 ? f0 : (field == 1 ? f1 : f2);
  const CUtensorMap* map = field == 0 ? &m0 : (field == 1 ? &m1 : &m2);
  const int kx0 = blockIdx.x * 32, y = blockIdx.y;
  if (y >= F.Nyr) return;                           // whole blocks
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  cplx<float>* tile = reinterpret_cast<cplx<float>*>(smem_raw + 128);     // [Nz][32]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) tma_load_3d(tile, map, 2 * kx0, y, 0, (unsigned)(Nz * 32 * sizeof(cplx<float>)), bar);
  const bool ok = mbar_wait(bar, 0);
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) {
      if (fault) atomicOr(fault, FAULT_ASYNC_WAIT);
      mbar_wait(bar, 0);                            // let the copy land before the CTA leaves
    }
    return;
  }
  const bool inv = inverse != 0;
  for (int i1 = w; i1 < N1; i1 += nw) {
    cplx<float> v[N2];
#pragma unroll
    for (int m = 0; m < N2; ++m) v[m] = tile[(i1 + N1 * m) * 32 + lane];
    reg_dft<float, N2>(v, tw, Nz, inv);
#pragma unroll
    for (int p = 0; p < N2; ++p) {
      const int k2 = brev_c<N2>(p);
      tile[(i1 + N1 * k2) * 32 + lane] = p == 0 ? v[p] : cmul(v[p], twid(tw, i1 * k2, Nz, inv));
    }
  }
  __syncthreads();
  const bool col_ok = kx0 + lane < Nxh;
  cplx<float>* col = F.base + (size_t)y * Px + kx0 + lane;
  const size_t zs = (size_t)F.Nyr * Px;
  for (int k2 = w; k2 < N2; k2 += nw) {
    cplx<float> u[N1];
#pragma unroll
    for (int i1 = 0; i1 < N1; ++i1) u[i1] = tile[(i1 + N1 * k2) * 32 + lane];
    reg_dft<float, N1>(u, tw, Nz, inv);
    if (col_ok) {
#pragma unroll
      for (int p = 0; p < N1; ++p) col[(size_t)(k2 + N2 * brev_c<N1>(p)) * zs] = u[p];
    }
  }
}

}  // namespace

// Default launch shapes of the transforms (discos_tune_transforms may replace
// them): 1024 / Nx row pairs per x-block on 256 threads; 8 columns per
// z-block (small blocks keep the launch within one wave at typical sizes),
// halved while the two buffers exceed 140 KB.
int default_fx_pairs(int Nx) {
  int pp = 1024 / Nx;
  return pp < 1 ? 1 : pp;
}
int max_tile_z(int Nz, size_t elem) {
  int tk = 16;
  while (tk > 1 && 2 * (size_t)tk * (Nz + 1) * elem > 140 * 1024) tk >>= 1;
  return tk;
}
// one radix-4 butterfly per thread: TK Nz / 4 threads, 64..256
int fz_threads(int TK, int Nz) {
  int t = TK * Nz / 4;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}
int default_tile_z(int Nz, size_t elem) {
  int tk = max_tile_z(Nz, elem);
  return tk > 8 ? 8 : tk;
}


// Register-resident x transforms for Nx >= 32: fx_pp row pairs (warps) per
// block, within 48 KB of shared memory.
template <typename T>
int x_warps_per_block(const Params& P) {
  const int Pn = P.Nx / 32;
  const size_t per_warp = 32 * (size_t)(Pn + 1) * sizeof(cplx<T>);
  int w = P.fx_pp < 1 ? 1 : (P.fx_pp > 16 ? 16 : P.fx_pp);
  while (w > 1 && w * per_warp > 48 * 1024) --w;
  return w;
}


// Staged x transforms: W warps per CTA so that a chunk (2 W rows) is about
// 16 KB (1 <= W <= 8); as many CTAs as fit on the SMs, at most one per chunk.
int staged_warps(size_t row_bytes) {
  int w = (int)(8192 / row_bytes);
  return w < 1 ? 1 : (w > 8 ? 8 : w);
}

// Persistent grid for kernel Kern with the given block and shared memory:
// the opt-in shared-memory attribute is set once per device, and the CTAs
// per SM come from the occupancy calculator.
template <auto Kern>
cudaError_t persistent_grid(int threads, size_t smem, int* grid) {
  static std::atomic<unsigned long long> attr_done{0};
  static int per_sm[64] = {0};
  static int sms[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!(attr_done.load() & (1ull << dev))) {
    e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[dev], Kern, threads, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    attr_done.fetch_or(1ull << dev);
  }
  const int b = per_sm[dev] < 1 ? 1 : per_sm[dev];
  *grid = b * (sms[dev] < 1 ? 1 : sms[dev]);
  return cudaSuccess;
}

template <typename T, int PP>
cudaError_t rfft_x_staged(const Params& P, const T* in, int R, cplx<T>* out, T scale, int Nyr, T add0, T add1,
                          const cplx<T>* tw, const T* add0x, cudaStream_t s) {
  constexpr int N = 32 * PP;
  const int W = staged_warps(N * sizeof(T)), C = 2 * W;
  const size_t sm = 32 + XS_NB * (size_t)C * N * sizeof(T) + (size_t)W * 32 * (PP + 1) * sizeof(cplx<T>);
  int grid = 0;
  cudaError_t e = persistent_grid<k_rfft_x_staged<T, PP>>(32 * W, sm, &grid);
  if (e != cudaSuccess) return e;
  const int nchunks = (R + C - 1) / C;
  if (grid > nchunks) grid = nchunks;
  k_rfft_x_staged<T, PP><<<grid, 32 * W, sm, s>>>(in, R, P.Px, out, scale, Nyr, add0, add1, tw, add0x, P.fault);
  return cudaSuccess;
}

template <typename T, int PP>
cudaError_t irfft_x_staged(const Params& P, const cplx<T>* in, int R, T* out, T scale, const cplx<T>* tw,
                           cudaStream_t s) {
  const int W = staged_warps(P.Px * sizeof(cplx<T>)), C = 2 * W;
  const size_t sm = 32 + XS_NB * (size_t)C * P.Px * sizeof(cplx<T>) + (size_t)W * 32 * (PP + 1) * sizeof(cplx<T>);
  int grid = 0;
  cudaError_t e = persistent_grid<k_irfft_x_staged<T, PP>>(32 * W, sm, &grid);
  if (e != cudaSuccess) return e;
  const int nchunks = (R + C - 1) / C;
  if (grid > nchunks) grid = nchunks;
  k_irfft_x_staged<T, PP><<<grid, 32 * W, sm, s>>>(in, R, P.Px, out, scale, tw, P.fault);
  return cudaSuccess;
}

// The staged path needs 16-byte aligned rows in and out (always true for
// the library's own buffers; a caller's grid may be offset).
bool staged_ok(const Params& P, const void* a, const void* b) {
  return P.fx_staged && P.Nx >= 32 && (((uintptr_t)a | (uintptr_t)b) & 15u) == 0;
}

#define DISCOS_X_STAGED(FN, ...)                                      \
  switch (P.Nx) {                                                     \
    case 32: e = FN<T, 1>(__VA_ARGS__); break;                        \
    case 64: e = FN<T, 2>(__VA_ARGS__); break;                        \
    case 128: e = FN<T, 4>(__VA_ARGS__); break;                       \
    case 256: e = FN<T, 8>(__VA_ARGS__); break;                       \
    default: e = FN<T, 16>(__VA_ARGS__); break;                       \
  }

#define DISCOS_X_DISPATCH(KERNEL, ...)                                                        \
  switch (P.Nx) {                                                                             \
    case 32: KERNEL<T, 1><<<nb, 32 * wpb, sm, s>>>(__VA_ARGS__); break;                       \
    case 64: KERNEL<T, 2><<<nb, 32 * wpb, sm, s>>>(__VA_ARGS__); break;                       \
    case 128: KERNEL<T, 4><<<nb, 32 * wpb, sm, s>>>(__VA_ARGS__); break;                      \
    case 256: KERNEL<T, 8><<<nb, 32 * wpb, sm, s>>>(__VA_ARGS__); break;                      \
    default: KERNEL<T, 16><<<nb, 32 * wpb, sm, s>>>(__VA_ARGS__); break;                      \
  }

// Shared by the Poisson and Stokes paths.
template <typename T>
cudaError_t fft_x_forward(const Params& P, const T* in, int R, cplx<T>* out, T scale, int Nyr, T add0, T add1,
                          const cplx<T>* tw, cudaStream_t s, const T* add0x) {
  int N = P.Nx, logN = 31 - __builtin_clz((unsigned)N);
  const int pairs = (R + 1) / 2;
  probe_begin(PROBE_FFT_X, s);
  if (staged_ok(P, in, out)) {
    cudaError_t e = cudaSuccess;
    DISCOS_X_STAGED(rfft_x_staged, P, in, R, out, scale, Nyr, add0, add1, tw, add0x, s)
    if (e != cudaSuccess) {
      probe_end(PROBE_FFT_X, s);
      return e;
    }
  } else if (N >= 32) {
    const int wpb = x_warps_per_block<T>(P);
    const int nb = (pairs + wpb - 1) / wpb;
    const size_t sm = (size_t)wpb * 32 * (N / 32 + 1) * sizeof(cplx<T>);
    DISCOS_X_DISPATCH(k_rfft_x_w, in, R, P.Px, out, scale, Nyr, add0, add1, tw, add0x)
  } else {
    int pp = P.fx_pp;
    int nb = (pairs + pp - 1) / pp;
    size_t sm = (2 * (size_t)pp * N + N / 2) * sizeof(cplx<T>) + 2 * (size_t)pp * sizeof(T);
    k_rfft_x<T><<<nb, P.fx_threads, sm, s>>>(in, R, N, logN, P.Px, out, scale, Nyr, add0, add1, tw, pp, add0x);
  }
  count_launches(1);
  probe_end(PROBE_FFT_X, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_x_inverse(const Params& P, const cplx<T>* in, int R, T* out, T scale, const cplx<T>* tw,
                          cudaStream_t s) {
  int N = P.Nx, logN = 31 - __builtin_clz((unsigned)N);
  const int pairs = (R + 1) / 2;
  probe_begin(PROBE_FFT_X, s);
  if (staged_ok(P, in, out)) {
    cudaError_t e = cudaSuccess;
    DISCOS_X_STAGED(irfft_x_staged, P, in, R, out, scale, tw, s)
    if (e != cudaSuccess) {
      probe_end(PROBE_FFT_X, s);
      return e;
    }
  } else if (N >= 32) {
    const int wpb = x_warps_per_block<T>(P);
    const int nb = (pairs + wpb - 1) / wpb;
    const size_t sm = (size_t)wpb * 32 * (N / 32 + 1) * sizeof(cplx<T>);
    DISCOS_X_DISPATCH(k_irfft_x_w, in, R, P.Px, out, scale, tw)
  } else {
    int pp = P.fx_pp;
    int nb = (pairs + pp - 1) / pp;
    size_t sm = (2 * (size_t)pp * N + N / 2) * sizeof(cplx<T>);
    k_irfft_x<T><<<nb, P.fx_threads, sm, s>>>(in, R, N, logN, P.Px, out, scale, tw, pp);
  }
  count_launches(1);
  probe_end(PROBE_FFT_X, s);
  return cudaGetLastError();
}
#undef DISCOS_X_DISPATCH
#undef DISCOS_X_STAGED

// z transforms: fz_tk x-mode columns per block (rounded up to whole warps).
template <typename T, int G>
void fft_z_dispatch(const Params& P, dim3 grid, int threads, cplx<T>* data, int Nyr, int inv, const cplx<T>* tw,
                    size_t field_stride, int mac, cudaStream_t s) {
  switch (P.Nz / G) {
    case 1: k_fft_z_w<T, G, 1><<<grid, threads, 0, s>>>(data, Nyr, P.Px, P.Nxh, inv, tw, field_stride, mac); break;
    case 2: k_fft_z_w<T, G, 2><<<grid, threads, 0, s>>>(data, Nyr, P.Px, P.Nxh, inv, tw, field_stride, mac); break;
    case 4: k_fft_z_w<T, G, 4><<<grid, threads, 0, s>>>(data, Nyr, P.Px, P.Nxh, inv, tw, field_stride, mac); break;
    case 8: k_fft_z_w<T, G, 8><<<grid, threads, 0, s>>>(data, Nyr, P.Px, P.Nxh, inv, tw, field_stride, mac); break;
    case 16: k_fft_z_w<T, G, 16><<<grid, threads, 0, s>>>(data, Nyr, P.Px, P.Nxh, inv, tw, field_stride, mac); break;
    default: k_fft_z_w<T, G, 32><<<grid, threads, 0, s>>>(data, Nyr, P.Px, P.Nxh, inv, tw, field_stride, mac); break;
  }
}


// The driver's tensor-map encoder, fetched once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::atomic<int> state{0};
  if (state.load() == 0) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess && p)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    state.store(fn ? 1 : 2);
  }
  return fn;
}

// Tensor map of one field's spectrum [Nz][Nyr][Px] (complex as 2 floats),
// box [32 complex][1][Nz].
bool encode_z_map(CUtensorMap* map, cplx<float>* base, int Px, int Nyr, int Nz) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * Px, (cuuint64_t)Nyr, (cuuint64_t)Nz};
  const cuuint64_t strides[2] = {(cuuint64_t)Px * sizeof(cplx<float>), (cuuint64_t)Nyr * Px * sizeof(cplx<float>)};
  const cuuint32_t box[3] = {64, 1, (cuuint32_t)Nz};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N1>
cudaError_t fft_z_tma_launch(const Params& P, const ZField* f, int nfields, int grid_y, bool inverse,
                             const cplx<float>* tw, cudaStream_t s) {
  CUtensorMap m[3];
  for (int i = 0; i < 3; ++i) {
    const ZField& g = f[i < nfields ? i : 0];
    if (!encode_z_map(&m[i], g.base, P.Px, g.Nyr, P.Nz)) return cudaErrorNotSupported;
  }
  const size_t sm = 128 + (size_t)P.Nz * 32 * sizeof(cplx<float>);
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !(done.load() & (1ull << dev))) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_z_tma<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    done.fetch_or(1ull << dev);
  }
  dim3 grid((P.Nxh + 31) / 32, grid_y, nfields);
  k_fft_z_tma<N1><<<grid, 256, sm, s>>>(m[0], m[1], m[2], f[0], f[nfields > 1 ? 1 : 0], f[nfields > 2 ? 2 : 0], P.Px,
                                         P.Nxh, inverse ? 1 : 0, tw, P.fault);
  return cudaGetLastError();
}

// The tiled z transform applies to single-precision spectra with
// 16 <= Nz <= 256 whose rows start on 16-byte boundaries.
bool z_tma_ok(const Params& P, const void* data) {
  return P.fz_tma && P.Nz >= 16 && P.Nz <= 256 && ((uintptr_t)data & 15u) == 0 && tensor_map_encoder() != nullptr;
}

cudaError_t fft_z_tma(const Params& P, const ZField* f, int nfields, int grid_y, bool inverse, const cplx<float>* tw,
                      cudaStream_t s) {
  switch (P.Nz) {
    case 16: return fft_z_tma_launch<1>(P, f, nfields, grid_y, inverse, tw, s);
    case 32: return fft_z_tma_launch<2>(P, f, nfields, grid_y, inverse, tw, s);
    case 64: return fft_z_tma_launch<4>(P, f, nfields, grid_y, inverse, tw, s);
    case 128: return fft_z_tma_launch<8>(P, f, nfields, grid_y, inverse, tw, s);
    default: return fft_z_tma_launch<16>(P, f, nfields, grid_y, inverse, tw, s);
  }
}

template <typename T>
cudaError_t fft_z_launch(const Params& P, cplx<T>* data, int Nyr, int grid_y, int nfields, size_t field_stride,
                         bool inverse, const cplx<T>* tw, int mac, cudaStream_t s) {
  // lanes per column: 8 (float, Nz <= 256), else 16; never more than Nz
  int G = (sizeof(T) == 4 && P.Nz <= 256) ? 8 : 16;
  if (G > P.Nz) G = P.Nz;
  const int cpw = 32 / G;
  const int wpb = P.fz_tk <= cpw ? 1 : P.fz_tk / cpw;
  dim3 grid((P.Nxh + cpw * wpb - 1) / (cpw * wpb), grid_y, nfields);
  const int inv = inverse ? 1 : 0;
  probe_begin(PROBE_FFT_Z, s);
  if constexpr (std::is_same<T, float>::value) {
    if (z_tma_ok(P, data)) {
      ZField f[3];
      int nf = nfields;
      if (mac) {
        const int Ny = Nyr;
        f[0] = ZField{data, Ny};
        f[1] = ZField{data + (size_t)P.Nz * Ny * P.Px, Ny + 1};
        f[2] = ZField{data + (size_t)P.Nz * (2 * Ny + 1) * P.Px, Ny};
        nf = 3;
      } else {
        for (int i = 0; i < nfields && i < 3; ++i) f[i] = ZField{data + (size_t)i * field_stride, Nyr};
      }
      cudaError_t e = nf <= 3 ? fft_z_tma(P, f, nf, grid_y, inverse, tw, s) : cudaErrorNotSupported;
      if (e == cudaSuccess) {
        count_launches(1);
        probe_end(PROBE_FFT_Z, s);
        return cudaSuccess;
      }
      if (e != cudaErrorNotSupported) {
        probe_end(PROBE_FFT_Z, s);
        return e;
      }
      (void)cudaGetLastError();
    }
  }
  if (G == 8) fft_z_dispatch<T, 8>(P, grid, 32 * wpb, data, Nyr, inv, tw, field_stride, mac, s);
  else fft_z_dispatch<T, 16>(P, grid, 32 * wpb, data, Nyr, inv, tw, field_stride, mac, s);
  count_launches(1);
  probe_end(PROBE_FFT_Z, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_z(const Params& P, cplx<T>* data, int Nyr, int nfields, size_t field_stride, bool inverse,
                  const cplx<T>* tw, cudaStream_t s) {
  return fft_z_launch<T>(P, data, Nyr, Nyr, nfields, field_stride, inverse, tw, 0, s);
}

template <typename T>
cudaError_t fft_z_mac(const Params& P, cplx<T>* data, bool inverse, const cplx<T>* tw, cudaStream_t s) {
  return fft_z_launch<T>(P, data, P.Ny, P.Ny + 1, 3, 0, inverse, tw, 1, s);
}

// One transform-solve-transform pass: phi = A^-1 (scale rho + wall terms)
// with the ghost-cell terms add0 / add1 on the wall rows.
template <typename T>
cudaError_t poisson_pass(const Params& P, Workspace& W, const T* rho, T* phi, T scale, T add0, T add1,
                         cudaStream_t s, const T* add0x) {
  const int Ny = P.Ny, Nz = P.Nz;
  cplx<T>* S = reinterpret_cast<cplx<T>*>(W.spec);
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(W.tw_x);
  const cplx<T>* twz = reinterpret_cast<const cplx<T>*>(W.tw_z);
  cudaError_t e = fft_x_forward<T>(P, rho, Nz * Ny, S, scale, Ny, add0, add1, twx, s, add0x);
  if (e != cudaSuccess) return e;
  e = fft_z<T>(P, S, Ny, 1, 0, false, twz, s);
  if (e != cudaSuccess) return e;
  e = launch_poisson_y<T>(P, W, S, s);
  if (e != cudaSuccess) return e;
  e = fft_z<T>(P, S, Ny, 1, 0, true, twz, s);
  if (e != cudaSuccess) return e;
  return fft_x_inverse<T>(P, S, Nz * Ny, phi, T(1), twx, s);
}

template <typename T>
cudaError_t launch_poisson(const Params& P, Workspace& W, const T* rho, T* phi, cudaStream_t s) {
  const double fourpi_lB = 4.0 * M_PI * P.lB;
  // ghost-cell terms of the wall rows (Eqs. esbc1, esbc3)
  const T add0 = P.bc[0] == DISCOS_BC_DIRICHLET ? T(2.0 * P.phi_b[0]) : T(-P.slope[0]);
  const T add1 = P.bc[1] == DISCOS_BC_DIRICHLET ? T(2.0 * P.phi_b[1]) : T(P.slope[1]);
  if (P.strip) return launch_poisson_strip<T>(P, W, rho, phi, T(fourpi_lB), add1, s);
  const int sweeps = (sizeof(T) == sizeof(float) && W.rref) ? P.max_refine : 0;
  if (sweeps == 0) return poisson_pass<T>(P, W, rho, phi, T(fourpi_lB), add0, add1, s, static_cast<const T*>(nullptr));
  // mixed precision with residual refinement: keep rho (phi may alias it),
  // solve, then correct with the double-precision residual (k_refine.cu); the
  // corrections accumulate in double, so the residual can fall below the
  // rounding of a single-precision potential
  const size_t G = (size_t)P.Nx * P.Ny * P.Nz;
  T* rho_keep = reinterpret_cast<T*>(W.rref);
  T* res = reinterpret_cast<T*>(W.rres);
  cudaError_t e = cudaMemcpyAsync(rho_keep, rho, sizeof(T) * G, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_fill_zero<double>(W.rnorm, 2 * (DISCOS_MAX_REFINE + 1), s);
  if (e == cudaSuccess) e = poisson_pass<T>(P, W, rho_keep, phi, T(fourpi_lB), add0, add1, s, static_cast<const T*>(nullptr));
  if (e == cudaSuccess) e = launch_convert<double, T>(W.phi64, phi, G, s);
  for (int it = 0; it < sweeps && e == cudaSuccess; ++it) {
    e = launch_poisson_residual<T, double>(P, rho_keep, W.phi64, res, W.rnorm + 2 * it, s);
    if (e == cudaSuccess) e = poisson_pass<T>(P, W, res, res, T(1), T(0), T(0), s, static_cast<const T*>(nullptr));
    if (e == cudaSuccess) e = launch_accumulate<T>(W.phi64, res, G, s);
  }
  if (e == cudaSuccess) e = launch_poisson_residual<T, double>(P, rho_keep, W.phi64, (T*)nullptr, W.rnorm + 2 * sweeps, s);
  if (e == cudaSuccess) e = launch_convert<T, double>(phi, W.phi64, G, s);
  return e;
}

// Launch-shape autotuner of the transforms: times each candidate shape of the
// x transform (row pairs per block, threads) and of the z transform (columns
// per block) on the handle's own potential and spectrum buffers at the
// Poisson sizes, and keeps the fastest in P.  Blocks until done.
template <typename T>
cudaError_t tune_transforms_t(Params& P, Workspace& W, cudaStream_t s, float* best_ms) {
  const int N = P.Nx, R = P.Nz * P.Ny;
  T* grid = reinterpret_cast<T*>(W.phi);
  cplx<T>* S = reinterpret_cast<cplx<T>*>(W.spec);
  const cplx<T>* twx = reinterpret_cast<const cplx<T>*>(W.tw_x);
  const cplx<T>* twz = reinterpret_cast<const cplx<T>*>(W.tw_z);
  cudaError_t e = launch_fill_zero<T>(grid, (size_t)P.Nx * P.Ny * P.Nz, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto time_it = [&](auto&& launch) -> float {
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 1e30f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    return ms / 10.0f;
  };
  Params Q = P;
  Q.fx_staged = 0;
  float bx = 1e30f, bz = 1e30f;
  int best_pp = P.fx_pp, best_th = P.fx_threads, best_tk = P.fz_tk;
  int last_pp = 0;
  for (int vals = 128; vals <= 2048 && e == cudaSuccess; vals *= 2) {
    const int pp = vals / N < 1 ? 1 : vals / N;
    if (pp == last_pp) continue;
    if ((2 * (size_t)pp * N + N / 2) * sizeof(cplx<T>) + 2 * (size_t)pp * sizeof(T) > 48 * 1024) break;
    last_pp = pp;
    int th = pp * N / 4;
    th = th < 32 ? 32 : (th > 256 ? 256 : th);
    Q.fx_pp = pp;
    Q.fx_threads = th;
    const float ms = time_it([&] { return fft_x_forward<T>(Q, grid, R, S, T(1), P.Ny, T(0), T(0), twx, s, nullptr); });
    if (ms < bx) { bx = ms; best_pp = pp; best_th = th; }
  }
  // the bulk-staged kernel (launch shape fixed by its chunk size)
  bool best_staged = false;
  if (N >= 32 && e == cudaSuccess) {
    Q = P;
    Q.fx_staged = 1;
    const float ms = time_it([&] { return fft_x_forward<T>(Q, grid, R, S, T(1), P.Ny, T(0), T(0), twx, s, nullptr); });
    if (ms < bx) { bx = ms; best_staged = true; }
  }
  // z: at least one 32-byte sector of consecutive x-modes per row access
  // (4 columns in float, 2 in double); narrower tiles can win on an
  // L2-resident trial spectrum and lose on the step's larger ones.  With a
  // fluid the trial is the three-field Stokes spectrum, the largest one.
  Q = P;
  Q.fz_tma = 0;
  const int tk0 = (int)(32 / sizeof(cplx<T>));
  const bool mac = W.st_l1 != nullptr;   // the Stokes factors exist only with a fluid
  bool best_tma = false;
  if (std::is_same<T, float>::value && P.Nz >= 16 && P.Nz <= 256 && e == cudaSuccess) {
    Q.fz_tma = 1;
    const float ms = time_it([&] {
      return mac ? fft_z_mac<T>(Q, S, false, twz, s) : fft_z<T>(Q, S, P.Ny, 1, 0, false, twz, s);
    });
    if (ms < bz) { bz = ms; best_tma = true; }
    Q.fz_tma = 0;
  }
  for (int tk = tk0; tk <= max_tile_z(P.Nz, sizeof(cplx<T>)) && e == cudaSuccess; tk *= 2) {
    Q.fz_tk = tk;
    const float ms = time_it([&] {
      return mac ? fft_z_mac<T>(Q, S, false, twz, s) : fft_z<T>(Q, S, P.Ny, 1, 0, false, twz, s);
    });
    if (ms < bz) { bz = ms; best_tk = tk; best_tma = false; }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  P.fx_pp = best_pp;
  P.fx_threads = best_th;
  P.fx_staged = best_staged ? 1 : 0;
  P.fz_tk = best_tk;
  P.fz_tma = best_tma ? 1 : 0;
  best_ms[0] = bx;
  best_ms[1] = bz;
  return cudaSuccess;
}

cudaError_t tune_transforms(Params& P, Workspace& W, bool mixed, cudaStream_t s, float* best_ms) {
  return mixed ? tune_transforms_t<float>(P, W, s, best_ms) : tune_transforms_t<double>(P, W, s, best_ms);
}

template cudaError_t launch_poisson<float>(const Params&, Workspace&, const float*, float*, cudaStream_t);
template cudaError_t launch_poisson<double>(const Params&, Workspace&, const double*, double*, cudaStream_t);
template cudaError_t fft_x_forward<float>(const Params&, const float*, int, cplx<float>*, float, int, float, float, const cplx<float>*, cudaStream_t, const float*);
template cudaError_t fft_x_forward<double>(const Params&, const double*, int, cplx<double>*, double, int, double, double, const cplx<double>*, cudaStream_t, const double*);
template cudaError_t poisson_pass<float>(const Params&, Workspace&, const float*, float*, float, float, float, cudaStream_t, const float*);
template cudaError_t poisson_pass<double>(const Params&, Workspace&, const double*, double*, double, double, double, cudaStream_t, const double*);
template cudaError_t fft_x_inverse<float>(const Params&, const cplx<float>*, int, float*, float, const cplx<float>*, cudaStream_t);
template cudaError_t fft_x_inverse<double>(const Params&, const cplx<double>*, int, double*, double, const cplx<double>*, cudaStream_t);
template cudaError_t fft_z<float>(const Params&, cplx<float>*, int, int, size_t, bool, const cplx<float>*, cudaStream_t);
template cudaError_t fft_z<double>(const Params&, cplx<double>*, int, int, size_t, bool, const cplx<double>*, cudaStream_t);
template cudaError_t fft_z_mac<float>(const Params&, cplx<float>*, bool, const cplx<float>*, cudaStream_t);
template cudaError_t fft_z_mac<double>(const Params&, cplx<double>*, bool, const cplx<double>*, cudaStream_t);

}  // namespace discos
