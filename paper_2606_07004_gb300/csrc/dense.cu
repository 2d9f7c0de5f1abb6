// Dense and small-matrix kernels (see dense.cuh).  Arithmetic is FP64, except
// the FP32 instances of the Hutch++ split kernels (mixed-precision OSLQ).
#include "dense.cuh"
#include "krylov.cuh"
#include "profile.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace ld {

// ===========================================================================
// Hutch++ QR: A = orth(Y) by two rounds of Cholesky QR (the QR step of
// Algorithms 2 and 3: an orthonormal basis of span(Y)).  For full-rank Y
// this gives the thin QR factor with positive diag(R), the same columns as a
// Householder QR with that sign convention.
// ===========================================================================
constexpr int kGramThreads = 256;
constexpr int kGramRows = 256;   // rows per tile (one partial per tile)
constexpr int kGramChunk = 32;   // rows staged in shared memory at a time

__device__ __forceinline__ void unrank_upper(int q, int s, int& i, int& j) {
  i = 0;
  int rem = q;
  while (rem >= s - i) { rem -= s - i; ++i; }
  j = i + rem;
}

// Accumulator of the Gram and A^T G sums per element type: FP64 FMA for
// FP64 blocks; for FP32 blocks the compensated dot (Dot2) of FP32 inputs,
// whose partial is read out in FP64 (error ~ (rows eps_32)^2 of the sum of
// |products|, far below FP32 rounding).
template <typename TY> struct GramAcc;
template <> struct GramAcc<double> { using type = AccD; };
template <> struct GramAcc<float> { using type = AccF; };

// Per-tile partial Gram sums sum_rows y_i y_j (i <= j), written [pair][tile].
// Thread t owns pairs t + q * blockDim.x for q < NP, NP the smallest count
// that covers all pairs (a compile-time loop: the FP64 pipe sees no
// predicated-off multiply-adds; spare slots repeat pair (0, 0) and are not
// written).
template <int NP, typename TY>
__global__ void __launch_bounds__(kGramThreads) k_gram(const TY* __restrict__ Y, int ldy,
                                                       int n, int s, int ntiles,
                                                       double* __restrict__ part) {
  __shared__ double sy_raw[kGramChunk * kMaxSketch];
  TY* sy = reinterpret_cast<TY*>(sy_raw);
  // Rows staged at a time: the buffer's capacity for s columns (32 for the
  // largest sketch, more for small ones: fewer barriers per tile).
  const int chunk = kGramChunk * (kMaxSketch / s);
  const int npairs = s * (s + 1) / 2;
  int pi[NP], pj[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    int idx = threadIdx.x + q * blockDim.x;
    if (idx < npairs) unrank_upper(idx, s, pi[q], pj[q]);
    else { pi[q] = 0; pj[q] = 0; }
  }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    typename GramAcc<TY>::type acc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q].zero();
    const int row0 = tile * kGramRows;
    const int row1 = min(row0 + kGramRows, n);
    for (int c0 = row0; c0 < row1; c0 += chunk) {
      const int rows = min(chunk, row1 - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < rows * s; e += blockDim.x) {
        int r = e / s, i = e - r * s;
        sy[r * s + i] = Y[(size_t)(c0 + r) * ldy + i];
      }
      __syncthreads();
      const TY* row = sy;
      for (int r = 0; r < rows; ++r, row += s) {
#pragma unroll
        for (int q = 0; q < NP; ++q) acc[q].fma(row[pi[q]], row[pj[q]]);
      }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      int idx = threadIdx.x + q * blockDim.x;
      if (idx < npairs) part[(size_t)idx * ntiles + tile] = acc[q].value();
    }
  }
}

// Sum the tile partials of each entry in a fixed order: out[e] for e < count.
// With sym_s > 0 the entries are upper-triangle pairs of an sym_s x sym_s
// matrix and both (i,j) and (j,i) of out are written.
__global__ void __launch_bounds__(128) k_reduce_rows(const double* __restrict__ part, int ntiles,
                                                     int sym_s, double* __restrict__ out) {
  __shared__ double sh[128];
  const int e = blockIdx.x;
  const double* src = part + (size_t)e * ntiles;
  double a = 0.0;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) a += src[t];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (sym_s > 0) {
      int i, j;
      unrank_upper(e, sym_s, i, j);
      out[i * sym_s + j] = sh[0];
      out[j * sym_s + i] = sh[0];
    } else {
      out[e] = sh[0];
    }
  }
}

// Cholesky C = R^T R of the s x s Gram matrix, dropping a column whose pivot
// R_jj^2 is <= thr_rel * max_i C_ii (its R row and Rinv column become zero),
// then Rinv = R^{-1} restricted to the kept columns.  One CTA.
__global__ void __launch_bounds__(256) k_chol_inv(const double* __restrict__ C, int s,
                                                  double thr_rel, double* __restrict__ Rinv,
                                                  int* __restrict__ keep_out) {
  __shared__ double R[kMaxSketch * kMaxSketch];
  __shared__ int keep[kMaxSketch];
  __shared__ double thr;
  double* Ri = Rinv;  // written column by column by the thread that owns it
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) { R[e] = C[e]; Ri[e] = 0.0; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < s; ++i) mx = fmax(mx, R[i * s + i]);
    thr = thr_rel * mx;
  }
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (threadIdx.x == 0) {
      double piv = R[j * s + j];
      for (int k = 0; k < j; ++k) piv -= R[k * s + j] * R[k * s + j];
      keep[j] = piv > thr;
      R[j * s + j] = keep[j] ? sqrt(piv) : 0.0;
    }
    __syncthreads();
    for (int l = j + 1 + threadIdx.x; l < s; l += blockDim.x) {
      if (keep[j]) {
        double v = R[j * s + l];
        for (int k = 0; k < j; ++k) v -= R[k * s + j] * R[k * s + l];
        R[j * s + l] = v / R[j * s + j];
      } else {
        R[j * s + l] = 0.0;
      }
    }
    __syncthreads();
  }
  // Upper-triangular inverse, one column per thread: R Rinv = I.  The zero
  // fill above is made visible to every thread before columns are written.
  __threadfence_block();
  __syncthreads();
  for (int l = threadIdx.x; l < s; l += blockDim.x) {
    if (!keep[l]) continue;
    for (int i = l; i >= 0; --i) {
      if (!keep[i]) { Ri[i * s + l] = 0.0; continue; }
      double v = (i == l) ? 1.0 : 0.0;
      for (int k = i + 1; k <= l; ++k) v -= R[i * s + k] * Ri[k * s + l];
      Ri[i * s + l] = v / R[i * s + i];
    }
  }
  for (int i = threadIdx.x; i < s; i += blockDim.x) keep_out[i] = keep[i];
}

// A[row, l] = sum_{i <= l} Y[row, i] Rinv[i, l]; A may alias Y.  A chunk of
// 32 rows is staged in shared memory (row stride odd, so the lanes' reads of
// one column spread over the banks); warp w computes output columns
// [4w, 4w + 4) of all 32 rows, lane = row, so every lane of a warp runs the
// same triangular loop (i <= 4w + 3; the extra terms multiply zeros of the
// upper-triangular Rinv and change nothing).  FP32 blocks take Rinv rounded
// to FP32 (a slightly different triangular preconditioner: the second
// round orthonormalises what the first leaves).  Dynamic shared memory:
// s * s + 32 * (s | 1) elements.
constexpr int kApplyCols = 4;
template <typename TY>
__global__ void __launch_bounds__(512) k_apply_rinv(const TY* Y, int ldy, int n, int s,
                                                    const double* __restrict__ Rinv, TY* A,
                                                    int lda) {
  extern __shared__ double smem_ar[];
  const int S1 = s | 1;
  TY* sr = reinterpret_cast<TY*>(smem_ar);
  TY* sy = sr + s * s;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) sr[e] = (TY)Rinv[e];
  const int lane = threadIdx.x & 31;
  const int l0 = (threadIdx.x >> 5) * kApplyCols;
  for (int c0 = blockIdx.x * 32; c0 < n; c0 += gridDim.x * 32) {
    const int rows = min(32, n - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * s; e += blockDim.x) {
      const int r = e / s, i = e - r * s;
      sy[r * S1 + i] = Y[(size_t)(c0 + r) * ldy + i];
    }
    __syncthreads();
    if (lane < rows && l0 < s) {
      TY acc[kApplyCols];
#pragma unroll
      for (int q = 0; q < kApplyCols; ++q) acc[q] = TY(0);
      const int lmax = min(l0 + kApplyCols, s);
      for (int i = 0; i < lmax; ++i) {
        const TY y = sy[lane * S1 + i];
#pragma unroll
        for (int q = 0; q < kApplyCols; ++q)
          if (l0 + q < s) acc[q] = fma(y, sr[i * s + l0 + q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < kApplyCols; ++q)
        if (l0 + q < s) A[(size_t)(c0 + lane) * lda + l0 + q] = acc[q];
    }
  }
}

size_t orth_workspace_doubles(int n, int s) {
  int ntiles = div_up(n, kGramRows);
  size_t npairs = (size_t)s * (s + 1) / 2;
  return npairs * ntiles + 2 * (size_t)s * s + 64;
}

// Persistent grids: 4 CTAs per SM, or for CTAs of fewer than 256 threads
// (small sketches: one thread per Gram pair, one warp per 4 columns) enough
// CTAs for 32 warps per SM, up to 16 (with 4 CTAs of 64 threads an SM held 8
// warps, and these loops idled) -- never more than the SM can hold at once
// with the kernel's shared memory and registers: a grid past that runs its
// last CTAs as a second wave, each with a whole CTA's share of the tiles
// (16 CTAs of 16 KB asked for, 14 resident: the Gram took twice its time).
template <typename Kern>
static int grid_for(Kern kern, int tiles, int threads = 256, size_t dyn_smem = 0) {
  int per_sm = threads >= 256 ? 4 : std::min(16, std::max(4, 1024 / std::max(32, threads)));
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, threads, dyn_smem) == cudaSuccess &&
      fit > 0)
    per_sm = std::min(per_sm, fit);
  else
    (void)cudaGetLastError();
  return std::max(1, std::min(tiles, per_sm * sm_count()));
}

// Pairs per thread of the Gram and A^T G kernels: the smallest instance that
// covers `per` (the pair count over at most kGramThreads threads; up to 9 for
// the Gram of 64 columns, 16 for A^T G of 64 x 64).
static int pairs_instance(int per) {
  static const int kInst[] = {1, 2, 3, 4, 6, 8, 12, 16};
  for (int v : kInst)
    if (v >= per) return v;
  return 16;
}

template <typename TY>
using GramKern = void (*)(const TY*, int, int, int, int, double*);
template <typename TY>
static GramKern<TY> gram_kernel(int np) {
  switch (np) {
    case 1: return k_gram<1, TY>;
    case 2: return k_gram<2, TY>;
    case 3: return k_gram<3, TY>;
    case 4: return k_gram<4, TY>;
    case 6: return k_gram<6, TY>;
    case 8: return k_gram<8, TY>;
    default: return k_gram<12, TY>;  // 64 columns: 2080 pairs, 9 per thread
  }
}

template <typename TY>
static int orth_t(int n, int s, const TY* Y, int ldy, TY* A, int lda, double* ws,
                  int* keep_dev, int* s_eff_host, cudaStream_t st) {
  if (s < 1 || s > kMaxSketch || n < 1) {
    set_error("orth: s=%d must be in [1, %d]", s, kMaxSketch);
    return LOGDET_EINVAL;
  }
  const int ntiles = div_up(n, kGramRows);
  const int npairs = s * (s + 1) / 2;
  double* part = ws;
  double* C = part + (size_t)npairs * ntiles;
  double* Rinv = C + (size_t)s * s;
  int* keep = keep_dev;
  int* keep_tmp = nullptr;
  if (!keep) {
    LD_CUDA(cudaMallocAsync(&keep_tmp, sizeof(int) * s, st));
    keep = keep_tmp;
  }
  const TY* src = Y;
  int ldsrc = ldy;
  // Gram: one thread per (i <= j) pair while they fit in one CTA, else as
  // few threads as keep the pairs per thread at their minimum.  Apply: one
  // warp per 4 output columns.
  const int gram_np = pairs_instance(div_up(npairs, kGramThreads));
  const int gram_threads = std::min(kGramThreads, div_up(div_up(npairs, gram_np), 32) * 32);
  const GramKern<TY> gram = gram_kernel<TY>(gram_np);
  const int apply_threads = 32 * div_up(s, kApplyCols);
  const size_t apply_smem = sizeof(TY) * ((size_t)s * s + 32 * (size_t)(s | 1));
  if (apply_smem > 48 * 1024)
    LD_CUDA(cudaFuncSetAttribute(k_apply_rinv<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)apply_smem));
  for (int round = 0; round < 2; ++round) {
    ProfScope prof(KC_QR, st, 2.0 * n * (double)s * s * 2.0, 2.0 * sizeof(TY) * n * s);
    prof_count();
    prof_count();
    prof_count();
    gram<<<grid_for(gram, ntiles, gram_threads), gram_threads, 0, st>>>(src, ldsrc, n, s, ntiles,
                                                                         part);
    LD_CHECK_LAUNCH();
    k_reduce_rows<<<npairs, 128, 0, st>>>(part, ntiles, s, C);
    LD_CHECK_LAUNCH();
    // R14: |R_ii| <= 1e-6 max_j |y_j|  <=>  R_ii^2 <= 1e-12 max_j C_jj.
    k_chol_inv<<<1, 256, 0, st>>>(C, s, 1e-12, Rinv, keep);
    LD_CHECK_LAUNCH();
    k_apply_rinv<TY><<<grid_for(k_apply_rinv<TY>, div_up(n, 32), apply_threads, apply_smem),
                       apply_threads, apply_smem, st>>>(src, ldsrc, n, s, Rinv, A, lda);
    LD_CHECK_LAUNCH();
    src = A;
    ldsrc = lda;
  }
  if (s_eff_host) {
    std::vector<int> h(s);
    LD_CUDA(cudaMemcpyAsync(h.data(), keep, sizeof(int) * s, cudaMemcpyDeviceToHost, st));
    LD_CUDA(cudaStreamSynchronize(st));
    int c = 0;
    for (int i = 0; i < s; ++i) c += h[i] != 0;
    *s_eff_host = c;
  }
  if (keep_tmp) LD_CUDA(cudaFreeAsync(keep_tmp, st));
  return LOGDET_OK;
}

int orth_fp64(int n, int s, const double* Y, int ldy, double* A, int lda, double* ws,
              int* keep_dev, int* s_eff_host, cudaStream_t st) {
  return orth_t<double>(n, s, Y, ldy, A, lda, ws, keep_dev, s_eff_host, st);
}

int orth_f32(int n, int s, const float* Y, int ldy, float* A, int lda, double* ws,
             int* keep_dev, int* s_eff_host, cudaStream_t st) {
  return orth_t<float>(n, s, Y, ldy, A, lda, ws, keep_dev, s_eff_host, st);
}

// ===========================================================================
// Hutch++ residual probes: Z = G - A (A^T G), G generated from the probe hash.
// ===========================================================================
// Per-tile partials of A^T G, written [i * r + j][tile]; thread t owns pairs
// t + q * blockDim.x for q < NP (compile-time, as in k_gram).
template <int NP, typename TY>
__global__ void __launch_bounds__(kGramThreads) k_atg(const TY* __restrict__ A, int lda,
                                                      int n, int s, int r, uint64_t key,
                                                      const uint64_t* __restrict__ keyp,
                                                      int ntiles, double* __restrict__ part,
                                                      int gaussian) {
  if (keyp) key = *keyp;
  __shared__ double sa_raw[kGramChunk * kMaxSketch];
  __shared__ double sg_raw[kGramChunk * kMaxSketch];
  TY* sa = reinterpret_cast<TY*>(sa_raw);
  TY* sg = reinterpret_cast<TY*>(sg_raw);
  const int chunk = kGramChunk * (kMaxSketch / max(s, r));  // rows staged at a time
  const int npairs = s * r;
  int pi[NP], pj[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    int idx = threadIdx.x + q * blockDim.x;
    pi[q] = idx < npairs ? idx / r : 0;
    pj[q] = idx < npairs ? idx - (idx / r) * r : 0;
  }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    typename GramAcc<TY>::type acc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q].zero();
    const int row0 = tile * kGramRows;
    const int row1 = min(row0 + kGramRows, n);
    for (int c0 = row0; c0 < row1; c0 += chunk) {
      const int rows = min(chunk, row1 - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < rows * s; e += blockDim.x) {
        int rr = e / s, i = e - rr * s;
        sa[rr * s + i] = A[(size_t)(c0 + rr) * lda + i];
      }
      for (int e = threadIdx.x; e < rows * r; e += blockDim.x) {
        int rr = e / r, j = e - rr * r;
        sg[rr * r + j] = (TY)probe_value(key, (uint32_t)j, (uint32_t)(c0 + rr), gaussian);
      }
      __syncthreads();
      const TY* ra = sa;
      const TY* rg = sg;
      for (int rr = 0; rr < rows; ++rr, ra += s, rg += r) {
#pragma unroll
        for (int q = 0; q < NP; ++q) acc[q].fma(ra[pi[q]], rg[pj[q]]);
      }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      int idx = threadIdx.x + q * blockDim.x;
      if (idx < npairs) part[(size_t)idx * ntiles + tile] = acc[q].value();
    }
  }
}

// Rows of A that k_project stages at a time: the buffer's capacity for s
// columns (at least kGramChunk).
__host__ __device__ inline int project_chunk(int s) {
  return kGramChunk * (kMaxSketch / (s > 0 ? s : kMaxSketch));
}

// X[row, zcol0 + j] = g(row, j) - sum_i A[row, i] B[i, j] (FP32 blocks: B
// and g rounded to FP32, the s-term sum in FP32).
template <typename TY>
__global__ void __launch_bounds__(256) k_project(const TY* A, int lda, int n, int s, int r,
                                                 uint64_t key, const uint64_t* __restrict__ keyp,
                                                 const double* __restrict__ Bm,
                                                 TY* X, int ldx, int zcol0, int gaussian) {
  if (keyp) key = *keyp;
  __shared__ double sb_raw[kMaxSketch * kMaxSketch];
  __shared__ double sa_raw[kGramChunk * kMaxSketch];
  TY* sb = reinterpret_cast<TY*>(sb_raw);
  TY* sa = reinterpret_cast<TY*>(sa_raw);
  for (int e = threadIdx.x; e < s * r; e += blockDim.x) sb[e] = (TY)Bm[e];
  const int chunk = project_chunk(s);  // rows staged at a time
  for (int c0 = blockIdx.x * chunk; c0 < n; c0 += gridDim.x * chunk) {
    const int rows = min(chunk, n - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * s; e += blockDim.x) {
      int rr = e / s, i = e - rr * s;
      sa[rr * s + i] = A[(size_t)(c0 + rr) * lda + i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * r; e += blockDim.x) {
      int rr = e / r, j = e - rr * r;
      TY acc = TY(0);
      for (int i = 0; i < s; ++i) acc = fma(sa[rr * s + i], sb[i * r + j], acc);
      TY g = (TY)probe_value(key, (uint32_t)j, (uint32_t)(c0 + rr), gaussian);
      X[(size_t)(c0 + rr) * ldx + zcol0 + j] = g - acc;
    }
  }
}

int reduce_partials_fp64(const double* part, int nrows, int ntiles, double* out, cudaStream_t st) {
  ProfScope prof(KC_SCALAR, st);
  k_reduce_rows<<<nrows, 128, 0, st>>>(part, ntiles, 0, out);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

size_t project_workspace_doubles(int n, int s, int r) {
  int ntiles = div_up(n, kGramRows);
  return (size_t)s * r * ntiles + (size_t)s * r + 64;
}

template <typename TY>
using AtgKern = void (*)(const TY*, int, int, int, int, uint64_t, const uint64_t*, int, double*,
                         int);
template <typename TY>
static AtgKern<TY> atg_kernel(int np) {
  switch (np) {
    case 1: return k_atg<1, TY>;
    case 2: return k_atg<2, TY>;
    case 3: return k_atg<3, TY>;
    case 4: return k_atg<4, TY>;
    case 6: return k_atg<6, TY>;
    case 8: return k_atg<8, TY>;
    case 12: return k_atg<12, TY>;
    default: return k_atg<16, TY>;
  }
}

template <typename TY>
static int project_residual_t(int n, int s, int r, const TY* A, int lda, uint64_t key, TY* X,
                              int ldx, int zcol0, double* ws, cudaStream_t st, int gaussian,
                              const uint64_t* keyp) {
  if (s > kMaxSketch || r > kMaxSketch || r < 1) {
    set_error("project: s=%d r=%d out of range", s, r);
    return LOGDET_EINVAL;
  }
  const int ntiles = div_up(n, kGramRows);
  double* part = ws;
  double* Bm = ws + (size_t)s * r * ntiles;
  ProfScope prof(KC_PROJECT, st, 4.0 * n * (double)s * r, sizeof(TY) * n * (2.0 * s + r));
  if (s > 0) {
    prof_count();
    prof_count();
    // As few threads as keep the per-thread pair count at its minimum.
    const int np = s * r, per = pairs_instance(div_up(np, kGramThreads));
    const int atg_threads = std::min(kGramThreads, div_up(div_up(np, per), 32) * 32);
    const AtgKern<TY> atg = atg_kernel<TY>(per);
    atg<<<grid_for(atg, ntiles, atg_threads), atg_threads, 0, st>>>(A, lda, n, s, r, key, keyp,
                                                                     ntiles, part, gaussian);
    LD_CHECK_LAUNCH();
    k_reduce_rows<<<s * r, 128, 0, st>>>(part, ntiles, 0, Bm);
    LD_CHECK_LAUNCH();
  }
  k_project<TY><<<grid_for(k_project<TY>, div_up(n, project_chunk(s))), 256, 0, st>>>(
      A, lda, n, s, r, key, keyp, Bm, X, ldx, zcol0, gaussian);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

int project_residual_fp64(int n, int s, int r, const double* A, int lda, uint64_t key,
                          double* X, int ldx, int zcol0, double* ws, cudaStream_t st,
                          int gaussian, const uint64_t* keyp) {
  return project_residual_t<double>(n, s, r, A, lda, key, X, ldx, zcol0, ws, st, gaussian, keyp);
}

int project_residual_f32(int n, int s, int r, const float* A, int lda, uint64_t key, float* X,
                         int ldx, int zcol0, double* ws, cudaStream_t st, int gaussian,
                         const uint64_t* keyp) {
  return project_residual_t<float>(n, s, r, A, lda, key, X, ldx, zcol0, ws, st, gaussian, keyp);
}

// ===========================================================================
// Column norms (partials in the Krylov layout [ld][ntiles]).
// ===========================================================================
template <typename T>
__global__ void __launch_bounds__(512) k_colnorm(const T* __restrict__ X, int n, int ld,
                                                  int tile_rows, int ntiles,
                                                  typename PartOf<T>::type* __restrict__ part) {
  constexpr int V = Vec16<T>::N;
  using Acc = typename AccOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* smem = reinterpret_cast<Acc*>(smem_raw);
  const int G = ld / V;
  const int R = blockDim.x / G;
  const int r = threadIdx.x / G, g = threadIdx.x - (threadIdx.x / G) * G;
  const bool live = r < R;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    Acc acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v].zero();
    const int row0 = tile * tile_rows, row1 = min(row0 + tile_rows, n);
    if (live) {
      for (int row = row0 + r; row < row1; row += R) {
        typename Compute<T>::type x[V];
        load_vec<T>(X + (size_t)row * ld + g * V, x);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v].fma(x[v], x[v]);
      }
    }
    __syncthreads();
    if (live) {
#pragma unroll
      for (int v = 0; v < V; ++v) smem[threadIdx.x * V + v] = acc[v];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ld; c += blockDim.x) {
      int gg = c / V, v = c - gg * V;
      Acc t;
      t.zero();
      for (int rr = 0; rr < R; ++rr) t.add(smem[(rr * G + gg) * V + v]);
      put_part(part + (size_t)c * ntiles + tile, t);
    }
    __syncthreads();
  }
}

template <typename T>
int colnorm_partials(const T* X, int n, int ld, int tile_rows, int ntiles,
                     typename PartOf<T>::type* part, int threads, cudaStream_t st) {
  using Acc = typename AccOf<T>::type;
  size_t smem = (size_t)threads * Vec16<T>::N * sizeof(Acc);
  ProfScope prof(KC_OTHER, st, 2.0 * n * (double)ld, (double)n * ld * sizeof(T));
  k_colnorm<T><<<grid_for(k_colnorm<T>, ntiles, threads, smem), threads, smem, st>>>(
      X, n, ld, tile_rows, ntiles, part);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}
template int colnorm_partials<double>(const double*, int, int, int, int, double*, int, cudaStream_t);
template int colnorm_partials<float>(const float*, int, int, int, int, float2*, int, cudaStream_t);
template int colnorm_partials<bf16>(const bf16*, int, int, int, int, float2*, int, cudaStream_t);
template int colnorm_partials<f32x2>(const f32x2*, int, int, int, int, float2*, int, cudaStream_t);

// ===========================================================================
// Gauss quadrature of a symmetric tridiagonal (Sec. 3.1): eigenvalues theta_k
// and first eigenvector components tau_k by implicit symmetric QR steps with
// a Wilkinson shift (Golub and Van Loan, "Matrix Computations", Sec. 8.3),
// carrying only the first row of the accumulated rotations (Golub and
// Welsch, Math. Comp. 1969).  One thread per probe; its d, e, z arrays live
// in shared memory, interleaved across the CTA's threads (element k of
// thread t at k * S + t), and the bulge chase carries the entries it has just
// updated in registers.
// ===========================================================================
__device__ double tridiag_gauss_log(double* d, double* e, double* z, int S, int m,
                                    double clamp_lo, bool* nonpos) {
  // d[0..m) diagonal, e[0..m-1) off-diagonal, z = e_1 on entry; stride S.
#define TD(k) d[(k) * S]
#define TE(k) e[(k) * S]
#define TZ(k) z[(k) * S]
  const double eps = 2.220446049250313e-16;
  int hi = m - 1;
  int iters = 0;
  while (hi > 0) {
    // Deflate negligible off-diagonals at the bottom.
    if (fabs(TE(hi - 1)) <= eps * (fabs(TD(hi - 1)) + fabs(TD(hi)))) {
      TE(hi - 1) = 0.0;
      --hi;
      iters = 0;
      continue;
    }
    // Find the top of the unreduced block ending at hi.
    int lo = hi - 1;
    while (lo > 0 && fabs(TE(lo - 1)) > eps * (fabs(TD(lo - 1)) + fabs(TD(lo)))) --lo;
    if (lo > 0) TE(lo - 1) = 0.0;
    if (++iters > 60) { *nonpos = true; break; }  // unconverged: flagged
    // Wilkinson shift from the trailing 2x2 block.
    const double t = TE(hi - 1);
    const double delta = 0.5 * (TD(hi - 1) - TD(hi));
    const double den = delta + copysign(hypot(delta, t), delta == 0.0 ? 1.0 : delta);
    const double mu = TD(hi) - t * t / den;
    double a = TD(lo), b = TE(lo), zc = TZ(lo);  // d[k], e[k], z[k] of the current k
    double x = a - mu;
    double bz = b;
    for (int k = lo; k < hi; ++k) {
      // Givens pair (c, s) with c x - s bz = r, s x + c bz = 0: one reciprocal
      // square root (the entries are O(1) for the scaled operators); hypot
      // only for arguments near underflow.
      const double rr2 = x * x + bz * bz;
      double rr, c, s;
      if (rr2 > 1e-280) {
        const double ri = rsqrt(rr2);
        rr = rr2 * ri;
        c = x * ri;
        s = -bz * ri;
      } else {
        rr = hypot(x, bz);
        c = (rr == 0.0) ? 1.0 : x / rr;
        s = (rr == 0.0) ? 0.0 : -bz / rr;
      }
      if (k > lo) TE(k - 1) = rr;
      const double cc = TD(k + 1);
      const double dk = c * c * a - 2.0 * c * s * b + s * s * cc;
      const double dk1 = s * s * a + 2.0 * c * s * b + c * c * cc;
      const double ek = c * s * (a - cc) + (c * c - s * s) * b;
      TD(k) = dk;
      TE(k) = ek;
      const double z1 = TZ(k + 1);
      TZ(k) = c * zc - s * z1;
      zc = s * zc + c * z1;
      if (k + 1 < hi) {
        const double en = TE(k + 1);
        bz = -s * en;
        b = c * en;
        x = ek;
      }
      a = dk1;
    }
    TD(hi) = a;
    TZ(hi) = zc;
  }
  double sum = 0.0;
  for (int k = 0; k < m; ++k) {
    double th = TD(k);
    if (!(th > 0.0)) { *nonpos = true; th = clamp_lo; }
    sum += TZ(k) * TZ(k) * log(th);
  }
  return sum;
#undef TD
#undef TE
#undef TZ
}

// ---------------------------------------------------------------------------
// The Gauss rule's value sum_k tau_k^2 log(theta_k) is e_1^T log(T) e_1.  For
// SPD T it follows from log(theta) = int_0^inf [1/(1+s) - 1/(theta+s)] ds as
//   e_1^T log(T) e_1 = int_R s [1/(1+s) - r(s)] du,   s = e^u,
//   r(s) = e_1^T (T + s I)^{-1} e_1 = 1 / d_1,
// with d_1 from the continued fraction d_m = t_m + s,
// d_i = t_i + s - b_i^2 / d_{i+1} (the pivots of T + s I = U D U^T, all
// positive for SPD T).  The integrand is analytic in the strip |Im u| < pi
// and decays like s / lambda_min(T) as u -> -inf and like lambda_max(T) / s
// as u -> +inf, so the trapezoid rule with step h = 1/2 on u in [-60, 39.5]
// (200 nodes) has discretisation error ~exp(-2 pi^2 / h) < 1e-17 and
// truncation error < 1e-17 for spectra in [1e-9, 1] (the scaled operators
// J = Q / alpha have lambda_max <= 1).  One CTA per probe, one node per
// thread, node values added in a fixed-order tree.  A T that is not SPD
// (a non-positive pivot at s = 0, possible only from FP32 rounding) takes
// the implicit-QR rule above, which clamps and flags non-positive Ritz values.
// ---------------------------------------------------------------------------
constexpr int kQuadThreads = 256;
constexpr int kQuadNodes = 200;
constexpr double kQuadULo = -60.0;
constexpr double kQuadH = 0.5;

__global__ void __launch_bounds__(kQuadThreads) k_gauss_quad(
    const double* __restrict__ alpha, const double* __restrict__ beta, int ldab,
    const int* __restrict__ msteps, int m, int nprobe, double clamp_lo, double* __restrict__ out,
    uint32_t* __restrict__ status) {
  extern __shared__ double sq[];  // a[m], b2[m], fallback d, e, z [3m]
  __shared__ double fv[kQuadThreads];
  __shared__ int s_spd;
  const int p = blockIdx.x;
  if (p >= nprobe) return;
  int mp = msteps ? msteps[p] : m;
  if (mp > m) mp = m;
  if (mp <= 0) {
    if (threadIdx.x == 0) out[p] = 0.0;
    return;
  }
  double* a = sq;
  double* b2 = sq + m;
  for (int k = threadIdx.x; k < mp; k += blockDim.x) {
    a[k] = alpha[(size_t)p * ldab + k];
    const double b = (k + 1 < mp) ? beta[(size_t)p * ldab + k] : 0.0;
    b2[k] = b * b;
  }
  if (threadIdx.x == 0) s_spd = 1;
  __syncthreads();
  const int t = threadIdx.x;
  if (t == kQuadNodes) {
    // Pivots at s = 0: all positive iff T is SPD (Sylvester's law of inertia).
    double d = a[mp - 1];
    bool ok = d > 0.0;
    for (int i = mp - 2; i >= 0 && ok; --i) {
      d = a[i] - b2[i] / d;
      ok = d > 0.0;
    }
    if (!ok) s_spd = 0;
  }
  double f = 0.0;
  if (t < kQuadNodes) {
    const double sn = exp(kQuadULo + kQuadH * t);
    double d = a[mp - 1] + sn;
    for (int i = mp - 2; i >= 0; --i) d = (a[i] + sn) - b2[i] / d;
    f = sn * (1.0 / (1.0 + sn) - 1.0 / d);
  }
  fv[t] = f;
  __syncthreads();
  for (int w = kQuadThreads / 2; w > 0; w >>= 1) {
    if (t < w) fv[t] += fv[t + w];
    __syncthreads();
  }
  if (s_spd) {
    if (t == 0) out[p] = kQuadH * fv[0];
    return;
  }
  if (t == 0) {
    double* d = sq + 2 * m;
    double* e = d + m;
    double* z = e + m;
    for (int k = 0; k < mp; ++k) {
      d[k] = alpha[(size_t)p * ldab + k];
      e[k] = (k + 1 < mp) ? beta[(size_t)p * ldab + k] : 0.0;
      z[k] = (k == 0) ? 1.0 : 0.0;
    }
    bool nonpos = false;
    out[p] = tridiag_gauss_log(d, e, z, 1, mp, clamp_lo, &nonpos);
    if (nonpos && status) atomicOr(status + p, LOGDET_ST_NONPOS_RITZ);
  }
}

int gauss_quadrature_log(const double* alpha, const double* beta, int ldab, const int* msteps,
                         int m, int nprobe, double clamp_lo, double* out, uint32_t* status,
                         cudaStream_t st) {
  if (m < 1 || m > kMaxSteps) {
    set_error("gauss quadrature: m=%d must be in [1, %d]", m, kMaxSteps);
    return LOGDET_EINVAL;
  }
  const size_t smem = (size_t)5 * m * sizeof(double);
  ProfScope prof(KC_SMALL, st);
  k_gauss_quad<<<nprobe, kQuadThreads, smem, st>>>(alpha, beta, ldab, msteps, m, nprobe, clamp_lo,
                                                   out, status);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

// ===========================================================================
// log(H) e_1 by inverse scaling and squaring (Kenney and Laub 1989; Higham,
// "Evaluating Pade approximants of the matrix logarithm", SIMAX 2001): take
// square roots A <- A^{1/2} (product form of the Denman-Beavers iteration)
// until |A - I|_1 <= 0.25, then log(H) = 2^s log(I + X), X = A - I, with the
// [8/8] Pade approximant in its partial-fraction form
//   log(I + X) ~ sum_j w_j X (I + x_j X)^{-1}
// (x_j, w_j the 8-point Gauss-Legendre rule on [0, 1]).  Only the first
// column is formed.  One CTA per probe.  The four m x m work matrices sit in
// shared memory when they fit (m <= 80); for m <= 113 the two that the
// inversions and products work on (Y, W) stay in shared memory and the other
// two (M, T) in the global workspace; beyond that all four are global.
// (One-warp CTAs were measured 4x slower: FP64 issues at 2 lanes per clock
// per SM on this part, so a probe's work needs the whole CTA's warps in
// flight, not cheaper barriers.)
// ===========================================================================
constexpr int kLogThreads = 256;
constexpr int kPadeNodes = 8;

struct GLRule { double x[kPadeNodes], w[kPadeNodes]; };

// Barrier of the CTA; a one-warp CTA needs only a warp barrier.
__device__ __forceinline__ void cta_bar() {
  if (blockDim.x == 32) __syncwarp();
  else __syncthreads();
}

// Row-major element loop over an m x m matrix without a division per step:
// thread t visits e = t, t + blockDim.x, ... as (i, j) = (e / m, e % m).
__device__ __forceinline__ void ij_first(int m, int& i, int& j) {
  i = (int)threadIdx.x / m;
  j = (int)threadIdx.x - i * m;
}
__device__ __forceinline__ void ij_next(int m, int& i, int& j) {
  j += blockDim.x;
  while (j >= m) { j -= m; ++i; }
}

// Gauss-Jordan inversion in place with partial (row) pivoting; A row-major m x m.
__device__ bool cta_invert(double* A, int m, int* perm, double* fcol) {
  __shared__ int s_piv;
  __shared__ bool s_ok;
  if (threadIdx.x == 0) s_ok = true;
  for (int k = 0; k < m; ++k) {
    cta_bar();
    if (threadIdx.x < 32) {  // pivot: largest |A_ik|, i >= k, smallest index on ties
      double best = -1.0;
      int bi = k;
      for (int i = k + (int)threadIdx.x; i < m; i += 32) {
        const double v = fabs(A[i * m + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        s_piv = bi;
        perm[k] = bi;
        if (!(best > 0.0)) s_ok = false;
      }
    }
    cta_bar();
    const int p = s_piv;
    if (p != k) {
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double t = A[k * m + j];
        A[k * m + j] = A[p * m + j];
        A[p * m + j] = t;
      }
    }
    cta_bar();
    const double piv = A[k * m + k];
    const double ipiv = (piv != 0.0) ? 1.0 / piv : 0.0;
    cta_bar();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      A[k * m + j] = (j == k) ? ipiv : A[k * m + j] * ipiv;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) fcol[i] = (i == k) ? 0.0 : A[i * m + k];
    cta_bar();
    int i, j;
    for (ij_first(m, i, j); i < m; ij_next(m, i, j)) {
      if (i == k) continue;
      const double f = fcol[i];
      if (j == k) A[i * m + j] = -f * A[k * m + k];
      else A[i * m + j] = fma(-f, A[k * m + j], A[i * m + j]);
    }
  }
  cta_bar();
  for (int k = m - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double t = A[i * m + k];
        A[i * m + k] = A[i * m + p];
        A[i * m + p] = t;
      }
    }
    cta_bar();
  }
  return s_ok;
}

// max_j sum_i |A_ij - delta_ij|
__device__ double cta_norm1_minus_identity(const double* A, int m, double* red) {
  double mx = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += fabs(A[i * m + j] - (i == j ? 1.0 : 0.0));
    mx = fmax(mx, s);
  }
  red[threadIdx.x] = mx;
  cta_bar();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    cta_bar();
  }
  double r = red[0];
  cta_bar();
  return r;
}

// smem_mats: how many of the four work matrices are in dynamic shared memory
// (4: Y, M, W, T; 2: Y and W; 0: none).  The global workspace holds 4 mmax^2
// doubles per probe whatever the split.
__global__ void __launch_bounds__(kLogThreads) k_hesslog(const double* __restrict__ H, int ldh,
                                                         const int* __restrict__ msteps, int mmax,
                                                         double* __restrict__ cout, int ldc,
                                                         double* __restrict__ ws,
                                                         uint32_t* __restrict__ status,
                                                         GLRule gl, int smem_mats) {
  extern __shared__ double dyn[];
  __shared__ double red[kLogThreads];
  __shared__ int perm[kMaxSteps];
  __shared__ double fcol[kMaxSteps];
  __shared__ double rhs[kMaxSteps];
  __shared__ double acc[kMaxSteps];
  const int p = blockIdx.x;
  int m = msteps ? msteps[p] : mmax;
  if (m > mmax) m = mmax;
  double* c = cout + (size_t)p * ldc;
  if (m <= 0) {
    for (int i = threadIdx.x; i < ldc; i += blockDim.x) c[i] = 0.0;
    return;
  }
  const size_t mm = (size_t)m * m;
  double* wsp = ws + (size_t)p * 4 * ((size_t)mmax * mmax);
  double *Yb, *Mb, *Wb, *Tb;  // current matrix (square-rooted in place), DB M, inverse, product
  if (smem_mats == 4) {
    Yb = dyn; Mb = dyn + mm; Wb = dyn + 2 * mm; Tb = dyn + 3 * mm;
  } else if (smem_mats == 2) {
    Yb = dyn; Wb = dyn + mm; Mb = wsp; Tb = wsp + mm;
  } else {
    Yb = wsp; Mb = wsp + mm; Wb = wsp + 2 * mm; Tb = wsp + 3 * mm;
  }
  const double* Hp = H + (size_t)p * ldh * mmax;
  int i, j;
  // Row-major copy of the leading m x m block of the column-major H.
  for (ij_first(m, i, j); i < m; ij_next(m, i, j)) Yb[i * m + j] = Hp[(size_t)j * ldh + i];
  cta_bar();
  bool ok = true;
  int nroots = 0;
  while (cta_norm1_minus_identity(Yb, m, red) > 0.25 && nroots < 64) {
    // Product-form Denman-Beavers: M0 = Y0 = A;
    //   Y <- Y (I + M^{-1}) / 2,  M <- (I + (M + M^{-1}) / 2) / 2,  Y -> A^{1/2}.
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Mb[e] = Yb[e];
    cta_bar();
    bool conv = false;
    double prev = 1e300;
    for (int it = 0; it < 100; ++it) {
      for (int e = threadIdx.x; e < m * m; e += blockDim.x) Wb[e] = Mb[e];
      cta_bar();
      if (!cta_invert(Wb, m, perm, fcol)) { ok = false; break; }
      cta_bar();
      for (ij_first(m, i, j); i < m; ij_next(m, i, j)) {
        double v = 0.0;
        for (int k = 0; k < m; ++k) v = fma(Yb[i * m + k], Wb[k * m + j], v);
        Tb[i * m + j] = 0.5 * (Yb[i * m + j] + v);
      }
      cta_bar();
      for (ij_first(m, i, j); i < m; ij_next(m, i, j)) {
        const int e = i * m + j;
        Yb[e] = Tb[e];
        Mb[e] = 0.25 * (Mb[e] + Wb[e]) + (i == j ? 0.5 : 0.0);
      }
      cta_bar();
      double dev = cta_norm1_minus_identity(Mb, m, red);
      // Converged at rounding level, or stagnating there.
      if (dev <= 1e-15 * m || (dev < 1e-9 && dev > 0.5 * prev)) { conv = true; break; }
      prev = dev;
    }
    if (!conv) { ok = false; break; }
    ++nroots;
  }
  // X = A - I ; rhs = X e_1 ; c = 2^s sum_j w_j (I + x_j X)^{-1} rhs
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    rhs[r] = Yb[r * m + 0] - (r == 0 ? 1.0 : 0.0);
    acc[r] = 0.0;
  }
  cta_bar();
  for (int q = 0; q < kPadeNodes && ok; ++q) {
    const double xq = gl.x[q];
    for (ij_first(m, i, j); i < m; ij_next(m, i, j)) {
      const int e = i * m + j;
      Wb[e] = (i == j ? 1.0 : 0.0) + xq * (Yb[e] - (i == j ? 1.0 : 0.0));
    }
    cta_bar();
    if (!cta_invert(Wb, m, perm, fcol)) { ok = false; break; }
    cta_bar();
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      double v = 0.0;
      for (int k = 0; k < m; ++k) v = fma(Wb[r * m + k], rhs[k], v);
      acc[r] = fma(gl.w[q], v, acc[r]);
    }
    cta_bar();
  }
  const double scale = ldexp(1.0, nroots);
  for (int r = threadIdx.x; r < ldc; r += blockDim.x) c[r] = (r < m && ok) ? scale * acc[r] : 0.0;
  if (!ok && threadIdx.x == 0 && status) atomicOr(status + p, LOGDET_ST_LOG_FAILED);
}

// ===========================================================================
// Banded Hessenberg matrices (the IOP window k gives upper bandwidth k - 1):
// log(H) e_1 by the resolvent quadrature used for the Gauss rules,
//   log(H) e_1 = int_R s [ e_1 / (1 + s) - (H + s I)^{-1} e_1 ] du,  s = e^u,
// (log(lambda) = int_0^inf [1/(1+s) - 1/(lambda+s)] ds on each eigenvalue),
// trapezoid rule with step 1/2 on u in [-60, 60]: 241 nodes, discretisation
// error ~exp(-2 pi^2 / h) and truncation error < 1e-16 for spectra in
// [1e-9, 1e9] off the negative real axis.  Each node is one banded solve of
// (H + s I) x = e_1 by Gaussian elimination with partial pivoting between
// adjacent rows (the only rows with an entry in the pivot column), O(m k)
// work; one node per thread, the node vectors added in node order.  This is
// O(241 m k) per probe against the ~40 dense O(m^3) inversions of inverse
// scaling and squaring, and its nodes spread over the whole CTA.
// ===========================================================================
constexpr int kResMaxBand = 8;
constexpr int kResNodes = 241;
constexpr int kResThreads = 256;
constexpr double kResULo = -60.0;
constexpr double kResH = 0.5;

size_t hesslog_band_workspace_doubles(int m, int nprobe) {
  return (size_t)nprobe * kResNodes * m * (kResMaxBand + 3) + 16;
}

// W = band + 2: the length of a row of U (band, diagonal and one fill entry).
template <int W>
__global__ void __launch_bounds__(kResThreads) k_hesslog_band(
    const double* __restrict__ H, int ldh, const int* __restrict__ msteps, int mmax,
    double* __restrict__ cout, int ldc, double* __restrict__ ws, uint32_t* __restrict__ status) {
  constexpr int band = W - 2;
  extern __shared__ double hb[];  // hb[j * W + l] = H(j - band + l, j), l = 0..band+1
  __shared__ int s_fail;
  const int p = blockIdx.x;
  int m = msteps ? msteps[p] : mmax;
  if (m > mmax) m = mmax;
  double* c = cout + (size_t)p * ldc;
  if (m <= 0) {
    for (int i = threadIdx.x; i < ldc; i += blockDim.x) c[i] = 0.0;
    return;
  }
  const double* Hp = H + (size_t)p * ldh * mmax;
  for (int e = threadIdx.x; e < m * W; e += blockDim.x) {
    const int j = e / W, l = e - j * W, i = j - band + l;
    hb[e] = (i >= 0 && i < m) ? Hp[(size_t)j * ldh + i] : 0.0;
  }
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  const size_t NN = kResNodes;
  double* U = ws + (size_t)p * NN * mmax * (kResMaxBand + 3);  // [m][W][node]
  double* R = U + (size_t)mmax * W * NN;                       // [m][node]
  const int t = threadIdx.x;
  if (t < kResNodes) {
    const double s = exp(kResULo + kResH * t);
    // Entry (i, j) of H + s I inside the band (0 outside).
    auto A = [&](int i, int j) -> double {
      const int l = i - j + band;
      if (j >= m || l < 0 || l > band + 1) return 0.0;
      return hb[j * W + l] + (i == j ? s : 0.0);
    };
    double act[W], nxt[W];
#pragma unroll
    for (int q = 0; q < W; ++q) act[q] = A(0, q);
    double ract = 1.0;
    bool bad = false;
    for (int j = 0; j < m; ++j) {
      double rn = 0.0;
      if (j + 1 < m) {
#pragma unroll
        for (int q = 0; q < W; ++q) nxt[q] = A(j + 1, j + q);
        if (fabs(nxt[0]) > fabs(act[0])) {
#pragma unroll
          for (int q = 0; q < W; ++q) {
            const double tmp = act[q];
            act[q] = nxt[q];
            nxt[q] = tmp;
          }
          rn = ract;
          ract = 0.0;
        }
      }
      if (!(fabs(act[0]) > 0.0) || !isfinite(act[0])) bad = true;
#pragma unroll
      for (int q = 0; q < W; ++q) U[((size_t)j * W + q) * NN + t] = act[q];
      R[(size_t)j * NN + t] = ract;
      if (j + 1 < m) {
        const double lm = nxt[0] / act[0];
#pragma unroll
        for (int q = 0; q + 1 < W; ++q) nxt[q] = fma(-lm, act[q + 1], nxt[q + 1]);
        nxt[W - 1] = 0.0;
        rn = fma(-lm, ract, rn);
#pragma unroll
        for (int q = 0; q < W; ++q) act[q] = nxt[q];
        ract = rn;
      }
    }
    // Back substitution; R[j] becomes x_j.
    for (int j = m - 1; j >= 0 && !bad; --j) {
      double v = R[(size_t)j * NN + t];
#pragma unroll
      for (int q = 1; q < W; ++q)
        if (j + q < m) v = fma(-U[((size_t)j * W + q) * NN + t], R[(size_t)(j + q) * NN + t], v);
      const double x = v / U[(size_t)j * W * NN + t];
      if (!isfinite(x)) bad = true;
      R[(size_t)j * NN + t] = x;
    }
    // Node value s (e_1 / (1 + s) - x).
    for (int j = 0; j < m; ++j) {
      const double x = R[(size_t)j * NN + t];
      R[(size_t)j * NN + t] = s * ((j == 0 ? 1.0 / (1.0 + s) : 0.0) - x);
    }
    if (bad) atomicOr(&s_fail, 1);
  }
  __syncthreads();
  const bool ok = s_fail == 0;
  for (int j = threadIdx.x; j < ldc; j += blockDim.x) {
    double v = 0.0;
    if (j < m && ok) {
      for (int q = 0; q < kResNodes; ++q) v += R[(size_t)j * NN + q];
      v *= kResH;
    }
    c[j] = v;
  }
  if (!ok && threadIdx.x == 0 && status) atomicOr(status + p, LOGDET_ST_LOG_FAILED);
}

// Gauss-Legendre nodes and weights on [0, 1] by Newton's method on P_N.
static GLRule gauss_legendre01() {
  GLRule g;
  const int N = kPadeNodes;
  for (int i = 0; i < N; ++i) {
    double x = cos(M_PI * (i + 0.75) / (N + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= N; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = N * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= N; ++k) {
        double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = N * (x * p1 - p0) / (x * x - 1.0);
    }
    g.x[i] = 0.5 * (x + 1.0);
    g.w[i] = 1.0 / ((1.0 - x * x) * dp * dp);  // = (2/((1-x^2)P'^2)) / 2 on [0,1]
  }
  return g;
}

size_t hesslog_workspace_doubles(int m, int nprobe, int band) {
  const size_t dense = (size_t)nprobe * 4 * m * m + 16;
  if (band < 0 || band > kResMaxBand) return dense;
  return std::max(dense, hesslog_band_workspace_doubles(m, nprobe));
}

int hessenberg_log_e1(const double* H, int ldh, const int* msteps, int m, int nprobe, double* c,
                      int ldc, double* ws, uint32_t* status, cudaStream_t st, int band) {
  if (m < 1 || m > kMaxSteps) {
    set_error("hessenberg log: m=%d must be in [1, %d]", m, kMaxSteps);
    return LOGDET_EINVAL;
  }
  if (band >= 0 && band <= kResMaxBand && band + 1 < m) {
    const size_t smem = sizeof(double) * (size_t)m * (band + 2);
    ProfScope prof(KC_SMALL, st);
#define LD_RES_CASE(B)                                                                   \
  case B:                                                                                \
    k_hesslog_band<B + 2><<<nprobe, kResThreads, smem, st>>>(H, ldh, msteps, m, c, ldc, ws, \
                                                             status);                    \
    break;
    switch (band) {
      LD_RES_CASE(0) LD_RES_CASE(1) LD_RES_CASE(2) LD_RES_CASE(3) LD_RES_CASE(4)
      LD_RES_CASE(5) LD_RES_CASE(6) LD_RES_CASE(7) LD_RES_CASE(8)
    }
#undef LD_RES_CASE
    LD_CHECK_LAUNCH();
    return LOGDET_OK;
  }
  static const GLRule gl = gauss_legendre01();
  // Work matrices in shared memory as far as they fit (see k_hesslog).
  const size_t mat = sizeof(double) * (size_t)m * m;
  const int smem_mats = 4 * mat <= 200 * 1024 ? 4 : 2 * mat <= 200 * 1024 ? 2 : 0;
  const size_t smem = smem_mats * mat;
  const int threads = kLogThreads;
  if (smem > 48 * 1024)
    LD_CUDA(cudaFuncSetAttribute(k_hesslog, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope prof(KC_SMALL, st);
  k_hesslog<<<nprobe, threads, smem, st>>>(H, ldh, msteps, m, c, ldc, ws, status, gl, smem_mats);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

// ===========================================================================
// Probe fill and block conversion.
// ===========================================================================
template <typename T>
__global__ void k_probe_fill(uint64_t key, const uint64_t* __restrict__ keyp, int n, int ncols,
                             int col0, T* out, int ld, int gaussian) {
  if (keyp) key = *keyp;
  const size_t total = (size_t)n * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int row = (int)(e / ld), c = (int)(e - (size_t)row * ld);
    double v = 0.0;
    if (c < ncols) v = probe_value(key, (uint32_t)(col0 + c), (uint32_t)row, gaussian);
    out[e] = cvt<T>(v);
  }
}

template <typename T>
int probe_fill(uint64_t key, int n, int ncols, int col0, T* out, int ld, cudaStream_t st,
               int gaussian, const uint64_t* keyp) {
  ProfScope prof(KC_OTHER, st, 0.0, (double)n * ld * sizeof(T));
  k_probe_fill<T><<<4 * sm_count(), 256, 0, st>>>(key, keyp, n, ncols, col0, out, ld, gaussian);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}
template int probe_fill<double>(uint64_t, int, int, int, double*, int, cudaStream_t, int,
                                 const uint64_t*);
template int probe_fill<float>(uint64_t, int, int, int, float*, int, cudaStream_t, int,
                                 const uint64_t*);
template int probe_fill<bf16>(uint64_t, int, int, int, bf16*, int, cudaStream_t, int,
                                 const uint64_t*);
template int probe_fill<f32x2>(uint64_t, int, int, int, f32x2*, int, cudaStream_t, int,
                                 const uint64_t*);

__global__ void k_fill_double(double* out, size_t count, double value) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = value;
}

int fill_double(double* out, size_t count, double value, cudaStream_t st) {
  ProfScope prof(KC_OTHER, st);
  k_fill_double<<<std::max(1, std::min(div_up((int)count, 256), 64)), 256, 0, st>>>(out, count, value);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* in, int ldin, Tout* out, int ldout, int n, int cols) {
  const size_t total = (size_t)n * ldout;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int row = (int)(e / ldout), c = (int)(e - (size_t)row * ldout);
    out[e] = (c < cols) ? cvt<Tout>(in[(size_t)row * ldin + c]) : cvt<Tout>(0.0);
  }
}

template <typename Tin, typename Tout>
int convert_block(const Tin* in, int ldin, Tout* out, int ldout, int n, int cols,
                  cudaStream_t st) {
  ProfScope prof(KC_OTHER, st, 0.0, (double)n * (ldin * sizeof(Tin) + ldout * sizeof(Tout)));
  k_convert<Tin, Tout><<<4 * sm_count(), 256, 0, st>>>(in, ldin, out, ldout, n, cols);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}
template int convert_block<double, double>(const double*, int, double*, int, int, int, cudaStream_t);
template int convert_block<double, float>(const double*, int, float*, int, int, int, cudaStream_t);
template int convert_block<float, double>(const float*, int, double*, int, int, int, cudaStream_t);
template int convert_block<double, bf16>(const double*, int, bf16*, int, int, int, cudaStream_t);
template int convert_block<bf16, double>(const bf16*, int, double*, int, int, int, cudaStream_t);
template int convert_block<double, f32x2>(const double*, int, f32x2*, int, int, int, cudaStream_t);
template int convert_block<f32x2, double>(const f32x2*, int, double*, int, int, int, cudaStream_t);

// ===========================================================================
// OSA-IOP sketch assembly: Y[:, p] = sum_j w[j][p] V_j[:, p]
// ===========================================================================
// Thread-level work: one vector chunk (Vec16<T>::N columns) of one row, the
// m basis blocks read four at a time (independent loads in flight), each
// column's sum over j in increasing order.  V has row stride ldv and block
// stride n * ldv; columns [0, ncols) are assembled (ncols and ldv multiples
// of N, V aligned to the chunk).
//
// FP64 blocks: FP64 fused multiply-adds, w read as vectors.  FP32 / BF16
// blocks: the FP64 pipe of this GPU (1/64 of the FP32 rate) would bound the
// kernel at m n ncols FMAs, so each sum runs in double-float arithmetic on
// the FP32 pipe instead: w_j split once per CTA into hi + lo floats (shared
// memory), the product with x (exact in hi: an FMA gives its rounding
// error) added by an error-free two-sum into a (hi, lo) pair; relative error
// about 2^-44 per sum, returned as hi + lo in FP64.  (Tables of more than
// kSketchSmemW weights, m ncols > 4096, take the FP64 form.)
constexpr int kSketchSmemW = 4096;

template <typename T, bool kDF>
__global__ void k_sketch_assemble(const T* __restrict__ V, int n, int ncols, int ldv, int m,
                                  const double* __restrict__ w, double* __restrict__ Y,
                                  int ldy) {
  constexpr int N = Vec16<T>::N;
  using CT = typename Compute<T>::type;
  __shared__ float2 sw[kDF ? kSketchSmemW : 1];
  if constexpr (kDF) {
    for (int i = threadIdx.x; i < m * ncols; i += blockDim.x) {
      const double x = w[i];
      const float hi = (float)x;
      sw[i] = make_float2(hi, (float)(x - (double)hi));
    }
    __syncthreads();
  }
  const int chunks = ncols / N;
  const size_t total = (size_t)n * chunks;
  const size_t stride_v = (size_t)n * ldv;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / chunks), p0 = (int)(e - (size_t)row * chunks) * N;
    const T* v0 = V + (size_t)row * ldv + p0;
    double acc[N];
    float sh[N], sl[N];
#pragma unroll
    for (int c = 0; c < N; ++c) acc[c] = 0.0, sh[c] = 0.f, sl[c] = 0.f;
    auto term = [&](int j, const CT (&x)[N]) {
      if constexpr (kDF) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
          const float2 wj = sw[j * ncols + p0 + c];
          if constexpr (std::is_same<T, f32x2>::value) {
            // double-float x: the product's cross term w_hi x_lo joins the
            // error word (w_lo x_lo is below the pair's precision)
            const float p = __fmul_rn(wj.x, x[c].hi);
            float pe = __fmaf_rn(wj.x, x[c].hi, -p);
            pe = __fmaf_rn(wj.y, x[c].hi, pe);
            pe = __fmaf_rn(wj.x, x[c].lo, pe);
            const float t = __fadd_rn(sh[c], p);
            const float z = __fsub_rn(t, sh[c]);
            const float err = __fadd_rn(__fsub_rn(sh[c], __fsub_rn(t, z)), __fsub_rn(p, z));
            sl[c] = __fadd_rn(sl[c], __fadd_rn(err, pe));
            sh[c] = t;
          } else {
            const float p = wj.x * x[c];
            float pe = fmaf(wj.x, x[c], -p);
            pe = fmaf(wj.y, x[c], pe);
            const float t = sh[c] + p;
            const float z = t - sh[c];
            const float err = (sh[c] - (t - z)) + (p - z);
            sl[c] += err + pe;
            sh[c] = t;
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < N; c += 2) {
          const double2 wv = *reinterpret_cast<const double2*>(w + (size_t)j * ncols + p0 + c);
          acc[c] = fma(wv.x, (double)x[c], acc[c]);
          acc[c + 1] = fma(wv.y, (double)x[c + 1], acc[c + 1]);
        }
      }
    };
    int j = 0;
    for (; j + 4 <= m; j += 4) {
      CT x[4][N];
#pragma unroll
      for (int u = 0; u < 4; ++u) load_vec<T>(v0 + (size_t)(j + u) * stride_v, x[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) term(j + u, x[u]);
    }
    for (; j < m; ++j) {
      CT x[N];
      load_vec<T>(v0 + (size_t)j * stride_v, x);
      term(j, x);
    }
#pragma unroll
    for (int c = 0; c < N; ++c) {
      if constexpr (kDF) acc[c] = (double)sh[c] + (double)sl[c];
      if (p0 + c < ldy) Y[(size_t)row * ldy + p0 + c] = acc[c];
    }
  }
}

template <typename T>
int sketch_assemble(const T* V, int n, int ld, int m, const double* w, double* Y, int ldy,
                    cudaStream_t st) {
  return sketch_assemble_cols<T>(V, n, ld, ld, m, w, Y, ldy, st);
}

// The same for ncols columns of basis blocks with leading dimension ldv (a
// column slice of a wider basis).
template <typename T>
int sketch_assemble_cols(const T* V, int n, int ncols, int ldv, int m, const double* w, double* Y,
                         int ldy, cudaStream_t st) {
  constexpr uintptr_t kAlign = sizeof(typename Vec16<T>::type);
  if (ncols % Vec16<T>::N || ldv % Vec16<T>::N || (reinterpret_cast<uintptr_t>(V) % kAlign)) {
    set_error("sketch assembly: columns %d / stride %d not in whole vector chunks", ncols, ldv);
    return LOGDET_EINVAL;
  }
  ProfScope prof(KC_OTHER, st, 2.0 * n * (double)ncols * m,
                 (double)n * ncols * (m * sizeof(T) + 8.0));
  bool launched = false;
  if constexpr (!std::is_same<T, double>::value) {
    if ((size_t)m * ncols <= (size_t)kSketchSmemW) {
      k_sketch_assemble<T, true><<<8 * sm_count(), 256, 0, st>>>(V, n, ncols, ldv, m, w, Y, ldy);
      launched = true;
    }
  }
  if (!launched)
    k_sketch_assemble<T, false><<<8 * sm_count(), 256, 0, st>>>(V, n, ncols, ldv, m, w, Y, ldy);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}
template int sketch_assemble_cols<double>(const double*, int, int, int, int, const double*, double*,
                                          int, cudaStream_t);
template int sketch_assemble_cols<float>(const float*, int, int, int, int, const double*, double*,
                                         int, cudaStream_t);
template int sketch_assemble_cols<bf16>(const bf16*, int, int, int, int, const double*, double*,
                                        int, cudaStream_t);
template int sketch_assemble_cols<f32x2>(const f32x2*, int, int, int, int, const double*, double*,
                                         int, cudaStream_t);

template int sketch_assemble<double>(const double*, int, int, int, const double*, double*, int, cudaStream_t);
template int sketch_assemble<float>(const float*, int, int, int, const double*, double*, int, cudaStream_t);
template int sketch_assemble<bf16>(const bf16*, int, int, int, const double*, double*, int, cudaStream_t);
template int sketch_assemble<f32x2>(const f32x2*, int, int, int, const double*, double*, int, cudaStream_t);

}  // namespace ld

// ===========================================================================
// Allocation-free Hessenberg logarithm.
//
// Some callers cannot allocate device memory while they run: hosts whose
// device memory is handed out once at start-up under a fixed budget,
// callers running under an external allocator (a framework's caching pool)
// that owns all device memory and forbids cudaMalloc/cudaFree, and loops
// that must not pay for cudaFree, which synchronises the whole device.  For
// them the same Hessenberg-log kernel can run on scratch that lives in this
// file: a statically sized device array, loaded once with the library and
// held by every GPU that loads it until the process exits.
//
// Limits: nprobe <= kNoAllocMaxProbes (status words), and when the four m x m
// work matrices do not fit in shared memory (m >= 81: 4 m^2 doubles above
// 200 KiB), 4 m^2 nprobe doubles must fit in kNoAllocMatDoubles (8 MiB).
// Larger requests are rejected.  All calls share the one array; two calls
// whose kernels overlap on the GPU (different streams, no ordering between
// them) race on it.  The array's device address is looked up once per device
// and kept for the life of the process, so the entry point must not be used
// after a reset of that device (cudaDeviceReset) in the same process.
// ===========================================================================
namespace ld {

constexpr size_t kNoAllocMatDoubles = (size_t)1 << 20;  // 8 MiB of work matrices
constexpr int kNoAllocMaxProbes = 4096;                 // 16 KiB of status words
constexpr size_t kNoAllocBytes = kNoAllocMatDoubles * sizeof(double) + kNoAllocMaxProbes * sizeof(uint32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the first call on a device does it; make that first call
// before any stream capture).
int noalloc_scratch(void** out) {
  int dev = 0;
  LD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range for the allocation-free path", dev);
    return LOGDET_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      return LOGDET_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return LOGDET_OK;
}
}  // namespace

}  // namespace ld

extern "C" int logdet_hessenberg_log_e1_noalloc(const double* H, int32_t ldh,
                                                const int32_t* msteps, int32_t m,
                                                int32_t nprobe, double* c, uint32_t* status,
                                                void* cuda_stream) {
  using namespace ld;
  if (!H || !c || m < 1 || m > kMaxSteps || nprobe < 1 || ldh < m) {
    set_error("hessenberg_log_e1_noalloc: bad arguments (1 <= m <= %d, ldh >= m)", kMaxSteps);
    return LOGDET_EINVAL;
  }
  if (nprobe > kNoAllocMaxProbes) {
    set_error("hessenberg_log_e1_noalloc: nprobe=%d exceeds the static limit %d", nprobe,
              kNoAllocMaxProbes);
    return LOGDET_EINVAL;
  }
  const bool fits_smem = 4 * sizeof(double) * (size_t)m * m <= 200 * 1024;
  if (!fits_smem && 4 * (size_t)m * m * nprobe > kNoAllocMatDoubles) {
    set_error("hessenberg_log_e1_noalloc: 4*m^2*nprobe = %zu doubles exceeds the static "
              "scratch of %zu doubles (m=%d, nprobe=%d)",
              4 * (size_t)m * m * nprobe, kNoAllocMatDoubles, m, nprobe);
    return LOGDET_EINVAL;
  }
  void* base = nullptr;
  LD_TRY(noalloc_scratch(&base));
  double* ws = static_cast<double*>(base);
  uint32_t* st_words = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) +
                                                   kNoAllocMatDoubles * sizeof(double));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // Status words accumulate with atomicOr: they must start at zero.  The work
  // matrices are written before they are read and need no clearing.
  LD_CUDA(cudaMemsetAsync(st_words, 0, sizeof(uint32_t) * nprobe, st));
  LD_TRY(hessenberg_log_e1(H, ldh, msteps, m, nprobe, c, m, ws, st_words, st));
  uint32_t acc = 0, buf[256];
  for (int p0 = 0; p0 < nprobe; p0 += 256) {
    const int cnt = std::min(256, nprobe - p0);
    LD_CUDA(cudaMemcpyAsync(buf, st_words + p0, sizeof(uint32_t) * cnt, cudaMemcpyDeviceToHost, st));
    LD_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < cnt; ++i) acc |= buf[i];
  }
  if (status) *status = acc;
  return LOGDET_OK;
}
