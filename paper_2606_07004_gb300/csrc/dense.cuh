// Dense and small-matrix kernels of the estimators: Hutch++ QR and
// projection (FP64, or FP32 with compensated sums for FP32 blocks), batched
// tridiagonal Gauss rules, batched Hessenberg logarithms, OSA-IOP sketch
// assembly and quadratic forms (FP64).
#pragma once

#include "common.cuh"

namespace ld {

constexpr int kMaxSketch = 64;  // s <= 64 columns per QR
constexpr int kMaxSteps = 256;  // m <= 256 Krylov steps (small solves)

// Workspace sizes (doubles) for orth() on n rows and s columns.
size_t orth_workspace_doubles(int n, int s);

// A = orth(Y) by two rounds of Cholesky QR.  Y and A may alias.  `ws` must
// hold orth_workspace_doubles(n, s) doubles.  keep_dev (s ints, optional)
// receives 1 for kept columns.  s_eff_host receives the kept count (one
// device-to-host copy, stream-synchronising) when non-null.
int orth_fp64(int n, int s, const double* Y, int ldy, double* A, int lda, double* ws,
              int* keep_dev, int* s_eff_host, cudaStream_t st);

// The same split for FP32 blocks (mixed-precision solves): Gram and A^T G
// sums are compensated FP32 dots (Dot2) read out in FP64, the Cholesky
// factor and its inverse FP64, the applies and the residual in FP32.  A is
// orthonormal to FP32 rounding, the accuracy the FP32 Krylov runs start
// from in any case.  s_eff_host as for orth_fp64.
int orth_f32(int n, int s, const float* Y, int ldy, float* A, int lda, double* ws,
             int* keep_dev, int* s_eff_host, cudaStream_t st);
int project_residual_f32(int n, int s, int r, const float* A, int lda, uint64_t key, float* X,
                         int ldx, int zcol0, double* ws, cudaStream_t st, int gaussian = 0,
                         const uint64_t* keyp = nullptr);

// Z = G - A (A^T G) with G the probe block of (key, columns 0..r-1)
// generated on the fly; written into X[:, zcol0 .. zcol0+r) (leading dim ldx).
// With keyp non-null the kernels read the key from device memory at run time
// instead (graph replays with a new seed).
int project_residual_fp64(int n, int s, int r, const double* A, int lda, uint64_t key,
                          double* X, int ldx, int zcol0, double* ws, cudaStream_t st,
                          int gaussian = 0, const uint64_t* keyp = nullptr);
size_t project_workspace_doubles(int n, int s, int r);

// out[i] = sum_t part[i * ntiles + t] for i < nrows (FP64 partials).
int reduce_partials_fp64(const double* part, int nrows, int ntiles, double* out, cudaStream_t st);

// Per-column squared norms of a block (FP64 or FP32 elements): partials
// [ld][ntiles] in the Krylov layout, for k_init_sigma.
template <typename T>
int colnorm_partials(const T* X, int n, int ld, int tile_rows, int ntiles,
                     typename PartOf<T>::type* part, int threads, cudaStream_t st);

// Gauss quadrature sum_k tau_k^2 log(theta_k) of symmetric tridiagonals.
int gauss_quadrature_log(const double* alpha, const double* beta, int ldab, const int* msteps,
                         int m, int nprobe, double clamp_lo, double* out, uint32_t* status,
                         cudaStream_t st);

// c_p = log(H_p) e_1 for nprobe upper Hessenberg matrices (column-major,
// leading dim ldh, H_p at H + p*ldh*m).  band >= 0: the matrices are zero
// above upper bandwidth `band` (IOP window k: band = k - 1), which selects
// the resolvent quadrature for band <= 8 and band + 1 < m; otherwise
// inverse scaling and squaring.  ws: hesslog_workspace_doubles(m, nprobe, band).
size_t hesslog_workspace_doubles(int m, int nprobe, int band = -1);
int hessenberg_log_e1(const double* H, int ldh, const int* msteps, int m, int nprobe,
                      double* c, int ldc, double* ws, uint32_t* status, cudaStream_t st,
                      int band = -1);

// Probe fill, columns col0..col0+ncols of stream key (keyp: as for
// project_residual_fp64).
template <typename T>
int probe_fill(uint64_t key, int n, int ncols, int col0, T* out, int ld, cudaStream_t st,
               int gaussian = 0, const uint64_t* keyp = nullptr);

// out[i] = value for i < count.
int fill_double(double* out, size_t count, double value, cudaStream_t st);

// Copy/convert a block with the same layout (FP64 <-> FP32).
template <typename Tin, typename Tout>
int convert_block(const Tin* in, int ldin, Tout* out, int ldout, int n, int cols,
                  cudaStream_t st);

// OSA-IOP sketch: Y[:, p] = sum_{j=1}^{m_p} w[j][p] V_j[:, p], V_j = V + (j-1)*n*ld.
template <typename T>
int sketch_assemble(const T* V, int n, int ld, int m, const double* w, double* Y, int ldy,
                    cudaStream_t st);
// The same for ncols columns of basis blocks of leading dimension ldv.
template <typename T>
int sketch_assemble_cols(const T* V, int n, int ncols, int ldv, int m, const double* w, double* Y,
                         int ldy, cudaStream_t st);

}  // namespace ld
