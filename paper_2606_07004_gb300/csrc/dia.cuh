// Diagonal fast path of the SpMM pass for FP32 blocks (see dia.cu).
#pragma once

#include "handle.cuh"
#include "krylov.cuh"

namespace ld {

constexpr int kDiaBandGap = 8;    // offsets at most this far apart share a staged band
constexpr int kDiaMaxExt = 16;    // largest band extent handled
constexpr int kDiaRows = 8;       // rows a CTA computes at once (CTA = 8 x width / 4 threads)
constexpr int kDiaSmemTarget = 56 * 1024;  // staged bytes per CTA (several CTAs per SM)

// At handle creation (host CSR): record the diagonal structure when every
// entry lies on at most kMaxDiags diagonals and the bands are narrow.
int dia_build(logdet_ctx* h, const int* rowptr, const int* colind);

// Values of Q / c per diagonal, [ndiag][n] (0 where a row has no entry on a
// diagonal); the division in FP64 as for the CSR values.
int dia_values_f32(const logdet_ctx* h, double c, float* out, cudaStream_t st);

// Tile rows of the diagonal path for a slice of `width` FP32 columns; 0 when
// the matrix or the slice does not take it.
int dia_tile_rows(const logdet_ctx* h, int width);

// Fill the job's tensor map for x (n x ld FP32, box of width columns and
// box_rows rows).
int dia_encode_x(SpmmJob<float>& J, const float* x, int n, int ld, int width, int box_rows);

// Batched launch of diagonal-path jobs (all with dia != nullptr), with the
// CTA size of the jobs' CSR geometry.
int launch_spmm_dia(const SpmmBatch<float>& b, int threads, cudaStream_t s);

}  // namespace ld
