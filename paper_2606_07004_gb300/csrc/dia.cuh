// Line-sweep path of the SpMM pass for FP32 blocks of stencil matrices (see
// dia.cu).
#pragma once

#include "handle.cuh"
#include "krylov.cuh"

namespace ld {

constexpr int kSweepMaxA = 3;           // lines -A..A held at once: at most 7
constexpr int kPlaneMaxA = 2;           // plane sweep: planes -A..A, in-plane radii
constexpr int kPlaneMaxR = 4;           //   |dy| <= 2, |dx| <= kPlaneMaxR
constexpr int kSweepMaxCw = 16;         // extra rows of a line window
constexpr int kSweepMinL = 32;          // shortest line
constexpr int kSweepPrefetch = 2;       // windows loaded ahead of the sweep
constexpr int kSweepSmemBudget = 110 * 1024;  // per CTA (two CTAs per SM)

// Diagonal values per row, padded to a multiple of four (one 16-byte vector
// per four diagonals).
__host__ __device__ inline int dia_pad(int ndiag) { return (ndiag + 3) & ~3; }

// Grid structure of host CSR arrays (sorted columns, n >= 4096), see
// DiaInfo: a 2D line structure if there is one, else a 3D grid stencil;
// false (and *out zeroed) when there is neither.  Host only.
bool dia_detect(int n, const int* rowptr, const int* colind, DiaInfo* out);

// At handle creation (host CSR): record the grid structure when every entry
// lies on at most kMaxDiags diagonals that fit one (see DiaInfo): a 2D line
// structure if there is one, else a 3D grid stencil.
int dia_build(logdet_ctx* h, const int* rowptr, const int* colind);

// Values of Q / c per row and diagonal, [n][dia_pad(ndiag)] (0 where a row
// has no entry on a diagonal); the division in FP64 as for the CSR values.
int dia_values_f32(const logdet_ctx* h, double c, float* out, cudaStream_t st);

// Sweep geometry of a block slice of `width` FP32 columns processed by CTAs
// of `threads`: points per segment or tile T (dim 2: a multiple of the row
// groups), lines or planes per unit, segments or tiles per line or plane,
// lines or planes, units.  Returns false when the matrix or
// the slice does not take the sweep (then the CSR path runs).
struct SweepGeom {
  int T, kc, nseg, nlines, units;
  int tx, ty, txs;  // plane sweep: tile tx (= 1 << txs) x ty points
};
bool dia_sweep_geom(const logdet_ctx* h, int width, int threads, SweepGeom* g);

// Fill the job's tensor maps: x (n x ld FP32; box of width columns and
// T + cw rows, or a 3D box of tx + 2 Ax by ty + 2 Ay points of one plane)
// and the values (box of T rows, or tx by ty points).
int dia_encode(SpmmJob<float>& J, const float* x, int n, int ld, int width);

// Batched launch of sweep jobs (all with dia != nullptr), CTAs of `threads`.
int launch_spmm_dia(const SpmmBatch<float>& b, int threads, cudaStream_t s);

}  // namespace ld
