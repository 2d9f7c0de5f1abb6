// Krylov step kernels: the per-step block passes and the per-probe scalar
// updates shared by Lanczos (OSLQ, Sec. 3.1) and Arnoldi-IOP (Algorithm 1).
//
// Vectors are stored unnormalised: the basis vector v_j of probe p is
// sigma_j[p] * u_j[:, p], with u_j the stored column and sigma_j a per-probe
// FP64 scalar.  One step j of a block of probes is
//
//   pass 1  (k_spmm)    y = A u_j                     (A = Q/alpha or Q/gamma)
//                       d_i = u_i^T y  for the window vectors u_i
//   scalar  (k_coef)    H_{i,j} = sigma_i sigma_j d_i  (Lanczos: alpha_j)
//                       coefficients of pass 2
//   pass 2  (k_update)  u_{j+1} = a (y - sum_i c_i u_i),  |u_{j+1}|^2 [, u_1^T u_{j+1}]
//   scalar  (k_norm)    h = sigma_j |u_{j+1}| / a, sigma_{j+1} = sigma_j / (a h)
//
// a is 1 unless sigma drifts out of range, then an exact power of two.  In
// exact arithmetic this is the normalised recurrence of the paper: only the
// rounding of the stored vectors differs.
//
// Every kernel takes a batch of independent jobs (blocks of probes, possibly
// on different matrices) in one launch; a single solve is a batch of one.
// Per-tile partial sums are reduced in a fixed order, so a job's result does
// not depend on what else is in the batch.
#pragma once

#include "common.cuh"

namespace ld {

constexpr int kMaxWin = 9;    // window vectors per pass (window k <= 8, plus slack)
constexpr int kMaxJobs = 24;  // jobs per batched launch
// Rows longer than this are split across a whole CTA.  Measured on the
// 2M-row power-law graph (SpMM, OSA-IOP m = 20, FP32, window 4): threshold
// 64 (24k split rows) 55.8 ms, 128 46.2, 256 43.3, 512 43.0, 1024 48.8,
// 2048 59.2; window 8 151.9 -> 108.7 ms and FP64 138.1 -> 114.1 ms at 256:
// each split row pays two CTA barriers and its item's dot reduction, while
// a row of up to 256 entries takes 64 four-gather batches in one row group.
constexpr int kSplitRowNnz = 256;
constexpr int kRedThreads = 256;  // threads of one scalar reduction (a k_scalar CTA)

// ---------------------------------------------------------------------------
// pass 1: SpMM with fused window dots
// ---------------------------------------------------------------------------
template <typename T>
struct SpmmJob {
  const int* rowptr;
  const int* colind;
  const typename ValOf<T>::type* vals;  // matrix values (FP32 for BF16 blocks)
  const T* x;                      // gather source, n x ld
  T* y;                            // output, n x ld (may be null: dots only is not supported)
  const T* dotv[kMaxWin];          // vectors dotted with y, n x ld each
  typename PartOf<T>::type* part;  // [ndots][ld][ntiles]
  const double* colscale;          // optional [ld]: y[:,p] *= colscale[p]
  const double* colshift;          // optional [ld]: y[:,p] += colshift[p] * x[:,p] (before scale)
  // Work items.  nullptr: ntiles uniform tiles of tile_rows rows, partial
  // slot = tile.  Otherwise ntiles items in launch order, each {r0, r1, slot,
  // 0}: rows [r0, r1) spread over the CTA's row groups (r1 > r0), or, with
  // r1 < 0, the single long row r0 whose nonzeros all row groups share; slot
  // is the item's partial index (the items in row order), so results do not
  // depend on the launch order.
  const int4* items;
  int n, ld, ndots, tile_rows, ntiles;
  int col_off, width;              // columns [col_off, col_off+width) of the block (width % vec == 0)
  int b;                           // live columns in this slice (accounting only)
  long long nnz;                   // (accounting only)
  // Line- and plane-sweep paths (FP32 blocks of a matrix with grid
  // structure, see dia.cu); dia == nullptr: CSR path.  dim 2: the rows are
  // cut into segments of dia_T rows within each line of L rows; dim 3: each
  // plane into tiles of dia_tx x dia_ty points.  A unit is one segment or
  // tile position swept over dia_kc consecutive lines or planes, and ntiles
  // counts the units (their index is the partial slot).  dia: values per row and diagonal
  // [n][dia_pad(ndiag)]; tmap: x, box of width columns x (dia_T + cw) rows;
  // vmap: the values, box of dia_T rows; err: set if a bounded wait gives up.
  const float* dia;
  int* err;
  int dia_T, dia_kc, dia_nseg, dia_nlines;
  int dia_tx, dia_ty, dia_txs;     // plane sweep: tile of tx (= 1 << txs) x ty points, T = tx ty
  DiaInfo dinfo;
  CUtensorMap tmap;
  CUtensorMap vmap;
};

template <typename T>
struct SpmmBatch {
  int njobs, total_tiles;
  int tile_start[kMaxJobs + 1];
  SpmmJob<T> jobs[kMaxJobs];
};

// ---------------------------------------------------------------------------
// pass 2: window update with fused norm (and optional dot with u_1)
// ---------------------------------------------------------------------------
template <typename T>
struct UpdJob {
  const T* y;
  const T* basis[kMaxWin];
  const double* coef;              // [nbasis][ld]
  const double* ycoef;             // [ld]
  T* out;
  const T* extra;                  // optional: dot out with extra
  typename PartOf<T>::type* part;  // [1 or 2][ld][ntiles]
  int n, ld, nbasis, tile_rows, ntiles;
  int col_off, width;              // column slice, as in SpmmJob
  int b;                           // live columns in this slice (accounting only)
};

template <typename T>
struct UpdBatch {
  int njobs, total_tiles;
  int tile_start[kMaxJobs + 1];
  UpdJob<T> jobs[kMaxJobs];
};

// ---------------------------------------------------------------------------
// per-probe scalar state of one Krylov run over a block (device arrays)
// ---------------------------------------------------------------------------
struct KrylovState {
  int method;        // 0 = Lanczos (3-term), 1 = IOP window k
  int b, ld, m, k;   // probes, leading dim, max steps, window
  double tol;
  double rescale_lim;  // |log2 sigma| beyond which a power-of-two rescale is applied
  double* alpha;     // Lanczos: [p*m + j-1]
  double* beta;      // Lanczos: [p*m + j-1]  (beta_j, j = 1..m-1)
  double* H;         // IOP: [p*(m+1)*m + (j-1)*(m+1) + (i-1)]  column-major H(i,j)
  double* sig;       // [p*(m+2) + j]  sigma_j, j = 1..m+1
  double* edot;      // optional [p*(m+2) + j]  u_1^T u_j
  double* coef;      // [kMaxWin][ld]  pass-2 coefficients (window order)
  double* ycoef;     // [ld]
  int* meff;         // [p] completed steps
  int* active;       // [p]
  uint32_t* status;  // [p] status bits
  double* dbuf;      // [kMaxWin][ld] reduced dots of the current scalar step
  unsigned* cnt;     // [ld] arrival counters (zero between launches)
};

struct ScalarJob {
  KrylovState st;
  const void* part;   // partials to reduce
  int part_f32;       // 1 = float2 (compensated FP32) partials
  int ntiles;
  int step;           // j (1-based)
  int ndots;          // number of dots in part
  int win_lo;         // first window index i (1-based) for IOP / Lanczos
  int last;           // 1 = last step (no pass 2 follows)
};

struct ScalarBatch {
  int njobs;
  int probe_start[kMaxJobs + 1];
  ScalarJob jobs[kMaxJobs];
};

// ---------------------------------------------------------------------------
// persistent Krylov run: every remaining step of one run in one cooperative
// launch, for blocks small enough that launch gaps, not the passes, set the
// step time.  A step is pass 1, a grid barrier, the coefficients, pass 2, a
// grid barrier, the norms: every CTA reduces the partials itself (a warp per
// dot, in the operand order of the 256-thread reduction) and runs the
// per-probe recurrences in shared memory, so it needs no barrier after them.
// The passes are the step kernels' own tile loops in the same CTA size and
// tile geometry, so results are bit-identical to the step-by-step path.
// Measured on GB300 (2D Laplacian 64^2, FP64, 30 steps): 0.90 ms per run,
// about what the 4 kernels per step of the step path take: each phase is
// latency-bound like a kernel boundary, and the partial sums every CTA
// reduces are FP64 additions, which GB300 issues at 2 lanes per clock per
// SM (the FP64 pipe was 48 % busy).  Opt-in: LOGDET_KRYLOV_PERSISTENT=1.
// ---------------------------------------------------------------------------
template <typename Job>
struct OneJob {  // a batch of one job (the members the tile loops read)
  int njobs, total_tiles;
  int tile_start[2];
  Job jobs[1];
};

template <typename T>
struct PersistRun {
  SpmmJob<T> sj;   // pass-1 job: fields that do not change with the step
  UpdJob<T> uj;    // pass-2 job: the same
  ScalarJob cj;    // scalar jobs: st, part, part_f32
  T* X0;           // u_1
  T* ring;         // ring of nring blocks for u_2, u_3, ... (no Vfull)
  T* Vfull;        // or the full basis, u_j at Vfull + (j-1) blk
  size_t blk;      // n * ld
  int nring, method, k, m, j0, track_e, ntiles;
  unsigned* bar;   // [2]: arrivals and generation of the grid barrier (zero at launch)
  int* err;        // set to 1 when a barrier wait gives up
  unsigned nwait;  // arrivals that complete a barrier (the grid size)
  long long limit_ns;  // bound of one barrier wait (global timer)
};

// Cooperative launch of the run (CTA size threads; nd_max / nb_max: the
// most window dots / basis vectors a step of it takes).  LOGDET_ECUDA when
// the launch is refused.
template <typename T>
int launch_krylov_run(const PersistRun<T>& P, int threads, int nd_max, int nb_max,
                      cudaStream_t s);

// Tile geometry for a block of leading dimension ld with elements of
// `vec` entries per 16-byte load: threads per CTA and rows per tile.
struct TileGeom {
  int threads;   // CTA size
  int rows_per_iter;
  int tile_rows;
};
// Geometry for a slice of `width` columns.  threads_hint (a multiple of both
// 32 and width/vec, <= 512) and iters_hint (rows per tile = rows per CTA
// iteration x iters) override the defaults when valid.  Without iters_hint,
// a block of n rows (n > 0) too short to give two tiles per SM gets shallower
// tiles (down to one row per thread group), so that small problems still
// spread over the whole GPU.
TileGeom tile_geom(int width, int vec, int threads_hint = 0, int iters_hint = 0, int n = 0);

// Tunable layout of a Krylov run: the block's columns are processed as
// `split` slices of ld/split columns, with the CTA size and tile depth above.
struct TuneCfg {
  int split = 1;
  int threads = 0;  // 0 = default
  int iters = 0;    // 0 = default
};

// Launchers (krylov.cu).  `grid_cap` bounds the persistent grid.
template <typename T> int launch_spmm(const SpmmBatch<T>& b, int threads, cudaStream_t s);
template <typename T> int launch_update(const UpdBatch<T>& b, int threads, cudaStream_t s);
enum ScalarKind { SK_INIT = 0, SK_COEF = 1, SK_NORM = 2 };
int launch_coef(const ScalarBatch& b, cudaStream_t s);
int launch_norm(const ScalarBatch& b, cudaStream_t s);
int launch_init_sigma(const ScalarBatch& b, cudaStream_t s);

int sm_count();

// Job of global tile gt in a batch (tile_start ascending).
template <typename Batch>
__device__ __forceinline__ int find_job(const Batch& B, int gt) {
  int j = 0;
  while (j + 1 < B.njobs && gt >= B.tile_start[j + 1]) ++j;
  return j;
}

// Reduce the per-thread accumulators of all rows of the CTA for one dot and
// write one partial per column.  smem holds blockDim.x * V accumulators.
// The CTA owns columns [col_off, col_off + width) of the block; partials are
// indexed by the block column.
template <typename T, typename Acc>
__device__ __forceinline__ void cta_reduce_write(Acc* smem, const Acc (&acc)[Vec16<T>::N],
                                                 bool live, int G, int R, int col_off, int width,
                                                 typename PartOf<T>::type* dst, int ntiles,
                                                 int tile) {
  constexpr int V = Vec16<T>::N;
  __syncthreads();
  if (live) {
#pragma unroll
    for (int v = 0; v < V; ++v) smem[threadIdx.x * V + v] = acc[v];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < width; c += blockDim.x) {
    int g = c / V, v = c - (c / V) * V;
    Acc t;
    t.zero();
    for (int rr = 0; rr < R; ++rr) t.add(smem[(rr * G + g) * V + v]);
    put_part(dst + (size_t)(col_off + c) * ntiles + tile, t);
  }
}

}  // namespace ld
