// Diagonal fast path of the SpMM pass for FP32 blocks.
//
// Stencil operators (the Laplacians, the Matérn operator) keep every entry on
// a few diagonals.  Instead of gathering x rows through the column indices
// (one dependent round trip per batch of nonzeros), a CTA stages, for a tile
// of T output rows, one block of x rows per band of nearby diagonals with a
// TMA 2D copy (cp.async.bulk.tensor, completion on an mbarrier), and reads
// every neighbour from shared memory.  Rows outside the matrix are filled
// with zeros by the copy; the values per diagonal are 0 where a row has no
// entry.  Each row sums over the diagonals in ascending offset order, which
// is the CSR column order of the CSR path, so y is the same FP32 sum.
#include "dia.cuh"
#include "profile.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

namespace ld {

// ---------------------------------------------------------------------------
// Structure
// ---------------------------------------------------------------------------
int dia_build(logdet_ctx* h, const int* rowptr, const int* colind) {
  memset(&h->dia, 0, sizeof h->dia);
  const int n = h->n;
  if (n < 4096 || h->nnz <= 0) return LOGDET_OK;
  std::vector<int> offs;
  for (int i = 0; i < n; ++i) {
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      const int o = colind[q] - i;
      if (std::find(offs.begin(), offs.end(), o) == offs.end()) {
        offs.push_back(o);
        if ((int)offs.size() > kMaxDiags) return LOGDET_OK;  // not diagonal-structured
      }
    }
  }
  std::sort(offs.begin(), offs.end());
  DiaInfo d;
  memset(&d, 0, sizeof d);
  d.ndiag = (int)offs.size();
  for (int k = 0; k < d.ndiag; ++k) d.off[k] = offs[k];
  int lo = offs[0], prev = offs[0];
  d.band_lo[0] = lo;
  int nb = 0;
  for (int k = 0; k < d.ndiag; ++k) {
    if (k > 0 && offs[k] - prev > kDiaBandGap) {
      d.maxext = std::max(d.maxext, prev - lo);
      lo = offs[k];
      d.band_lo[++nb] = lo;
    }
    d.diag_band[k] = nb;
    d.diag_shift[k] = offs[k] - lo;
    prev = offs[k];
  }
  d.maxext = std::max(d.maxext, prev - lo);
  d.nbands = nb + 1;
  if (d.maxext > kDiaMaxExt) return LOGDET_OK;
  // CSR entry -> diagonal index.
  std::vector<int> slot((size_t)h->nnz);
  for (int i = 0; i < n; ++i)
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q)
      slot[q] = (int)(std::lower_bound(offs.begin(), offs.end(), colind[q] - i) - offs.begin());
  if (cudaMalloc(&h->dia_slot, sizeof(int) * slot.size()) != cudaSuccess) {
    cudaGetLastError();
    h->dia_slot = nullptr;
    return LOGDET_OK;  // the CSR path still works
  }
  if (cudaMemcpy(h->dia_slot, slot.data(), sizeof(int) * slot.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    set_error("copy of the diagonal map failed");
    return LOGDET_ECUDA;
  }
  h->dia = d;
  return LOGDET_OK;
}

template <typename V>
__global__ void k_dia_values(const int* __restrict__ rowptr, const int* __restrict__ slot,
                             const V* __restrict__ vals, int n, double c, float* __restrict__ out) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x)
    for (int q = rowptr[row]; q < rowptr[row + 1]; ++q)
      out[(size_t)slot[q] * n + row] = (float)((double)vals[q] / c);
}

int dia_values_f32(const logdet_ctx* h, double c, float* out, cudaStream_t st) {
  const int n = h->n;
  LD_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)h->dia.ndiag * n, st));
  ProfScope prof(KC_OTHER, st);
  const int blocks = std::max(1, std::min(div_up(n, 256), 8 * sm_count()));
  if (h->vals_dtype == LOGDET_VALS_F64)
    k_dia_values<double><<<blocks, 256, 0, st>>>(h->rowptr, h->dia_slot, (const double*)h->vals,
                                                 n, c, out);
  else
    k_dia_values<float><<<blocks, 256, 0, st>>>(h->rowptr, h->dia_slot, (const float*)h->vals, n,
                                                c, out);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

// T rows per tile: the staged bands (nbands x (T + maxext) rows x width
// floats) kept near kDiaSmemTarget, T a multiple of kDiaRows in [8, 128].
int dia_tile_rows(const logdet_ctx* h, int width) {
  const DiaInfo& d = h->dia;
  if (d.ndiag == 0 || !h->dia_slot || width % 4 || width > 256 || width < 4) return 0;
  const int row_bytes = width * 4;
  int T = kDiaSmemTarget / (d.nbands * row_bytes) - d.maxext;
  T = T / kDiaRows * kDiaRows;
  T = std::max(kDiaRows, std::min(T, 128));
  if (T + d.maxext > 256) T = (256 - d.maxext) / kDiaRows * kDiaRows;
  return T;
}

// ---------------------------------------------------------------------------
// Tensor maps
// ---------------------------------------------------------------------------
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

int dia_encode_x(SpmmJob<float>& J, const float* x, int n, int ld, int width, int box_rows) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  });
  if (!g_encode) {
    set_error("cuTensorMapEncodeTiled is not available");
    return LOGDET_ECUDA;
  }
  if (((uintptr_t)x & 15) || (ld * 4) % 16 || width > 256 || width < 4 || width % 4 ||
      box_rows > 256 || box_rows < 1) {
    set_error("diagonal path: block not aligned for TMA");
    return LOGDET_EINVAL;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)width, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(&J.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(x), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LOGDET_ECUDA;
  }
  return LOGDET_OK;
}

// ---------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
constexpr int kDiaWaitLimit = 1 << 20;  // try_wait polls before a wait is abandoned

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait for the barrier's phase to complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase) {
  for (int i = 0; i < kDiaWaitLimit; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}
// 2D tiled copy of the box at (x = column, y = row) into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// ---------------------------------------------------------------------------
// y = A x and the window dots for FP32 blocks of a diagonal-structured
// matrix.  Same tiles, CTA shape, per-thread row order and partial slots as
// k_spmm (thread (r, g) owns rows r, r + R, ... of the tile and 16-byte chunk
// g), so the result is bit-identical to the CSR path.  A tile is processed in
// sub-tiles of dia_T rows: thread 0 arms the mbarrier with the byte count and
// issues one TMA copy per band (dia_T + maxext rows from row r0 + band_lo);
// every thread waits on the barrier with a bounded poll; the CTA decides
// together (__syncthreads_or) to go on or, if a wait gave up, to wait once
// more for the copies in flight, set the job's error flag and return.
// ---------------------------------------------------------------------------
template <int NDOT>
__global__ void __launch_bounds__(512) k_spmm_dia(const __grid_constant__ SpmmBatch<float> B) {
  constexpr int V = 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  float* stage = reinterpret_cast<float*>(smem_raw + 128);
  AccF* red = reinterpret_cast<AccF*>(smem_raw + 128);  // reused for the dot reduction
  const uint32_t bar_a = smem_addr(bar);
  if (threadIdx.x == 0) {
    mbar_init(bar_a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int gt = blockIdx.x; gt < B.total_tiles; gt += gridDim.x) {
    const int jb = find_job(B, gt);
    const SpmmJob<float>& J = B.jobs[jb];
    const DiaInfo& D = J.dinfo;
    const int tile = gt - B.tile_start[jb];
    const int G = J.width / V;
    const int R = blockDim.x / G;
    const int r = threadIdx.x / G;
    const int g = threadIdx.x - r * G;
    const bool live = r < R;
    const int row0 = tile * J.tile_rows;
    const int row1 = min(row0 + J.tile_rows, J.n);
    const int col0 = J.col_off + g * V;
    const int ndots = J.ndots;
    const int rows_box = J.dia_T + D.maxext;
    // Band regions start on 128-byte boundaries (TMA destinations).
    const int band_floats = (rows_box * J.width + 31) / 32 * 32;
    const bool has_scale = J.colscale != nullptr, has_shift = J.colshift != nullptr;
    int dz = 0;  // the main diagonal (every row stores it)
    for (int d = 0; d < D.ndiag; ++d)
      if (D.off[d] == 0) dz = d;

    AccF acc[NDOT > 0 ? NDOT : 1][V];
#pragma unroll
    for (int d = 0; d < (NDOT > 0 ? NDOT : 1); ++d)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[d][v].zero();

    for (int s0 = row0; s0 < row1; s0 += J.dia_T) {
      __syncthreads();  // the previous sub-tile's reads of the stage are done
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar_a, (uint32_t)(D.nbands * rows_box * J.width * (int)sizeof(float)));
        for (int b = 0; b < D.nbands; ++b)
          tma_load_2d(smem_addr(stage + (size_t)b * band_floats), &J.tmap, J.col_off,
                      s0 + D.band_lo[b], bar_a);
      }
      const bool ok = mbar_wait_bounded(bar_a, phase);
      if (__syncthreads_or(!ok)) {
        mbar_wait_bounded(bar_a, phase);  // let copies in flight land before leaving
        if (threadIdx.x == 0) atomicExch(J.err, 1);
        return;
      }
      phase ^= 1;
      if (live) {
        const int s1 = min(s0 + J.dia_T, row1);
        for (int row = s0 + r; row < s1; row += R) {
          const int rr = row - s0;
          float s[V] = {0.f, 0.f, 0.f, 0.f};
          for (int d = 0; d < D.ndiag; ++d) {
            const float a = __ldg(J.dia + (size_t)d * J.n + row);
            const float4 xv = *reinterpret_cast<const float4*>(
                stage + (size_t)D.diag_band[d] * band_floats +
                (size_t)(rr + D.diag_shift[d]) * J.width + g * V);
            s[0] = fmaf(a, xv.x, s[0]);
            s[1] = fmaf(a, xv.y, s[1]);
            s[2] = fmaf(a, xv.z, s[2]);
            s[3] = fmaf(a, xv.w, s[3]);
          }
          if (has_shift || has_scale) {
            const float4 xr = *reinterpret_cast<const float4*>(
                stage + (size_t)D.diag_band[dz] * band_floats +
                (size_t)(rr + D.diag_shift[dz]) * J.width + g * V);
            const float xs[V] = {xr.x, xr.y, xr.z, xr.w};
#pragma unroll
            for (int v = 0; v < V; ++v) {
              if (has_shift) s[v] = fmaf((float)J.colshift[col0 + v], xs[v], s[v]);
              if (has_scale) s[v] = s[v] * (float)J.colscale[col0 + v];
            }
          }
          store_vec<float>(J.y + (size_t)row * J.ld + col0, s);
#pragma unroll
          for (int d = 0; d < NDOT; ++d) {
            if (d < ndots) {
              float u[V];
              load_vec<float>(J.dotv[d] + (size_t)row * J.ld + col0, u);
#pragma unroll
              for (int v = 0; v < V; ++v) acc[d][v].fma(u[v], s[v]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int d = 0; d < NDOT; ++d) {
      if (d < ndots)
        cta_reduce_write<float, AccF>(red, acc[d], live, G, R, J.col_off, J.width,
                                      J.part + (size_t)d * J.ld * J.ntiles, J.ntiles, tile);
    }
  }
}

static size_t dia_smem_bytes(const SpmmBatch<float>& b, int threads) {
  size_t mx = 0;
  for (int j = 0; j < b.njobs; ++j) {
    const SpmmJob<float>& J = b.jobs[j];
    const size_t band = ((size_t)(J.dia_T + J.dinfo.maxext) * J.width + 31) / 32 * 32;
    const size_t stage = (size_t)J.dinfo.nbands * band * 4;
    mx = std::max(mx, stage);
  }
  const size_t red = (size_t)threads * 4 * sizeof(AccF);
  return 128 + std::max(mx, red);
}

int launch_spmm_dia(const SpmmBatch<float>& b, int threads, cudaStream_t s) {
  int nd = 0;
  double flops = 0.0, bytes = 0.0;
  for (int j = 0; j < b.njobs; ++j) {
    const SpmmJob<float>& J = b.jobs[j];
    nd = std::max(nd, J.ndots);
    const double vb = (double)J.n * J.b * 4;
    const int extra_reads = J.ndots - ((J.ndots > 0 && J.dotv[0] == J.x) ? 1 : 0);
    flops += 2.0 * (double)J.nnz * J.b + 2.0 * (double)J.n * J.b * J.ndots;
    bytes += 4.0 * (J.n + 1) + (double)J.nnz * 8 + vb * (2 + extra_reads);
  }
  const size_t smem = dia_smem_bytes(b, threads);
  ProfScope prof(KC_SPMM, s, flops, bytes);
#define LD_DIA_CASE(ND)                                                                      \
  {                                                                                          \
    auto kern = k_spmm_dia<ND>;                                                              \
    if (smem > 48 * 1024)                                                                    \
      LD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    int per_sm = 0;                                                                          \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);             \
    if (per_sm < 1) per_sm = 1;                                                              \
    const int grid = std::max(1, std::min(b.total_tiles, per_sm * sm_count()));              \
    kern<<<grid, threads, smem, s>>>(b);                                                     \
    break;                                                                                   \
  }
  do {
    if (nd == 0) LD_DIA_CASE(0)
    if (nd == 1) LD_DIA_CASE(1)
    if (nd == 2) LD_DIA_CASE(2)
    if (nd <= 4) LD_DIA_CASE(4)
    LD_DIA_CASE(kMaxWin)
  } while (0);
#undef LD_DIA_CASE
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

}  // namespace ld
