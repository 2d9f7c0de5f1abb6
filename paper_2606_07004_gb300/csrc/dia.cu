// Sweep paths of the SpMM pass for FP32 blocks of grid stencil matrices.
//
// Line sweep (2D grid stencils: the 2D Laplacians, the Matérn operator
// (kappa^2 I + L)^2).  Every entry lies on a few diagonals whose offsets are
// line * L + c, with L the grid's row length, |line| <= A and c in a short
// range [cmin, cmin + cw].  Output row i needs x rows from the lines
// i/L - A .. i/L + A.  A CTA owns a segment of T consecutive rows within a
// line and sweeps it over kc consecutive lines (a "unit").  It keeps the
// 2A + 1 line windows the current line needs (T + cw rows of x each) in a
// ring of shared-memory slots; moving to the next line needs one new
// window, which a TMA 2D copy (cp.async.bulk.tensor, completion on the
// slot's mbarrier) brings in, with the values of the new line, ahead of the
// computation.  So each x row crosses from L2 to the SM about (T + cw) / T
// times per pass instead of once per diagonal line.
//
// Plane sweep (3D grid stencils on an L x ny x nz grid).  The same with
// tiles of tx x ty points of a plane in place of segments, planes in place
// of lines, and a 4D TMA box (columns, x, y, z) holding the tile and its
// halo in place of a 2D box.
//
// Points outside the matrix (or the grid) are filled with zeros by the copy;
// the value of a diagonal is 0 where a row has no entry (and, in 3D, no
// entry wraps across a grid edge).  Each row sums over the diagonals in
// ascending offset order, the CSR column order, so y is the same FP32 sum as
// on the CSR path; the window dots are accumulated per unit (the unit is the
// partial slot), so they differ from the CSR path's only by the order of
// their compensated partial sums.
#include "dia.cuh"
#include "profile.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <type_traits>
#include <vector>

namespace ld {

// ---------------------------------------------------------------------------
// Structure
// ---------------------------------------------------------------------------
// Runs fn(i0, i1) over row ranges of [0, n) on up to 8 host threads (the
// structure passes are linear in nnz; a 2M-row stencil takes tens of ms on
// one core).  Returns the AND of the ranges' results.
template <typename Fn>
static bool rows_parallel(int n, Fn fn) {
  const int nt = std::max(1, std::min(8, std::min((int)std::thread::hardware_concurrency(),
                                                  n / 65536)));
  if (nt == 1) return fn(0, n);
  std::vector<char> ok(nt, 1);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    const int i0 = (int)((long long)n * t / nt), i1 = (int)((long long)n * (t + 1) / nt);
    th.emplace_back([&, t, i0, i1] { ok[t] = fn(i0, i1) ? 1 : 0; });
  }
  for (auto& x : th) x.join();
  for (char c : ok)
    if (!c) return false;
  return true;
}

// Nearest line of offset o for stride L (ties toward zero).
static int nearest_line(int o, int L) {
  const int a = o >= 0 ? o : -o;
  const int l = (a + (L - 1) / 2) / L;
  return o >= 0 ? l : -l;
}

// 3D grid stencil: L = the smallest offset magnitude above kPlaneMaxR (the
// grid's row length), P (the plane stride, a multiple of L with ny = P / L
// >= 2 and nz = n / P >= 2) = the first of the offset magnitudes and their
// halves, in ascending order, for which every offset splits as
// dz P + dy L + dx (nearest) with |dz| <= kPlaneMaxA, |dy| <= 2,
// |dx| <= kPlaneMaxR and no entry's grid neighbour wraps across a line or
// plane edge (so that reading a zero-filled point outside the grid stands
// for "no entry").
static bool plane_split(const std::vector<int>& offs, int n, int L, int P, DiaInfo* d) {
  if (P % L || P / L < 2 || n % P || n / P < 2) return false;
  memset(d, 0, sizeof *d);
  d->ndiag = (int)offs.size();
  d->dim = 3;
  d->L = L;
  d->P = P;
  d->ny = P / L;
  d->nz = n / P;
  for (int q = 0; q < d->ndiag; ++q) {
    const int o = offs[q];
    d->off[q] = o;
    d->line[q] = nearest_line(o, P);
    const int rem = o - d->line[q] * P;
    d->dy[q] = nearest_line(rem, L);
    d->dx[q] = rem - d->dy[q] * L;
    d->A = std::max(d->A, std::abs(d->line[q]));
    d->Ay = std::max(d->Ay, std::abs(d->dy[q]));
    d->Ax = std::max(d->Ax, std::abs(d->dx[q]));
  }
  return d->A <= kPlaneMaxA && d->Ay <= 2 && d->Ax <= kPlaneMaxR;
}

static bool plane_structure(const std::vector<int>& offs, int n, const int* rowptr,
                            const int* colind, DiaInfo* out) {
  int L = INT_MAX;
  std::vector<int> cand;
  for (int o : offs) {
    const int a = std::abs(o);
    if (a > kPlaneMaxR) L = std::min(L, a);
    if (a > 0) {
      cand.push_back(a);
      if (a % 2 == 0) cand.push_back(a / 2);
    }
  }
  if (L == INT_MAX) return false;
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  // A plane stride can split every offset within the radii and still not be
  // the grid's (half the true plane, say): then some entry wraps in its view,
  // and the next candidate is tried.
  auto no_wrap = [&](const DiaInfo& d) {
    const int nd = (int)offs.size();
    return rows_parallel(n, [&](int i0, int i1) {
      for (int i = i0; i < i1; ++i) {
        const int x = i % L, y = (i / L) % d.ny;
        int k = 0;
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
          const int o = colind[q] - i;
          while (k < nd && offs[k] < o) ++k;  // (every offset is in offs)
          if (x + d.dx[k] < 0 || x + d.dx[k] >= L || y + d.dy[k] < 0 || y + d.dy[k] >= d.ny)
            return false;
        }
      }
      return true;
    });
  };
  DiaInfo d;
  for (int P : cand)
    if (plane_split(offs, n, L, P, &d) && no_wrap(d)) {
      *out = d;
      return true;
    }
  return false;
}

bool dia_detect(int n, const int* rowptr, const int* colind, DiaInfo* out) {
  memset(out, 0, sizeof *out);
  if (n < 4096 || rowptr[n] <= 0) return false;
  // Distinct offsets, kept sorted: a row's offsets ascend with its columns,
  // so one forward walk per row finds (or places) each (linear in nnz); row
  // ranges on several threads, their sets merged.
  const int nt_max = 8;
  std::vector<std::vector<int>> part(nt_max);
  std::mutex pm;
  int next_part = 0;
  const bool few = rows_parallel(n, [&](int i0, int i1) {
    std::vector<int> offs;
    for (int i = i0; i < i1; ++i) {
      size_t k = 0;
      for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        if (q > rowptr[i] && colind[q] <= colind[q - 1]) return false;  // unsorted row
        const int o = colind[q] - i;
        while (k < offs.size() && offs[k] < o) ++k;
        if (k == offs.size() || offs[k] != o) {
          offs.insert(offs.begin() + k, o);
          if ((int)offs.size() > kMaxDiags) return false;  // not a stencil
        }
        ++k;
      }
    }
    std::lock_guard<std::mutex> lk(pm);
    part[next_part++] = std::move(offs);
    return true;
  });
  if (!few) return false;
  std::vector<int> offs;
  for (const auto& v : part) offs.insert(offs.end(), v.begin(), v.end());
  std::sort(offs.begin(), offs.end());
  offs.erase(std::unique(offs.begin(), offs.end()), offs.end());
  if ((int)offs.size() > kMaxDiags) return false;
  const int nd = (int)offs.size();
  // Line stride: the candidate (an offset's magnitude) with the smallest ring
  // (2A + 1 windows of a nominal 32 + cw rows); among equal rings the one
  // with the smallest sum of |c| (the grid's own row length, not a
  // neighbouring diagonal's offset).
  DiaInfo best;
  memset(&best, 0, sizeof best);
  long long best_cost = LLONG_MAX, best_sc = LLONG_MAX;
  for (int k = 0; k < nd; ++k) {
    const int L = offs[k] >= 0 ? offs[k] : -offs[k];
    if (L < kSweepMinL) continue;
    DiaInfo d;
    memset(&d, 0, sizeof d);
    d.ndiag = nd;
    d.dim = 2;
    d.L = L;
    int cmin = INT_MAX, cmax = INT_MIN;
    for (int q = 0; q < nd; ++q) {
      d.off[q] = offs[q];
      d.line[q] = nearest_line(offs[q], L);
      const int c = offs[q] - d.line[q] * L;
      d.A = std::max(d.A, d.line[q] >= 0 ? d.line[q] : -d.line[q]);
      cmin = std::min(cmin, c);
      cmax = std::max(cmax, c);
    }
    d.cmin = cmin;
    d.cw = cmax - cmin;
    if (d.A > kSweepMaxA || d.cw > kSweepMaxCw) continue;
    long long sc = 0;
    for (int q = 0; q < nd; ++q) {
      const int c = offs[q] - d.line[q] * L;
      d.cpos[q] = c - cmin;
      sc += c >= 0 ? c : -c;
    }
    const long long cost = (long long)(2 * d.A + 1) * (32 + d.cw);
    if (cost < best_cost || (cost == best_cost && sc < best_sc)) {
      best_cost = cost;
      best_sc = sc;
      best = d;
    }
  }
  if (best.ndiag == 0 && !plane_structure(offs, n, rowptr, colind, &best)) return false;
  *out = best;
  return true;
}

int dia_build(logdet_ctx* h, const int* rowptr, const int* colind) {
  memset(&h->dia, 0, sizeof h->dia);
  const int n = h->n;
  if (h->nnz <= 0) return LOGDET_OK;
  DiaInfo best;
  if (!dia_detect(n, rowptr, colind, &best)) return LOGDET_OK;
  const int nd = best.ndiag;
  const int* offs = best.off;
  // CSR entry -> diagonal index (a forward walk per row, as above).
  std::vector<int> slot((size_t)h->nnz);
  rows_parallel(n, [&](int i0, int i1) {
    for (int i = i0; i < i1; ++i) {
      int k = 0;
      for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        const int o = colind[q] - i;
        while (k < nd && offs[k] < o) ++k;
        slot[q] = k;
      }
    }
    return true;
  });
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
  h->dia = best;
  return LOGDET_OK;
}

template <typename V>
__global__ void k_dia_values(const int* __restrict__ rowptr, const int* __restrict__ slot,
                             const V* __restrict__ vals, int n, int dp, double c,
                             float* __restrict__ out) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x)
    for (int q = rowptr[row]; q < rowptr[row + 1]; ++q)
      out[(size_t)row * dp + slot[q]] = (float)((double)vals[q] / c);
}

int dia_values_f32(const logdet_ctx* h, double c, float* out, cudaStream_t st) {
  const int n = h->n;
  const int dp = dia_pad(h->dia.ndiag);
  LD_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)dp * n, st));
  ProfScope prof(KC_OTHER, st);
  const int blocks = std::max(1, std::min(div_up(n, 256), 8 * sm_count()));
  if (h->vals_dtype == LOGDET_VALS_F64)
    k_dia_values<double><<<blocks, 256, 0, st>>>(h->rowptr, h->dia_slot, (const double*)h->vals,
                                                 n, dp, c, out);
  else
    k_dia_values<float><<<blocks, 256, 0, st>>>(h->rowptr, h->dia_slot, (const float*)h->vals, n,
                                                dp, c, out);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

// Points of one x window: dim 2, T + cw rows; dim 3, the tile of tx x ty
// points with its halo of Ax, Ay on each side.
__host__ __device__ inline int sweep_win_points(const DiaInfo& d, int T, int tx, int ty) {
  return d.dim == 3 ? (tx + 2 * d.Ax) * (ty + 2 * d.Ay) : T + d.cw;
}
// Floats of one ring slot: the x window (its points x width floats), then the
// values of T points; each part rounded up to 128 bytes (TMA destinations).
__host__ __device__ inline int sweep_win_floats(int points, int width) {
  return (points * width + 31) / 32 * 32;
}
static int sweep_slot_floats(const DiaInfo& d, int T, int tx, int ty, int width) {
  return sweep_win_floats(sweep_win_points(d, T, tx, ty), width) +
         (T * dia_pad(d.ndiag) + 31) / 32 * 32;
}
// Shared memory of a CTA: barriers, the window-offset table (nr rotations x
// kMaxDiags), the dot reduction (threads x 4 accumulators), the ring.
static size_t sweep_smem_bytes(int nr, int slot_floats, int threads) {
  const size_t tab = ((size_t)nr * kMaxDiags * 4 + 127) / 128 * 128;
  const size_t red = ((size_t)threads * 4 * sizeof(AccF) + 127) / 128 * 128;
  return 128 + tab + red + (size_t)nr * slot_floats * sizeof(float);
}

bool dia_sweep_geom(const logdet_ctx* h, int width, int threads, SweepGeom* out) {
  const DiaInfo& d = h->dia;
  if (d.ndiag == 0 || !h->dia_slot || width % 4 || width < 4 || width > 256) return false;
  const int G = width / 4;
  const int R = threads / G;
  if (R < 1 || threads > 512) return false;
  const int nr = 2 * d.A + 1 + kSweepPrefetch;
  SweepGeom g;
  memset(&g, 0, sizeof g);
  if (d.dim == 3) {
    // Tile tx x ty (tx a power of two): the smallest DRAM-to-SM traffic per
    // point, (tx + 2 Ax)(ty + 2 Ay) / (tx ty) times the tiles' overhang of
    // the grid, that fits the budget; at least R points, and tiles of at
    // least 2R points (two per thread) are preferred.
    double best = 1e30;
    for (int txs = 5; txs >= 3; --txs) {
      const int tx = 1 << txs;
      if (tx > 8 && tx / 2 >= d.L) continue;
      for (int ty = 1; ty <= 16 && ty <= d.ny; ++ty) {
        const int T = tx * ty;
        if (T < R || tx + 2 * d.Ax > 256 || ty + 2 * d.Ay > 256) continue;
        if (sweep_smem_bytes(nr, sweep_slot_floats(d, T, tx, ty, width), threads) >
            (size_t)kSweepSmemBudget)
          continue;
        const double over = (double)((d.L + tx - 1) / tx * tx) / d.L *
                            ((double)((d.ny + ty - 1) / ty * ty) / d.ny);
        double cost = (double)(tx + 2 * d.Ax) * (ty + 2 * d.Ay) / T * over;
        if (T < 2 * R) cost *= 1.15;
        if (cost < best) {
          best = cost;
          g.T = T;
          g.tx = tx;
          g.ty = ty;
          g.txs = txs;
        }
      }
    }
    if (g.T == 0) return false;
    g.nseg = (d.L + g.tx - 1) / g.tx * ((d.ny + g.ty - 1) / g.ty);
    g.nlines = d.nz;
  } else {
    for (int m = 1;; ++m) {
      const int t = R * m;
      if (t + d.cw > 256 || (m > 1 && t > d.L)) break;
      if (sweep_smem_bytes(nr, sweep_slot_floats(d, t, 0, 0, width), threads) >
          (size_t)kSweepSmemBudget)
        break;
      g.T = t;
    }
    if (g.T == 0) return false;
    g.nseg = (d.L + g.T - 1) / g.T;
    g.nlines = (h->n + d.L - 1) / d.L;
  }
  // About eight units per SM; at least 4A lines or planes per unit (each
  // unit first loads 2A windows that only fill the ring).
  const int chunks = std::max(1, 8 * sm_count() / g.nseg);
  g.kc = (g.nlines + chunks - 1) / chunks;
  g.kc = std::min(g.nlines, std::max(g.kc, 4 * d.A));
  g.units = g.nseg * ((g.nlines + g.kc - 1) / g.kc);
  *out = g;
  return true;
}

// ---------------------------------------------------------------------------
// Tensor maps
// ---------------------------------------------------------------------------
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

static int encode_2d(CUtensorMap* map, const float* base, int inner, int outer, int pitch,
                     int box_inner, int box_outer) {
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LOGDET_ECUDA;
  }
  return LOGDET_OK;
}

// 4D map of an L x ny x nz grid of rows of `inner` floats (pitch floats
// apart), box of box_inner x bx x by x 1.
static int encode_grid(CUtensorMap* map, const float* base, const DiaInfo& d, int inner,
                       int pitch, int box_inner, int bx, int by) {
  const cuuint64_t dims[4] = {(cuuint64_t)inner, (cuuint64_t)d.L, (cuuint64_t)d.ny,
                              (cuuint64_t)d.nz};
  const cuuint64_t rowb = (cuuint64_t)pitch * sizeof(float);
  const cuuint64_t strides[3] = {rowb, rowb * d.L, rowb * d.P};
  const cuuint32_t box[4] = {(cuuint32_t)box_inner, (cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LOGDET_ECUDA;
  }
  return LOGDET_OK;
}

int dia_encode(SpmmJob<float>& J, const float* x, int n, int ld, int width) {
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
  const DiaInfo& d = J.dinfo;
  const int T = J.dia_T;
  const int dp = dia_pad(d.ndiag);
  const bool grid3 = d.dim == 3;
  const int bx = J.dia_tx + 2 * d.Ax, by = J.dia_ty + 2 * d.Ay;
  const int box_rows = T + d.cw;
  // TMA: 16-byte aligned bases and row pitches; the innermost box extent and
  // every innermost coordinate (J.col_off for x, 0 for the values) a
  // multiple of four floats; box extents at most 256.
  if (((uintptr_t)x & 15) || ((uintptr_t)J.dia & 15) || (ld * 4) % 16 || width > 256 ||
      width < 4 || width % 4 || J.col_off % 4 || T < 1 || dp > 256 ||
      (grid3 ? (bx > 256 || by > 256 || J.dia_tx * J.dia_ty != T ||
                (long long)d.P * d.nz != n)
             : box_rows > 256)) {
    set_error("grid sweep: block not aligned for TMA");
    return LOGDET_EINVAL;
  }
  if (grid3) {
    LD_TRY(encode_grid(&J.tmap, x, d, ld, ld, width, bx, by));
    return encode_grid(&J.vmap, J.dia, d, dp, dp, dp, J.dia_tx, J.dia_ty);
  }
  LD_TRY(encode_2d(&J.tmap, x, ld, n, ld, width, box_rows));
  return encode_2d(&J.vmap, J.dia, dp, n, dp, dp, T);
}

// ---------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
// A wait gives up after wait_ns of the global timer (2 s in normal use), or
// after kDiaWaitPolls polls whatever the timer says.
constexpr int kDiaWaitPolls = 1 << 24;
constexpr unsigned long long kDiaWaitNs = 2000000000ull;

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
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the barrier's phase to complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase,
                                                  unsigned long long wait_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < kDiaWaitPolls; i += 32) {
    for (int k = 0; k < 32; ++k)
      if (mbar_try_wait(bar, phase)) return true;
    if (global_ns() - t0 > wait_ns) return false;
  }
  return false;
}
// 4D tiled copy of the box at (column, x, y, z) into shared memory.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c, int x,
                                            int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
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
// Units.  Unit u of a job covers segment u % nseg (rows seg0 .. seg0 + segT
// of every line; plane sweep: tile u % nseg of every plane) over the lines
// or planes k0 .. k0 + nl - 1, chunk u / nseg.  A CTA takes units
// gu = blockIdx.x, + gridDim.x, ... of the batch; window q of a unit
// (q = 0 .. nl + 2A - 1) holds line or plane k0 - A + q, and from q = 2A on
// it also carries the values of line or plane k0 + q - 2A.
// ---------------------------------------------------------------------------
// (plane sweep: seg0, segT hold the tile origin x0, y0)
struct SwUnit {
  int gu, jb, seg0, segT, k0, nl;
};

template <int DIM>
__device__ __forceinline__ void sw_unit(SwUnit& U, const SpmmBatch<float>& B, int gu) {
  U.gu = gu;
  if (gu >= B.total_tiles) return;
  U.jb = find_job(B, gu);
  const SpmmJob<float>& J = B.jobs[U.jb];
  const DiaInfo& D = J.dinfo;
  const int u = gu - B.tile_start[U.jb];
  const int seg = u % J.dia_nseg, chunk = u / J.dia_nseg;
  if constexpr (DIM == 3) {
    const int nsx = (D.L + J.dia_tx - 1) >> J.dia_txs;
    const int sy = seg / nsx, sx = seg - sy * nsx;
    U.seg0 = sx << J.dia_txs;  // x0
    U.segT = sy * J.dia_ty;    // y0
  } else {
    U.seg0 = seg * J.dia_T;
    U.segT = min(J.dia_T, D.L - U.seg0);
  }
  U.k0 = chunk * J.dia_kc;
  U.nl = min(J.dia_kc, J.dia_nlines - U.k0);
}

// Thread 0: arm the slot's barrier with the window's byte count and issue
// its copies (dim 2: T + cw rows of line k0 - A + q; dim 3: the tile and
// its halo in plane k0 - A + q; from q = 2A on also the values of line or
// plane k0 + q - 2A).
template <int DIM>
__device__ __forceinline__ void sw_issue(const SpmmBatch<float>& B, const SwUnit& U, int q,
                                         float* slot, uint32_t bar, unsigned extra_tx) {
  const SpmmJob<float>& J = B.jobs[U.jb];
  const DiaInfo& D = J.dinfo;
  const int T = J.dia_T;
  const int dp = dia_pad(D.ndiag);
  const bool vals = q >= 2 * D.A;
  const int wp = sweep_win_points(D, T, J.dia_tx, J.dia_ty);
  const uint32_t bytes =
      (uint32_t)((wp * J.width + (vals ? T * dp : 0)) * (int)sizeof(float)) + extra_tx;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, bytes);
  const uint32_t vdst = smem_addr(slot + sweep_win_floats(wp, J.width));
  if constexpr (DIM == 3) {
    tma_load_4d(smem_addr(slot), &J.tmap, J.col_off, U.seg0 - D.Ax, U.segT - D.Ay,
                U.k0 - D.A + q, bar);
    if (vals) tma_load_4d(vdst, &J.vmap, 0, U.seg0, U.segT, U.k0 + q - 2 * D.A, bar);
  } else {
    tma_load_2d(smem_addr(slot), &J.tmap, J.col_off, U.seg0 + (U.k0 - D.A + q) * D.L + D.cmin,
                bar);
    if (vals) tma_load_2d(vdst, &J.vmap, 0, U.seg0 + (U.k0 + q - 2 * D.A) * D.L, bar);
  }
}

// ---------------------------------------------------------------------------
// y = A x and the window dots for FP32 blocks of a matrix with grid
// structure.  Thread (r, g) owns points r, r + R, ... of the segment or tile
// and 16-byte column chunk g (R = threads / G, G = width / 4).
//
// Ring protocol (uniform across the CTA): load t (a window) goes to slot
// t % nr and completes phase (t / nr) & 1 of that slot's mbarrier.  The
// producer issues load t once load t - nr has been released, i.e. the CTA
// has passed a barrier after its last read: window q of a unit is released
// by the barrier that starts line q + 1 (all its windows by the barrier
// after the unit's last line).  One barrier per line: after the threads
// have waited for the line's new window, the barrier also releases the
// window the previous line read last, and after the line thread 0 refills
// that slot, so nr - 2A - 2 windows beyond the current line's are in
// flight while it is computed.  Waits are bounded (wait_ns of the global
// timer): if one gives up, the CTA decides together (__syncthreads_or),
// waits once more for every copy still in flight, sets the job's error flag
// and returns.
//
// The window-offset table: entry [rot][d] is the byte offset (from the
// start of dynamic shared memory) of the first x row diagonal d reads when
// the current line's window 0 is load index rot (mod nr).
// ---------------------------------------------------------------------------
// MAXT: the largest CTA the instance takes (320 or 512); with at most two
// dots, two CTAs per SM are asked for (the register budget follows).  NDC:
// the diagonal count when every job of the launch has it (5: 2D Laplacian,
// 13: Matérn), fixed at compile time, which removes a third of the
// instructions; 7: the 3D Laplacian; 0 = any count up to kMaxDiags.  DIM:
// 2 = line sweep, 3 = plane sweep (see DiaInfo).
template <int NDOT, int MAXT, int NDC, int DIM>
__global__ void __launch_bounds__(MAXT, NDOT <= 2 ? 2 : 1)
    k_spmm_sweep(const __grid_constant__ SpmmBatch<float> B, int slot_floats, int nr,
                 unsigned extra_tx, unsigned long long wait_ns) {
  constexpr int kDiags = NDC > 0 ? NDC : kMaxDiags;
  constexpr int V = 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const uint32_t bar0 = smem_addr(smem_raw);  // nr barriers, 8 bytes apart
  int* xo_tab = reinterpret_cast<int*>(smem_raw + 128);
  const int tab_bytes = (nr * kMaxDiags * 4 + 127) / 128 * 128;
  AccF* red = reinterpret_cast<AccF*>(smem_raw + 128 + tab_bytes);
  const int red_bytes = ((int)blockDim.x * V * (int)sizeof(AccF) + 127) / 128 * 128;
  // Shared-memory addresses below are byte offsets from smem_raw (32-bit
  // arithmetic, immediate offsets where they are compile-time).
  const int ring_bytes = 128 + tab_bytes + red_bytes;
  float* ring = reinterpret_cast<float*>(smem_raw + ring_bytes);

  SwUnit C;
  sw_unit<DIM>(C, B, blockIdx.x);
  if (C.gu >= B.total_tiles) return;
  if (threadIdx.x == 0) {
    for (int q = 0; q < nr; ++q) mbar_init(bar0 + 8 * q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // Producer state (every thread keeps it; thread 0 issues).
  SwUnit P = C;
  int pq = 0, issued = 0, pslot = 0;  // pslot = issued % nr
  auto produce = [&](int released) {
    while (P.gu < B.total_tiles && issued < released + nr) {
      if (threadIdx.x == 0)
        sw_issue<DIM>(B, P, pq, ring + (size_t)pslot * slot_floats, bar0 + 8 * pslot, extra_tx);
      ++issued;
      if (++pslot == nr) pslot = 0;
      if (++pq == P.nl + 2 * B.jobs[P.jb].dinfo.A) {
        sw_unit<DIM>(P, B, P.gu + gridDim.x);
        pq = 0;
      }
    }
  };
  produce(0);

  // Dot accumulators: columns (0, 1) and (2, 3) of the thread's chunk.
  AccF2 acc[NDOT > 0 ? NDOT : 1][2];
#pragma unroll
  for (int d = 0; d < (NDOT > 0 ? NDOT : 1); ++d) acc[d][0].zero(), acc[d][1].zero();

  // Constants of the current job.
  int cur_jb = -1, G = 1, R = 1, r = 0, g = 0, width = 0, nd = 0, dp = 0, A = 0, L = 0;
  int win_floats = 0, dself = 0, col0 = 0, ldy = 0, ndots = 0, n = 0;
  int PL = 0, txs = 0, tmask = 0, WX = 0, hoff = 0;  // plane sweep: P, tile shape, halo offset
  float* yv = nullptr;
  float csh[V], csc[V];
  bool has_shift = false, has_scale = false;
  unsigned selfmask = 0;
  bool live = false;

  // Consumer state: every load is waited for once, in order.  wnext is the
  // index of the next load to wait for, wslot = wnext % nr, bit s of
  // phases the parity its slot completes next; rslot = (t0 + j) % nr for
  // the current unit's window 0 t0 and line j.
  int t0 = 0, wnext = 0, wslot = 0, rslot = 0;
  uint32_t phases = 0;
  while (C.gu < B.total_tiles) {
    const SpmmJob<float>& J = B.jobs[C.jb];
    if (C.jb != cur_jb) {
      cur_jb = C.jb;
      const DiaInfo& D = J.dinfo;
      G = J.width / V;
      R = blockDim.x / G;
      r = threadIdx.x / G;
      g = threadIdx.x - r * G;
      live = r < R;
      width = J.width;
      nd = NDC > 0 ? NDC : D.ndiag;
      dp = dia_pad(nd);
      A = D.A;
      L = D.L;
      n = J.n;
      win_floats = sweep_win_floats(sweep_win_points(D, J.dia_T, J.dia_tx, J.dia_ty), width);
      if constexpr (DIM == 3) {
        PL = D.P;
        txs = J.dia_txs;
        tmask = J.dia_tx - 1;
        WX = J.dia_tx + 2 * D.Ax;
        hoff = D.Ay * WX + D.Ax;
      }
      for (int d = 0; d < nd; ++d)
        if (D.off[d] == 0) dself = d;
      col0 = J.col_off + g * V;
      // The thread's column shift and scale, converted once per job (the
      // conversion from FP64 runs on the FP64 pipe, slow on this GPU).
      has_shift = J.colshift != nullptr;
      has_scale = J.colscale != nullptr;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        csh[v] = has_shift ? (float)J.colshift[col0 + v] : 0.f;
        csc[v] = has_scale ? (float)J.colscale[col0 + v] : 1.f;
      }
      ldy = J.ld;
      yv = J.y;
      ndots = J.ndots;
      selfmask = 0;
      for (int d = 0; d < ndots; ++d)
        if (J.dotv[d] == J.x) selfmask |= 1u << d;
      // (every read of the previous table ended before the last barrier)
      for (int e = threadIdx.x; e < nr * kMaxDiags; e += blockDim.x) {
        const int rot = e / kMaxDiags, d = e - rot * kMaxDiags;
        const int pos = DIM == 3 ? D.dy[d] * (J.dia_tx + 2 * D.Ax) + D.dx[d] : D.cpos[d];
        xo_tab[e] = d < nd ? ring_bytes + (((rot + A + D.line[d]) % nr) * slot_floats +
                                           pos * width) * (int)sizeof(float)
                           : 0;
      }
      __syncthreads();
    }
    const int nwin = C.nl + 2 * A;
    for (int j = 0; j < C.nl; ++j) {
      // Windows of line k0 + j: loads t0 + j .. t0 + j + 2A (only the last
      // is new after the first line).  Every thread waits (try_wait
      // suspends the thread until the phase completes or a time limit
      // passes); the barrier then also marks line j - 1's reads done,
      // releasing window t0 + j - 1.
      const int tw = t0 + j + 2 * A;
      bool ok = true;
      while (ok && wnext <= tw) {
        ok = mbar_wait_bounded(bar0 + 8 * wslot, (phases >> wslot) & 1u, wait_ns);
        if (ok) {
          phases ^= 1u << wslot;
          ++wnext;
          if (++wslot == nr) wslot = 0;
        }
      }
      if (__syncthreads_or(!ok)) {
        // Copies still in flight: loads wnext .. issued - 1 (distinct slots).
        for (int t = wnext, sl = wslot; t < issued; ++t) {
          mbar_wait_bounded(bar0 + 8 * sl, (phases >> sl) & 1u, wait_ns);
          if (++sl == nr) sl = 0;
        }
        if (threadIdx.x == 0) atomicExch(J.err, 1);
        return;
      }
      if (live) {
        const int* xt = xo_tab + rslot * kMaxDiags;
        int xo[kDiags + 3 & ~3];
#pragma unroll
        for (int q = 0; q < (kDiags + 3) / 4; ++q) {
          if (NDC > 0 || 4 * q < nd) {
            const int4 o = reinterpret_cast<const int4*>(xt)[q];
            xo[4 * q] = o.x;
            xo[4 * q + 1] = o.y;
            xo[4 * q + 2] = o.z;
            xo[4 * q + 3] = o.w;
          } else {
            xo[4 * q] = xo[4 * q + 1] = xo[4 * q + 2] = xo[4 * q + 3] = 0;
          }
        }
        const int xself = xt[dself];
        const int vslot = rslot + 2 * A < nr ? rslot + 2 * A : rslot + 2 * A - nr;
        const int vs_b = ring_bytes + (vslot * slot_floats + win_floats) * (int)sizeof(float);
        // First row of the segment (dim 2) or tile (dim 3) in this line or
        // plane, and its point count.
        const int rowbase =
            DIM == 3 ? (C.k0 + j) * PL + C.segT * L + C.seg0 : C.seg0 + (C.k0 + j) * L;
        const int npts = DIM == 3 ? J.dia_T : C.segT;
        // plane sweep: the tile's points inside the grid
        const int wx = DIM == 3 ? min(tmask + 1, L - C.seg0) : 0;
        const int wy = DIM == 3 ? min(J.dia_ty, J.dinfo.ny - C.segT) : 0;
        // kRows rows of the segment per thread at a time (rows rr, rr + R,
        // ...): independent FMA chains interleave.  Each row's sum, y and
        // dot updates are those of one row at a time, in row order.
        auto rows_loop = [&](auto krows) {
        constexpr int kRows = decltype(krows)::value;
        // Window vectors other than x itself are loaded before the sums, so
        // that their latency overlaps them (up to four; more would spill).
        constexpr bool kEarly = NDOT <= 4;
        for (int rr = r; rr < npts; rr += kRows * R) {
          if (DIM == 2 && rowbase + rr >= n) break;
          // Point rq (its window position) and row rowq (global) of each of
          // the thread's kRows points; an absent point re-reads point rr
          // (dim 2) or its smem position and the tile's first row (dim 3).
          bool on[kRows];
          int rq[kRows], rowq3[DIM == 3 ? kRows : 1];
#pragma unroll
          for (int q = 0; q < kRows; ++q) {
            const int p = rr + q * R;
            if constexpr (DIM == 3) {
              on[q] = p < npts && (p & tmask) < wx && (p >> txs) < wy;
              rq[q] = p < npts ? p : rr;
              rowq3[q] = on[q] ? rowbase + (p >> txs) * L + (p & tmask) : rowbase;
            } else {
              on[q] = p < npts && rowbase + p < n;
              rq[q] = on[q] ? p : rr;
            }
          }
          // x, y and the window vectors move as pairs of packed columns
          // (16 bytes = two f32x2 pairs); the row sums use fma.rn.f32x2,
          // lane for lane the fmaf of the scalar form.
          ulonglong2 u[kRows][NDOT > 0 ? NDOT : 1];
#pragma unroll
          for (int q = 0; q < kRows; ++q)
#pragma unroll
            for (int d = 0; d < NDOT; ++d)
              if (kEarly && d < ndots && !((selfmask >> d) & 1u))
                u[q][d] = __ldg(reinterpret_cast<const ulonglong2*>(
                    J.dotv[d] +
                    (size_t)(DIM == 3 ? rowq3[DIM == 3 ? q : 0] : rowbase + rq[q]) * ldy + col0));
          int xb[kRows], vb[kRows];  // byte offsets of the row's chunk and values
#pragma unroll
          for (int q = 0; q < kRows; ++q) {
            const int wpos = DIM == 3 ? (rq[q] >> txs) * WX + (rq[q] & tmask) + hoff : rq[q];
            xb[q] = (wpos * width + g * V) * (int)sizeof(float);
            vb[q] = vs_b + rq[q] * dp * (int)sizeof(float);
          }
          unsigned long long s2[kRows][2];
#pragma unroll
          for (int q = 0; q < kRows; ++q) s2[q][0] = s2[q][1] = 0ull;
          float4 av[kRows];
#pragma unroll
          for (int d = 0; d < kDiags; ++d) {
            if (NDC > 0 || d < nd) {
#pragma unroll
              for (int q = 0; q < kRows; ++q) {
                if (d % 4 == 0)
                  av[q] = *reinterpret_cast<const float4*>(smem_raw + vb[q] + 4 * d);
                const float a = d % 4 == 0   ? av[q].x
                                : d % 4 == 1 ? av[q].y
                                : d % 4 == 2 ? av[q].z
                                             : av[q].w;
                const unsigned long long a2 = f2_pack(a, a);
                const ulonglong2 xv =
                    *reinterpret_cast<const ulonglong2*>(smem_raw + xb[q] + xo[d]);
                s2[q][0] = f2_fma(a2, xv.x, s2[q][0]);
                s2[q][1] = f2_fma(a2, xv.y, s2[q][1]);
              }
            }
          }
#pragma unroll
          for (int q = 0; q < kRows; ++q) {
            if (!on[q]) continue;
            const int row = DIM == 3 ? rowq3[DIM == 3 ? q : 0] : rowbase + rq[q];
            const ulonglong2 xs2 = *reinterpret_cast<const ulonglong2*>(smem_raw + xb[q] + xself);
            if (has_shift || has_scale) {
              float sc[V], xs[V];
              f2_unpack(s2[q][0], sc[0], sc[1]);
              f2_unpack(s2[q][1], sc[2], sc[3]);
              f2_unpack(xs2.x, xs[0], xs[1]);
              f2_unpack(xs2.y, xs[2], xs[3]);
#pragma unroll
              for (int v = 0; v < V; ++v) {
                if (has_shift) sc[v] = fmaf(csh[v], xs[v], sc[v]);
                if (has_scale) sc[v] = sc[v] * csc[v];
              }
              s2[q][0] = f2_pack(sc[0], sc[1]);
              s2[q][1] = f2_pack(sc[2], sc[3]);
            }
            *reinterpret_cast<ulonglong2*>(yv + (size_t)row * ldy + col0) =
                make_ulonglong2(s2[q][0], s2[q][1]);
#pragma unroll
            for (int d = 0; d < NDOT; ++d) {
              if (d < ndots) {
                const bool self = (selfmask >> d) & 1u;
                if (!kEarly && !self)
                  u[q][d] = __ldg(reinterpret_cast<const ulonglong2*>(
                      J.dotv[d] + (size_t)row * ldy + col0));
                const ulonglong2 uu = self ? xs2 : u[q][d];
                acc[d][0].fma(uu.x, s2[q][0]);
                acc[d][1].fma(uu.y, s2[q][1]);
              }
            }
          }
        }
        };
        // (pairs with at most two dots, in CTAs of up to 320 threads only:
        // the larger ones run at two per SM on 64 registers, and four dots'
        // early loads for two rows exceed the 168 registers a thread of a
        // 320-thread CTA can have)
        if (NDOT <= 2 && MAXT <= 320 && npts >= 2 * R)
          rows_loop(std::integral_constant<int, 2>{});
        else
          rows_loop(std::integral_constant<int, 1>{});
      }
      const bool last = j == C.nl - 1;
      if (last) {
        const int unit = C.gu - B.tile_start[C.jb];
#pragma unroll
        for (int d = 0; d < NDOT; ++d) {
          if (d < ndots) {
            const AccF a4[V] = {acc[d][0].lo(), acc[d][0].hi(), acc[d][1].lo(), acc[d][1].hi()};
            cta_reduce_write<float, AccF>(red, a4, live, G, R, J.col_off, width,
                                          J.part + (size_t)d * ldy * J.ntiles, J.ntiles, unit);
          }
        }
#pragma unroll
        for (int d = 0; d < (NDOT > 0 ? NDOT : 1); ++d) acc[d][0].zero(), acc[d][1].zero();
        __syncthreads();  // every read of the unit's windows is done
        produce(t0 + nwin);
      } else {
        produce(t0 + j);  // window t0 + j - 1: released by this line's barrier
      }
      if (++rslot == nr) rslot = 0;
    }
    // The next unit's window 0 follows this unit's last 2A windows.
    rslot += 2 * A;
    if (rslot >= nr) rslot -= nr;
    t0 += nwin;
    sw_unit<DIM>(C, B, C.gu + gridDim.x);
  }
}

// Ring slot size (floats, a multiple of 32) and the largest A of a launch.
// The ring holds 2A + 1 + kSweepPrefetch slots: measured on GB300, deeper
// prefetch (up to 8 windows, one CTA per SM or two) gives the same time, so
// the kernel is bound by issue, not by the latency of the copies.
static void sweep_launch_geom(const SpmmBatch<float>& b, int* slot_floats, int* amax) {
  int sf = 0, a = 0;
  for (int j = 0; j < b.njobs; ++j) {
    const SpmmJob<float>& J = b.jobs[j];
    sf = std::max(sf, sweep_slot_floats(J.dinfo, J.dia_T, J.dia_tx, J.dia_ty, J.width));
    a = std::max(a, J.dinfo.A);
  }
  *slot_floats = (sf + 31) / 32 * 32;
  *amax = a;
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
  int slot_floats = 0, amax = 0;
  sweep_launch_geom(b, &slot_floats, &amax);
  // Test hook: LOGDET_TEST_SWEEP_STALL=1 arms every barrier for 16 bytes
  // more than its copies deliver, so that every wait runs out (after 20 ms)
  // and the solve fails with LOGDET_ETIMEOUT; nothing faults or hangs.
  const char* stall_env = getenv("LOGDET_TEST_SWEEP_STALL");
  const bool stall = stall_env && stall_env[0] == '1';
  const unsigned extra_tx = stall ? 16u : 0u;
  const unsigned long long wait_ns = stall ? 20000000ull : kDiaWaitNs;
  // Every job of a launch has the same dimension (launch_spmm_jobs splits).
  const int dim = b.jobs[0].dinfo.dim;
  int ndc = b.jobs[0].dinfo.ndiag;
  for (int j = 1; j < b.njobs; ++j)
    if (b.jobs[j].dinfo.ndiag != ndc) ndc = 0;
  if (dim == 3 ? ndc != 7 : (ndc != 5 && ndc != 13)) ndc = 0;
  ProfScope prof(KC_SPMM, s, flops, bytes);
#define LD_SW_KERN(ND, NC, DM) \
  (threads <= 320 ? k_spmm_sweep<ND, 320, NC, DM> : k_spmm_sweep<ND, 512, NC, DM>)
#define LD_SW_CASE(ND)                                                                       \
  {                                                                                          \
    auto kern = dim == 3 ? (ndc == 7 ? LD_SW_KERN(ND, 7, 3) : LD_SW_KERN(ND, 0, 3))           \
                         : ndc == 13 ? LD_SW_KERN(ND, 13, 2)                                  \
                         : ndc == 5  ? LD_SW_KERN(ND, 5, 2)                                   \
                                     : LD_SW_KERN(ND, 0, 2);                                  \
    const int nr = 2 * amax + 1 + kSweepPrefetch;                                            \
    const size_t smem = sweep_smem_bytes(nr, slot_floats, threads);                          \
    if (smem > 48 * 1024)                                                                    \
      LD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    int per_sm = 0;                                                                          \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);             \
    if (per_sm < 1) per_sm = 1;                                                              \
    const int grid = std::max(1, std::min(b.total_tiles, per_sm * sm_count()));              \
    kern<<<grid, threads, smem, s>>>(b, slot_floats, nr, extra_tx, wait_ns);                 \
    break;                                                                                   \
  }
  do {
    if (nd == 0) LD_SW_CASE(0)
    if (nd == 1) LD_SW_CASE(1)
    if (nd == 2) LD_SW_CASE(2)
    if (nd <= 4) LD_SW_CASE(4)
    LD_SW_CASE(kMaxWin)
  } while (0);
#undef LD_SW_CASE
#undef LD_SW_KERN
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

}  // namespace ld
