// Krylov step kernels (see krylov.cuh for the recurrence they implement).
#include "handle.cuh"
#include "krylov.cuh"
#include "profile.cuh"

#include <algorithm>
#include <cstdlib>
#include <vector>

namespace ld {

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

static int gcd_int(int a, int b) { while (b) { int t = a % b; a = b; b = t; } return a; }

// Threads per CTA: a multiple of both 32 (full warps) and of the chunks per
// row G = ld / vec, so every lane of every warp owns a (row, chunk) slot.
TileGeom tile_geom(int width, int vec, int threads_hint, int iters_hint, int n) {
  TileGeom g;
  int G = width / vec;
  int lcm = G / gcd_int(G, 32) * 32;          // smallest CTA with whole rows and warps
  int threads = lcm;
  while (threads < 256 && threads + lcm <= 512) threads += lcm;
  if (threads > 512) threads = std::max(1, 512 / G) * G;  // very wide blocks: idle lanes accepted
  if (G > 512) threads = 512;                               // (not reached for ld <= 1024)
  if (threads_hint > 0 && threads_hint <= 512 && threads_hint % 32 == 0 && threads_hint % G == 0)
    threads = threads_hint;
  g.threads = threads;
  g.rows_per_iter = threads / G;
  // 32 rows per thread and tile (the depth the autotuner picks on GB300 for
  // narrow and wide blocks alike; shallower tiles spend the update pass on
  // per-tile reductions: 20-column blocks 13.7 -> 10.4 ms per 4M-row solve).
  int iters = 32;
  if (n > 0) {
    const long long want = 2LL * sm_count();  // tiles
    const int fit = (int)std::max<long long>(1, n / (want * g.rows_per_iter));
    if (fit < iters) iters = fit;
  }
  if (iters_hint > 0 && iters_hint <= 256) iters = iters_hint;
  g.tile_rows = g.rows_per_iter * iters;
  return g;
}


// ---------------------------------------------------------------------------
// pass 1: y = A x (CSR order per row) and d_i += dotv_i . y
//
// Thread (r, g) of a tile owns row r (stepping by R rows) and the vector
// chunk g of the probe columns.  A row's gathers of x are issued four at a
// time (one memory round trip per four nonzeros), then the remainder.  The
// CSR arrays are read through the read-only cache; measured on GB300 this
// beats staging each tile's CSR slice in shared memory, which takes L1
// capacity away from the gathers of x.
// ---------------------------------------------------------------------------
constexpr int kGather = 4;
constexpr int kPrefetch = 8;  // entries of a row whose x rows are prefetched

// Checked builds (LOGDET_CHECKED): bounds checks on the indices the passes
// take from memory -- work-item rows and slots, row ranges from rowptr,
// column indices -- before they address anything.  A violation sets a bit
// of g_violations (logdet_checked_report) and the access is redirected in
// range (column 0, an empty row range, slot 0); nothing traps.  In other
// builds the checks are the identity.
enum : unsigned { kViolItem = 1u, kViolRowRange = 2u, kViolColumn = 4u, kViolSlot = 8u };
#ifdef LOGDET_CHECKED
__device__ unsigned int g_violations;
__device__ __forceinline__ int chk_col(int c, int n) {
  if ((unsigned)c >= (unsigned)n) {
    atomicOr(&g_violations, kViolColumn);
    return 0;
  }
  return c;
}
__device__ __forceinline__ void chk_range(int& q0, int& q1, long long nnz) {
  if (q0 < 0 || q1 < q0 || (long long)q1 > nnz) {
    atomicOr(&g_violations, kViolRowRange);
    q0 = q1 = 0;
  }
}
__device__ __forceinline__ int chk_slot(int t, int nslots) {
  if ((unsigned)t >= (unsigned)nslots) {
    atomicOr(&g_violations, kViolSlot);
    return 0;
  }
  return t;
}
__device__ __forceinline__ void chk_item(int& r0, int& r1, bool split, int n) {
  if (r0 < 0 || r0 >= n || (!split && (r1 < r0 || r1 > n))) {
    atomicOr(&g_violations, kViolItem);
    r0 = 0;
    r1 = split ? -1 : 0;
  }
}
#else
__device__ __forceinline__ int chk_col(int c, int) { return c; }
__device__ __forceinline__ void chk_range(int&, int&, long long) {}
__device__ __forceinline__ int chk_slot(int t, int) { return t; }
__device__ __forceinline__ void chk_item(int&, int&, bool, int) {}
#endif

// L2 prefetch of the 16-byte-aligned chunk at p (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.L2 [%0];" ::"l"(p));
}

// Programmatic dependent launch of the step kernels: a step kernel may be
// launched while its predecessor in the stream still runs (its CTAs get
// resident early, which hides the launch latency of small steps).  On entry
// it waits for the predecessor grid to complete and its writes to be
// visible, then lets its own successor launch.  A launch without the
// attribute, or after a kernel that does not trigger, orders as usual.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Vector load of block data: through the non-coherent path for the step
// kernels (the block is read-only while they run), through L2 only (.cg)
// when COH, for the persistent run, whose blocks other CTAs write between
// its phases.
template <bool COH, typename T>
__device__ __forceinline__ void load_v(const T* p, typename Compute<T>::type (&v)[Vec16<T>::N]) {
  if constexpr (!COH) {
    load_vec<T>(p, v);
  } else {
    using V = typename Vec16<T>::type;
    const V t = __ldcg(reinterpret_cast<const V*>(p));
    if constexpr (std::is_same<T, double>::value) { v[0] = t.x; v[1] = t.y; }
    else if constexpr (std::is_same<T, float>::value) { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
    else if constexpr (std::is_same<T, f32x2>::value) { v[0] = dfloat(t.x, t.y); v[1] = dfloat(t.z, t.w); }
    else {
      const uint32_t w[2] = {t.x, t.y};
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
      }
    }
  }
}

// Blocks whose passes are bound by memory latency and computed on the FP32
// pipe (FP32, BF16 and double-float entries: a double-float thread holds two
// entries where an FP32 one holds four, so their registers match); FP64
// blocks are bound by the FP64 pipe and take the register-rich instances.
template <typename T>
constexpr bool narrow_block() { return !std::is_same<T, double>::value; }

// FP64 instances with the full dot window hold two CTAs per SM: at 85
// registers one 480-thread CTA fit, and the update pass of OSA-IOP k = 8
// then ran at half the FP64 and HBM peaks (a few spilled registers cost
// less than the second CTA gains).  0 leaves every other instance's
// register choice to the compiler, as without the hint.
template <typename T, int N>
constexpr int fp64_wide_min_ctas() { return (std::is_same<T, double>::value && N >= kMaxWin) ? 2 : 0; }

// Pass 1 over the tiles (or work items) gt0, gt0 + stride, ... of a batch,
// each by the whole CTA; the dynamic shared memory holds blockDim.x * V
// accumulators.  Batch: SpmmBatch or any type with the same members.
// PF: the row-start L2 prefetch below (always for FP32, BF16 and
// double-float blocks; for FP64 blocks an instance of its own, launched for
// matrices cut into work items).
template <typename T, int NDOT, typename Batch, bool COH = false, bool PF = narrow_block<T>()>
__device__ __forceinline__ void spmm_tiles(const Batch& B, int gt0, int stride,
                                           unsigned char* smem_raw) {
  constexpr int V = Vec16<T>::N;
  using Acc = typename AccOf<T>::type;
  using CT = typename Compute<T>::type;
  Acc* smem = reinterpret_cast<Acc*>(smem_raw);
  for (int gt = gt0; gt < B.total_tiles; gt += stride) {
    const int jb = find_job(B, gt);
    const SpmmJob<T>& J = B.jobs[jb];
    const int G = J.width / V;
    const int R = blockDim.x / G;
    const int r = threadIdx.x / G;
    const int g = threadIdx.x - r * G;
    const bool live = r < R;
    int tile = gt - B.tile_start[jb];
    int row0 = tile * J.tile_rows;
    int row1 = min(row0 + J.tile_rows, J.n);
    bool split = false;
    if (J.items) {
      const int4 it = __ldg(J.items + tile);
      row0 = it.x;
      row1 = it.y;
      tile = chk_slot(it.z, J.ntiles);
      split = it.y < 0;
      chk_item(row0, row1, split, J.n);
    }
    const int col0 = J.col_off + g * V;
    const int ndots = J.ndots;

    Acc acc[NDOT > 0 ? NDOT : 1][V];
#pragma unroll
    for (int d = 0; d < (NDOT > 0 ? NDOT : 1); ++d)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[d][v].zero();

    const bool has_scale = J.colscale != nullptr, has_shift = J.colshift != nullptr;
    if (split) {
      // One long row: row group r takes nonzeros q0 + r, q0 + r + R, ...;
      // the groups' sums are added in group order by group 0.
      const int row = row0;
      const T* xcol = J.x + col0;
      CT s[V];
#pragma unroll
      for (int v = 0; v < V; ++v) s[v] = CT(0);
      if (live) {
        int q0 = __ldg(J.rowptr + row), q1 = __ldg(J.rowptr + row + 1);
        chk_range(q0, q1, J.nnz);
        int q = q0 + r;
        for (; q + (kGather - 1) * R < q1; q += kGather * R) {
          int c[kGather];
          CT a[kGather], xv[kGather][V];
#pragma unroll
          for (int u = 0; u < kGather; ++u) {
            c[u] = chk_col(__ldg(J.colind + q + u * R), J.n);
            a[u] = __ldg(J.vals + q + u * R);
          }
#pragma unroll
          for (int u = 0; u < kGather; ++u) load_v<COH, T>(xcol + (size_t)c[u] * J.ld, xv[u]);
#pragma unroll
          for (int u = 0; u < kGather; ++u)
#pragma unroll
            for (int v = 0; v < V; ++v) s[v] = fma(a[u], xv[u][v], s[v]);
        }
        for (; q < q1; q += R) {
          const int c = chk_col(__ldg(J.colind + q), J.n);
          const CT a = __ldg(J.vals + q);
          CT xv[V];
          load_v<COH, T>(xcol + (size_t)c * J.ld, xv);
#pragma unroll
          for (int v = 0; v < V; ++v) s[v] = fma(a, xv[v], s[v]);
        }
      }
      CT* sred = reinterpret_cast<CT*>(smem_raw);
      __syncthreads();
      if (live) {
#pragma unroll
        for (int v = 0; v < V; ++v) sred[threadIdx.x * V + v] = s[v];
      }
      __syncthreads();
      if (live && r == 0) {
        CT t[V];
#pragma unroll
        for (int v = 0; v < V; ++v) t[v] = CT(0);
        for (int rr = 0; rr < R; ++rr)
#pragma unroll
          for (int v = 0; v < V; ++v) t[v] += sred[(rr * G + g) * V + v];
        if (has_shift || has_scale) {
          CT xr[V];
          load_v<COH, T>(xcol + (size_t)row * J.ld, xr);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            if (has_shift) t[v] = fma(CT(J.colshift[col0 + v]), xr[v], t[v]);
            if (has_scale) t[v] = t[v] * CT(J.colscale[col0 + v]);
          }
        }
        store_vec<T>(J.y + (size_t)row * J.ld + col0, t);
#pragma unroll
        for (int d = 0; d < NDOT; ++d) {
          if (d < ndots) {
            CT u[V];
            load_v<COH, T>(J.dotv[d] + (size_t)row * J.ld + col0, u);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[d][v].fma(u[v], t[v]);
          }
        }
      }
    } else if (live) {
      // FP32, BF16 and double-float blocks with at most one dot
      // (memory-latency bound, and with registers to spare) are software
      // pipelined: the next row's range and the next batch's column indices
      // are requested before the current gathers are consumed, one round
      // trip per batch instead of two (measured 39.3 -> 32.7 ms per Matérn
      // solve).  With more dots, or
      // FP64, the extra registers cost more occupancy than the overlap gains
      // (power-law graph, four dots: 435 -> 720 ms per solve).  The
      // accumulation order is the same either way.
      constexpr bool kPipe = narrow_block<T>() && NDOT <= 1;
      const T* xcol = J.x + col0;
      // Other than FP64: the thread's column shift and scale converted from
      // FP64 once per tile, not once per row (the conversion runs on the
      // FP64 pipe: per row it kept that pipe 21-31 % busy).
      CT csh[V], csc[V];
      if constexpr (!std::is_same<T, double>::value) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          csh[v] = has_shift ? CT(J.colshift[col0 + v]) : CT(0);
          csc[v] = has_scale ? CT(J.colscale[col0 + v]) : CT(1);
        }
      }
      int row = row0 + r;
      int q0 = 0, q1 = 0;
      if (kPipe && row < row1) {
        q0 = __ldg(J.rowptr + row);
        q1 = __ldg(J.rowptr + row + 1);
        chk_range(q0, q1, J.nnz);
      }
      for (; row < row1; row += R) {
        int nq0 = 0, nq1 = 0;
        if constexpr (kPipe) {
          if (row + R < row1) {
            nq0 = __ldg(J.rowptr + row + R);
            nq1 = __ldg(J.rowptr + row + R + 1);
            chk_range(nq0, nq1, J.nnz);
          }
        } else {
          q0 = __ldg(J.rowptr + row);
          q1 = __ldg(J.rowptr + row + 1);
          chk_range(q0, q1, J.nnz);
        }
        // Latency-bound blocks: the x rows of the row's first kPrefetch
        // entries, and the row of each window vector, are requested into L2
        // in one wave before the row's own loads (one round trip for their
        // indices).  The gathers that follow, one batch and then the tail
        // one entry at a time, and the dot loads then wait for DRAM once per
        // row instead of once per batch and per tail entry (most rows of a
        // power-law graph are shorter than a batch).  FP64 blocks, bound by
        // the FP64 pipe on regular matrices, prefetch only for matrices cut
        // into work items (irregular rows), whose pass waits on loads too;
        // as a runtime switch the prefetch cost the single-dot FP64 instance
        // a spill, so it is an instance of its own.  The arithmetic is
        // unchanged.
        if constexpr (PF) {
#pragma unroll
          for (int u = 0; u < kPrefetch; ++u) {
            if (q0 + u < q1) prefetch_l2(xcol + (size_t)chk_col(__ldg(J.colind + q0 + u), J.n) * J.ld);
          }
#pragma unroll
          for (int d = 0; d < NDOT; ++d)
            if (d < ndots) prefetch_l2(J.dotv[d] + (size_t)row * J.ld + col0);
        }
        // FP32, BF16 and double-float blocks with two window dots: the row's
        // window vectors are requested before its gathers, so their latency
        // overlaps them (the dot products keep their order).  Measured on the 2M-row
        // power-law graph (OSA-IOP k = 2, m = 100): SpMM 334 -> 295 ms per
        // solve.  The instance for up to four dots keeps late loads: early
        // loads of all four cost the second CTA per SM (428 -> 666 ms), and
        // of the first two, at two CTAs per SM, still lost (427 -> 584 ms).
        constexpr bool kEarlyDots = narrow_block<T>() && NDOT == 2;
        CT ue[kEarlyDots ? NDOT : 1][V];
        if constexpr (kEarlyDots) {
#pragma unroll
          for (int d = 0; d < NDOT; ++d)
            if (d < ndots) load_v<COH, T>(J.dotv[d] + (size_t)row * J.ld + col0, ue[d]);
        }
        CT s[V];
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] = CT(0);
        int q = q0;
        if constexpr (kPipe) {
          int c[kGather];
          CT a[kGather];
          if (q + kGather <= q1) {
#pragma unroll
            for (int u = 0; u < kGather; ++u) {
              c[u] = chk_col(__ldg(J.colind + q + u), J.n);
              a[u] = __ldg(J.vals + q + u);
            }
          }
          for (; q + kGather <= q1; q += kGather) {
            CT xv[kGather][V];
#pragma unroll
            for (int u = 0; u < kGather; ++u) load_v<COH, T>(xcol + (size_t)c[u] * J.ld, xv[u]);
            const bool more = q + 2 * kGather <= q1;
            int cn[kGather];
            CT an[kGather];
            if (more) {
#pragma unroll
              for (int u = 0; u < kGather; ++u) {
                cn[u] = chk_col(__ldg(J.colind + q + kGather + u), J.n);
                an[u] = __ldg(J.vals + q + kGather + u);
              }
            }
#pragma unroll
            for (int u = 0; u < kGather; ++u)
#pragma unroll
              for (int v = 0; v < V; ++v) s[v] = fma(a[u], xv[u][v], s[v]);
            if (more) {
#pragma unroll
              for (int u = 0; u < kGather; ++u) {
                c[u] = cn[u];
                a[u] = an[u];
              }
            }
          }
        } else {
          for (; q + kGather <= q1; q += kGather) {
            int c[kGather];
            CT a[kGather], xv[kGather][V];
#pragma unroll
            for (int u = 0; u < kGather; ++u) {
              c[u] = chk_col(__ldg(J.colind + q + u), J.n);
              a[u] = __ldg(J.vals + q + u);
            }
#pragma unroll
            for (int u = 0; u < kGather; ++u) load_v<COH, T>(xcol + (size_t)c[u] * J.ld, xv[u]);
#pragma unroll
            for (int u = 0; u < kGather; ++u)
#pragma unroll
              for (int v = 0; v < V; ++v) s[v] = fma(a[u], xv[u][v], s[v]);
          }
        }
        for (; q < q1; ++q) {
          const int c = chk_col(__ldg(J.colind + q), J.n);
          const CT a = __ldg(J.vals + q);
          CT xv[V];
          load_v<COH, T>(xcol + (size_t)c * J.ld, xv);
#pragma unroll
          for (int v = 0; v < V; ++v) s[v] = fma(a, xv[v], s[v]);
        }
        if (has_shift || has_scale) {
          CT xr[V];
          load_v<COH, T>(xcol + (size_t)row * J.ld, xr);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            if constexpr (std::is_same<T, double>::value) {
              if (has_shift) s[v] = fma(CT(J.colshift[col0 + v]), xr[v], s[v]);
              if (has_scale) s[v] = s[v] * CT(J.colscale[col0 + v]);
            } else {
              if (has_shift) s[v] = fma(csh[v], xr[v], s[v]);
              if (has_scale) s[v] = s[v] * csc[v];
            }
          }
        }
        store_vec<T>(J.y + (size_t)row * J.ld + col0, s);
#pragma unroll
        for (int d = 0; d < NDOT; ++d) {
          if (d < ndots) {
            CT u[V];
            if constexpr (kEarlyDots) {
#pragma unroll
              for (int v = 0; v < V; ++v) u[v] = ue[d][v];
            } else {
              load_v<COH, T>(J.dotv[d] + (size_t)row * J.ld + col0, u);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) acc[d][v].fma(u[v], s[v]);
          }
        }
        q0 = nq0;
        q1 = nq1;
      }
    }
#pragma unroll
    for (int d = 0; d < NDOT; ++d) {
      if (d < ndots)
        cta_reduce_write<T, Acc>(smem, acc[d], live, G, R, J.col_off, J.width,
                                 J.part + (size_t)d * J.ld * J.ntiles, J.ntiles, tile);
    }
    __syncthreads();
  }
}

template <typename T, int NDOT, bool PF>
__global__ void __launch_bounds__(512, fp64_wide_min_ctas<T, NDOT>())
    k_spmm(const __grid_constant__ SpmmBatch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_entry();
  spmm_tiles<T, NDOT, SpmmBatch<T>, false, PF>(B, blockIdx.x, gridDim.x, smem_raw);
}

// FP32, BF16 and double-float blocks: the pass is bound by the latency of
// its dependent loads (row range -> column indices -> gathers of x), so resident warps
// count for more than registers.  A register cap that fits three 352-thread
// CTAs per SM instead of two (two instead of one for the full window)
// trades a few spilled accumulators for 50% more loads in flight.  Measured
// on the 2M-row power-law graph, OSA-IOP m = 20, mixed FP32, SpMM time:
// window 4 82.5 -> 55.5 ms (8-shift group 403 -> 282 ms), window 2
// 58.4 -> 43.7 ms, window 8 176 -> 151 ms; a cap of 48 lost again (58.1 ms).
// The same caps on the update pass lost (window 4 11.6 -> 13.0 ms, window 8
// 26.4 -> 38.4 ms): it streams, and keeps its registers.  Register
// allocation does not change the arithmetic: results are bitwise the same.
// (Double-float blocks with the software-pipelined single-dot loop keep 64:
// at 56 that instance spilled its prefetched row.)
template <typename T, int NDOT>
constexpr int lo_spmm_regs() {
  return NDOT > 4 ? 88 : (std::is_same<T, f32x2>::value && NDOT <= 1) ? 64 : 56;
}

template <typename T, int NDOT>
__global__ void __maxnreg__((lo_spmm_regs<T, NDOT>()))
    k_spmm_lo(const __grid_constant__ SpmmBatch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_entry();
  spmm_tiles<T, NDOT>(B, blockIdx.x, gridDim.x, smem_raw);
}

// PF: matrices cut into work items (FP64 blocks take the prefetching
// instance there; the other block types always prefetch).
template <typename T, int NDOT, bool PF>
constexpr auto spmm_kernel() {
  if constexpr (!narrow_block<T>()) return k_spmm<T, NDOT, PF>;
  else return k_spmm_lo<T, NDOT>;
}

// ---------------------------------------------------------------------------
// pass 2: out = ycoef*y - sum_i coef_i basis_i;  |out|^2 [; extra . out]
//
// EX: the batch has jobs with the extra dot (OSA-IOP's u_1 . u_{j+1});
// without it the instance carries no code for it.  For FP64 blocks a column
// scale ycoef != 1 (a power of two once sigma drifted, 0 for an inactive
// probe) is applied to y in place before the row loop (y is this step's
// pass-1 output and nothing reads it after this pass), so the loop issues
// only the FMAs the update needs; the product is the one the loop would
// form, so results do not change.
// ---------------------------------------------------------------------------
// load_vec through L2 only (ld.global.cg), for FP64 data this kernel may
// have written earlier: the non-coherent path of load_vec must not read it.
template <typename T>
__device__ __forceinline__ void load_vec_cg(const T* p, typename Compute<T>::type (&v)[Vec16<T>::N]) {
  static_assert(std::is_same<T, double>::value, "coherent vector loads are used for FP64 blocks");
  const double2 t = __ldcg(reinterpret_cast<const double2*>(p));
  v[0] = t.x;
  v[1] = t.y;
}

// FP64 update instances held at two CTAs per SM: the full window (see
// fp64_wide_min_ctas) and the software-pipelined NB <= 2 loop below (its
// prefetched row fits 64 registers).
template <typename T, int NB>
constexpr int update_min_ctas() {
  return (std::is_same<T, double>::value && (NB >= kMaxWin || NB <= 2)) ? 2 : 0;
}

// Pass 2 over the tiles gt0, gt0 + stride, ... of a batch (UpdBatch or a
// type with the same members), each by the whole CTA.
template <typename T, int NB, bool EX, typename Batch, bool COH = false>
__device__ __forceinline__ void update_tiles(const Batch& B, int gt0, int stride,
                                             unsigned char* smem_raw) {
  constexpr int V = Vec16<T>::N;
  using Acc = typename AccOf<T>::type;
  using CT = typename Compute<T>::type;
  Acc* smem = reinterpret_cast<Acc*>(smem_raw);
  for (int gt = gt0; gt < B.total_tiles; gt += stride) {
    const int jb = find_job(B, gt);
    const UpdJob<T>& J = B.jobs[jb];
    const int tile = gt - B.tile_start[jb];
    const int G = J.width / V;
    const int R = blockDim.x / G;
    const int r = threadIdx.x / G;
    const int g = threadIdx.x - r * G;
    const bool live = r < R;
    const int row0 = tile * J.tile_rows;
    const int row1 = min(row0 + J.tile_rows, J.n);
    const int col0 = J.col_off + g * V;
    const int nb = J.nbasis;
    const bool has_extra = EX && J.extra != nullptr;

    Acc nrm[V], ex[V];
#pragma unroll
    for (int v = 0; v < V; ++v) { nrm[v].zero(); ex[v].zero(); }

    if (live) {
      CT cf[NB > 0 ? NB : 1][V];
      CT yc[V];
      bool unit = true;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        double a = J.ycoef[col0 + v];
        yc[v] = CT(a);
        unit = unit && (a == 1.0);
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int v = 0; v < V; ++v)
          cf[i][v] = (i < nb) ? CT(J.coef[i * J.ld + col0 + v]) : CT(0);

      // FP64: scale y in place where ycoef != 1 (rows and chunk of this
      // thread only), then read y through L2 so the loop sees those stores.
      constexpr bool kPre = std::is_same<T, double>::value;
      if constexpr (kPre) {
        if (!unit) {
          T* yw = const_cast<T*>(J.y);
          for (int row = row0 + r; row < row1; row += R) {
            const size_t off = (size_t)row * J.ld + col0;
            CT o[V];
            load_vec_cg<T>(yw + off, o);
#pragma unroll
            for (int v = 0; v < V; ++v) o[v] = o[v] * yc[v];
            store_vec<T>(yw + off, o);
          }
        }
      }
      auto load_y = [&](size_t off, CT (&o)[V]) {
        if constexpr (kPre) load_vec_cg<T>(J.y + off, o);
        else load_v<COH, T>(J.y + off, o);
      };
      const bool scale_in_loop = !kPre && !unit;

      // kU rows per thread at a time (rows row, row + R): every load of
      // both rows is issued before their arithmetic, doubling the bytes in
      // flight of the HBM-bound FP32 pass; each row's operations, and the
      // order in which the rows enter the norm, are those of one row at a
      // time.  (FP64 is bound by its ALU; BF16 blocks measured 2x slower
      // with two rows: their registers cost occupancy.)
      constexpr int kU = ((std::is_same<T, float>::value || std::is_same<T, f32x2>::value) && NB <= 4) ? 2 : 1;
      if constexpr (kU > 1) {
      for (int row = row0 + r; row < row1; row += kU * R) {
        bool on[kU];
        size_t off[kU];
#pragma unroll
        for (int q = 0; q < kU; ++q) {
          on[q] = row + q * R < row1;
          off[q] = (size_t)(on[q] ? row + q * R : row) * J.ld + col0;
        }
        CT o[kU][V], ub[kU][NB > 0 ? NB : 1][V], ue[kU][V];
#pragma unroll
        for (int q = 0; q < kU; ++q) {
          load_y(off[q], o[q]);
#pragma unroll
          for (int i = 0; i < NB; ++i)
            if (i < nb) load_v<COH, T>(J.basis[i] + off[q], ub[q][i]);
          if (has_extra) load_v<COH, T>(J.extra + off[q], ue[q]);
        }
#pragma unroll
        for (int q = 0; q < kU; ++q) {
          if (!on[q]) continue;
          if (scale_in_loop) {
#pragma unroll
            for (int v = 0; v < V; ++v) o[q][v] = o[q][v] * yc[v];
          }
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            if (i < nb) {
#pragma unroll
              for (int v = 0; v < V; ++v) o[q][v] = fma(-cf[i][v], ub[q][i][v], o[q][v]);
            }
          }
          store_vec<T>(J.out + off[q], o[q]);
#pragma unroll
          for (int v = 0; v < V; ++v) nrm[v].fma(o[q][v], o[q][v]);
          if (has_extra) {
#pragma unroll
            for (int v = 0; v < V; ++v) ex[v].fma(ue[q][v], o[q][v]);
          }
        }
      }
      } else if constexpr (std::is_same<T, double>::value && NB <= 2) {
      // FP64 with up to two basis vectors: the next row's loads are issued
      // before this row's arithmetic, so the FP64 pipe works while they are
      // in flight (one row at a time left it and HBM both half idle).  The
      // operations and their order per row are those of the loop below.
      CT py[V], pu[NB][V], pe[V];
      int row = row0 + r;
      if (row < row1) {
        const size_t off = (size_t)row * J.ld + col0;
        load_y(off, py);
#pragma unroll
        for (int i = 0; i < NB; ++i)
          if (i < nb) load_v<COH, T>(J.basis[i] + off, pu[i]);
        if (has_extra) load_v<COH, T>(J.extra + off, pe);
      }
      for (; row < row1; row += R) {
        const size_t off = (size_t)row * J.ld + col0;
        CT o[V], u[NB][V], e[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          o[v] = py[v];
          e[v] = pe[v];
#pragma unroll
          for (int i = 0; i < NB; ++i) u[i][v] = pu[i][v];
        }
        if (row + R < row1) {
          const size_t noff = off + (size_t)R * J.ld;
          load_y(noff, py);
#pragma unroll
          for (int i = 0; i < NB; ++i)
            if (i < nb) load_v<COH, T>(J.basis[i] + noff, pu[i]);
          if (has_extra) load_v<COH, T>(J.extra + noff, pe);
        }
        if (scale_in_loop) {
#pragma unroll
          for (int v = 0; v < V; ++v) o[v] = o[v] * yc[v];
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i < nb) {
#pragma unroll
            for (int v = 0; v < V; ++v) o[v] = fma(-cf[i][v], u[i][v], o[v]);
          }
        }
        store_vec<T>(J.out + off, o);
#pragma unroll
        for (int v = 0; v < V; ++v) nrm[v].fma(o[v], o[v]);
        if (has_extra) {
#pragma unroll
          for (int v = 0; v < V; ++v) ex[v].fma(e[v], o[v]);
        }
      }
      } else {
      for (int row = row0 + r; row < row1; row += R) {
        const size_t off = (size_t)row * J.ld + col0;
        CT o[V];
        load_y(off, o);
        if (scale_in_loop) {
#pragma unroll
          for (int v = 0; v < V; ++v) o[v] = o[v] * yc[v];
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          if (i < nb) {
            CT u[V];
            load_v<COH, T>(J.basis[i] + off, u);
#pragma unroll
            for (int v = 0; v < V; ++v) o[v] = fma(-cf[i][v], u[v], o[v]);
          }
        }
        store_vec<T>(J.out + off, o);
#pragma unroll
        for (int v = 0; v < V; ++v) nrm[v].fma(o[v], o[v]);
        if (has_extra) {
          CT u[V];
          load_v<COH, T>(J.extra + off, u);
#pragma unroll
          for (int v = 0; v < V; ++v) ex[v].fma(u[v], o[v]);
        }
      }
      }
    }
    cta_reduce_write<T, Acc>(smem, nrm, live, G, R, J.col_off, J.width, J.part, J.ntiles, tile);
    if (has_extra)
      cta_reduce_write<T, Acc>(smem, ex, live, G, R, J.col_off, J.width,
                               J.part + (size_t)J.ld * J.ntiles,
                               J.ntiles, tile);
    __syncthreads();
  }
}

template <typename T, int NB, bool EX>
__global__ void __launch_bounds__(512, update_min_ctas<T, NB>())
    k_update(const __grid_constant__ UpdBatch<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_entry();
  update_tiles<T, NB, EX>(B, blockIdx.x, gridDim.x, smem_raw);
}

// ---------------------------------------------------------------------------
// Scalar kernels.  One CTA per (probe, dot) reduces that dot's ntiles
// partials in a fixed order; the last CTA of a probe to finish (an arrival
// counter behind a fence) runs the probe's scalar recurrence on the reduced
// values.  Which CTA arrives last does not change any value.
// ---------------------------------------------------------------------------
constexpr int kRedLanes = 4;  // independent accumulators per thread


// Sum of the ntiles partials of (dot d, column p) by a CTA of kRedThreads
// threads: thread t adds tiles t + kRedThreads*(kRedLanes*i + l) into
// accumulator l, the lanes are combined in order, then a shared-memory tree.
// Returns the value to every thread.
template <typename Acc, typename PartT>
__device__ double reduce_partials(const PartT* part, int ld, int ntiles, int d, int p, Acc* sh) {
  const int t = threadIdx.x;
  const PartT* src = part + ((size_t)d * ld + p) * ntiles;
  Acc a[kRedLanes];
#pragma unroll
  for (int l = 0; l < kRedLanes; ++l) a[l].zero();
  const int stride = kRedThreads * kRedLanes;
  for (int base = t; base < ntiles; base += stride) {
#pragma unroll
    for (int l = 0; l < kRedLanes; ++l) {
      const int i = base + l * kRedThreads;
      if (i < ntiles) {
        Acc o;
        get_part(src + i, o);
        a[l].add(o);
      }
    }
  }
#pragma unroll
  for (int l = 1; l < kRedLanes; ++l) a[0].add(a[l]);
  sh[t] = a[0];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
      Acc x = sh[t];
      x.add(sh[t + w]);
      sh[t] = x;
    }
    __syncthreads();
  }
  const double r = sh[0].value();
  __syncthreads();
  return r;
}

__device__ __forceinline__ int find_probe_job(const ScalarBatch& B, int gp) {
  int j = 0;
  while (j + 1 < B.njobs && gp >= B.probe_start[j + 1]) ++j;
  return j;
}

// Power-of-two factor keeping the stored vectors near unit norm when sigma drifts.
// Sigma within 2^+-(lim - 1) is well inside the limit whatever log2 rounds
// to, so the answer 1 needs no FP64 logarithm there.
__device__ __forceinline__ double rescale_factor(double sigma, double lim) {
  const long long e = (long long)lim - 1;  // 2^+-e built from its bits (1 <= e <= 1000)
  const double lo = __longlong_as_double((1023 - e) << 52), hi = __longlong_as_double((1023 + e) << 52);
  if (sigma >= lo && sigma <= hi) return 1.0;
  double l2 = log2(sigma);
  if (fabs(l2) <= lim) return 1.0;
  return exp2(rint(l2));
}

__device__ void scalar_init(const ScalarJob& J, int p, const double* D) {
  const KrylovState& S = J.st;
  const double nn = D[0];
  const int m2 = S.m + 2;
  S.status[p] = 0;
  S.meff[p] = 0;
  if (nn > 0.0 && p < S.b) {
    S.sig[p * m2 + 1] = 1.0 / sqrt(nn);
    S.active[p] = 1;
  } else {
    S.sig[p * m2 + 1] = 0.0;
    S.active[p] = 0;
  }
  if (S.edot) S.edot[p * m2 + 1] = nn;
}

__device__ void scalar_coef(const ScalarJob& J, int p, const double* D) {
  const KrylovState& S = J.st;
  const int j = J.step;
  const int m2 = S.m + 2;
  const double* sg = S.sig + p * m2;
  double* coef = S.coef;
  if (!S.active[p]) {
    S.ycoef[p] = 0.0;
    for (int t = 0; t < kMaxWin; ++t) coef[t * S.ld + p] = 0.0;
    return;
  }
  S.meff[p] = j;
  const double sj = sg[j];
  const double a = rescale_factor(sj, S.rescale_lim);
  if (S.method == 0) {
    const double al = sj * sj * D[0];
    S.alpha[p * S.m + j - 1] = al;
    if (j >= 2) {
      coef[0 * S.ld + p] = a * S.beta[p * S.m + j - 2] * sg[j - 1] / sj;
      coef[1 * S.ld + p] = a * al;
    } else {
      coef[0 * S.ld + p] = a * al;
    }
  } else {
    double* Hc = S.H + (size_t)p * (S.m + 1) * S.m + (size_t)(j - 1) * (S.m + 1);
    for (int t = 0; t < J.ndots; ++t) {
      const int i = J.win_lo + t;
      Hc[i - 1] = sg[i] * sj * D[t];
      coef[t * S.ld + p] = a * sg[i] * sg[i] * D[t];
    }
  }
  S.ycoef[p] = a;
}

__device__ void scalar_norm(const ScalarJob& J, int p, const double* D) {
  const KrylovState& S = J.st;
  if (!S.active[p]) return;
  const double nn = D[0];
  const double ee = J.ndots > 1 ? D[1] : 0.0;
  const int j = J.step;
  const int m2 = S.m + 2;
  double* sg = S.sig + p * m2;
  const double a = S.ycoef[p];
  const double h = sg[j] * sqrt(nn) / a;
  bool stop;
  if (S.method == 0) {
    S.beta[p * S.m + j - 1] = h;
    stop = !(h > S.tol);          // beta_j <= tol
  } else {
    S.H[(size_t)p * (S.m + 1) * S.m + (size_t)(j - 1) * (S.m + 1) + j] = h;
    stop = h < S.tol;
  }
  if (stop) {
    S.active[p] = 0;
    S.status[p] |= LOGDET_ST_BREAKDOWN;
    sg[j + 1] = 0.0;
  } else {
    sg[j + 1] = sg[j] / (a * h);
  }
  if (S.edot) S.edot[p * m2 + j + 1] = ee;
}

// Dot d of probe p of a scalar job by one CTA: reduce its partials; the last
// of the probe's dots to arrive runs the recurrence.
template <typename Acc, typename PartT>
__device__ void scalar_item(const ScalarJob& J, int kind, int p, int d, Acc* sh) {
  const KrylovState& S = J.st;
  const double v = reduce_partials<Acc, PartT>(static_cast<const PartT*>(J.part), S.ld, J.ntiles,
                                               d, p, sh);
  if (threadIdx.x == 0) {
    S.dbuf[d * S.ld + p] = v;
    __threadfence();
    const unsigned ticket = atomicAdd(S.cnt + p, 1u);
    if (ticket == (unsigned)(J.ndots - 1)) {
      S.cnt[p] = 0;
      __threadfence();
      double D[kMaxWin];
      for (int t = 0; t < J.ndots; ++t) D[t] = __ldcg(S.dbuf + t * S.ld + p);
      if (kind == SK_INIT) scalar_init(J, p, D);
      else if (kind == SK_COEF) scalar_coef(J, p, D);
      else scalar_norm(J, p, D);
    }
  }
}

template <typename Acc, typename PartT>
__device__ void scalar_body(const ScalarBatch& B, int kind, Acc* sh) {
  const int gp = blockIdx.x;
  const int d = blockIdx.y;
  const int jb = find_probe_job(B, gp);
  const ScalarJob& J = B.jobs[jb];
  const int p = gp - B.probe_start[jb];
  if (d >= J.ndots) return;
  scalar_item<Acc, PartT>(J, kind, p, d, sh);
}

__global__ void __launch_bounds__(kRedThreads) k_scalar(const __grid_constant__ ScalarBatch B,
                                                        int kind, int f32) {
  __shared__ AccD shd[kRedThreads];
  __shared__ AccF shf[kRedThreads];
  pdl_entry();
  if (f32) scalar_body<AccF, float2>(B, kind, shf);
  else scalar_body<AccD, double>(B, kind, shd);
}

// ---------------------------------------------------------------------------
// Persistent Krylov run (see krylov.cuh).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of the cooperative run: a counter and a generation
// word.  Every wait is bounded (P.limit_ns of the global timer, 2^26 polls);
// a CTA that gives up, or sees that another one did, sets / keeps P.err and
// the whole CTA returns false, so every CTA leaves the kernel.
template <typename T>
__device__ bool run_barrier(const PersistRun<T>& P) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = P.bar + 1;
    volatile int* err = P.err;
    int ok = 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(P.bar, 1u) + 1u;
    if (arrived == P.nwait) {
      atomicExch(P.bar, 0u);
      __threadfence();
      atomicAdd(P.bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned polls = 0;
      while (*gen == g0) {
        if (*err || ++polls > (1u << 26) ||
            (long long)(global_ns() - t0) > P.limit_ns) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (!ok) atomicExch(P.err, 1);
    __threadfence();
    s_ok = ok && !*err;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T* run_ptr(const PersistRun<T>& P, int i) {
  if (P.Vfull) return P.Vfull + (size_t)(i - 1) * P.blk;
  if (i == 1) return P.X0;
  return P.ring + (size_t)((i - 2) % P.nring) * P.blk;
}

// One warp's copy of reduce_partials for (dot d, column p): lane L stands in
// for the reduction threads L, L + 32, ..., L + 224, each accumulating the
// same tiles into the same lanes, then the same tree (the first three levels
// within a lane, the last five by shuffles), so the value is bit-identical
// to the 256-thread reduction of k_scalar.  Partials are read through L2.
template <typename Acc>
__device__ __forceinline__ Acc shfl_down_acc(const Acc& a, int w);
template <>
__device__ __forceinline__ AccD shfl_down_acc<AccD>(const AccD& a, int w) {
  AccD o;
  o.s = __shfl_down_sync(0xffffffffu, a.s, w);
  return o;
}
template <>
__device__ __forceinline__ AccF shfl_down_acc<AccF>(const AccF& a, int w) {
  AccF o;
  o.s = __shfl_down_sync(0xffffffffu, a.s, w);
  o.e = __shfl_down_sync(0xffffffffu, a.e, w);
  return o;
}

template <typename Acc, typename PartT>
__device__ double warp_reduce_partials(const PartT* part, int ld, int ntiles, int d, int p) {
  static_assert(kRedThreads == 256, "the warp copy stands in for 8 threads per lane");
  const int L = threadIdx.x & 31;
  const PartT* src = part + ((size_t)d * ld + p) * ntiles;
  // Slots (reduction threads) that hold data: the others stay +0, and the
  // additions of +0 that the 256-thread tree makes leave a value unchanged
  // (accumulators start at +0 and never become -0), so they are skipped.
  int nz = min(ntiles, kRedThreads);
  Acc v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int t = L + 32 * k;
    Acc a[kRedLanes];
#pragma unroll
    for (int l = 0; l < kRedLanes; ++l) a[l].zero();
    if (t < nz) {
      for (int base = t; base < ntiles; base += kRedThreads * kRedLanes) {
#pragma unroll
        for (int l = 0; l < kRedLanes; ++l) {
          const int i = base + l * kRedThreads;
          if (i < ntiles) {
            const PartT x = __ldcg(src + i);
            Acc o;
            get_part(&x, o);
            a[l].add(o);
          }
        }
      }
#pragma unroll
      for (int l = 1; l < kRedLanes; ++l) a[0].add(a[l]);
    }
    v[k] = a[0];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)                       // w = 128
    if (L + 32 * k + 128 < nz) v[k].add(v[k + 4]);
  nz = min(nz, 128);
#pragma unroll
  for (int k = 0; k < 2; ++k)                       // w = 64
    if (L + 32 * k + 64 < nz) v[k].add(v[k + 2]);
  nz = min(nz, 64);
  if (L + 32 < nz) v[0].add(v[1]);                  // w = 32
  nz = min(nz, 32);
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {               // w = 16 .. 1
    const Acc o = shfl_down_acc(v[0], w);
    if (L + w < nz) v[0].add(o);                    // (implies L < w: nz <= 2w here)
    nz = min(nz, w);
  }
  return __shfl_sync(0xffffffffu, v[0].value(), 0);
}

// Shared-memory state of a persistent run: every CTA keeps the per-probe
// scalars the recurrences read (recent sigmas, the last beta, the active
// flags) and the pass-2 coefficients, and runs the recurrences itself, so a
// step needs two grid barriers (after each pass) instead of four.
constexpr int kRunMaxLd = 128;         // ld <= 2 * kMaxSketch
constexpr int kSgRing = kMaxWin + 3;   // sigma_{j-k+1} .. sigma_{j+1}

struct RunShared {
  double sg[kRunMaxLd][kSgRing];
  double cf[kMaxWin * kRunMaxLd];      // pass-2 coefficients, [t][ld] as in KrylovState::coef
  double yc[kRunMaxLd];
  double D[kMaxWin][kRunMaxLd];
  double beta_prev[kRunMaxLd];
  int act[kRunMaxLd];
};

// The coefficient step of probe p (the expressions of scalar_coef, with the
// sigmas and beta from shared memory); CTA 0 also writes the history.
__device__ __forceinline__ void run_coef(const KrylovState& S, RunShared& R, int p, int j, int lo,
                                         int nd, bool writer) {
  const int ld = S.ld;
  if (!R.act[p]) {
    R.yc[p] = 0.0;
    for (int t = 0; t < kMaxWin; ++t) R.cf[t * ld + p] = 0.0;
    return;
  }
  if (writer) S.meff[p] = j;
  const double* sg = R.sg[p];
  const double sj = sg[j % kSgRing];
  const double a = rescale_factor(sj, S.rescale_lim);
  if (S.method == 0) {
    const double al = sj * sj * R.D[0][p];
    if (writer) S.alpha[p * S.m + j - 1] = al;
    if (j >= 2) {
      R.cf[0 * ld + p] = a * R.beta_prev[p] * sg[(j - 1) % kSgRing] / sj;
      R.cf[1 * ld + p] = a * al;
    } else {
      R.cf[0 * ld + p] = a * al;
    }
  } else {
    double* Hc = S.H + (size_t)p * (S.m + 1) * S.m + (size_t)(j - 1) * (S.m + 1);
    for (int t = 0; t < nd; ++t) {
      const int i = lo + t;
      const double si = sg[i % kSgRing];
      if (writer) Hc[i - 1] = si * sj * R.D[t][p];
      R.cf[t * ld + p] = a * si * si * R.D[t][p];
    }
  }
  R.yc[p] = a;
}

// The norm step of probe p (the expressions of scalar_norm).
__device__ __forceinline__ void run_norm(const KrylovState& S, RunShared& R, int p, int j, int nd2,
                                         bool writer) {
  if (!R.act[p]) return;
  const double nn = R.D[0][p];
  const double ee = nd2 > 1 ? R.D[1][p] : 0.0;
  const int m2 = S.m + 2;
  const double a = R.yc[p];
  const double sgj = R.sg[p][j % kSgRing];
  const double h = sgj * sqrt(nn) / a;
  bool stop;
  if (S.method == 0) {
    R.beta_prev[p] = h;
    if (writer) S.beta[p * S.m + j - 1] = h;
    stop = !(h > S.tol);
  } else {
    if (writer) S.H[(size_t)p * (S.m + 1) * S.m + (size_t)(j - 1) * (S.m + 1) + j] = h;
    stop = h < S.tol;
  }
  double next;
  if (stop) {
    R.act[p] = 0;
    if (writer) {
      S.active[p] = 0;
      S.status[p] |= LOGDET_ST_BREAKDOWN;
    }
    next = 0.0;
  } else {
    next = sgj / (a * h);
  }
  R.sg[p][(j + 1) % kSgRing] = next;
  if (writer) {
    S.sig[p * m2 + j + 1] = next;
    if (S.edot) S.edot[p * m2 + j + 1] = ee;
  }
}

template <typename T, int NDOT, int NB, bool EX>
__global__ void __maxnreg__(128) k_krylov_run(const __grid_constant__ PersistRun<T> P) {
  using Acc = typename AccOf<T>::type;
  using PartT = typename PartOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ OneJob<SpmmJob<T>> sb;
  __shared__ OneJob<UpdJob<T>> ub;
  __shared__ RunShared R;
  const KrylovState& S = P.cj.st;
  const int ld = S.ld;
  const int m2 = S.m + 2;
  const bool writer = blockIdx.x == 0;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // start state (written by the kernels before this launch)
  for (int p = threadIdx.x; p < ld; p += blockDim.x) {
    R.sg[p][P.j0 % kSgRing] = __ldcg(S.sig + p * m2 + P.j0);
    R.act[p] = __ldcg(S.active + p);
    R.beta_prev[p] = 0.0;
  }
  if (threadIdx.x == 0) {
    sb.njobs = 1;
    sb.total_tiles = P.ntiles;
    sb.tile_start[0] = 0;
    sb.tile_start[1] = P.ntiles;
    sb.jobs[0] = P.sj;
    ub.njobs = 1;
    ub.total_tiles = P.ntiles;
    ub.tile_start[0] = 0;
    ub.tile_start[1] = P.ntiles;
    ub.jobs[0] = P.uj;
    ub.jobs[0].coef = R.cf;   // this CTA's copy of the coefficients
    ub.jobs[0].ycoef = R.yc;
  }
  // Pass-1 and pass-2 partials live in separate buffers: with no barrier
  // after the reductions, a CTA may start the next pass while another one
  // still reads the previous pass's partials.
  const PartT* part = static_cast<const PartT*>(P.cj.part);
  const PartT* part2 = P.uj.part;
  for (int j = P.j0; j <= P.m; ++j) {
    // the step's jobs, as KRun::spmm_jobs / upd_jobs build them
    const int lo = P.method == 0 ? j : max(1, j - P.k + 1);
    const int nd = P.method == 0 ? 1 : j - lo + 1;
    if (threadIdx.x == 0) {
      SpmmJob<T>& J = sb.jobs[0];
      J.x = run_ptr(P, j);
      J.ndots = nd;
      if (P.method == 0) J.dotv[0] = run_ptr(P, j);
      else
        for (int i = lo; i <= j; ++i) J.dotv[i - lo] = run_ptr(P, i);
    }
    __syncthreads();
    spmm_tiles<T, NDOT, OneJob<SpmmJob<T>>, true>(sb, blockIdx.x, gridDim.x, smem_raw);
    if (!run_barrier(P)) return;
    // coefficients: every CTA reduces all dots and runs every recurrence
    for (int it = warp; it < ld * nd; it += nwarps) {
      const int p = it / nd, d = it - p * nd;
      const double v = warp_reduce_partials<Acc, PartT>(part, ld, P.ntiles, d, p);
      if ((threadIdx.x & 31) == 0) R.D[d][p] = v;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < ld; p += blockDim.x) run_coef(S, R, p, j, lo, nd, writer);
    __syncthreads();
    if (j >= P.m) break;
    if (threadIdx.x == 0) {
      UpdJob<T>& U = ub.jobs[0];
      if (P.method == 0) {
        if (j >= 2) {
          U.nbasis = 2;
          U.basis[0] = run_ptr(P, j - 1);
          U.basis[1] = run_ptr(P, j);
        } else {
          U.nbasis = 1;
          U.basis[0] = run_ptr(P, j);
        }
      } else {
        U.nbasis = j - lo + 1;
        for (int i = lo; i <= j; ++i) U.basis[i - lo] = run_ptr(P, i);
      }
      U.out = run_ptr(P, j + 1);
    }
    __syncthreads();
    update_tiles<T, NB, EX, OneJob<UpdJob<T>>, true>(ub, blockIdx.x, gridDim.x, smem_raw);
    if (!run_barrier(P)) return;
    const int nd2 = P.track_e ? 2 : 1;
    for (int it = warp; it < ld * nd2; it += nwarps) {
      const int p = it / nd2, d = it - p * nd2;
      const double v = warp_reduce_partials<Acc, PartT>(part2, ld, P.ntiles, d, p);
      if ((threadIdx.x & 31) == 0) R.D[d][p] = v;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < ld; p += blockDim.x) run_norm(S, R, p, j, nd2, writer);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Resident CTAs per SM of (kernel, CTA size, shared memory), looked up once
// per thread and shape instead of once per launch.
template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, int total_tiles) {
  struct Entry { const void* f; int threads; size_t smem; int per_sm; };
  thread_local std::vector<Entry> cache;
  int per_sm = 0;
  const void* f = reinterpret_cast<const void*>(kernel);
  for (const Entry& e : cache)
    if (e.f == f && e.threads == threads && e.smem == smem) per_sm = e.per_sm;
  if (per_sm == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    cache.push_back(Entry{f, threads, smem, per_sm});
  }
  return std::max(1, std::min(total_tiles, per_sm * sm_count()));
}

// Launch with programmatic stream serialization (see pdl_entry).
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename T>
int launch_spmm(const SpmmBatch<T>& b, int threads, cudaStream_t s) {
  int nd = 0;
  bool items = false;
  for (int j = 0; j < b.njobs; ++j) {
    nd = std::max(nd, b.jobs[j].ndots);
    items = items || b.jobs[j].items != nullptr;
  }
  using Acc = typename AccOf<T>::type;
  size_t smem = (size_t)threads * Vec16<T>::N * sizeof(Acc);
  double flops = 0.0, bytes = 0.0;
  for (int j = 0; j < b.njobs; ++j) {
    const SpmmJob<T>& J = b.jobs[j];
    const double vb = (double)J.n * J.b * sizeof(T);
    const int extra_reads = J.ndots - ((J.ndots > 0 && J.dotv[0] == J.x) ? 1 : 0);
    flops += 2.0 * (double)J.nnz * J.b + 2.0 * (double)J.n * J.b * J.ndots;
    bytes += 4.0 * (J.n + 1) + (double)J.nnz * (4 + sizeof(typename ValOf<T>::type)) +
             vb * (2 + extra_reads);
  }
  ProfScope prof(KC_SPMM, s, flops, bytes);
#define LD_SPMM_CASE(ND)                                                      \
  {                                                                           \
    auto kern = items ? spmm_kernel<T, ND, true>() : spmm_kernel<T, ND, false>(); \
    int grid = persistent_grid(kern, threads, smem, b.total_tiles);           \
    launch_pdl(kern, dim3(grid), dim3(threads), smem, s, b);                  \
    break;                                                                    \
  }
  do {
    if (nd == 0) LD_SPMM_CASE(0)
    if (nd == 1) LD_SPMM_CASE(1)
    if (nd == 2) LD_SPMM_CASE(2)
    if (nd <= 4) LD_SPMM_CASE(4)
    LD_SPMM_CASE(kMaxWin)
  } while (0);
#undef LD_SPMM_CASE
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

template <typename T>
int launch_update(const UpdBatch<T>& b, int threads, cudaStream_t s) {
  int nb = 0;
  bool ex = false;
  for (int j = 0; j < b.njobs; ++j) {
    nb = std::max(nb, b.jobs[j].nbasis);
    ex = ex || b.jobs[j].extra != nullptr;
  }
  using Acc = typename AccOf<T>::type;
  size_t smem = (size_t)threads * Vec16<T>::N * sizeof(Acc);
  double flops = 0.0, bytes = 0.0;
  for (int j = 0; j < b.njobs; ++j) {
    const UpdJob<T>& J = b.jobs[j];
    const int ex = J.extra ? 1 : 0;
    const double vb = (double)J.n * J.b * sizeof(T);
    flops += 2.0 * (double)J.n * J.b * (J.nbasis + 1 + ex);
    bytes += vb * (2 + J.nbasis + ex);
  }
  ProfScope prof(KC_UPDATE, s, flops, bytes);
#define LD_UPD_CASE(NB)                                                       \
  {                                                                           \
    auto kern = ex ? k_update<T, NB, true> : k_update<T, NB, false>;          \
    int grid = persistent_grid(kern, threads, smem, b.total_tiles);           \
    launch_pdl(kern, dim3(grid), dim3(threads), smem, s, b);                  \
    break;                                                                    \
  }
  do {
    if (nb <= 1) LD_UPD_CASE(1)
    if (nb == 2) LD_UPD_CASE(2)
    if (nb <= 4) LD_UPD_CASE(4)
    LD_UPD_CASE(kMaxWin)
  } while (0);
#undef LD_UPD_CASE
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

// Test hook: LOGDET_TEST_KRUN_STALL=1 makes every barrier of a persistent run
// wait for one arrival more than the grid has, with a 20 ms bound, so that
// every wait runs out (the error path, exercised without a fault).
static bool krun_stall_test() {
  const char* e = std::getenv("LOGDET_TEST_KRUN_STALL");
  return e && e[0] == '1';
}

template <typename T>
int launch_krylov_run(const PersistRun<T>& P0, int threads, int nd_max, int nb_max,
                      cudaStream_t s) {
  using Acc = typename AccOf<T>::type;
  PersistRun<T> P = P0;
  const size_t smem = (size_t)threads * Vec16<T>::N * sizeof(Acc);
  auto cls = [](int w) { return w <= 1 ? 1 : w == 2 ? 2 : w <= 4 ? 4 : kMaxWin; };
  const int cd = cls(nd_max), cb = cls(nb_max);
  void* kern = nullptr;
#define LD_KRUN(ND, NB, EX)                                                     \
  if (cd == ND && cb == NB && (P.track_e != 0) == EX)                         \
    kern = reinterpret_cast<void*>(k_krylov_run<T, ND, NB, EX>);
  LD_KRUN(1, 2, false)
  LD_KRUN(1, 1, false) LD_KRUN(1, 1, true)
  LD_KRUN(2, 2, false) LD_KRUN(2, 2, true)
  LD_KRUN(4, 4, false) LD_KRUN(4, 4, true)
  LD_KRUN(kMaxWin, kMaxWin, false) LD_KRUN(kMaxWin, kMaxWin, true)
#undef LD_KRUN
  if (!kern || threads % 32 || threads > 512) {
    set_error("no persistent Krylov kernel for %d dots / %d basis vectors at %d threads", nd_max,
              nb_max, threads);
    return LOGDET_EINVAL;
  }
  int per_sm = 0;
  LD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) {
    set_error("persistent Krylov kernel does not fit an SM at %d threads", threads);
    return LOGDET_ECUDA;
  }
  if (P.sj.ld > kRunMaxLd) {
    set_error("persistent Krylov run: block width %d above %d", P.sj.ld, kRunMaxLd);
    return LOGDET_EINVAL;
  }
  const int work = P.ntiles;
  const int grid = std::max(1, std::min(work, per_sm * sm_count()));
  const bool stall = krun_stall_test();
  P.nwait = (unsigned)grid + (stall ? 1u : 0u);
  P.limit_ns = stall ? 20000000LL : 2000000000LL;
  LD_CUDA(cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned), s));
  ProfScope prof(KC_KRUN, s);
  void* args[] = {&P};
  cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, smem, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("persistent Krylov launch failed: %s", cudaGetErrorString(e));
    return LOGDET_ECUDA;
  }
  return LOGDET_OK;
}

template int launch_krylov_run<double>(const PersistRun<double>&, int, int, int, cudaStream_t);
template int launch_krylov_run<float>(const PersistRun<float>&, int, int, int, cudaStream_t);

static int total_probes(const ScalarBatch& b) { return b.probe_start[b.njobs]; }

static int launch_scalar(const ScalarBatch& b, int kind, cudaStream_t s) {
  int nd = 1, f32 = b.jobs[0].part_f32;
  for (int j = 0; j < b.njobs; ++j) nd = std::max(nd, b.jobs[j].ndots);
  ProfScope prof(KC_SCALAR, s);
  launch_pdl(k_scalar, dim3(total_probes(b), nd), dim3(kRedThreads), 0, s, b, kind, f32);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}

int launch_coef(const ScalarBatch& b, cudaStream_t s) { return launch_scalar(b, SK_COEF, s); }
int launch_norm(const ScalarBatch& b, cudaStream_t s) { return launch_scalar(b, SK_NORM, s); }
int launch_init_sigma(const ScalarBatch& b, cudaStream_t s) { return launch_scalar(b, SK_INIT, s); }

template int launch_spmm<double>(const SpmmBatch<double>&, int, cudaStream_t);
template int launch_spmm<float>(const SpmmBatch<float>&, int, cudaStream_t);
template int launch_spmm<bf16>(const SpmmBatch<bf16>&, int, cudaStream_t);
template int launch_spmm<f32x2>(const SpmmBatch<f32x2>&, int, cudaStream_t);
template int launch_update<double>(const UpdBatch<double>&, int, cudaStream_t);
template int launch_update<float>(const UpdBatch<float>&, int, cudaStream_t);
template int launch_update<bf16>(const UpdBatch<bf16>&, int, cudaStream_t);
template int launch_update<f32x2>(const UpdBatch<f32x2>&, int, cudaStream_t);

}  // namespace ld

// ---------------------------------------------------------------------------
// C-ABI: state of the checks of a checked build
// ---------------------------------------------------------------------------
extern "C" int logdet_checked_report(int32_t* checked, uint32_t* device_violations,
                                     uint64_t* canary_bytes) {
  if (!checked || !device_violations || !canary_bytes) {
    ld::set_error("checked_report: NULL argument");
    return LOGDET_EINVAL;
  }
  unsigned v = 0;
#ifdef LOGDET_CHECKED
  *checked = 1;
  LD_CUDA(cudaDeviceSynchronize());
  LD_CUDA(cudaMemcpyFromSymbol(&v, ld::g_violations, sizeof v));
#else
  *checked = 0;
#endif
  *device_violations = v;
  *canary_bytes = ld::canary_fault_count();
  return LOGDET_OK;
}
