// Matrix-free gridded operators (see grid.cuh): handle creation with the
// Gershgorin interval, the scaled expanded table, the convolution kernel and
// the pass-1 dot partials.
#include "grid.cuh"
#include "krylov.cuh"
#include "profile.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace ld {

// ---------------------------------------------------------------------------
// Handle: validation, expanded table, Gershgorin interval (Sec. 2.1)
// ---------------------------------------------------------------------------
int create_grid_handle(int nx, int ny, int R, const double* w, logdet_handle* out) {
  if (!out) { set_error("out is NULL"); return LOGDET_EINVAL; }
  *out = nullptr;
  if (nx < 1 || ny < 1 || (long long)nx * ny >= (1LL << 31) || R < 0 || R > kMaxGridRadius || !w) {
    set_error("grid operator: need nx, ny >= 1, nx * ny < 2^31, 0 <= radius <= %d, table",
              kMaxGridRadius);
    return LOGDET_EINVAL;
  }
  for (int i = 0; i < (R + 1) * (R + 1); ++i)
    if (!std::isfinite(w[i])) { set_error("grid operator: non-finite table entry %d", i); return LOGDET_EINVAL; }
  logdet_ctx* h = new logdet_ctx();
  auto fail = [&](int code) { destroy_handle(h); return code; };
  if (cudaGetDevice(&h->device) != cudaSuccess) { set_error("no CUDA device"); delete h; return LOGDET_ECUDA; }
  int rc = ensure_pool(h->device);
  if (rc) { delete h; return rc; }
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    delete h;
    return LOGDET_ECUDA;
  }
  h->kind = 1;
  h->gx = nx;
  h->gy = ny;
  h->gr = R;
  h->n = nx * ny;
  h->owns = false;
  h->vals_dtype = LOGDET_VALS_F64;
  // Stored entries of the implied matrix (accounting): each nonzero offset
  // (dy, dx) occurs (ny - |dy|)(nx - |dx|) times.
  long long nnz = 0;
  for (int dy = -R; dy <= R; ++dy)
    for (int dx = -R; dx <= R; ++dx) {
      const double v = w[std::abs(dy) * (R + 1) + std::abs(dx)];
      if (v != 0.0 && std::abs(dy) < ny && std::abs(dx) < nx)
        nnz += (long long)(ny - std::abs(dy)) * (nx - std::abs(dx));
    }
  h->nnz = nnz;
  // Gershgorin: the off-diagonal sum is largest at the most central point;
  // summed in column order (dy, then dx ascending) as for a CSR row.
  const int yc = ny / 2, xc = nx / 2;
  double r = 0.0;
  for (int dy = -R; dy <= R; ++dy) {
    if (yc + dy < 0 || yc + dy >= ny) continue;
    for (int dx = -R; dx <= R; ++dx) {
      if (xc + dx < 0 || xc + dx >= nx || (dy == 0 && dx == 0)) continue;
      r += std::fabs(w[std::abs(dy) * (R + 1) + std::abs(dx)]);
    }
  }
  h->g_lo = w[0] - r;
  h->g_hi = w[0] + r;
  // Expanded table and per-row extents.
  const int L = grid_row_len(R);
  std::vector<double> tab((size_t)(R + 1) * L, 0.0);
  std::vector<int> rx(R + 1, -1);
  for (int dy = 0; dy <= R; ++dy)
    for (int dx = -R; dx <= R; ++dx) {
      const double v = w[dy * (R + 1) + std::abs(dx)];
      tab[(size_t)dy * L + dx + R] = v;
      if (v != 0.0) rx[dy] = std::max(rx[dy], std::abs(dx));
    }
  if (cudaMalloc(&h->gtab, sizeof(double) * tab.size()) != cudaSuccess ||
      cudaMalloc(&h->grx, sizeof(int) * rx.size()) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of the grid table failed");
    return fail(LOGDET_ENOMEM);
  }
  if (cudaMemcpy(h->gtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->grx, rx.data(), sizeof(int) * rx.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("copy of the grid table failed");
    return fail(LOGDET_ECUDA);
  }
  if (!(h->g_hi > 0.0)) {
    set_error("Gershgorin upper bound %g is not positive: not SPD", h->g_hi);
    return fail(LOGDET_ENOTSPD);
  }
  *out = h;
  return LOGDET_OK;
}

size_t grid_table_count(const logdet_ctx* h) {
  return (size_t)(h->gr + 1) * grid_row_len(h->gr);
}

template <typename CT>
__global__ void k_grid_table(const double* __restrict__ in, size_t count, double c,
                             CT* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (CT)(in[i] / c);
}

template <typename CT>
int grid_table(const logdet_ctx* h, double c, CT* out, cudaStream_t st) {
  const size_t count = grid_table_count(h);
  ProfScope prof(KC_OTHER, st);
  k_grid_table<CT><<<(int)std::min<size_t>(div_up((int)count, 256), 1024), 256, 0, st>>>(
      h->gtab, count, c, out);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}
template int grid_table<double>(const logdet_ctx*, double, double*, cudaStream_t);
template int grid_table<float>(const logdet_ctx*, double, float*, cudaStream_t);


// ---------------------------------------------------------------------------
// y = Q x.  A CTA owns work items (a block of kGridTY output rows, a segment
// of kGridTX * kGridP outputs along x, a vector chunk of V block columns) and
// keeps the expanded table in shared memory for all of them.  It stages each
// input row within R of the block once (segment plus halo), and warp ty then
// accumulates the row's contribution to output row y0 + ty: every lane runs
// a sliding window over dx for its kGridP consecutive outputs, one shared
// load of x and one of W per step feeding kGridP x V FMAs.  The loop over dx
// is unrolled by kGridP so that the window's register slots are static
// (position base + k lives in slot k mod kGridP).  Items are ordered chunk,
// segment, row block, so that CTAs running together share input rows in L2.
// ---------------------------------------------------------------------------
// Packed FP32 pairs (Blackwell's fma.rn.f32x2): two IEEE single-precision
// FMAs per instruction, each rounded exactly as fmaf.  The four block
// columns of a thread share the weight, so its FMAs go in pairs; this halves
// the FMA instruction count (measured: issue 80 % -> 50 % busy), and the
// FP32 FMA pipe remains the limit.
__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long dup_f32x2(float w) {
  unsigned long long d;
  asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(w));
  return d;
}

template <typename T>
__global__ void __launch_bounds__(kGridThreads) k_grid_apply(
    const typename Compute<T>::type* __restrict__ tab, const int* __restrict__ rx, int nx, int ny,
    int R, const T* __restrict__ x, T* __restrict__ y, int ld, const double* __restrict__ colshift,
    int nseg, int nchunk) {
  constexpr int V = Vec16<T>::N;
  constexpr int P = kGridP;
  using CT = typename Compute<T>::type;
  using VT = typename Vec16<T>::type;  // 16 bytes: V values of CT (T is double or float)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 2 * R + 1 + P;
  const int TX = kGridTX * P;
  const int SL = TX + 2 * R + 2 * P;  // staged positions per input row
  CT* wt = reinterpret_cast<CT*>(smem_raw);
  // Staged row after the table (16-byte aligned).  Position p sits at slot
  // p + p / P: the lanes of a warp read positions P apart, and the skew
  // spreads each quarter-warp's 16-byte reads over distinct banks.
  VT* xs = reinterpret_cast<VT*>(smem_raw + ((size_t)(R + 1) * L * sizeof(CT) + 15) / 16 * 16);
  const int t = threadIdx.x;
  const int tx = t % kGridTX, ty = t / kGridTX;
  for (int i = t; i < (R + 1) * L; i += blockDim.x) wt[i] = tab[i];
  const int nyb = (ny + kGridTY - 1) / kGridTY;
  const long long total = (long long)nyb * nseg * nchunk;
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int yb = (int)(it % nyb);
    const int seg = (int)((it / nyb) % nseg);
    const int chunk = (int)(it / ((long long)nyb * nseg));
    const int col0 = chunk * V;
    const int x0 = seg * TX;
    const int y0 = yb * kGridTY;
    const int yo = y0 + ty;
    CT acc[P][V];
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[q][v] = CT(0);
    const int y_lo = max(0, y0 - R), y_hi = min(ny - 1, y0 + kGridTY - 1 + R);
    for (int yy = y_lo; yy <= y_hi; ++yy) {
      __syncthreads();  // previous row consumed (and the table loaded)
      const T* xrow = x + (size_t)yy * nx * ld + col0;
      for (int i = t; i < SL; i += blockDim.x) {
        const int gxp = x0 - R + i;
        VT v;
        if (gxp >= 0 && gxp < nx) v = __ldg(reinterpret_cast<const VT*>(xrow + (size_t)gxp * ld));
        else memset(&v, 0, sizeof v);
        xs[i + i / P] = v;
      }
      __syncthreads();
      const int dy = abs(yy - yo);
      if (yo >= ny || dy > R) continue;
      const int rxd = rx[dy];
      if (rxd < 0) continue;
      const int base = tx * P + (R - rxd);
      const int Lc = (2 * rxd + 1 + P - 1) / P * P;
      const CT* wrow = wt + (size_t)dy * L + (R - rxd);
      if constexpr (std::is_same<T, float>::value) {
        // acc[q][0..3] as two packed pairs; the same window and order as below.
        unsigned long long win2[P][2];
        unsigned long long* acc2 = reinterpret_cast<unsigned long long*>(&acc[0][0]);
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const int pos = base + q;
          const VT v = xs[pos + pos / P];
          memcpy(win2[q], &v, sizeof v);
        }
        for (int s0 = 0; s0 < Lc; s0 += P) {
#pragma unroll
          for (int u = 0; u < P; ++u) {
            const unsigned long long w2 = dup_f32x2(wrow[s0 + u]);
#pragma unroll
            for (int q = 0; q < P; ++q) {
              acc2[2 * q] = fma_f32x2(w2, win2[(q + u) % P][0], acc2[2 * q]);
              acc2[2 * q + 1] = fma_f32x2(w2, win2[(q + u) % P][1], acc2[2 * q + 1]);
            }
            const int pos = base + s0 + u + P;
            const VT v = xs[pos + pos / P];
            memcpy(win2[u], &v, sizeof v);
          }
        }
      } else {
        CT win[P][V];
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const int pos = base + q;
          const VT v = xs[pos + pos / P];
          memcpy(win[q], &v, sizeof v);
        }
        for (int s0 = 0; s0 < Lc; s0 += P) {
#pragma unroll
          for (int u = 0; u < P; ++u) {
            const CT w = wrow[s0 + u];
#pragma unroll
            for (int q = 0; q < P; ++q)
#pragma unroll
              for (int c = 0; c < V; ++c) acc[q][c] = fma(w, win[(q + u) % P][c], acc[q][c]);
            const int pos = base + s0 + u + P;
            const VT v = xs[pos + pos / P];
            memcpy(win[u], &v, sizeof v);
          }
        }
      }
    }
    if (yo < ny) {
      // The shift of the thread's columns, converted once (for FP32 blocks
      // the conversion from FP64 runs on the FP64 pipe).
      CT csh[V];
#pragma unroll
      for (int c = 0; c < V; ++c) csh[c] = colshift ? CT(colshift[col0 + c]) : CT(0);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int xo = x0 + tx * P + q;
        if (xo >= nx) break;
        const size_t off = ((size_t)yo * nx + xo) * ld + col0;
        if (colshift) {
          CT xr[V];
          load_vec<T>(x + off, xr);
#pragma unroll
          for (int c = 0; c < V; ++c) acc[q][c] = fma(csh[c], xr[c], acc[q][c]);
        }
        store_vec<T>(y + off, acc[q]);
      }
    }
  }
}

static size_t grid_smem_bytes(int R, size_t ct) {
  const size_t tabn = (size_t)(R + 1) * grid_row_len(R);
  const size_t tab_bytes = (tabn * ct + 15) / 16 * 16;
  const size_t sl = (size_t)kGridTX * kGridP + 2 * R + 2 * kGridP;
  return tab_bytes + (sl + sl / kGridP + 1) * 16;
}

template <typename T>
int grid_apply(const logdet_ctx* h, const typename Compute<T>::type* tab, const T* x, T* y,
               int ld, const double* colshift, cudaStream_t st) {
  using CT = typename Compute<T>::type;
  constexpr int V = Vec16<T>::N;
  if (ld % V) {
    set_error("grid operator: leading dimension %d is not a multiple of %d", ld, V);
    return LOGDET_EINVAL;
  }
  const int R = h->gr;
  const size_t smem = grid_smem_bytes(R, sizeof(CT));
  if (smem > 48 * 1024)
    LD_CUDA(cudaFuncSetAttribute(k_grid_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  const int nseg = div_up(h->gx, kGridTX * kGridP);
  const int nchunk = ld / V;
  const long long items = (long long)div_up(h->gy, kGridTY) * nseg * nchunk;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_apply<T>, kGridThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int grid = (int)std::max<long long>(1, std::min<long long>(items, (long long)per_sm * sm_count()));
  // Accounting: 2 flop per (output, column, table entry); x staged once per
  // (output row, input row) segment, y written once.
  double taps = 0.0;
  {
    // |stencil| from the implied nnz: nnz ~ n * taps away from the edges.
    taps = (double)h->nnz / std::max(1, h->n);
  }
  ProfScope prof(KC_GRID, st, 2.0 * taps * h->n * ld, 2.0 * (double)h->n * ld * sizeof(T));
  k_grid_apply<T><<<grid, kGridThreads, smem, st>>>(tab, h->grx, h->gx, h->gy, R, x, y, ld,
                                                    colshift, nseg, nchunk);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}
template int grid_apply<double>(const logdet_ctx*, const double*, const double*, double*, int,
                                const double*, cudaStream_t);
template int grid_apply<float>(const logdet_ctx*, const float*, const float*, float*, int,
                               const double*, cudaStream_t);

// ---------------------------------------------------------------------------
// Pass-1 dots of a gridded operator: partials [d][ld][tile] of dotv_d . y,
// uniform tiles, thread (r, g) owning rows r, r + R, ... of a tile and the
// vector chunk g (the layout of the SpMM pass's fused dots).
// ---------------------------------------------------------------------------
struct DotsArgs {
  const void* dotv[kMaxWin];
};

template <typename T, int NDOT>
__global__ void __launch_bounds__(512) k_dots(const T* __restrict__ y, const __grid_constant__ DotsArgs A,
                                              int ndots, typename PartOf<T>::type* __restrict__ part,
                                              int n, int ld, int tile_rows, int ntiles) {
  constexpr int V = Vec16<T>::N;
  using Acc = typename AccOf<T>::type;
  using CT = typename Compute<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* smem = reinterpret_cast<Acc*>(smem_raw);
  const int G = ld / V;
  const int Rg = blockDim.x / G;
  const int r = threadIdx.x / G;
  const int g = threadIdx.x - r * G;
  const bool live = r < Rg;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * tile_rows, row1 = min(row0 + tile_rows, n);
    Acc acc[NDOT][V];
#pragma unroll
    for (int d = 0; d < NDOT; ++d)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[d][v].zero();
    if (live) {
      for (int row = row0 + r; row < row1; row += Rg) {
        CT yv[V];
        load_vec<T>(y + (size_t)row * ld + g * V, yv);
#pragma unroll
        for (int d = 0; d < NDOT; ++d) {
          if (d < ndots) {
            CT u[V];
            load_vec<T>(static_cast<const T*>(A.dotv[d]) + (size_t)row * ld + g * V, u);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[d][v].fma(u[v], yv[v]);
          }
        }
      }
    }
#pragma unroll
    for (int d = 0; d < NDOT; ++d)
      if (d < ndots)
        cta_reduce_write<T, Acc>(smem, acc[d], live, G, Rg, 0, ld, part + (size_t)d * ld * ntiles,
                                 ntiles, tile);
    __syncthreads();
  }
}

template <typename T>
int dots_pass(const T* y, const T* const* dotv, int ndots, typename PartOf<T>::type* part, int n,
              int ld, int tile_rows, int ntiles, int threads, cudaStream_t st) {
  if (ndots < 1) return LOGDET_OK;
  if (ndots > kMaxWin) {
    set_error("dots_pass: %d dots exceed %d", ndots, kMaxWin);
    return LOGDET_EINVAL;
  }
  DotsArgs A;
  memset(&A, 0, sizeof A);
  for (int d = 0; d < ndots; ++d) A.dotv[d] = dotv[d];
  using Acc = typename AccOf<T>::type;
  const size_t smem = (size_t)threads * Vec16<T>::N * sizeof(Acc);
  const int grid = std::max(1, std::min(ntiles, 4 * sm_count()));
  ProfScope prof(KC_SPMM, st, 2.0 * n * ld * ndots, (double)n * ld * sizeof(T) * (1 + ndots));
#define LD_DOTS_CASE(ND) \
  k_dots<T, ND><<<grid, threads, smem, st>>>(y, A, ndots, part, n, ld, tile_rows, ntiles); break;
  switch (ndots <= 1 ? 1 : ndots <= 2 ? 2 : ndots <= 4 ? 4 : 9) {
    case 1: LD_DOTS_CASE(1)
    case 2: LD_DOTS_CASE(2)
    case 4: LD_DOTS_CASE(4)
    default: LD_DOTS_CASE(9)
  }
#undef LD_DOTS_CASE
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}
template int dots_pass<double>(const double*, const double* const*, int, double*, int, int, int,
                               int, int, cudaStream_t);
template int dots_pass<float>(const float*, const float* const*, int, float2*, int, int, int, int,
                              int, cudaStream_t);

}  // namespace ld
