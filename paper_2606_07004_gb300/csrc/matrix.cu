// Matrix handles: CSR upload and validation, Gershgorin interval (Sec. 2.1),
// scaled value copies, error plumbing and the step-level SpMM entry point.
#include "handle.cuh"
#include "dia.cuh"
#include "krylov.cuh"
#include "profile.cuh"

#include <atomic>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <vector>

namespace ld {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}
const char* last_error() { return g_last_error.c_str(); }

int ensure_pool(int device) {
  static bool done[64] = {false};
  if (device >= 0 && device < 64 && !done[device]) {
    cudaMemPool_t pool;
    LD_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    LD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    done[device] = true;
  }
  return LOGDET_OK;
}

// Canary bytes found changed when checked builds release a buffer.
static std::atomic<unsigned long long> g_canary_bytes{0};
void canary_fault(size_t bytes_changed) { g_canary_bytes += bytes_changed; }
unsigned long long canary_fault_count() { return g_canary_bytes.load(); }

// ---------------------------------------------------------------------------
// Pinned host block cache (see handle.cuh).  At most kPinnedCacheMax bytes
// stay cached; beyond that a released block is freed.
// ---------------------------------------------------------------------------

namespace {
struct PinnedFree {
  void* p;
  size_t cap;
  cudaEvent_t ev;  // recorded on the releasing stream; nullptr = idle
};
std::mutex g_pin_mu;
std::vector<PinnedFree> g_pin_free;
size_t g_pin_cached = 0;
constexpr size_t kPinnedCacheMax = size_t(256) << 20;
}  // namespace

void* pinned_acquire(size_t bytes, size_t* cap) {
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (size_t i = 0; i < g_pin_free.size(); ++i) {
      PinnedFree& f = g_pin_free[i];
      if (f.cap != c) continue;
      if (f.ev && cudaEventQuery(f.ev) != cudaSuccess) continue;
      void* p = f.p;
      if (f.ev) cudaEventDestroy(f.ev);
      g_pin_cached -= c;
      g_pin_free.erase(g_pin_free.begin() + i);
      *cap = c;
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, c) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *cap = c;
  return p;
}

void pinned_release(void* p, size_t cap, cudaStream_t st) {
  if (!p) return;
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ev = nullptr;
  } else if (cudaEventRecord(ev, st) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(ev);
    ev = nullptr;
  }
  if (!ev) cudaStreamSynchronize(st);
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_cached + cap <= kPinnedCacheMax) {
      g_pin_free.push_back(PinnedFree{p, cap, ev});
      g_pin_cached += cap;
      return;
    }
  }
  if (ev) {
    cudaEventSynchronize(ev);
    cudaEventDestroy(ev);
  }
  cudaFreeHost(p);
}

// ---------------------------------------------------------------------------
// Gershgorin interval: per row a_ii -/+ sum_{j != i} |a_ij| (CSR order),
// min/max over rows.  Also checks the CSR structure on the device (the
// borrowed-pointer path): flag bits 1 = bad column/order, 2 = no diagonal,
// 4 = non-finite value, 8 = bad rowptr.
// ---------------------------------------------------------------------------
template <typename V>
__global__ void k_gershgorin(const int* __restrict__ rowptr, const int* __restrict__ colind,
                             const V* __restrict__ vals, int n, long long nnz,
                             double* __restrict__ lo_out, double* __restrict__ hi_out,
                             int* __restrict__ flags) {
  __shared__ double slo[256], shi[256];
  double lo = INFINITY, hi = -INFINITY;
  int fl = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p0 = rowptr[i], p1 = rowptr[i + 1];
    if (p0 < 0 || p1 < p0 || (long long)p1 > nnz) { fl |= 8; continue; }
    double d = 0.0, R = 0.0;
    bool has_d = false;
    int prev = -1;
    for (int p = p0; p < p1; ++p) {
      const int c = colind[p];
      const double a = (double)vals[p];
      if (c < 0 || c >= n || c <= prev) fl |= 1;
      prev = c;
      if (!isfinite(a)) fl |= 4;
      if (c == i) { d = a; has_d = true; }
      else R += fabs(a);
    }
    if (!has_d) fl |= 2;
    lo = fmin(lo, d - R);
    hi = fmax(hi, d + R);
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + w]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    lo_out[blockIdx.x] = slo[0];
    hi_out[blockIdx.x] = shi[0];
  }
  if (fl) atomicOr(flags, fl);
}

static int compute_gershgorin(logdet_ctx* h, bool check_structure) {
  const int blocks = std::max(1, std::min(div_up(h->n, 256), 4 * sm_count()));
  DevBuf<double> lo(h->stream), hi(h->stream);
  DevBuf<int> fl(h->stream);
  LD_TRY(lo.alloc(blocks));
  LD_TRY(hi.alloc(blocks));
  LD_TRY(fl.alloc(1));
  LD_CUDA(cudaMemsetAsync(fl.p, 0, sizeof(int), h->stream));
  ProfScope prof(KC_OTHER, h->stream);
  if (h->vals_dtype == LOGDET_VALS_F64)
    k_gershgorin<double><<<blocks, 256, 0, h->stream>>>(h->rowptr, h->colind, (const double*)h->vals,
                                                       h->n, h->nnz, lo.p, hi.p, fl.p);
  else
    k_gershgorin<float><<<blocks, 256, 0, h->stream>>>(h->rowptr, h->colind, (const float*)h->vals,
                                                      h->n, h->nnz, lo.p, hi.p, fl.p);
  LD_CHECK_LAUNCH();
  std::vector<double> hl(blocks), hh(blocks);
  int hf = 0;
  LD_CUDA(cudaMemcpyAsync(hl.data(), lo.p, sizeof(double) * blocks, cudaMemcpyDeviceToHost, h->stream));
  LD_CUDA(cudaMemcpyAsync(hh.data(), hi.p, sizeof(double) * blocks, cudaMemcpyDeviceToHost, h->stream));
  LD_CUDA(cudaMemcpyAsync(&hf, fl.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LD_CUDA(cudaStreamSynchronize(h->stream));
  if (check_structure && hf) {
    set_error("CSR validation failed on device (flags 0x%x: 1 column order/range, 2 missing "
              "diagonal, 4 non-finite value, 8 rowptr)", hf);
    return LOGDET_EINVAL;
  }
  double glo = INFINITY, ghi = -INFINITY;
  for (int b = 0; b < blocks; ++b) { glo = std::min(glo, hl[b]); ghi = std::max(ghi, hh[b]); }
  h->g_lo = glo;
  h->g_hi = ghi;
  if (!(ghi > 0.0)) {
    set_error("Gershgorin upper bound %g <= 0: matrix is not SPD", ghi);
    return LOGDET_ENOTSPD;
  }
  return LOGDET_OK;
}

template <typename V>
static int validate_host(int n, const int32_t* rowptr, const int32_t* colind, const V* vals) {
  if (rowptr[0] != 0) { set_error("rowptr[0] = %d, expected 0", rowptr[0]); return LOGDET_EINVAL; }
  for (int i = 0; i < n; ++i) {
    const int p0 = rowptr[i], p1 = rowptr[i + 1];
    if (p1 < p0) { set_error("rowptr decreases at row %d", i); return LOGDET_EINVAL; }
    bool has_d = false;
    int prev = -1;
    for (int p = p0; p < p1; ++p) {
      const int c = colind[p];
      if (c < 0 || c >= n) { set_error("row %d: column %d out of range", i, c); return LOGDET_EINVAL; }
      if (c <= prev) { set_error("row %d: columns not strictly increasing", i); return LOGDET_EINVAL; }
      prev = c;
      if (!std::isfinite((double)vals[p])) { set_error("row %d: non-finite value", i); return LOGDET_EINVAL; }
      if (c == i) has_d = true;
    }
    if (!has_d) { set_error("row %d has no stored diagonal entry", i); return LOGDET_EINVAL; }
  }
  return LOGDET_OK;
}

int create_handle(int32_t n, const int32_t* rowptr, const int32_t* colind, const void* vals,
                  int32_t vals_dtype, bool device_ptrs, logdet_handle* out) {
  if (!out) { set_error("out is NULL"); return LOGDET_EINVAL; }
  *out = nullptr;
  if (n < 1 || !rowptr || !colind || !vals) { set_error("n < 1 or NULL array"); return LOGDET_EINVAL; }
  if (vals_dtype != LOGDET_VALS_F64 && vals_dtype != LOGDET_VALS_F32) {
    set_error("vals_dtype %d unknown", vals_dtype);
    return LOGDET_EINVAL;
  }
  const size_t vsize = vals_dtype == LOGDET_VALS_F64 ? 8 : 4;
  logdet_ctx* h = new logdet_ctx();
  int rc = LOGDET_OK;
  auto fail = [&](int code) { destroy_handle(h); return code; };
  if (cudaGetDevice(&h->device) != cudaSuccess) { set_error("no CUDA device"); delete h; return LOGDET_ECUDA; }
  rc = ensure_pool(h->device);
  if (rc) { delete h; return rc; }
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("cudaStreamCreate failed");
    delete h;
    return LOGDET_ECUDA;
  }
  h->n = n;
  h->vals_dtype = vals_dtype;
  if (!device_ptrs) {
    const long long nnz = rowptr[n];
    if (nnz < 0) { set_error("rowptr[n] < 0"); return fail(LOGDET_EINVAL); }
    rc = vals_dtype == LOGDET_VALS_F64
             ? validate_host<double>(n, rowptr, colind, (const double*)vals)
             : validate_host<float>(n, rowptr, colind, (const float*)vals);
    if (rc) return fail(rc);
    h->nnz = nnz;
    h->owns = true;
    if (cudaMalloc(&h->rowptr, sizeof(int) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&h->colind, sizeof(int) * std::max<long long>(nnz, 1)) != cudaSuccess ||
        cudaMalloc(&h->vals, vsize * std::max<long long>(nnz, 1)) != cudaSuccess) {
      set_error("device allocation of the CSR arrays failed");
      return fail(LOGDET_ENOMEM);
    }
    if (cudaMemcpy(h->rowptr, rowptr, sizeof(int) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->colind, colind, sizeof(int) * nnz, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->vals, vals, vsize * nnz, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("copy of the CSR arrays failed");
      return fail(LOGDET_ECUDA);
    }
    rc = compute_gershgorin(h, false);
    if (!rc) rc = dia_build(h, rowptr, colind);
  } else {
    int last = 0;
    if (cudaMemcpy(&last, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("rowptr is not a readable device pointer");
      return fail(LOGDET_EINVAL);
    }
    if (last < 0) { set_error("rowptr[n] < 0"); return fail(LOGDET_EINVAL); }
    h->nnz = last;
    h->owns = false;
    h->rowptr = const_cast<int*>(rowptr);
    h->colind = const_cast<int*>(colind);
    h->vals = const_cast<void*>(vals);
    rc = compute_gershgorin(h, true);
  }
  if (rc) return fail(rc);
  // Row lengths: keep a host copy of rowptr only when some row is long.
  {
    std::vector<int> rp;
    const int* hp = rowptr;
    if (device_ptrs) {
      rp.resize((size_t)n + 1);
      if (cudaMemcpy(rp.data(), rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("copy of rowptr to the host failed");
        return fail(LOGDET_ECUDA);
      }
      hp = rp.data();
    }
    int mx = 0;
    for (int i = 0; i < n; ++i) mx = std::max(mx, hp[i + 1] - hp[i]);
    h->max_row_nnz = mx;
    if (mx > kSplitRowNnz) h->h_rowptr.assign(hp, hp + n + 1);
  }
  *out = h;
  return LOGDET_OK;
}

// Work items for tiles of tile_rows rows (see SpmmJob::items).  In row order,
// a row longer than kSplitRowNnz is an item of its own; the rows between long
// rows are cut into ranges of at most tile_rows rows and at most
// tile_rows * (mean row length) nonzeros, so that no item holds much more
// work than a uniform tile.  Items are launched in decreasing order of work
// (nonzeros + rows), so that persistent CTAs taking every grid-th item end
// with similar loads.
int spmm_items(logdet_ctx* h, int tile_rows, const int4** items, int* count) {
  *items = nullptr;
  *count = 0;
  if (h->max_row_nnz <= kSplitRowNnz || h->h_rowptr.empty()) return LOGDET_OK;
  std::lock_guard<std::mutex> lk(h->items_mu);
  auto it = h->items.find(tile_rows);
  if (it != h->items.end()) {
    *items = it->second.first;
    *count = it->second.second;
    return LOGDET_OK;
  }
  const int* rp = h->h_rowptr.data();
  const int n = h->n;
  const double mean = std::max(1.0, (double)h->nnz / n);
  const long long budget = std::max<long long>(tile_rows, (long long)(tile_rows * mean));
  std::vector<int4> list;
  std::vector<long long> cost;
  for (int r = 0; r < n;) {
    const int d = rp[r + 1] - rp[r];
    if (d > kSplitRowNnz) {
      list.push_back(make_int4(r, -1, (int)list.size(), 0));
      cost.push_back((long long)d + 1);
      ++r;
      continue;
    }
    const int r0 = r;
    long long sum = 0;
    while (r < n && r - r0 < tile_rows) {
      const int dr = rp[r + 1] - rp[r];
      if (dr > kSplitRowNnz) break;
      if (r > r0 && sum + dr > budget) break;
      sum += dr;
      ++r;
    }
    list.push_back(make_int4(r0, r, (int)list.size(), 0));
    cost.push_back(sum + (r - r0));
  }
  std::vector<int> order(list.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int4> launch(list.size());
  for (size_t i = 0; i < order.size(); ++i) launch[i] = list[order[i]];
  int4* d = nullptr;
  if (cudaMalloc(&d, sizeof(int4) * launch.size()) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu SpMM work items failed", launch.size());
    return LOGDET_ENOMEM;
  }
  if (cudaMemcpy(d, launch.data(), sizeof(int4) * launch.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    set_error("copy of the SpMM work items failed");
    return LOGDET_ECUDA;
  }
  h->items[tile_rows] = std::make_pair(d, (int)launch.size());
  *items = d;
  *count = (int)launch.size();
  return LOGDET_OK;
}

void destroy_handle(logdet_ctx* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->items) cudaFree(kv.second.first);
  if (h->gtab) cudaFree(h->gtab);
  if (h->grx) cudaFree(h->grx);
  if (h->dia_slot) cudaFree(h->dia_slot);
  if (h->owns) {
    if (h->rowptr) cudaFree(h->rowptr);
    if (h->colind) cudaFree(h->colind);
    if (h->vals) cudaFree(h->vals);
  }
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// Scaled copy of the values: out[i] = (T)(vals[i] / c), the division in FP64.
template <typename Vin, typename T>
__global__ void k_scale_vals(const Vin* __restrict__ in, long long nnz, double c, T* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (T)((double)in[i] / c);
}

template <typename T>
int scaled_values(logdet_ctx* h, double c, T* out, cudaStream_t st) {
  const int blocks = 4 * sm_count();
  ProfScope prof(KC_OTHER, st);
  if (h->vals_dtype == LOGDET_VALS_F64)
    k_scale_vals<double, T><<<blocks, 256, 0, st>>>((const double*)h->vals, h->nnz, c, out);
  else
    k_scale_vals<float, T><<<blocks, 256, 0, st>>>((const float*)h->vals, h->nnz, c, out);
  LD_CHECK_LAUNCH();
  return LOGDET_OK;
}
template int scaled_values<double>(logdet_ctx*, double, double*, cudaStream_t);
template int scaled_values<float>(logdet_ctx*, double, float*, cudaStream_t);

// One SpMM y = (vals * 1) x over a block (no dots), used by the step entry point
// and by the OSLQ sketch.
template <typename T>
int spmm_block(const int* rowptr, const int* colind, const typename ValOf<T>::type* vals, int n,
               const T* x, T* y, int ld, cudaStream_t st, const double* colshift, logdet_ctx* h) {
  TileGeom g = tile_geom(ld, Vec16<T>::N, 0, 0, n);
  SpmmBatch<T> B;
  memset(&B, 0, sizeof B);
  B.njobs = 1;
  SpmmJob<T>& J = B.jobs[0];
  J.rowptr = rowptr;
  J.colind = colind;
  J.vals = vals;
  J.x = x;
  J.y = y;
  J.n = n;
  J.ld = ld;
  J.ndots = 0;
  J.colshift = colshift;
  J.col_off = 0;
  J.width = ld;
  J.b = ld;
  J.nnz = h ? h->nnz : 0;  // (every caller passes the handle; the checked build bounds rows by it)
  J.tile_rows = g.tile_rows;
  J.ntiles = div_up(n, g.tile_rows);
  if (h) {
    int cnt = 0;
    LD_TRY(spmm_items(h, g.tile_rows, &J.items, &cnt));
    if (J.items) J.ntiles = cnt;
  }
  B.tile_start[0] = 0;
  B.tile_start[1] = J.ntiles;
  B.total_tiles = J.ntiles;
  return launch_spmm<T>(B, g.threads, st);
}
template int spmm_block<double>(const int*, const int*, const double*, int, const double*, double*, int,
                                cudaStream_t, const double*, logdet_ctx*);
template int spmm_block<float>(const int*, const int*, const float*, int, const float*, float*, int,
                                cudaStream_t, const double*, logdet_ctx*);
template int spmm_block<bf16>(const int*, const int*, const float*, int, const bf16*, bf16*, int,
                                cudaStream_t, const double*, logdet_ctx*);
template int spmm_block<f32x2>(const int*, const int*, const float*, int, const f32x2*, f32x2*, int,
                                 cudaStream_t, const double*, logdet_ctx*);

}  // namespace ld
