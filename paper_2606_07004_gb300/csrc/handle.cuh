// The matrix handle and small host-side helpers shared by the translation units.
#pragma once

#include "common.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

struct logdet_ctx {
  int device = 0;
  int n = 0;
  long long nnz = 0;
  int* rowptr = nullptr;
  int* colind = nullptr;
  void* vals = nullptr;
  int vals_dtype = LOGDET_VALS_F64;
  bool owns = false;
  double g_lo = 0.0, g_hi = 0.0;  // Gershgorin interval (unclamped)
  cudaStream_t stream = nullptr;
  // Irregular sparsity (some row longer than kSplitRowNnz): a host copy of
  // rowptr and, per tile depth, the SpMM work-item list built from it.
  int max_row_nnz = 0;
  std::vector<int> h_rowptr;
  std::mutex items_mu;
  std::map<int, std::pair<int4*, int>> items;  // tile_rows -> (device items, count)
  // Matrix-free gridded operator (kind == 1; see grid.cuh): no CSR arrays.
  int kind = 0;                  // 0 CSR, 1 grid operator
  int gx = 0, gy = 0, gr = 0;    // grid size and stencil radius
  double* gtab = nullptr;        // device expanded table of W (FP64)
  int* grx = nullptr;            // device [gr + 1]: last nonzero |dx| per |dy|
  // Diagonal structure (dia.ndiag > 0): CSR entry -> diagonal index.
  ld::DiaInfo dia{};
  int* dia_slot = nullptr;       // device [nnz]
};

namespace ld {

// Checked builds (LOGDET_CHECKED): every workspace buffer is allocated with
// kCanaryBytes of guard on each side, filled with kCanaryByte; release reads
// both guards back and counts any byte that changed (canary_fault_count).
constexpr size_t kCanaryBytes = 256;  // keeps the buffer 256-byte aligned
constexpr unsigned char kCanaryByte = 0xA5;
void canary_fault(size_t bytes_changed);
unsigned long long canary_fault_count();

// Stream-ordered device buffer freed when it goes out of scope.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t count = 0;
  cudaStream_t st;
  explicit DevBuf(cudaStream_t s) : st(s) {}
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
#ifdef LOGDET_CHECKED
  static constexpr size_t kGuard = kCanaryBytes;
#else
  static constexpr size_t kGuard = 0;
#endif
  cudaError_t raw_alloc() {
    void* base = nullptr;
    cudaError_t e = cudaMallocAsync(&base, count * sizeof(T) + 2 * kGuard, st);
    if (e != cudaSuccess) return e;
    p = reinterpret_cast<T*>(static_cast<unsigned char*>(base) + kGuard);
    if (kGuard) {
      cudaMemsetAsync(base, kCanaryByte, kGuard, st);
      cudaMemsetAsync(reinterpret_cast<unsigned char*>(p) + count * sizeof(T), kCanaryByte, kGuard,
                      st);
    }
    return cudaSuccess;
  }
  int alloc(size_t n) {
    release();
    count = std::max<size_t>(n, 1);
    cudaError_t e = raw_alloc();
    if (e == cudaErrorMemoryAllocation) {
      // The pool keeps freed memory (release threshold: never); memory it
      // holds unused in blocks of other sizes goes back once, then retry.
      cudaGetLastError();
      int dev = 0;
      cudaMemPool_t pool;
      if (cudaStreamSynchronize(st) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess &&
          cudaMemPoolTrimTo(pool, 0) == cudaSuccess)
        e = raw_alloc();
    }
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return LOGDET_ENOMEM;
    }
    return LOGDET_OK;
  }
  int zero() { return cudaMemsetAsync(p, 0, count * sizeof(T), st) == cudaSuccess ? LOGDET_OK : LOGDET_ECUDA; }
  void release() {
    if (!p) return;
    unsigned char* base = reinterpret_cast<unsigned char*>(p) - kGuard;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (kGuard && cudaStreamIsCapturing(st, &cap) == cudaSuccess &&
        cap == cudaStreamCaptureStatusNone) {  // (no reads back inside a graph capture)
      unsigned char g[2 * kCanaryBytes];
      if (cudaMemcpyAsync(g, base, kGuard, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
          cudaMemcpyAsync(g + kGuard, reinterpret_cast<unsigned char*>(p) + count * sizeof(T), kGuard,
                          cudaMemcpyDeviceToHost, st) == cudaSuccess &&
          cudaStreamSynchronize(st) == cudaSuccess) {
        size_t bad = 0;
        for (size_t i = 0; i < 2 * kGuard; ++i) bad += g[i] != kCanaryByte;
        if (bad) canary_fault(bad);
      }
    }
    cudaFreeAsync(base, st);
    p = nullptr;
  }
  ~DevBuf() { release(); }
};

int ensure_pool(int device);

// Pinned host blocks for per-solve results, kept in a process-wide cache
// instead of allocated and freed per solve (cudaFreeHost synchronises the
// whole device, which would stall solves queued behind the current one).
// A released block is handed out again only once the work queued on its
// stream at release time has finished.  Blocks come in power-of-two sizes
// (>= 4 KiB); acquire returns nullptr when pinned allocation fails.
void* pinned_acquire(size_t bytes, size_t* cap);
void pinned_release(void* p, size_t cap, cudaStream_t st);
int create_handle(int32_t n, const int32_t* rowptr, const int32_t* colind, const void* vals,
                  int32_t vals_dtype, bool device_ptrs, logdet_handle* out);
void destroy_handle(logdet_ctx* h);

template <typename T>
int scaled_values(logdet_ctx* h, double c, T* out, cudaStream_t st);

// SpMM work items of a matrix with irregular rows for tiles of tile_rows
// rows (see SpmmJob::items); *items = nullptr, *count = 0 for a matrix whose
// rows are all short (uniform row tiles).  Built once per tile depth.
int spmm_items(logdet_ctx* h, int tile_rows, const int4** items, int* count);

template <typename T>
int spmm_block(const int* rowptr, const int* colind, const typename ValOf<T>::type* vals, int n,
               const T* x, T* y, int ld, cudaStream_t st, const double* colshift = nullptr,
               logdet_ctx* h = nullptr);

}  // namespace ld
