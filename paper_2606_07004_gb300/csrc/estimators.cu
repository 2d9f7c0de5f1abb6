// OSLQ (Algorithm 3) and OSA-IOP (Algorithm 2 with Algorithm 1) on the
// device, and the C-ABI of liblogdet.
#include "dense.cuh"
#include "dia.cuh"
#include "grid.cuh"
#include "handle.cuh"
#include "krylov.cuh"
#include "profile.cuh"
#include "solve.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace ld {

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

int solve(logdet_ctx* h, const SolveCfg& c, cudaStream_t st, SolveOut& o) {
  memset(&o.res, 0, sizeof o.res);
  LD_TRY(validate_cfg(h, c));
  if (cudaSetDevice(h->device) != cudaSuccess) { set_error("cudaSetDevice failed"); return LOGDET_ECUDA; }
  Events ev;
  LD_CUDA(cudaEventCreate(&ev.a));
  LD_CUDA(cudaEventCreate(&ev.b));
  LD_CUDA(cudaEventRecord(ev.a, st));
  int rc = solve_blocking(h, c, st, o);
  if (rc) {
    cudaStreamSynchronize(st);
    return rc;
  }
  LD_CUDA(cudaEventRecord(ev.b, st));
  LD_CUDA(cudaEventSynchronize(ev.b));
  float ms = 0.f;
  LD_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
  o.res.device_ms = ms;
  LD_CUDA(cudaGetLastError());
  return LOGDET_OK;
}

static int run_estimator(int method, logdet_handle h, int32_t P, int32_t m, int32_t k, uint64_t seed,
                         const logdet_opts* opts, logdet_result* out) {
  if (!h || !out) { set_error("NULL handle or result"); return LOGDET_EINVAL; }
  SolveCfg c = make_solve_cfg(method, P, m, k, seed, opts);
  cudaStream_t st = (opts && opts->stream) ? (cudaStream_t)opts->stream : h->stream;
  SolveOut o;
  int rc = solve(h, c, st, o);
  if (rc) return rc;
  *out = o.res;
  if (opts && opts->per_probe)
    for (size_t i = 0; i < o.per_probe.size(); ++i) opts->per_probe[i] = o.per_probe[i];
  if (opts && opts->z_norm2)
    for (size_t i = 0; i < o.zn2.size(); ++i) opts->z_norm2[i] = o.zn2[i];
  return LOGDET_OK;
}

// Several shifts of one matrix in lockstep (solve_shifts); member t takes
// shift shifts[t] and seed seed0 + t, everything else from opts.
static int run_shifts(int method, logdet_handle h, int32_t nshift, const double* shifts, int32_t P,
                      int32_t m, int32_t k, uint64_t seed0, const logdet_opts* opts,
                      logdet_result* out) {
  if (!h || !out || !shifts) { set_error("NULL handle, shifts or results"); return LOGDET_EINVAL; }
  if (nshift < 1) { set_error("nshift=%d must be >= 1", nshift); return LOGDET_EINVAL; }
  std::vector<SolveCfg> cfgs;
  for (int t = 0; t < nshift; ++t) {
    SolveCfg c = make_solve_cfg(method, P, m, k, seed0 + (uint64_t)t, opts);
    c.shift = shifts[t];
    cfgs.push_back(c);
  }
  cudaStream_t st = (opts && opts->stream) ? (cudaStream_t)opts->stream : h->stream;
  if (cudaSetDevice(h->device) != cudaSuccess) { set_error("cudaSetDevice failed"); return LOGDET_ECUDA; }
  Events ev;
  LD_CUDA(cudaEventCreate(&ev.a));
  LD_CUDA(cudaEventCreate(&ev.b));
  LD_CUDA(cudaEventRecord(ev.a, st));
  std::vector<SolveOut> outs;
  LD_TRY(solve_shifts(h, cfgs, st, outs));
  LD_CUDA(cudaEventRecord(ev.b, st));
  LD_CUDA(cudaEventSynchronize(ev.b));
  float ms = 0.f;
  LD_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
  for (int t = 0; t < nshift; ++t) {
    out[t] = outs[t].res;
    out[t].device_ms = ms;
  }
  LD_CUDA(cudaGetLastError());
  return LOGDET_OK;
}

}  // namespace ld

// ===========================================================================
// C-ABI
// ===========================================================================
using namespace ld;

extern "C" {

void logdet_opts_default(logdet_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->precision = LOGDET_FP64;
  o->tol = kDefaultTol;
}

const char* logdet_strerror(int code) {
  switch (code) {
    case LOGDET_OK: return "ok";
    case LOGDET_PENDING: return "pending";
    case LOGDET_EINVAL: return "invalid argument";
    case LOGDET_ENOMEM: return "out of device memory or over budget";
    case LOGDET_ENOTSPD: return "matrix is not symmetric positive definite";
    case LOGDET_ETIMEOUT: return "timed out";
    case LOGDET_ECUDA: return "CUDA error";
    case LOGDET_ENOENT: return "unknown request";
    case LOGDET_ECANCEL: return "cancelled";
    default: return "unknown error code";
  }
}

const char* logdet_last_error(void) { return ld::last_error(); }

int logdet_create(int32_t n, const int32_t* rowptr, const int32_t* colind, const void* vals,
                  int32_t vals_dtype, logdet_handle* out) {
  return create_handle(n, rowptr, colind, vals, vals_dtype, false, out);
}

int logdet_create_device(int32_t n, const int32_t* rowptr_dev, const int32_t* colind_dev,
                         const void* vals_dev, int32_t vals_dtype, logdet_handle* out) {
  return create_handle(n, rowptr_dev, colind_dev, vals_dev, vals_dtype, true, out);
}

int logdet_create_grid(int32_t nx, int32_t ny, int32_t radius, const double* w,
                       logdet_handle* out) {
  return create_grid_handle(nx, ny, radius, w, out);
}

void logdet_destroy(logdet_handle h) { destroy_handle(h); }

int logdet_info(logdet_handle h, int32_t* n, int64_t* nnz, double* lo, double* hi) {
  if (!h) { set_error("NULL handle"); return LOGDET_EINVAL; }
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (lo) *lo = h->g_lo;
  if (hi) *hi = h->g_hi;
  return LOGDET_OK;
}

int logdet_grid_structure(logdet_handle h, int32_t* dim, int32_t* line_stride, int32_t* reach) {
  if (!h || !dim || !line_stride || !reach) {
    set_error("NULL handle or output pointer");
    return LOGDET_EINVAL;
  }
  const bool on = h->dia.ndiag > 0 && h->dia_slot;
  *dim = on ? h->dia.dim : 0;
  *line_stride = on ? h->dia.L : 0;
  *reach = on ? h->dia.A : 0;
  return LOGDET_OK;
}

int logdet_grid_structure_csr(int32_t n, const int32_t* rowptr, const int32_t* colind,
                              int32_t* dim, int32_t* line_stride, int32_t* reach) {
  if (n < 1 || !rowptr || !colind || !dim || !line_stride || !reach) {
    set_error("n < 1 or NULL pointer");
    return LOGDET_EINVAL;
  }
  ld::DiaInfo d;
  const bool on = ld::dia_detect(n, rowptr, colind, &d);
  *dim = on ? d.dim : 0;
  *line_stride = on ? d.L : 0;
  *reach = on ? d.A : 0;
  return LOGDET_OK;
}

int logdet_oslq(logdet_handle h, int32_t P, int32_t m, int32_t k, uint64_t seed,
                const logdet_opts* opts, logdet_result* out) {
  return run_estimator(0, h, P, m, k, seed, opts, out);
}

int logdet_osaiop(logdet_handle h, int32_t P, int32_t m, int32_t k, uint64_t seed,
                  const logdet_opts* opts, logdet_result* out) {
  return run_estimator(1, h, P, m, k, seed, opts, out);
}

int logdet_oslq_shifts(logdet_handle h, int32_t nshift, const double* shifts, int32_t P, int32_t m,
                       int32_t k, uint64_t seed0, const logdet_opts* opts, logdet_result* out) {
  return run_shifts(0, h, nshift, shifts, P, m, k, seed0, opts, out);
}

int logdet_osaiop_shifts(logdet_handle h, int32_t nshift, const double* shifts, int32_t P, int32_t m,
                         int32_t k, uint64_t seed0, const logdet_opts* opts, logdet_result* out) {
  return run_shifts(1, h, nshift, shifts, P, m, k, seed0, opts, out);
}

int logdet_probe_fill(uint64_t seed, int32_t stream, int32_t n, int32_t ncols, int32_t col0,
                      double* out_dev, int32_t ld, void* cuda_stream) {
  if (n < 1 || ncols < 0 || col0 < 0 || ld < ncols || !out_dev || stream < 0) {
    set_error("probe_fill: bad arguments");
    return LOGDET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  LD_TRY(probe_fill<double>(probe_key(seed, stream), n, ncols, col0, out_dev, ld, st));
  LD_CUDA(cudaStreamSynchronize(st));
  return LOGDET_OK;
}

int logdet_probe_fill_gaussian(uint64_t seed, int32_t stream, int32_t n, int32_t ncols,
                               int32_t col0, double* out_dev, int32_t ld, void* cuda_stream) {
  if (n < 1 || ncols < 0 || col0 < 0 || ld < ncols || !out_dev || stream < 0) {
    set_error("probe_fill_gaussian: bad arguments");
    return LOGDET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  LD_TRY(probe_fill<double>(probe_key(seed, stream), n, ncols, col0, out_dev, ld, st, 1));
  LD_CUDA(cudaStreamSynchronize(st));
  return LOGDET_OK;
}

int logdet_spmm(logdet_handle h, const double* x, double* y, int32_t b, int32_t ld, void* cuda_stream) {
  if (!h || !x || !y || b < 1 || ld < b || (ld & 1) || ((uintptr_t)x & 15) || ((uintptr_t)y & 15)) {
    set_error("spmm: need b >= 1, even ld >= b and 16-byte aligned blocks");
    return LOGDET_EINVAL;
  }
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : h->stream;
  if (h->kind == 1) {
    LD_TRY(grid_apply<double>(h, h->gtab, x, y, ld, nullptr, st));
    LD_CUDA(cudaStreamSynchronize(st));
    return LOGDET_OK;
  }
  DevBuf<double> v(st);
  const double* vals = (const double*)h->vals;
  if (h->vals_dtype != LOGDET_VALS_F64) {
    LD_TRY(v.alloc(h->nnz));
    LD_TRY(scaled_values<double>(h, 1.0, v.p, st));
    vals = v.p;
  }
  LD_TRY(spmm_block<double>(h->rowptr, h->colind, vals, h->n, x, y, ld, st, nullptr, h));
  LD_CUDA(cudaStreamSynchronize(st));
  return LOGDET_OK;
}

int logdet_quadform(logdet_handle h, const double* x, double shift, double* out,
                    void* cuda_stream) {
  if (!h || !x || !out || !std::isfinite(shift)) {
    set_error("quadform: NULL argument or non-finite shift");
    return LOGDET_EINVAL;
  }
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : h->stream;
  const int n = h->n, ld = 2;
  DevBuf<double> X(st), Y(st), part(st), red(st), cs(st);
  LD_TRY(X.alloc((size_t)n * ld));
  LD_TRY(Y.alloc((size_t)n * ld));
  LD_TRY(X.zero());
  LD_CUDA(cudaMemcpy2DAsync(X.p, ld * sizeof(double), x, sizeof(double), sizeof(double), n,
                            cudaMemcpyDeviceToDevice, st));
  LD_TRY(cs.alloc(ld));
  LD_TRY(fill_double(cs.p, ld, shift, st));
  if (h->kind == 1) {
    LD_TRY(grid_apply<double>(h, h->gtab, X.p, Y.p, ld, cs.p, st));
  } else {
    DevBuf<double> v(st);
    const double* vals = (const double*)h->vals;
    if (h->vals_dtype != LOGDET_VALS_F64) {
      LD_TRY(v.alloc(h->nnz));
      LD_TRY(scaled_values<double>(h, 1.0, v.p, st));
      vals = v.p;
    }
    LD_TRY(spmm_block<double>(h->rowptr, h->colind, vals, n, X.p, Y.p, ld, st, cs.p, h));
  }
  const TileGeom g = tile_geom(ld, Vec16<double>::N, 0, 0, n);
  const int ntiles = div_up(n, g.tile_rows);
  LD_TRY(part.alloc((size_t)ld * ntiles));
  LD_TRY(red.alloc(ld));
  const double* dv[1] = {X.p};
  LD_TRY(dots_pass<double>(Y.p, dv, 1, part.p, n, ld, g.tile_rows, ntiles, g.threads, st));
  LD_TRY(reduce_partials_fp64(part.p, ld, ntiles, red.p, st));
  LD_CUDA(cudaMemcpyAsync(out, red.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  LD_CUDA(cudaStreamSynchronize(st));
  return LOGDET_OK;
}

int logdet_orth(int32_t n, int32_t s, const double* y, int32_t ldy, double* a, int32_t lda,
                int32_t* s_eff, void* cuda_stream) {
  if (n < 1 || s < 1 || s > kMaxSketch || ldy < s || lda < s || !y || !a) {
    set_error("orth: bad arguments (1 <= s <= %d)", kMaxSketch);
    return LOGDET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<double> ws(st);
  LD_TRY(ws.alloc(orth_workspace_doubles(n, s)));
  int se = 0;
  LD_TRY(orth_fp64(n, s, y, ldy, a, lda, ws.p, nullptr, &se, st));
  if (s_eff) *s_eff = se;
  LD_CUDA(cudaStreamSynchronize(st));
  return LOGDET_OK;
}

int logdet_orth_f32(int32_t n, int32_t s, const float* y, int32_t ldy, float* a, int32_t lda,
                    int32_t* s_eff, void* cuda_stream) {
  if (n < 1 || s < 1 || s > kMaxSketch || ldy < s || lda < s || !y || !a) {
    set_error("orth_f32: bad arguments (1 <= s <= %d)", kMaxSketch);
    return LOGDET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<double> ws(st);
  LD_TRY(ws.alloc(orth_workspace_doubles(n, s)));
  int se = 0;
  LD_TRY(orth_f32(n, s, y, ldy, a, lda, ws.p, nullptr, &se, st));
  if (s_eff) *s_eff = se;
  LD_CUDA(cudaStreamSynchronize(st));
  return LOGDET_OK;
}

int logdet_gauss_quadrature_log(const double* alpha, const double* beta, const int32_t* msteps,
                                int32_t m, int32_t nprobe, double clamp_lo, double* out,
                                uint32_t* status, void* cuda_stream) {
  if (!alpha || !beta || !out || m < 1 || nprobe < 1) {
    set_error("gauss_quadrature_log: bad arguments");
    return LOGDET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<uint32_t> sd(st);
  LD_TRY(sd.alloc(nprobe));
  LD_TRY(sd.zero());
  LD_TRY(gauss_quadrature_log(alpha, beta, m, msteps, m, nprobe, clamp_lo, out, sd.p, st));
  std::vector<uint32_t> hs(nprobe);
  LD_CUDA(cudaMemcpyAsync(hs.data(), sd.p, sizeof(uint32_t) * nprobe, cudaMemcpyDeviceToHost, st));
  LD_CUDA(cudaStreamSynchronize(st));
  if (status) {
    uint32_t acc = 0;
    for (auto v : hs) acc |= v;
    *status = acc;
  }
  return LOGDET_OK;
}

static int hesslog_entry(const double* H, int32_t ldh, const int32_t* msteps, int32_t m,
                         int32_t nprobe, int32_t band, double* c, uint32_t* status,
                         void* cuda_stream) {
  if (!H || !c || m < 1 || nprobe < 1 || ldh < m) {
    set_error("hessenberg_log_e1: bad arguments");
    return LOGDET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<double> ws(st);
  DevBuf<uint32_t> sd(st);
  LD_TRY(ws.alloc(hesslog_workspace_doubles(m, nprobe, band)));
  LD_TRY(sd.alloc(nprobe));
  LD_TRY(sd.zero());
  LD_TRY(hessenberg_log_e1(H, ldh, msteps, m, nprobe, c, m, ws.p, sd.p, st, band));
  std::vector<uint32_t> hs(nprobe);
  LD_CUDA(cudaMemcpyAsync(hs.data(), sd.p, sizeof(uint32_t) * nprobe, cudaMemcpyDeviceToHost, st));
  LD_CUDA(cudaStreamSynchronize(st));
  if (status) {
    uint32_t acc = 0;
    for (auto v : hs) acc |= v;
    *status = acc;
  }
  return LOGDET_OK;
}

int logdet_hessenberg_log_e1(const double* H, int32_t ldh, const int32_t* msteps, int32_t m,
                             int32_t nprobe, double* c, uint32_t* status, void* cuda_stream) {
  return hesslog_entry(H, ldh, msteps, m, nprobe, -1, c, status, cuda_stream);
}

int logdet_hessenberg_log_e1_banded(const double* H, int32_t ldh, const int32_t* msteps,
                                    int32_t m, int32_t nprobe, int32_t band, double* c,
                                    uint32_t* status, void* cuda_stream) {
  if (band < 0) {
    set_error("hessenberg_log_e1_banded: band < 0");
    return LOGDET_EINVAL;
  }
  return hesslog_entry(H, ldh, msteps, m, nprobe, band, c, status, cuda_stream);
}

}  // extern "C"
