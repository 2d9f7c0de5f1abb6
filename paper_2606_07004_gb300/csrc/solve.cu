// Resumable OSLQ / OSA-IOP solves (see solve.cuh).
#include "profile.cuh"
#include "solve.cuh"
#include "grid.cuh"
#include "dia.cuh"
#include "tune.cuh"

#include <cmath>
#include <functional>
#include <cstdlib>
#include <cstring>

namespace ld {

// ---------------------------------------------------------------------------
// configuration checks and spectral bounds
// ---------------------------------------------------------------------------
void spectral_bounds(const logdet_ctx* h, const SolveCfg& c, double& lo, double& hi) {
  if (c.lam_lo > 0.0 && c.lam_hi > 0.0) {
    lo = c.lam_lo;
    hi = c.lam_hi;
    return;
  }
  // Gershgorin of Q + shift I is [lo + shift, hi + shift].
  hi = h->g_hi + c.shift;
  const double glo = h->g_lo + c.shift;
  lo = glo > 0.0 ? glo : kClampRel * hi;
}

int validate_cfg(const logdet_ctx* h, const SolveCfg& c) {
  if (c.P < (c.plain ? 1 : 3)) {
    set_error("num_probes must be >= %d", c.plain ? 1 : 3);
    return LOGDET_EINVAL;
  }
  if (c.m < 1 || c.m > h->n || c.m > kMaxSteps) {
    set_error("krylov_steps=%d must be in [1, min(n, %d)]", c.m, kMaxSteps);
    return LOGDET_EINVAL;
  }
  const int s = c.plain ? 0 : c.P / 3, r = c.plain ? c.P : c.P - 2 * s;
  if (s > kMaxSketch || r > kMaxSketch) {
    set_error("num_probes=%d: s and r must be <= %d", c.P, kMaxSketch);
    return LOGDET_EINVAL;
  }
  if (c.method != 0 && c.method != 1) { set_error("method %d unknown", c.method); return LOGDET_EINVAL; }
  if (!(c.shift >= 0.0) || !std::isfinite(c.shift)) {
    set_error("shift must be finite and >= 0");
    return LOGDET_EINVAL;
  }
  if (c.method == 0 && !(c.k == 0 || c.k == 2)) {
    set_error("OSLQ uses three-term Lanczos: iop_window must be 0 or 2");
    return LOGDET_EINVAL;
  }
  if (c.method == 1 && (c.k < 1 || c.k > kMaxWin - 1)) {
    set_error("iop_window=%d must be in [1, %d]", c.k, kMaxWin - 1);
    return LOGDET_EINVAL;
  }
  if (c.precision != LOGDET_FP64 && c.precision != LOGDET_MIXED_FP32 &&
      c.precision != LOGDET_MIXED_BF16VEC && c.precision != LOGDET_MIXED_F32X2) {
    set_error("precision %d unknown", c.precision);
    return LOGDET_EINVAL;
  }
  if (h->kind == 1 && (c.precision == LOGDET_MIXED_BF16VEC || c.precision == LOGDET_MIXED_F32X2)) {
    set_error("gridded operators support FP64 and mixed FP32 blocks only");
    return LOGDET_EINVAL;
  }
  if (c.block_width < 0) {
    set_error("block_width=%d must be >= 0", c.block_width);
    return LOGDET_EINVAL;
  }
  if (c.block_width > 0 && h->kind != 1) {
    // Every Krylov block (s + r probes; OSA-IOP's s sketch columns) rounded
    // up to whole 16-byte vectors must split into slices of the width.
    const int vec = precision_vec(c.precision);
    const int ld = round_up(s + r, vec), lds = std::max(round_up(s, vec), vec);
    bool ok = c.block_width % vec == 0;
    for (int w : {ld, c.method == 1 && s > 0 ? lds : ld})
      ok = ok && w % std::min(c.block_width, w) == 0;
    if (!ok) {
      set_error("block_width=%d must be a multiple of %d dividing the block widths %d and %d",
                c.block_width, vec, ld, lds);
      return LOGDET_EINVAL;
    }
  }
  double lo, hi;
  spectral_bounds(h, c, lo, hi);
  if (!(hi > 0.0) || !(lo > 0.0) || lo > hi) {
    set_error("spectral bounds [%g, %g] invalid", lo, hi);
    return LOGDET_ENOTSPD;
  }
  return LOGDET_OK;
}

// ---------------------------------------------------------------------------
// KState / KRun
// ---------------------------------------------------------------------------
int KState::alloc(int method, int b, int ld, int m, int k, double tol, double rescale_lim) {
  if (method == 0) {
    LD_TRY(alpha.alloc((size_t)ld * m));
    LD_TRY(beta.alloc((size_t)ld * m));
    LD_TRY(alpha.zero());
    LD_TRY(beta.zero());
  } else {
    LD_TRY(H.alloc((size_t)ld * (m + 1) * m));
    LD_TRY(H.zero());
  }
  LD_TRY(sig.alloc((size_t)ld * (m + 2)));
  LD_TRY(edot.alloc((size_t)ld * (m + 2)));
  LD_TRY(coef.alloc((size_t)kMaxWin * ld));
  LD_TRY(ycoef.alloc(ld));
  LD_TRY(dbuf.alloc((size_t)kMaxWin * ld));
  LD_TRY(meff.alloc(ld));
  LD_TRY(active.alloc(ld));
  LD_TRY(status.alloc(ld));
  LD_TRY(cnt.alloc(ld));
  LD_TRY(cnt.zero());
  LD_TRY(sig.zero());
  LD_TRY(edot.zero());
  LD_TRY(coef.zero());
  st.method = method;
  st.b = b;
  st.ld = ld;
  st.m = m;
  st.k = k;
  st.tol = tol;
  st.rescale_lim = rescale_lim;
  st.alpha = alpha.p;
  st.beta = beta.p;
  st.H = H.p;
  st.sig = sig.p;
  st.edot = edot.p;
  st.coef = coef.p;
  st.ycoef = ycoef.p;
  st.meff = meff.p;
  st.active = active.p;
  st.status = status.p;
  st.cnt = cnt.p;
  st.dbuf = dbuf.p;
  return LOGDET_OK;
}

template <typename T>
int KRun<T>::init(const int* rp, const int* ci, const typename ValOf<T>::type* v, int n_,
                  long long nnz_, int b_, int ld_,
                  int m_, int k_, int method_, bool track_e_, T* X0_, T* Vfull_, double tol,
                  TuneCfg tc) {
  rowptr = rp;
  colind = ci;
  vals = v;
  n = n_;
  nnz = nnz_;
  b = b_;
  ld = ld_;
  m = m_;
  k = k_;
  method = method_;
  track_e = track_e_;
  X0 = X0_;
  Vfull = Vfull_;
  tune = tc;
  if (tune.split < 1 || ld % tune.split || (ld / tune.split) % Vec16<T>::N) tune.split = 1;
  if (hctx && hctx->kind == 1) tune = TuneCfg();  // gridded operator: full-width default layout
  width = ld / tune.split;
  g = tile_geom(width, Vec16<T>::N, tune.threads, tune.iters, n);
  ntiles = div_up(n, g.tile_rows);
  nslots = ntiles;
  items = nullptr;
  if (hctx) {
    int cnt = 0;
    LD_TRY(spmm_items(hctx, g.tile_rows, &items, &cnt));
    if (items) nslots = cnt;
  }
  if constexpr (std::is_same<T, float>::value) {
    // Line sweep: FP32 blocks of a matrix with line structure; its units are
    // the partial slots.
    SweepGeom sg;
    if (diavals && !items && hctx && hctx->kind == 0 && !((uintptr_t)X0 & 15) &&
        !((uintptr_t)Vfull & 15) && dia_sweep_geom(hctx, width, g.threads, &sg)) {
      sweep = true;
      sw_T = sg.T;
      sw_kc = sg.kc;
      sw_nseg = sg.nseg;
      sw_nlines = sg.nlines;
      sw_tx = sg.tx;
      sw_ty = sg.ty;
      sw_txs = sg.txs;
      nslots = sg.units;
    }
  }
  blk = (size_t)n * ld;
  const int win = method == 0 ? 2 : k;
  if (method == 1 && win > kMaxWin - 1) {
    set_error("iop_window %d exceeds the supported maximum %d", k, kMaxWin - 1);
    return LOGDET_EINVAL;
  }
  ndmax = std::max(win, 2);
  nring = win + 1;
  LD_TRY(part.alloc((size_t)ndmax * ld * std::max(ntiles, nslots)));
  if (diavals) {
    LD_TRY(dia_err.alloc(1));
    LD_TRY(dia_err.zero());
  }
  LD_TRY(y.alloc(blk));
  if (!Vfull) LD_TRY(ring.alloc(blk * nring));
  LD_TRY(ks.alloc(method, b, ld, m, k, tol, rescale_limit<T>()));
  {
    // Column norms of the start block over the same tiles (full-width CTAs).
    const TileGeom gf = tile_geom(ld, Vec16<T>::N);
    LD_TRY(colnorm_partials<T>(X0, n, ld, g.tile_rows, ntiles, part.p, gf.threads, st));
  }
  std::vector<ScalarJob> jobs{scalar_job(0, 1)};
  std::vector<int> widths{ld};
  return launch_scalar_jobs(jobs, widths, SK_INIT, st);
}

template <typename T>
T* KRun<T>::ptr(int i) const {
  if (Vfull) return Vfull + (size_t)(i - 1) * blk;
  if (i == 1) return X0;
  return ring.p + (size_t)((i - 2) % nring) * blk;
}

template <typename T>
int KRun<T>::slice_live(int q) const {
  const int lo = q * width;
  return std::max(0, std::min(width, b - lo));
}

template <typename T>
int KRun<T>::spmm_jobs(int j, std::vector<SpmmJob<T>>& out) const {
  for (int q = 0; q < tune.split; ++q) {
    SpmmJob<T> J;
    memset(&J, 0, sizeof J);
    J.rowptr = rowptr;
    J.colind = colind;
    J.vals = vals;
    J.x = ptr(j);
    J.y = y.p;
    J.part = part.p;
    J.n = n;
    J.ld = ld;
    J.col_off = q * width;
    J.width = width;
    J.b = slice_live(q);
    J.nnz = nnz;
    J.tile_rows = g.tile_rows;
    J.ntiles = nslots;
    J.items = items;
    J.colshift = colshift;
    J.colscale = colscale;
    if (method == 0) {
      J.ndots = 1;
      J.dotv[0] = ptr(j);
    } else {
      const int lo = win_lo(j);
      J.ndots = j - lo + 1;
      for (int i = lo; i <= j; ++i) J.dotv[i - lo] = ptr(i);
    }
    if constexpr (std::is_same<T, float>::value) {
      if (sweep) {
        J.dia = diavals;
        J.err = dia_err.p;
        J.dia_T = sw_T;
        J.dia_kc = sw_kc;
        J.dia_nseg = sw_nseg;
        J.dia_nlines = sw_nlines;
        J.dia_tx = sw_tx;
        J.dia_ty = sw_ty;
        J.dia_txs = sw_txs;
        J.dinfo = hctx->dia;
        LD_TRY(dia_encode(J, ptr(j), n, ld, width));
      }
    }
    out.push_back(J);
  }
  return LOGDET_OK;
}

template <typename T>
int KRun<T>::grid_pass1(int j) {
  if constexpr (std::is_same<T, bf16>::value || std::is_same<T, f32x2>::value) {
    set_error("gridded operators take FP64 and FP32 blocks only");
    return LOGDET_EINVAL;
  } else {
    using CT = typename Compute<T>::type;
    LD_TRY(grid_apply<T>(hctx, static_cast<const CT*>(gtab), ptr(j), y.p, ld, colshift, st));
    const T* dv[kMaxWin];
    int nd = 0;
    if (method == 0) {
      dv[nd++] = ptr(j);
    } else {
      for (int i = win_lo(j); i <= j; ++i) dv[nd++] = ptr(i);
    }
    return dots_pass<T>(y.p, dv, nd, part.p, n, ld, g.tile_rows, ntiles, g.threads, st);
  }
}

template <typename T>
void KRun<T>::upd_jobs(int j, std::vector<UpdJob<T>>& out) const {
  for (int q = 0; q < tune.split; ++q) {
    UpdJob<T> U;
    memset(&U, 0, sizeof U);
    U.y = y.p;
    U.coef = ks.coef.p;
    U.ycoef = ks.ycoef.p;
    U.extra = track_e ? X0 : nullptr;
    U.part = part.p;
    U.n = n;
    U.ld = ld;
    U.col_off = q * width;
    U.width = width;
    U.b = slice_live(q);
    U.tile_rows = g.tile_rows;
    U.ntiles = ntiles;
    if (method == 0) {
      if (j >= 2) {
        U.nbasis = 2;
        U.basis[0] = ptr(j - 1);
        U.basis[1] = ptr(j);
      } else {
        U.nbasis = 1;
        U.basis[0] = ptr(j);
      }
    } else {
      const int lo = win_lo(j);
      U.nbasis = j - lo + 1;
      for (int i = lo; i <= j; ++i) U.basis[i - lo] = ptr(i);
    }
    U.out = ptr(j + 1);
    out.push_back(U);
  }
}

template <typename T>
ScalarJob KRun<T>::scalar_job(int j, int ndots, bool spmm_pass) const {
  ScalarJob sj;
  memset(&sj, 0, sizeof sj);
  sj.st = ks.st;
  sj.part = part.p;
  sj.part_f32 = std::is_same<T, double>::value ? 0 : 1;
  sj.ntiles = spmm_pass ? nslots : ntiles;
  sj.step = j;
  sj.ndots = ndots;
  sj.win_lo = j >= 1 ? win_lo(j) : 1;
  sj.last = j == m;
  return sj;
}

template <typename T>
bool KRun<T>::persistent_ok() const {
  if constexpr (std::is_same<T, bf16>::value || std::is_same<T, f32x2>::value) {
    return false;
  } else {
    // Opt-in: measured on GB300 (2D Laplacian 64^2, FP64) it issues as fast
    // as the step path, not faster (see krylov.cuh), so the step path stays
    // the default.
    const char* e = std::getenv("LOGDET_KRYLOV_PERSISTENT");
    if (!e || e[0] != '1') return false;
    if (sweep || items || (hctx && hctx->kind == 1) || tune.split != 1 || nslots != ntiles)
      return false;
    // the scalar reductions run one per warp (whole warps only)
    if (g.threads % 32 || g.threads > 512) return false;
    // from the first step (the run seeds its sigmas from sigma_1)
    return done_steps == 0 && ld <= 128 && blk * sizeof(T) <= kPersistMaxBlock;
  }
}

template <typename T>
int KRun<T>::issue_rest_persistent() {
  if constexpr (std::is_same<T, bf16>::value || std::is_same<T, f32x2>::value) {
    return LOGDET_EINVAL;
  } else {
    const int j = next_step();
    PersistRun<T> P;
    memset(&P, 0, sizeof P);
    std::vector<SpmmJob<T>> sj;
    std::vector<UpdJob<T>> uj;
    LD_TRY(spmm_jobs(j, sj));
    upd_jobs(j, uj);
    if (!krun_part2.p) LD_TRY(krun_part2.alloc((size_t)2 * ld * ntiles));
    P.sj = sj[0];
    P.uj = uj[0];
    P.uj.part = krun_part2.p;  // pass-2 partials apart from pass 1's
    P.cj = scalar_job(j, 1, true);
    P.X0 = X0;
    P.ring = ring.p;
    P.Vfull = Vfull;
    P.blk = blk;
    P.nring = nring;
    P.method = method;
    P.k = k;
    P.m = m;
    P.j0 = j;
    P.track_e = track_e ? 1 : 0;
    P.ntiles = ntiles;
    if (!krun_bar.p) LD_TRY(krun_bar.alloc(2));
    if (!dia_err.p) {
      LD_TRY(dia_err.alloc(1));
      LD_TRY(dia_err.zero());
    }
    P.bar = krun_bar.p;
    P.err = dia_err.p;
    const int nd_max = method == 0 ? 1 : std::min(k, m);
    const int nb_max = method == 0 ? 2 : std::min(k, m);
    LD_TRY(launch_krylov_run<T>(P, g.threads, nd_max, nb_max, st));
    done_steps = m;
    return LOGDET_OK;
  }
}

template struct KRun<double>;
template struct KRun<float>;
template struct KRun<bf16>;
template struct KRun<f32x2>;

// ---------------------------------------------------------------------------
// batched launches
// ---------------------------------------------------------------------------
template <typename T>
int launch_spmm_jobs(const std::vector<SpmmJob<T>>& jobs, int threads, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    // Sweep jobs launch apart from CSR jobs, line sweeps apart from plane
    // sweeps (same stream, in order).
    auto kind = [](const SpmmJob<T>& J) { return J.dia ? J.dinfo.dim : 0; };
    bool mixed = false;
    for (const auto& J : jobs) mixed |= kind(J) != kind(jobs[0]);
    if (mixed) {
      std::vector<SpmmJob<T>> part[4];
      for (const auto& J : jobs) part[kind(J)].push_back(J);
      for (int k : {0, 2, 3})
        if (!part[k].empty()) LD_TRY(launch_spmm_jobs<T>(part[k], threads, s));
      return LOGDET_OK;
    }
  }
  for (size_t i0 = 0; i0 < jobs.size(); i0 += kMaxJobs) {
    SpmmBatch<T> B;
    memset(&B, 0, sizeof B);
    const int nj = (int)std::min<size_t>(kMaxJobs, jobs.size() - i0);
    int t = 0;
    for (int q = 0; q < nj; ++q) {
      B.jobs[q] = jobs[i0 + q];
      B.tile_start[q] = t;
      t += jobs[i0 + q].ntiles;
    }
    B.njobs = nj;
    B.tile_start[nj] = t;
    B.total_tiles = t;
    if constexpr (std::is_same<T, float>::value) {
      if (B.jobs[0].dia) {
        LD_TRY(launch_spmm_dia(B, threads, s));
        continue;
      }
    }
    LD_TRY(launch_spmm<T>(B, threads, s));
  }
  return LOGDET_OK;
}

template <typename T>
int launch_update_jobs(const std::vector<UpdJob<T>>& jobs, int threads, cudaStream_t s) {
  for (size_t i0 = 0; i0 < jobs.size(); i0 += kMaxJobs) {
    UpdBatch<T> B;
    memset(&B, 0, sizeof B);
    const int nj = (int)std::min<size_t>(kMaxJobs, jobs.size() - i0);
    int t = 0;
    for (int q = 0; q < nj; ++q) {
      B.jobs[q] = jobs[i0 + q];
      B.tile_start[q] = t;
      t += jobs[i0 + q].ntiles;
    }
    B.njobs = nj;
    B.tile_start[nj] = t;
    B.total_tiles = t;
    LD_TRY(launch_update<T>(B, threads, s));
  }
  return LOGDET_OK;
}

template int launch_spmm_jobs<double>(const std::vector<SpmmJob<double>>&, int, cudaStream_t);
template int launch_spmm_jobs<float>(const std::vector<SpmmJob<float>>&, int, cudaStream_t);
template int launch_spmm_jobs<bf16>(const std::vector<SpmmJob<bf16>>&, int, cudaStream_t);
template int launch_spmm_jobs<f32x2>(const std::vector<SpmmJob<f32x2>>&, int, cudaStream_t);
template int launch_update_jobs<double>(const std::vector<UpdJob<double>>&, int, cudaStream_t);
template int launch_update_jobs<float>(const std::vector<UpdJob<float>>&, int, cudaStream_t);
template int launch_update_jobs<bf16>(const std::vector<UpdJob<bf16>>&, int, cudaStream_t);
template int launch_update_jobs<f32x2>(const std::vector<UpdJob<f32x2>>&, int, cudaStream_t);

int launch_scalar_jobs(const std::vector<ScalarJob>& jobs, const std::vector<int>& widths, int kind,
                       cudaStream_t s) {
  // Jobs with FP64 and FP32 partials go to separate launches.
  for (int f32 = 0; f32 < 2; ++f32) {
    ScalarBatch B;
    memset(&B, 0, sizeof B);
    int nj = 0, pcount = 0;
    auto flush = [&]() -> int {
      if (!nj) return LOGDET_OK;
      B.njobs = nj;
      B.probe_start[nj] = pcount;
      int rc = kind == SK_INIT ? launch_init_sigma(B, s)
                               : kind == SK_COEF ? launch_coef(B, s) : launch_norm(B, s);
      memset(&B, 0, sizeof B);
      nj = 0;
      pcount = 0;
      return rc;
    };
    for (size_t i = 0; i < jobs.size(); ++i) {
      if (jobs[i].part_f32 != f32) continue;
      B.jobs[nj] = jobs[i];
      B.probe_start[nj] = pcount;
      pcount += widths[i];
      ++nj;
      if (nj == kMaxJobs) LD_TRY(flush());
    }
    LD_TRY(flush());
  }
  return LOGDET_OK;
}

// ---------------------------------------------------------------------------
// small assembly kernels of OSA-IOP
// ---------------------------------------------------------------------------
// Sketch weights: w[j][p] = |s_p| c_j sigma_j (+ shift for j = 1), so that
// Y[:, p] = sum_j w[j][p] u_j = |s| V_m log(H_m) e_1 + shift s (Algorithm 1's
// return line with L's shift).
__global__ void k_iop_weights(const double* __restrict__ c, int ldc, const double* __restrict__ sig,
                              const double* __restrict__ edot, const int* __restrict__ meff,
                              int m, int ld, double shift, double* __restrict__ w) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * ld) return;
  const int j = e / ld + 1, p = e - (e / ld) * ld;
  const int m2 = m + 2;
  double v = 0.0;
  if (j <= meff[p]) {
    v = sqrt(edot[p * m2 + 1]) * c[(size_t)p * ldc + j - 1] * sig[p * m2 + j];
    if (j == 1) v += shift;
  }
  w[(size_t)(j - 1) * ld + p] = v;
}

// Quadratic form x^T L x = |x| sum_j c_j sigma_j (u_1^T u_j) + shift |x|^2.
__global__ void k_iop_qf(const double* __restrict__ c, int ldc, const double* __restrict__ sig,
                         const double* __restrict__ edot, const int* __restrict__ meff, int m,
                         int ld, double shift, double* __restrict__ qf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ld) return;
  const int m2 = m + 2;
  const int me = meff[p];
  if (me <= 0) { qf[p] = 0.0; return; }
  double acc = 0.0;
  for (int j = 1; j <= me; ++j)
    acc = fma(c[(size_t)p * ldc + j - 1] * sig[p * m2 + j], edot[p * m2 + j], acc);
  const double e1 = edot[p * m2 + 1];
  qf[p] = sqrt(e1) * acc + shift * e1;
}

// Hutch++ split shared by both estimators: A = orth(Y) into X64[:, 0:s],
// Z = G - A A^T G into X64[:, s:s+r].  No host synchronisation.
static int hutchpp_split(int n, int s, int r, const double* Y64, int lds, uint64_t key_g,
                         DevBuf<double>& X64, int ld, int* keep, cudaStream_t st, int gaussian,
                         const uint64_t* keyp_g) {
  LD_TRY(X64.alloc((size_t)n * ld));
  LD_TRY(X64.zero());
  DevBuf<double> ws(st);
  LD_TRY(ws.alloc(std::max(s ? orth_workspace_doubles(n, s) : 0,
                           project_workspace_doubles(n, s, r))));
  if (s > 0) LD_TRY(orth_fp64(n, s, Y64, lds, X64.p, ld, ws.p, keep, nullptr, st));
  LD_TRY(project_residual_fp64(n, s, r, X64.p, ld, key_g, X64.p, ld, s, ws.p, st, gaussian,
                               keyp_g));
  return LOGDET_OK;
}

// The split for an FP32 block computed in FP32 (compensated sums): A into
// X[:, 0:s], Z into X[:, s:s+r] of the block the Krylov run starts from, so
// the mixed path needs no FP64 copy of Y or of the block.
static int hutchpp_split_f32(int n, int s, int r, const float* Y, int lds, uint64_t key_g,
                             DevBuf<float>& X, int ld, int* keep, cudaStream_t st, int gaussian,
                             const uint64_t* keyp_g) {
  LD_TRY(X.alloc((size_t)n * ld));
  LD_TRY(X.zero());
  DevBuf<double> ws(st);
  LD_TRY(ws.alloc(std::max(orth_workspace_doubles(n, s), project_workspace_doubles(n, s, r))));
  LD_TRY(orth_f32(n, s, Y, lds, X.p, ld, ws.p, keep, nullptr, st));
  LD_TRY(project_residual_f32(n, s, r, X.p, ld, key_g, X.p, ld, s, ws.p, st, gaussian, keyp_g));
  return LOGDET_OK;
}

// ---------------------------------------------------------------------------
// Solve<T>
// ---------------------------------------------------------------------------
struct PinnedHost {
  void* p = nullptr;
  size_t cap = 0;
  cudaStream_t st = nullptr;
  ~PinnedHost() { pinned_release(p, cap, st); }
};

template <typename T>
struct Solve : ISolve {
  logdet_ctx* h;
  SolveCfg c;
  cudaStream_t st;
  int ph = PH_SETUP;
  int n, s, r, b, ld, lds, m, kk;
  double lo, hi, alpha, gamma, shift;
  DevBuf<typename ValOf<T>::type> vals;
  DevBuf<typename Compute<T>::type> gtabs;  // gridded operator: scaled table
  DevBuf<float> diav;                        // FP32 values per diagonal (diagonal fast path)
  DevBuf<T> Vst, Xc;
  DevBuf<double> X64, outv, cshift;
  DevBuf<int> keep;
  std::unique_ptr<KRun<T>> run;
  PinnedHost pin;
  double *h_out = nullptr, *h_edot = nullptr;
  int *h_meff = nullptr, *h_keep = nullptr;
  uint32_t *h_status = nullptr, *h_status1 = nullptr;
  int* h_err = nullptr;  // [2]: a diagonal-path wait gave up (phase 1, last run)
  cudaEvent_t ev_done = nullptr;
  const uint64_t* dev_keys = nullptr;  // graph plans: probe keys in device memory
  // Group member (solve_shifts): the Krylov phases run in one wide run over
  // every member's columns; start_run hands the start block to the group,
  // adopt takes this member's scalar history back from the wide run.
  bool grouped = false, awaiting = false;
  T* pend_x0 = nullptr;          // start block of the phase that waits for the group
  int pend_b = 0, pend_ld = 0;   // its live columns and width
  const T* vst_ext = nullptr;    // phase-1 basis: this member's columns of the group's
  int vst_ld = 0;                //   basis blocks (leading dimension vst_ld)

  Solve(logdet_ctx* h_, const SolveCfg& c_, cudaStream_t st_)
      : h(h_), c(c_), st(st_), vals(st_), gtabs(st_), diav(st_), Vst(st_), Xc(st_), X64(st_), outv(st_), cshift(st_),
        keep(st_) {
    n = h->n;
    s = c.plain ? 0 : c.P / 3;
    r = c.plain ? c.P : c.P - 2 * s;
    b = s + r;
    ld = round_up(b, Vec16<T>::N);
    lds = std::max(round_up(s, Vec16<T>::N), Vec16<T>::N);
    m = c.m;
    kk = c.method == 0 ? 2 : std::min(c.k, m);
    spectral_bounds(h, c, lo, hi);
    gamma = std::sqrt(lo * hi);        // Proposition 2.1
    alpha = c.method == 0 ? hi : lo;   // readings R1 / R2
    shift = std::log(gamma / alpha);
  }
  ~Solve() override {
    if (ev_done) cudaEventDestroy(ev_done);
  }

  const uint64_t* dkey(int i) const { return dev_keys ? dev_keys + i : nullptr; }
  void set_dev_keys(const uint64_t* keys) override { dev_keys = keys; }
  int prepare_host() override {
    if (!ev_done) LD_CUDA(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming));
    return alloc_pinned();
  }

  int alloc_pinned() {
    if (pin.p) return LOGDET_OK;
    const size_t bytes = sizeof(double) * ld + sizeof(double) * (size_t)ld * (m + 2) +
                         sizeof(int) * ld + sizeof(int) * (s + 1) + sizeof(uint32_t) * ld +
                         sizeof(uint32_t) * lds + 2 * sizeof(int) + 64;
    pin.st = st;
    pin.p = pinned_acquire(bytes, &pin.cap);
    if (!pin.p) {
      set_error("pinned host allocation of %zu bytes failed", bytes);
      return LOGDET_ENOMEM;
    }
    memset(pin.p, 0, bytes);
    char* q = static_cast<char*>(pin.p);
    h_out = reinterpret_cast<double*>(q);
    q += sizeof(double) * ld;
    h_edot = reinterpret_cast<double*>(q);
    q += sizeof(double) * (size_t)ld * (m + 2);
    h_meff = reinterpret_cast<int*>(q);
    q += sizeof(int) * ld;
    h_keep = reinterpret_cast<int*>(q);
    q += sizeof(int) * (s + 1);
    h_status = reinterpret_cast<uint32_t*>(q);
    q += sizeof(uint32_t) * ld;
    h_status1 = reinterpret_cast<uint32_t*>(q);
    q += sizeof(uint32_t) * lds;
    h_err = reinterpret_cast<int*>(q);
    return LOGDET_OK;
  }

  int phase() const override { return ph; }
  bool in_krylov() const override { return ph == PH_K1 || ph == PH_K2; }

  // ---- suspension (see ISolve) ----
  struct BufRef {  // one DevBuf of the solve, whatever its element type
    std::function<void*()> ptr;
    size_t bytes;  // allocated size (0: no buffer)
    std::function<void()> release;
    std::function<int()> realloc;  // the same element count again
  };
  struct Saved {
    void* old;
    size_t off, bytes;
  };
  std::vector<unsigned char> susp_host;
  std::vector<Saved> susp_list;
  bool is_susp = false;

  template <typename U>
  static BufRef ref(DevBuf<U>& b) {
    return {[&b] { return static_cast<void*>(b.p); }, b.p ? b.count * sizeof(U) : 0,
            [&b] { b.release(); }, [&b] { return b.alloc(b.count); }};
  }
  std::vector<BufRef> buffers() {
    std::vector<BufRef> v = {ref(vals), ref(gtabs), ref(diav), ref(Vst), ref(Xc),
                             ref(X64),  ref(outv),  ref(cshift), ref(keep)};
    if (run) {
      KRun<T>& R = *run;
      KState& K = R.ks;
      for (BufRef b : {ref(R.part), ref(R.y), ref(R.ring), ref(R.dia_err), ref(R.krun_bar),
                       ref(R.krun_part2), ref(K.alpha), ref(K.beta), ref(K.H), ref(K.sig),
                       ref(K.edot), ref(K.coef), ref(K.ycoef), ref(K.dbuf), ref(K.meff),
                       ref(K.active), ref(K.status), ref(K.cnt)})
        v.push_back(b);
    }
    return v;
  }
  bool suspended() const override { return is_susp; }

  int suspend() override {
    if (is_susp) return LOGDET_OK;
    LD_CUDA(cudaStreamSynchronize(st));
    std::vector<BufRef> bufs = buffers();
    size_t total = 0;
    for (const BufRef& b : bufs) total += b.bytes;
    susp_host.resize(total);
    susp_list.clear();
    size_t off = 0;
    for (const BufRef& b : bufs) {
      susp_list.push_back({b.ptr(), off, b.bytes});
      if (b.bytes)
        LD_CUDA(cudaMemcpyAsync(susp_host.data() + off, b.ptr(), b.bytes, cudaMemcpyDeviceToHost, st));
      off += b.bytes;
    }
    LD_CUDA(cudaStreamSynchronize(st));
    for (const BufRef& b : bufs) b.release();
    is_susp = true;
    return LOGDET_OK;
  }

  int resume() override {
    if (!is_susp) return LOGDET_OK;
    std::vector<BufRef> bufs = buffers();  // (same order; every pointer is null now)
    if (bufs.size() != susp_list.size()) {
      set_error("resume: the solve's buffer list changed while suspended");
      return LOGDET_ECUDA;
    }
    std::vector<std::pair<const void*, void*>> moved;
    for (size_t i = 0; i < bufs.size(); ++i) {
      const Saved& sv = susp_list[i];
      if (!sv.bytes) continue;
      if (bufs[i].realloc() != LOGDET_OK) {  // (the message is set)
        for (size_t j = 0; j < i; ++j) bufs[j].release();
        return LOGDET_ENOMEM;
      }
      void* q = bufs[i].ptr();
      LD_CUDA(cudaMemcpyAsync(q, susp_host.data() + sv.off, sv.bytes, cudaMemcpyHostToDevice, st));
      moved.push_back({sv.old, q});
    }
    LD_CUDA(cudaStreamSynchronize(st));
    // Raw pointers held next to the buffers: the run's inputs and its state table.
    auto fix = [&](auto& ptr) {
      for (const auto& mv : moved)
        if (static_cast<const void*>(ptr) == mv.first) {
          ptr = static_cast<std::remove_reference_t<decltype(ptr)>>(mv.second);
          return;
        }
    };
    if (run) {
      KRun<T>& R = *run;
      fix(R.X0);
      fix(R.Vfull);
      fix(R.vals);
      fix(R.colshift);
      fix(R.colscale);
      fix(R.diavals);
      fix(R.gtab);
      KrylovState& S = R.ks.st;
      fix(S.alpha);
      fix(S.beta);
      fix(S.H);
      fix(S.sig);
      fix(S.edot);
      fix(S.coef);
      fix(S.ycoef);
      fix(S.meff);
      fix(S.active);
      fix(S.status);
      fix(S.cnt);
      fix(S.dbuf);
    }
    fix(pend_x0);
    susp_host.clear();
    susp_host.shrink_to_fit();
    susp_list.clear();
    is_susp = false;
    return LOGDET_OK;
  }
  int krylov_threads() const override { return run ? run->g.threads : 0; }
  bool is_fp32() const override { return !std::is_same<T, double>::value; }
  int elem_kind() const override {
    return std::is_same<T, double>::value  ? 0
           : std::is_same<T, float>::value ? 1
           : std::is_same<T, bf16>::value  ? 2
                                           : 3;
  }
  cudaEvent_t done_event() const override { return ev_done; }
  size_t bytes_estimate() const override { return estimate_solve_bytes(h, c); }

  // Layout of the Krylov kernels for a block of width w: defaults, or the
  // autotuner's choice for this matrix.
  int layout(int w, bool track_e, TuneCfg* tc) {
    *tc = TuneCfg();
    if (h->kind == 1) return LOGDET_OK;
    if (c.block_width > 0) {  // the caller's slice width (validated to divide w)
      tc->split = w / std::min(c.block_width, w);
      return LOGDET_OK;
    }
    if (!c.autotune) return LOGDET_OK;
    const int nd = c.method == 0 ? 1 : kk, nb = c.method == 0 ? 2 : kk;
    return autotune_krylov<T>(h, vals.p, w, nd, nb, track_e ? 1 : 0,
                              st, tc);
  }

  // Start the Krylov run of the current phase on X0 (a group member only
  // records it for the group).
  int start_run(int b_, int ld_, int k_, int method_, bool track_e_, T* X0, T* Vfull, TuneCfg tc) {
    if (grouped) {
      pend_x0 = X0;
      pend_b = b_;
      pend_ld = ld_;
      awaiting = true;
      return LOGDET_OK;
    }
    return run->init(h->rowptr, h->colind, vals.p, n, h->nnz, b_, ld_, m, k_, method_, track_e_, X0,
                     Vfull, c.tol, tc);
  }

  double cscale() const { return c.method == 0 ? alpha : gamma; }
  // Group member: free the start block once the group has copied it.
  void release_start() {
    if (pend_x0 == Vst.p) Vst.release();
    else if (pend_x0 == Xc.p) Xc.release();
    else if (static_cast<void*>(pend_x0) == static_cast<void*>(X64.p)) X64.release();
  }

  // Group member: this member's per-probe scalar history (probes p0 ..
  // p0 + pend_ld - 1 of the wide run w) into a run of its own, then the next
  // phase.
  int adopt(const KRun<T>& w, int p0) {
    const int ldm = pend_ld;
    run.reset(new KRun<T>(st));
    KRun<T>& rr = *run;
    rr.m = m;
    rr.ld = ldm;
    rr.b = pend_b;
    rr.k = w.k;
    rr.method = w.method;
    rr.track_e = w.track_e;
    LD_TRY(rr.ks.alloc(w.method, pend_b, ldm, m, w.k, c.tol, rescale_limit<T>()));
    auto cp = [&](auto* dst, const auto* src, size_t cnt) {
      return cudaMemcpyAsync(dst, src, cnt * sizeof(*dst), cudaMemcpyDeviceToDevice, st);
    };
    const size_t pm2 = (size_t)m + 2;
    if (w.method == 0) {
      LD_CUDA(cp(rr.ks.alpha.p, w.ks.alpha.p + (size_t)p0 * m, (size_t)ldm * m));
      LD_CUDA(cp(rr.ks.beta.p, w.ks.beta.p + (size_t)p0 * m, (size_t)ldm * m));
    } else {
      const size_t hb = (size_t)(m + 1) * m;
      LD_CUDA(cp(rr.ks.H.p, w.ks.H.p + (size_t)p0 * hb, (size_t)ldm * hb));
    }
    LD_CUDA(cp(rr.ks.sig.p, w.ks.sig.p + (size_t)p0 * pm2, (size_t)ldm * pm2));
    LD_CUDA(cp(rr.ks.edot.p, w.ks.edot.p + (size_t)p0 * pm2, (size_t)ldm * pm2));
    LD_CUDA(cp(rr.ks.meff.p, w.ks.meff.p + p0, (size_t)ldm));
    LD_CUDA(cp(rr.ks.active.p, w.ks.active.p + p0, (size_t)ldm));
    LD_CUDA(cp(rr.ks.status.p, w.ks.status.p + p0, (size_t)ldm));
    if (w.dia_err.p) {
      LD_TRY(rr.dia_err.alloc(1));
      LD_CUDA(cp(rr.dia_err.p, w.dia_err.p, 1));
    }
    awaiting = false;
    pend_x0 = nullptr;
    ph = (c.method == 1 && ph == PH_K1) ? PH_MID : PH_FINISH;
    return LOGDET_OK;
  }

  // X0 for the next Krylov run from X64 (a copy in FP32 for the mixed path).
  int make_x0(T** X0) {
    if constexpr (std::is_same<T, double>::value) {
      *X0 = X64.p;
    } else {
      LD_TRY(Xc.alloc((size_t)n * ld));
      LD_TRY((convert_block<double, T>(X64.p, ld, Xc.p, ld, n, ld, st)));
      X64.release();
      *X0 = Xc.p;
    }
    return LOGDET_OK;
  }

  int setup() {
    LD_TRY(alloc_pinned());
    LD_TRY(keep.alloc(std::max(s, 1)));
    const double cscale = c.method == 0 ? alpha : gamma;
    if (h->kind == 1) {
      // Gridded operator: the table of W / c replaces the scaled CSR values.
      if constexpr (std::is_same<T, f32x2>::value) {
        set_error("gridded operators support FP64 and mixed FP32 blocks only");
        return LOGDET_EINVAL;
      } else {
        LD_TRY(gtabs.alloc(grid_table_count(h)));
        LD_TRY(grid_table<typename Compute<T>::type>(h, cscale, gtabs.p, st));
      }
    } else {
      LD_TRY(vals.alloc(h->nnz));
      LD_TRY(scaled_values<typename ValOf<T>::type>(h, cscale, vals.p, st));
      if (std::is_same<T, float>::value && h->dia.ndiag > 0 && h->dia_slot) {
        LD_TRY(diav.alloc((size_t)dia_pad(h->dia.ndiag) * n));
        LD_TRY(dia_values_f32(h, cscale, diav.p, st));
      }
    }
    if (c.shift != 0.0) {
      // (Q + shift I)/c applied as vals/c plus (shift/c) times the row's own entry.
      const size_t cnt = std::max(ld, lds);
      LD_TRY(cshift.alloc(cnt));
      LD_TRY(fill_double(cshift.p, cnt, c.shift / cscale, st));
    }
    run.reset(new KRun<T>(st));
    if (s == 0) {
      // Plain SLQ: no sketch; the residual probes are the probes themselves.
      LD_TRY(hutchpp_split(n, 0, r, nullptr, lds, probe_key(c.seed, 1), X64, ld, keep.p, st,
                           c.gaussian, dkey(1)));
      T* X0;
      LD_TRY(make_x0(&X0));
      run->colshift = cshift.p;
      run->hctx = h;
      run->gtab = gtabs.p;
      run->diavals = diav.p;
      TuneCfg tc;
      LD_TRY(layout(ld, c.method == 1, &tc));
      if (c.method == 0) {
        LD_TRY(start_run(b, ld, 2, 0, false, X0, nullptr, tc));
        ph = PH_K1;
      } else {
        LD_TRY(start_run(b, ld, kk, 1, true, X0, nullptr, tc));
        ph = PH_K2;
      }
      return LOGDET_OK;
    }
    if (c.method == 0) {
      // Algorithm 3: Y = J S, A = orth(Y), Z = (I - A A^T) G.
      DevBuf<T> S(st), Yt(st);
      LD_TRY(S.alloc((size_t)n * lds));
      LD_TRY(Yt.alloc((size_t)n * lds));
      LD_TRY(probe_fill<T>(probe_key(c.seed, 0), n, s, 0, S.p, lds, st, c.gaussian, dkey(0)));
      if constexpr (std::is_same<T, bf16>::value || std::is_same<T, f32x2>::value) {
        LD_TRY(spmm_block<T>(h->rowptr, h->colind, vals.p, n, S.p, Yt.p, lds, st, cshift.p, h));
      } else {
        if (h->kind == 1) LD_TRY(grid_apply<T>(h, gtabs.p, S.p, Yt.p, lds, cshift.p, st));
        else LD_TRY(spmm_block<T>(h->rowptr, h->colind, vals.p, n, S.p, Yt.p, lds, st, cshift.p, h));
      }
      S.release();
      T* X0;
      if constexpr (std::is_same<T, double>::value) {
        LD_TRY(hutchpp_split(n, s, r, Yt.p, lds, probe_key(c.seed, 1), X64, ld, keep.p, st, c.gaussian,
                             dkey(1)));
        LD_TRY(make_x0(&X0));
      } else if constexpr (std::is_same<T, float>::value) {
        LD_TRY(hutchpp_split_f32(n, s, r, Yt.p, lds, probe_key(c.seed, 1), Xc, ld, keep.p, st,
                                 c.gaussian, dkey(1)));
        Yt.release();
        X0 = Xc.p;
      } else {
        DevBuf<double> Y64(st);
        LD_TRY(Y64.alloc((size_t)n * lds));
        LD_TRY((convert_block<T, double>(Yt.p, lds, Y64.p, lds, n, lds, st)));
        Yt.release();
        LD_TRY(hutchpp_split(n, s, r, Y64.p, lds, probe_key(c.seed, 1), X64, ld, keep.p, st, c.gaussian,
                             dkey(1)));
        LD_TRY(make_x0(&X0));
      }
      run->colshift = cshift.p;
      run->hctx = h;
      run->gtab = gtabs.p;
      run->diavals = diav.p;
      TuneCfg tc;
      LD_TRY(layout(ld, false, &tc));
      LD_TRY(start_run(b, ld, 2, 0, false, X0, nullptr, tc));
    } else {
      // Algorithm 2, phase 1: each sketch column through Algorithm 1, basis kept.
      // (a group member fills only the start block; the group keeps the basis)
      LD_TRY(Vst.alloc((size_t)n * lds * (grouped ? 1 : m)));
      LD_TRY(probe_fill<T>(probe_key(c.seed, 0), n, s, 0, Vst.p, lds, st, c.gaussian, dkey(0)));
      run->colshift = cshift.p;
      run->hctx = h;
      run->gtab = gtabs.p;
      run->diavals = diav.p;
      TuneCfg tc;
      LD_TRY(layout(lds, false, &tc));
      LD_TRY(start_run(s, lds, kk, 1, false, Vst.p, Vst.p, tc));
    }
    ph = PH_K1;
    return LOGDET_OK;
  }

  int mid() {
    // Y = L S from the kept bases, then the Hutch++ split and phase 2.
    KRun<T>& r1 = *run;
    DevBuf<double> cc(st), ws(st), w(st), Y64(st);
    LD_TRY(cc.alloc((size_t)lds * m));
    LD_TRY(ws.alloc(hesslog_workspace_doubles(m, lds, kk - 1)));
    LD_TRY(w.alloc((size_t)m * lds));
    LD_TRY(hessenberg_log_e1(r1.ks.H.p, m + 1, r1.ks.meff.p, m, lds, cc.p, m, ws.p, r1.ks.status.p, st,
                             kk - 1));
    {
      ProfScope prof(KC_SMALL, st);
      k_iop_weights<<<div_up(m * lds, 256), 256, 0, st>>>(cc.p, m, r1.ks.sig.p, r1.ks.edot.p,
                                                          r1.ks.meff.p, m, lds, shift, w.p);
      LD_CHECK_LAUNCH();
    }
    LD_TRY(Y64.alloc((size_t)n * lds));
    if (grouped)
      LD_TRY(sketch_assemble_cols<T>(vst_ext, n, lds, vst_ld, m, w.p, Y64.p, lds, st));
    else
      LD_TRY(sketch_assemble<T>(Vst.p, n, lds, m, w.p, Y64.p, lds, st));
    LD_CUDA(cudaMemcpyAsync(h_status1, r1.ks.status.p, sizeof(uint32_t) * lds, cudaMemcpyDeviceToHost, st));
    if (r1.dia_err.p)
      LD_CUDA(cudaMemcpyAsync(h_err, r1.dia_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    run.reset();
    Vst.release();
    cc.release();
    ws.release();
    w.release();
    LD_TRY(hutchpp_split(n, s, r, Y64.p, lds, probe_key(c.seed, 1), X64, ld, keep.p, st, c.gaussian,
                             dkey(1)));
    Y64.release();
    T* X0;
    LD_TRY(make_x0(&X0));
    run.reset(new KRun<T>(st));
    run->colshift = cshift.p;
    run->hctx = h;
    run->gtab = gtabs.p;
    run->diavals = diav.p;
    TuneCfg tc;
    LD_TRY(layout(ld, true, &tc));
    LD_TRY(start_run(b, ld, kk, 1, true, X0, nullptr, tc));
    ph = PH_K2;
    return LOGDET_OK;
  }

  int finish() {
    KRun<T>& rr = *run;
    LD_TRY(outv.alloc(ld));
    if (c.method == 0) {
      LD_TRY(gauss_quadrature_log(rr.ks.alpha.p, rr.ks.beta.p, m, rr.ks.meff.p, m, ld, lo / alpha,
                                  outv.p, rr.ks.status.p, st));
    } else {
      DevBuf<double> cc(st), ws(st);
      LD_TRY(cc.alloc((size_t)ld * m));
      LD_TRY(ws.alloc(hesslog_workspace_doubles(m, ld, kk - 1)));
      LD_TRY(hessenberg_log_e1(rr.ks.H.p, m + 1, rr.ks.meff.p, m, ld, cc.p, m, ws.p, rr.ks.status.p,
                               st, kk - 1));
      ProfScope prof(KC_SMALL, st);
      k_iop_qf<<<div_up(ld, 64), 64, 0, st>>>(cc.p, m, rr.ks.sig.p, rr.ks.edot.p, rr.ks.meff.p, m,
                                               ld, shift, outv.p);
      LD_CHECK_LAUNCH();
    }
    LD_CUDA(cudaMemcpyAsync(h_out, outv.p, sizeof(double) * ld, cudaMemcpyDeviceToHost, st));
    LD_CUDA(cudaMemcpyAsync(h_meff, rr.ks.meff.p, sizeof(int) * ld, cudaMemcpyDeviceToHost, st));
    LD_CUDA(cudaMemcpyAsync(h_status, rr.ks.status.p, sizeof(uint32_t) * ld, cudaMemcpyDeviceToHost, st));
    if (rr.dia_err.p)
      LD_CUDA(cudaMemcpyAsync(h_err + 1, rr.dia_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LD_CUDA(cudaMemcpyAsync(h_edot, rr.ks.edot.p, sizeof(double) * ld * (m + 2), cudaMemcpyDeviceToHost, st));
    if (s > 0) LD_CUDA(cudaMemcpyAsync(h_keep, keep.p, sizeof(int) * s, cudaMemcpyDeviceToHost, st));
    if (!ev_done) LD_CUDA(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming));
    LD_CUDA(cudaEventRecord(ev_done, st));
    // Device buffers are released in stream order; the copies above read them first.
    run.reset();
    vals.release();
    gtabs.release();
    diav.release();
    cshift.release();
    X64.release();
    Xc.release();
    outv.release();
    keep.release();
    ph = PH_WAIT;
    return LOGDET_OK;
  }

  int run_phase() override {
    NvtxRange nv(ph == PH_SETUP ? "logdet setup" : ph == PH_MID ? "logdet mid" : "logdet finish");
    int rc = LOGDET_OK;
    if (ph == PH_SETUP) rc = setup();
    else if (ph == PH_MID) rc = mid();
    else if (ph == PH_FINISH) rc = finish();
    if (rc) ph = PH_FAILED;
    return rc;
  }

  int add_pass1(void* vec, std::vector<ScalarJob>& coef, std::vector<int>& widths) override {
    auto& v = *static_cast<std::vector<SpmmJob<T>>*>(vec);
    const int j = run->next_step();
    if (h->kind == 1) LD_TRY(run->grid_pass1(j));
    else LD_TRY(run->spmm_jobs(j, v));
    coef.push_back(run->scalar_job(j, run->pass1_dots(j), true));
    widths.push_back(run->ld);
    return LOGDET_OK;
  }

  bool add_pass2(void* vec, std::vector<ScalarJob>& norm, std::vector<int>& widths) override {
    const int j = run->next_step();
    if (!run->has_pass2(j)) return false;
    auto& v = *static_cast<std::vector<UpdJob<T>>*>(vec);
    run->upd_jobs(j, v);
    norm.push_back(run->scalar_job(j, run->track_e ? 2 : 1));
    widths.push_back(run->ld);
    return true;
  }

  void step_issued() override {
    run->done_steps++;
    if (run->finished()) ph = (c.method == 1 && ph == PH_K1) ? PH_MID : PH_FINISH;
  }

  int issue_krylov_rest() override {
    if (!run || !run->persistent_ok()) return 1;
    NvtxRange nv("logdet persistent krylov run");
    const int rc = run->issue_rest_persistent();
    if (rc) {
      ph = PH_FAILED;
      return rc;
    }
    ph = (c.method == 1 && ph == PH_K1) ? PH_MID : PH_FINISH;
    return LOGDET_OK;
  }

  int assemble(SolveOut& o) override {
    memset(&o.res, 0, sizeof o.res);
    if (h_err && (h_err[0] || h_err[1])) {
      set_error("a bounded device wait gave up (a staged copy of the diagonal SpMM path, or "
                "a grid barrier of the persistent Krylov run)");
      return LOGDET_ETIMEOUT;
    }
    uint32_t status = 0;
    int s_eff = 0;
    for (int i = 0; i < s; ++i) s_eff += h_keep[i] != 0;
    if (s_eff < s) status |= LOGDET_ST_RANK_DEFICIENT;
    int smin = 1 << 30, smax = 0;
    for (int p = 0; p < b; ++p) {
      status |= h_status[p];
      if (h_meff[p] > 0) {
        smin = std::min(smin, h_meff[p]);
        smax = std::max(smax, h_meff[p]);
      }
    }
    if (c.method == 1)
      for (int p = 0; p < s; ++p) status |= h_status1[p];
    if (smax == 0) smin = 0;
    double tr_sub = 0.0, tr_res = 0.0;
    o.per_probe.assign(b, 0.0);
    o.zn2.assign(r, 0.0);
    for (int i = 0; i < s; ++i) {
      o.per_probe[i] = h_out[i];
      tr_sub += h_out[i];
    }
    for (int j = 0; j < r; ++j) {
      const double z2 = h_edot[(size_t)(s + j) * (m + 2) + 1];
      o.zn2[j] = z2;
      if (c.method == 0) {
        o.per_probe[s + j] = h_out[s + j];
        tr_res += z2 * h_out[s + j];
      } else {
        o.per_probe[s + j] = z2 > 0.0 ? h_out[s + j] / z2 : 0.0;
        tr_res += h_out[s + j];
      }
    }
    tr_res /= r;
    logdet_result& R = o.res;
    R.log_alpha = std::log(alpha);
    R.log_gamma = c.method == 0 ? 0.0 : std::log(gamma);
    R.tr_sub = tr_sub;
    R.tr_res = tr_res;
    R.logdet = n * R.log_alpha + tr_sub + tr_res;
    R.s = s;
    R.r = r;
    R.s_eff = s_eff;
    R.steps_min = smin;
    R.steps_max = smax;
    R.status_bits = status;
    ph = PH_DONE;
    return LOGDET_OK;
  }
};

size_t estimate_solve_bytes(const logdet_ctx* h, const SolveCfg& c) {
  const bool f32 = c.precision != LOGDET_FP64;  // FP32 matrix values
  const bool b16 = c.precision == LOGDET_MIXED_BF16VEC;
  const bool df = c.precision == LOGDET_MIXED_F32X2;
  const size_t es = b16 ? 2 : (f32 && !df) ? 4 : 8;
  const int vec = precision_vec(c.precision);
  const size_t n = h->n;
  const int s = c.plain ? 0 : c.P / 3, r = c.plain ? c.P : c.P - 2 * s, b = s + r;
  const size_t ld = round_up(b, vec), lds = std::max(round_up(s, vec), vec);
  const int m = c.m, k = c.method == 0 ? 2 : std::min(c.k, c.m);
  // Scaled values, plus (FP32 blocks of a grid stencil) the values per row
  // and diagonal of the sweep paths.
  const bool sweep_vals = f32 && !b16 && !df && h->kind == 0 && h->dia.ndiag > 0 && h->dia_slot;
  const size_t vals = (h->kind == 1 ? grid_table_count(h) * 8 : (size_t)h->nnz * (f32 ? 4 : 8)) +
                      (sweep_vals ? (size_t)dia_pad(h->dia.ndiag) * n * 4 : 0);
  const TileGeom g = tile_geom((int)ld, vec, 0, 0, (int)n);
  const size_t ntiles = div_up((int)n, g.tile_rows);
  const size_t part = (size_t)std::max(k, 2) * ld * ntiles * (f32 ? 8 : 8);
  const size_t kstate = ld * (m + 2) * 8 * 4 + ld * (size_t)(m + 1) * m * 8 + 64 * ld;
  const size_t split = n * ld * 8 + 8 * std::max(orth_workspace_doubles((int)n, s),
                                                 project_workspace_doubles((int)n, s, r));
  size_t peak;
  if (c.method == 0) {
    const size_t setup = 2 * n * lds * es + (f32 ? n * lds * 8 : 0) + split;
    const size_t krylov = (f32 ? n * ld * es : n * ld * 8) + part + n * ld * es * 4 + kstate;
    peak = vals + std::max(setup, krylov + (f32 ? 0 : 0));
  } else {
    const size_t phase1 = n * lds * m * es + part + n * lds * es + kstate +
                          hesslog_workspace_doubles(m, (int)lds, k - 1) * 8 + n * lds * 8;
    const size_t phase2 = (f32 ? n * ld * es : n * ld * 8) + part + n * ld * es * (k + 2) + kstate +
                          hesslog_workspace_doubles(m, (int)ld, k - 1) * 8;
    peak = vals + std::max(phase1, std::max(split + n * lds * 8, phase2));
  }
  return peak + (16u << 20);
}

std::unique_ptr<ISolve> make_solve(logdet_ctx* h, const SolveCfg& c, cudaStream_t st, int* rc) {
  *rc = validate_cfg(h, c);
  if (*rc) return nullptr;
  if (c.precision == LOGDET_FP64) return std::unique_ptr<ISolve>(new Solve<double>(h, c, st));
  if (c.precision == LOGDET_MIXED_BF16VEC) return std::unique_ptr<ISolve>(new Solve<bf16>(h, c, st));
  if (c.precision == LOGDET_MIXED_F32X2) return std::unique_ptr<ISolve>(new Solve<f32x2>(h, c, st));
  return std::unique_ptr<ISolve>(new Solve<float>(h, c, st));
}

SolveCfg make_solve_cfg(int method, int32_t P, int32_t m, int32_t k, uint64_t seed,
                        const logdet_opts* opts) {
  SolveCfg c;
  c.method = method;
  c.P = P;
  c.m = m;
  c.k = k;
  c.seed = seed;
  if (opts) {
    c.precision = opts->precision;
    c.tol = opts->tol > 0.0 ? opts->tol : kDefaultTol;
    c.lam_lo = opts->lambda_lo;
    c.lam_hi = opts->lambda_hi;
    c.shift = opts->shift;
    c.autotune = opts->autotune;
    c.plain = opts->plain_slq;
    c.gaussian = opts->gaussian_probes;
    c.block_width = opts->block_width;
  }
  return c;
}

// ---------------------------------------------------------------------------
// Several diagonal shifts of one matrix in lockstep
// ---------------------------------------------------------------------------
// The Krylov phases of the members run as one run over a wide block: member
// t owns columns [t w, (t + 1) w) (w its block width); the values are member
// 0's (Q / c_0), and column p of member t is scaled by c_0 / c_t after the
// shift sigma_t / c_0, so y = (Q + sigma_t I) x / c_t as in the member's own
// run.  Everything else of a member's solve (sketch, Hutch++ split, small
// solves, assembly) is its own.  One gather of the SpMM pass then fetches
// the x row of every member at once.  GroupSolve is the resumable form: the
// blocking call drives it with issue_solve, the server steps it like any
// other solve.
template <typename T>
struct GroupSolve : ISolve {
  logdet_ctx* h;
  cudaStream_t st;
  std::vector<std::unique_ptr<Solve<T>>> ms;
  std::unique_ptr<KRun<T>> w;  // the wide run of the current Krylov phase
  DevBuf<T> Vw, Xw;            // phase-1 basis (OSA-IOP) or start block of the wide run
  DevBuf<double> csc, csh;     // per-column scale c_0 / c_t and shift s_t / c_0
  int ph = PH_SETUP;
  bool phase1 = false;
  int wm = 0, ldw = 0;

  GroupSolve(logdet_ctx* h_, const std::vector<SolveCfg>& cfgs, cudaStream_t st_)
      : h(h_), st(st_), Vw(st_), Xw(st_), csc(st_), csh(st_) {
    for (const SolveCfg& c : cfgs) {
      ms.emplace_back(new Solve<T>(h_, c, st_));
      ms.back()->grouped = true;
    }
  }

  int phase() const override { return ph; }
  bool in_krylov() const override { return ph == PH_K1 || ph == PH_K2; }
  int krylov_threads() const override { return w ? w->g.threads : 0; }
  bool is_fp32() const override { return !std::is_same<T, double>::value; }
  int elem_kind() const override { return ms[0]->elem_kind(); }
  cudaEvent_t done_event() const override { return ms.back()->done_event(); }
  size_t bytes_estimate() const override {
    size_t b = 0;
    for (const auto& m : ms) b += m->bytes_estimate();
    return b;
  }
  void set_dev_keys(const uint64_t*) override {}
  int prepare_host() override {
    for (auto& m : ms) LD_TRY(m->prepare_host());
    return LOGDET_OK;
  }
  int suspend() override {
    set_error("shift groups are not suspended");
    return LOGDET_EINVAL;
  }
  int resume() override { return LOGDET_OK; }
  bool suspended() const override { return false; }
  int issue_krylov_rest() override { return 1; }
  int members() const override { return (int)ms.size(); }
  int assemble(SolveOut& o) override { return ms[0]->assemble(o); }
  int assemble_member(int t, SolveOut& o) override { return ms[t]->assemble(o); }

  // Every member's current non-Krylov phase; when they all wait for the
  // group, the wide run of the next Krylov phase starts.
  int run_phase() override {
    const int rc = step_members();
    if (rc) ph = PH_FAILED;
    return rc;
  }

  int step_members() {
    for (auto& m : ms)
      if (m->ph == PH_SETUP || m->ph == PH_MID || m->ph == PH_FINISH) LD_TRY(m->run_phase());
    for (auto& m : ms)
      if (m->ph == PH_FAILED) return LOGDET_ECUDA;
    if (ms[0]->ph == PH_WAIT) {
      for (auto& m : ms)
        if (m->ph != PH_WAIT) {
          set_error("shift group: members out of step");
          return LOGDET_ECUDA;
        }
      ph = PH_WAIT;
      return LOGDET_OK;
    }
    // every mid (OSA-IOP) has read the phase-1 basis: it goes in stream order
    Vw.release();
    return start_wide();
  }

  int start_wide() {
    const int R = (int)ms.size();
    Solve<T>& m0 = *ms[0];
    phase1 = m0.c.method == 1 && m0.ph == PH_K1;
    wm = m0.pend_ld;
    ldw = R * wm;
    const int n = m0.n, m = m0.m;
    const int method = m0.c.method == 0 ? 0 : 1;
    const bool track_e = m0.c.method == 1 && !phase1;
    for (auto& sv : ms)
      if (!sv->awaiting || sv->ph != m0.ph || sv->pend_ld != wm || sv->pend_b != m0.pend_b) {
        set_error("shift group: members out of step");
        return LOGDET_EINVAL;
      }
    T* X0w;
    if (phase1) {
      LD_TRY(Vw.alloc((size_t)n * ldw * m));
      X0w = Vw.p;
    } else {
      LD_TRY(Xw.alloc((size_t)n * ldw));
      X0w = Xw.p;
    }
    for (int t = 0; t < R; ++t) {
      LD_CUDA(cudaMemcpy2DAsync(X0w + (size_t)t * wm, sizeof(T) * ldw, ms[t]->pend_x0, sizeof(T) * wm,
                                sizeof(T) * wm, n, cudaMemcpyDeviceToDevice, st));
      ms[t]->release_start();
    }
    std::vector<double> hsc((size_t)ldw), hsh((size_t)ldw);
    const double c0 = m0.cscale();
    for (int t = 0; t < R; ++t)
      for (int q = 0; q < wm; ++q) {
        hsc[(size_t)t * wm + q] = c0 / ms[t]->cscale();
        hsh[(size_t)t * wm + q] = ms[t]->c.shift / c0;
      }
    LD_TRY(csc.alloc(ldw));
    LD_TRY(csh.alloc(ldw));
    LD_CUDA(cudaMemcpyAsync(csc.p, hsc.data(), sizeof(double) * ldw, cudaMemcpyHostToDevice, st));
    LD_CUDA(cudaMemcpyAsync(csh.p, hsh.data(), sizeof(double) * ldw, cudaMemcpyHostToDevice, st));
    // (the host arrays must outlive the copies: the copies are pageable, so
    // they complete before cudaMemcpyAsync returns)
    w.reset(new KRun<T>(st));
    w->colshift = csh.p;
    w->colscale = csc.p;
    w->hctx = h;
    w->diavals = m0.diav.p;
    TuneCfg tc;
    LD_TRY(m0.layout(ldw, track_e, &tc));
    LD_TRY(w->init(h->rowptr, h->colind, m0.vals.p, n, h->nnz, ldw, ldw, m, m0.kk, method, track_e,
                   X0w, phase1 ? Vw.p : nullptr, m0.c.tol, tc));
    if (m0.pend_b < wm)  // each member's padding columns stay out of the run, as in its own
      for (int t = 0; t < R; ++t)
        LD_CUDA(cudaMemsetAsync(w->ks.active.p + (size_t)t * wm + m0.pend_b, 0,
                                sizeof(*w->ks.active.p) * (wm - m0.pend_b), st));
    ph = m0.ph;  // PH_K1 or PH_K2
    return LOGDET_OK;
  }

  int add_pass1(void* vec, std::vector<ScalarJob>& coef, std::vector<int>& widths) override {
    auto& v = *static_cast<std::vector<SpmmJob<T>>*>(vec);
    const int j = w->next_step();
    LD_TRY(w->spmm_jobs(j, v));
    coef.push_back(w->scalar_job(j, w->pass1_dots(j), true));
    widths.push_back(w->ld);
    return LOGDET_OK;
  }

  bool add_pass2(void* vec, std::vector<ScalarJob>& norm, std::vector<int>& widths) override {
    const int j = w->next_step();
    if (!w->has_pass2(j)) return false;
    auto& v = *static_cast<std::vector<UpdJob<T>>*>(vec);
    w->upd_jobs(j, v);
    norm.push_back(w->scalar_job(j, w->track_e ? 2 : 1));
    widths.push_back(w->ld);
    return true;
  }

  void step_issued() override {
    w->done_steps++;
    if (!w->finished()) return;
    // every member takes its probes' scalar history back
    for (int t = 0; t < (int)ms.size(); ++t) {
      if (ms[t]->adopt(*w, t * wm)) {
        ph = PH_FAILED;
        return;
      }
      if (phase1) {
        ms[t]->vst_ext = Vw.p + (size_t)t * wm;
        ms[t]->vst_ld = ldw;
      }
    }
    w.reset();
    Xw.release();
    csc.release();
    csh.release();
    ph = ms[0]->ph;  // PH_MID or PH_FINISH
  }
};

template <typename T>
static int solve_shifts_t(logdet_ctx* h, const std::vector<SolveCfg>& cfgs, cudaStream_t st,
                          std::vector<SolveOut>& outs) {
  GroupSolve<T> g(h, cfgs, st);
  LD_TRY(issue_solve(&g, st));
  LD_CUDA(cudaEventSynchronize(g.done_event()));
  outs.resize(cfgs.size());
  for (int t = 0; t < g.members(); ++t) LD_TRY(g.assemble_member(t, outs[t]));
  return LOGDET_OK;
}

int shift_runs(logdet_ctx* h, const std::vector<SolveCfg>& cfgs,
               std::vector<std::pair<size_t, size_t>>& runs) {
  runs.clear();
  if (cfgs.empty()) {
    set_error("shift group: no shifts");
    return LOGDET_EINVAL;
  }
  if (h->kind == 1) {
    set_error("shift group: gridded operators take one shift per solve");
    return LOGDET_EINVAL;
  }
  for (const SolveCfg& c : cfgs) LD_TRY(validate_cfg(h, c));
  // Members per run: at most kMaxGroupWidth block columns, and (about R
  // solves' device memory) at most 85 % of the device's memory.  The split
  // depends only on the shapes and the device, so results do not depend on
  // what else is allocated.
  const int vec = precision_vec(cfgs[0].precision);
  const int s = cfgs[0].plain ? 0 : cfgs[0].P / 3, r = cfgs[0].plain ? cfgs[0].P : cfgs[0].P - 2 * s;
  const int width = std::max(round_up(s + r, vec), std::max(round_up(s, vec), vec));
  size_t free_b = 0, total_b = 0;
  LD_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t each = estimate_solve_bytes(h, cfgs[0]);
  const size_t by_mem = std::max<size_t>(1, (size_t)(0.85 * (double)total_b) / std::max<size_t>(each, 1));
  const int cap = (int)std::max<size_t>(1, std::min<size_t>(kMaxGroupWidth / width, by_mem));
  const int nruns = div_up((int)cfgs.size(), cap);
  const size_t per_run = (size_t)div_up((int)cfgs.size(), nruns);  // balanced runs
  for (size_t t0 = 0; t0 < cfgs.size(); t0 += per_run)
    runs.push_back({t0, std::min(cfgs.size(), t0 + per_run)});
  return LOGDET_OK;
}

std::unique_ptr<ISolve> make_group_solve(logdet_ctx* h, const std::vector<SolveCfg>& cfgs,
                                         cudaStream_t st, int* rc) {
  *rc = LOGDET_OK;
  if (cfgs.empty()) {
    *rc = LOGDET_EINVAL;
    return nullptr;
  }
  if (cfgs[0].precision == LOGDET_FP64)
    return std::unique_ptr<ISolve>(new GroupSolve<double>(h, cfgs, st));
  if (cfgs[0].precision == LOGDET_MIXED_BF16VEC)
    return std::unique_ptr<ISolve>(new GroupSolve<bf16>(h, cfgs, st));
  if (cfgs[0].precision == LOGDET_MIXED_F32X2)
    return std::unique_ptr<ISolve>(new GroupSolve<f32x2>(h, cfgs, st));
  return std::unique_ptr<ISolve>(new GroupSolve<float>(h, cfgs, st));
}

int solve_shifts(logdet_ctx* h, const std::vector<SolveCfg>& cfgs, cudaStream_t st,
                 std::vector<SolveOut>& outs) {
  std::vector<std::pair<size_t, size_t>> runs;
  LD_TRY(shift_runs(h, cfgs, runs));
  outs.clear();
  for (const auto& rg : runs) {
    const std::vector<SolveCfg> part(cfgs.begin() + rg.first, cfgs.begin() + rg.second);
    std::vector<SolveOut> po;
    int rc;
    if (cfgs[0].precision == LOGDET_FP64) rc = solve_shifts_t<double>(h, part, st, po);
    else if (cfgs[0].precision == LOGDET_MIXED_BF16VEC) rc = solve_shifts_t<bf16>(h, part, st, po);
    else if (cfgs[0].precision == LOGDET_MIXED_F32X2) rc = solve_shifts_t<f32x2>(h, part, st, po);
    else rc = solve_shifts_t<float>(h, part, st, po);
    if (rc) {
      cudaStreamSynchronize(st);
      return rc;
    }
    for (SolveOut& o : po) outs.push_back(std::move(o));
  }
  return LOGDET_OK;
}

// The blocking path: one solve advanced step by step with batches of one.
int solve_blocking(logdet_ctx* h, const SolveCfg& c, cudaStream_t st, SolveOut& o) {
  int rc = LOGDET_OK;
  std::unique_ptr<ISolve> sv = make_solve(h, c, st, &rc);
  if (!sv) return rc;
  rc = issue_solve(sv.get(), st);
  if (rc) {
    cudaStreamSynchronize(st);
    return rc;
  }
  LD_CUDA(cudaEventSynchronize(sv->done_event()));
  return sv->assemble(o);
}

// One Krylov step of a solve whose blocks hold T: pass 1, its scalar
// kernel, then (where the step has one) pass 2 and its scalar kernel.
template <typename T>
static int issue_step_t(ISolve* sv, int th, cudaStream_t st) {
  thread_local std::vector<SpmmJob<T>> sp;
  thread_local std::vector<UpdJob<T>> up;
  thread_local std::vector<ScalarJob> sj;
  thread_local std::vector<int> widths;
  sp.clear(); up.clear(); sj.clear(); widths.clear();
  LD_TRY(sv->add_pass1(&sp, sj, widths));
  LD_TRY(launch_spmm_jobs<T>(sp, th, st));
  LD_TRY(launch_scalar_jobs(sj, widths, SK_COEF, st));
  sj.clear(); widths.clear();
  if (sv->add_pass2(&up, sj, widths)) {
    LD_TRY(launch_update_jobs<T>(up, th, st));
    LD_TRY(launch_scalar_jobs(sj, widths, SK_NORM, st));
  }
  return LOGDET_OK;
}

int issue_solve(ISolve* sv, cudaStream_t st) {
  int rc = LOGDET_OK;
  while (sv->phase() != PH_WAIT) {
    if (sv->phase() == PH_FAILED) return rc ? rc : LOGDET_ECUDA;
    if (!sv->in_krylov()) {
      rc = sv->run_phase();
      if (rc) return rc;
      continue;
    }
    {
      // Small runs: every remaining step in one persistent launch.
      const int pr = sv->issue_krylov_rest();
      if (pr < 0) return pr;
      if (pr == 0) continue;
    }
    NvtxRange nv("logdet krylov step");
    const int th = sv->krylov_threads();
    switch (sv->elem_kind()) {
      case 0: LD_TRY(issue_step_t<double>(sv, th, st)); break;
      case 1: LD_TRY(issue_step_t<float>(sv, th, st)); break;
      case 2: LD_TRY(issue_step_t<bf16>(sv, th, st)); break;
      default: LD_TRY(issue_step_t<f32x2>(sv, th, st)); break;
    }
    sv->step_issued();
  }
  return LOGDET_OK;
}

}  // namespace ld
