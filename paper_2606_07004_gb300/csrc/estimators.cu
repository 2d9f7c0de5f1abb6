// OSLQ (Algorithm 3) and OSA-IOP (Algorithm 2 with Algorithm 1) on the
// device, and the C-ABI of liblogdet.
#include "dense.cuh"
#include "handle.cuh"
#include "krylov.cuh"
#include "profile.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace ld {

constexpr double kDefaultTol = 1e-12;
constexpr double kClampRel = 1e-6;  // lambda_lo = 1e-6 * lambda_hi when Gershgorin's lo <= 0

struct SolveCfg {
  int method = 0;  // 0 OSLQ, 1 OSA-IOP
  int P = 0, m = 0, k = 2;
  uint64_t seed = 0;
  double tol = kDefaultTol;
  double lam_lo = 0.0, lam_hi = 0.0;
  int precision = LOGDET_FP64;
};

struct SolveOut {
  logdet_result res;
  std::vector<double> per_probe;  // s + r
  std::vector<double> zn2;        // r
};

// Device arrays of one Krylov run (see KrylovState).
struct KState {
  DevBuf<double> alpha, beta, H, sig, edot, coef, ycoef;
  DevBuf<int> meff, active;
  DevBuf<uint32_t> status, cnt;
  DevBuf<double> dbuf;
  KrylovState st{};
  explicit KState(cudaStream_t s)
      : alpha(s), beta(s), H(s), sig(s), edot(s), coef(s), ycoef(s), meff(s), active(s), status(s),
        cnt(s), dbuf(s) {}
  int alloc(int method, int b, int ld, int m, int k, double tol, double rescale_lim) {
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
    LD_TRY(meff.alloc(ld));
    LD_TRY(active.alloc(ld));
    LD_TRY(status.alloc(ld));
    LD_TRY(cnt.alloc(ld));
    LD_TRY(dbuf.alloc((size_t)kMaxWin * ld));
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
};

template <typename T> constexpr double rescale_limit();
template <> constexpr double rescale_limit<double>() { return 200.0; }
template <> constexpr double rescale_limit<float>() { return 20.0; }

// Run m Krylov steps on the block X0 (n x ld, b live columns).  method 0:
// three-term Lanczos (window fixed at 2); method 1: IOP with window k.  With
// Vfull non-null the basis is kept: u_j = Vfull + (j-1)*n*ld and X0 == Vfull.
// track_e: accumulate u_1^T u_j for the OSA-IOP quadratic forms.
template <typename T>
int krylov_block(const int* rowptr, const int* colind, const T* vals, int n, long long nnz, int b,
                 int ld, int m, int k, int method, bool track_e, T* X0, T* Vfull, KState& ks,
                 cudaStream_t st) {
  using Part = typename PartOf<T>::type;
  constexpr bool f32 = std::is_same<T, float>::value;
  const TileGeom g = tile_geom(ld, Vec16<T>::N);
  const int ntiles = div_up(n, g.tile_rows);
  const size_t blk = (size_t)n * ld;
  const int win = method == 0 ? 2 : k;
  const int ndmax = std::max(win, 2);
  if (win > kMaxWin - 1 && method == 1) {
    set_error("iop_window %d exceeds the supported maximum %d", k, kMaxWin - 1);
    return LOGDET_EINVAL;
  }
  DevBuf<Part> part(st);
  DevBuf<T> y(st), ring(st);
  LD_TRY(part.alloc((size_t)ndmax * ld * ntiles));
  LD_TRY(y.alloc(blk));
  const int nring = win + 1;
  if (!Vfull) LD_TRY(ring.alloc(blk * nring));
  auto ptr = [&](int i) -> T* {
    if (Vfull) return Vfull + (size_t)(i - 1) * blk;
    if (i == 1) return X0;
    return ring.p + (size_t)((i - 2) % nring) * blk;
  };

  ScalarBatch sb;
  memset(&sb, 0, sizeof sb);
  sb.njobs = 1;
  sb.probe_start[0] = 0;
  sb.probe_start[1] = ld;
  ScalarJob& sj = sb.jobs[0];
  sj.st = ks.st;
  sj.part = part.p;
  sj.part_f32 = f32 ? 1 : 0;
  sj.ntiles = ntiles;

  LD_TRY(colnorm_partials<T>(X0, n, ld, g.tile_rows, ntiles, part.p, g.threads, st));
  sj.ndots = 1;
  LD_TRY(launch_init_sigma(sb, st));

  SpmmBatch<T> pb;
  memset(&pb, 0, sizeof pb);
  pb.njobs = 1;
  pb.tile_start[0] = 0;
  pb.tile_start[1] = ntiles;
  pb.total_tiles = ntiles;
  SpmmJob<T>& pj = pb.jobs[0];
  pj.rowptr = rowptr;
  pj.colind = colind;
  pj.vals = vals;
  pj.y = y.p;
  pj.part = part.p;
  pj.n = n;
  pj.ld = ld;
  pj.b = b;
  pj.nnz = nnz;
  pj.tile_rows = g.tile_rows;
  pj.ntiles = ntiles;

  UpdBatch<T> ub;
  memset(&ub, 0, sizeof ub);
  ub.njobs = 1;
  ub.tile_start[0] = 0;
  ub.tile_start[1] = ntiles;
  ub.total_tiles = ntiles;
  UpdJob<T>& uj = ub.jobs[0];
  uj.y = y.p;
  uj.coef = ks.coef.p;
  uj.ycoef = ks.ycoef.p;
  uj.extra = track_e ? X0 : nullptr;
  uj.part = part.p;
  uj.n = n;
  uj.ld = ld;
  uj.b = b;
  uj.tile_rows = g.tile_rows;
  uj.ntiles = ntiles;

  for (int j = 1; j <= m; ++j) {
    const int win_lo = method == 0 ? j : std::max(1, j - k + 1);
    // pass 1
    pj.x = ptr(j);
    if (method == 0) {
      pj.ndots = 1;
      pj.dotv[0] = ptr(j);
    } else {
      pj.ndots = j - win_lo + 1;
      for (int i = win_lo; i <= j; ++i) pj.dotv[i - win_lo] = ptr(i);
    }
    LD_TRY(launch_spmm<T>(pb, g.threads, st));
    sj.step = j;
    sj.ndots = pj.ndots;
    sj.win_lo = win_lo;
    sj.last = j == m;
    LD_TRY(launch_coef(sb, st));
    if (j == m) break;
    // pass 2
    if (method == 0) {
      if (j >= 2) {
        uj.nbasis = 2;
        uj.basis[0] = ptr(j - 1);
        uj.basis[1] = ptr(j);
      } else {
        uj.nbasis = 1;
        uj.basis[0] = ptr(j);
      }
    } else {
      uj.nbasis = j - win_lo + 1;
      for (int i = win_lo; i <= j; ++i) uj.basis[i - win_lo] = ptr(i);
    }
    uj.out = ptr(j + 1);
    LD_TRY(launch_update<T>(ub, g.threads, st));
    sj.ndots = track_e ? 2 : 1;
    LD_TRY(launch_norm(sb, st));
  }
  return LOGDET_OK;
}

// OSA-IOP sketch weights: w[j][p] = |s_p| c_j sigma_j (+ shift for j = 1).
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

// OSA-IOP quadratic form x^T L x = |x| sum_j c_j sigma_j (u_1^T u_j) + shift |x|^2.
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

static void spectral_bounds(const logdet_ctx* h, const SolveCfg& c, double& lo, double& hi) {
  if (c.lam_lo > 0.0 && c.lam_hi > 0.0) {
    lo = c.lam_lo;
    hi = c.lam_hi;
    return;
  }
  hi = h->g_hi;
  lo = h->g_lo > 0.0 ? h->g_lo : kClampRel * hi;
}

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

template <typename T>
static int to_block(const double* X64, int ld, int n, DevBuf<T>& out, cudaStream_t st) {
  LD_TRY(out.alloc((size_t)n * ld));
  return convert_block<double, T>(X64, ld, out.p, ld, n, ld, st);
}

// Hutch++ split shared by both estimators: A = orth(Y) into X64[:, 0:s],
// Z = G - A A^T G into X64[:, s:s+r].
static int hutchpp_split(int n, int s, int r, const double* Y64, int lds, uint64_t key_g,
                         DevBuf<double>& X64, int ld, int* s_eff, uint32_t* status, cudaStream_t st) {
  LD_TRY(X64.alloc((size_t)n * ld));
  LD_TRY(X64.zero());
  DevBuf<double> ws(st);
  DevBuf<int> keep(st);
  LD_TRY(ws.alloc(std::max(orth_workspace_doubles(n, s), project_workspace_doubles(n, s, r))));
  LD_TRY(keep.alloc(s));
  LD_TRY(orth_fp64(n, s, Y64, lds, X64.p, ld, ws.p, keep.p, s_eff, st));
  if (*s_eff < s) *status |= LOGDET_ST_RANK_DEFICIENT;
  LD_TRY(project_residual_fp64(n, s, r, X64.p, ld, key_g, X64.p, ld, s, ws.p, st));
  return LOGDET_OK;
}

template <typename T>
static int collect(const KState& ks, int b, int ld, int m, const double* dev_vals,
                   std::vector<double>& vals, std::vector<double>& e1, uint32_t& status,
                   int& smin, int& smax, cudaStream_t st) {
  std::vector<int> meff(ld);
  std::vector<uint32_t> stt(ld);
  std::vector<double> ed((size_t)ld * (m + 2));
  vals.resize(ld);
  LD_CUDA(cudaMemcpyAsync(vals.data(), dev_vals, sizeof(double) * ld, cudaMemcpyDeviceToHost, st));
  LD_CUDA(cudaMemcpyAsync(meff.data(), ks.meff.p, sizeof(int) * ld, cudaMemcpyDeviceToHost, st));
  LD_CUDA(cudaMemcpyAsync(stt.data(), ks.status.p, sizeof(uint32_t) * ld, cudaMemcpyDeviceToHost, st));
  LD_CUDA(cudaMemcpyAsync(ed.data(), ks.edot.p, sizeof(double) * ld * (m + 2), cudaMemcpyDeviceToHost, st));
  LD_CUDA(cudaStreamSynchronize(st));
  e1.resize(ld);
  smin = 1 << 30;
  smax = 0;
  for (int p = 0; p < ld; ++p) {
    e1[p] = ed[(size_t)p * (m + 2) + 1];
    if (p < b) {
      status |= stt[p];
      if (meff[p] > 0) {
        smin = std::min(smin, meff[p]);
        smax = std::max(smax, meff[p]);
      }
    }
  }
  if (smax == 0) smin = 0;
  return LOGDET_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 3 (OSLQ)
// ---------------------------------------------------------------------------
template <typename T>
int oslq_impl(logdet_ctx* h, const SolveCfg& c, SolveOut& o, cudaStream_t st) {
  const int n = h->n, s = c.P / 3, r = c.P - 2 * (c.P / 3), b = s + r;
  const int V = Vec16<T>::N;
  const int ld = round_up(b, V), lds = round_up(s, V);
  double lo, hi;
  spectral_bounds(h, c, lo, hi);
  const double alpha = hi;  // J = Q / lambda_max bound
  uint32_t status = 0;
  DevBuf<T> jv(st);
  LD_TRY(jv.alloc(h->nnz));
  LD_TRY(scaled_values<T>(h, alpha, jv.p, st));
  // Sketch Y = J S.
  DevBuf<double> X64(st);
  int s_eff = 0;
  {
    DevBuf<T> S(st), Yt(st);
    LD_TRY(S.alloc((size_t)n * lds));
    LD_TRY(Yt.alloc((size_t)n * lds));
    LD_TRY(probe_fill<T>(probe_key(c.seed, 0), n, s, 0, S.p, lds, st));
    LD_TRY(spmm_block<T>(h->rowptr, h->colind, jv.p, n, S.p, Yt.p, lds, st));
    S.release();
    if constexpr (std::is_same<T, double>::value) {
      LD_TRY(hutchpp_split(n, s, r, Yt.p, lds, probe_key(c.seed, 1), X64, ld, &s_eff, &status, st));
    } else {
      DevBuf<double> Y64(st);
      LD_TRY(Y64.alloc((size_t)n * lds));
      LD_TRY((convert_block<T, double>(Yt.p, lds, Y64.p, lds, n, lds, st)));
      Yt.release();
      LD_TRY(hutchpp_split(n, s, r, Y64.p, lds, probe_key(c.seed, 1), X64, ld, &s_eff, &status, st));
    }
  }
  DevBuf<T> Xc(st);
  T* X0;
  if constexpr (std::is_same<T, double>::value) {
    X0 = X64.p;
  } else {
    LD_TRY(to_block<T>(X64.p, ld, n, Xc, st));
    X64.release();
    X0 = Xc.p;
  }
  KState ks(st);
  LD_TRY(ks.alloc(0, b, ld, c.m, 2, c.tol, rescale_limit<T>()));
  LD_TRY(krylov_block<T>(h->rowptr, h->colind, jv.p, n, h->nnz, b, ld, c.m, 2, 0, false, X0, nullptr, ks, st));
  DevBuf<double> K(st);
  LD_TRY(K.alloc(ld));
  LD_TRY(gauss_quadrature_log(ks.alpha.p, ks.beta.p, c.m, ks.meff.p, c.m, ld, lo / alpha, K.p,
                              ks.status.p, st));
  std::vector<double> Kh, e1;
  int smin, smax;
  LD_TRY(collect<T>(ks, b, ld, c.m, K.p, Kh, e1, status, smin, smax, st));
  double tr_sub = 0.0, tr_res = 0.0;
  o.per_probe.assign(b, 0.0);
  o.zn2.assign(r, 0.0);
  for (int i = 0; i < s; ++i) {
    o.per_probe[i] = Kh[i];
    tr_sub += Kh[i];
  }
  for (int j = 0; j < r; ++j) {
    o.per_probe[s + j] = Kh[s + j];
    o.zn2[j] = e1[s + j];
    tr_res += e1[s + j] * Kh[s + j];
  }
  tr_res /= r;
  logdet_result& R = o.res;
  R.log_alpha = std::log(alpha);
  R.log_gamma = 0.0;
  R.tr_sub = tr_sub;
  R.tr_res = tr_res;
  R.logdet = n * R.log_alpha + tr_sub + tr_res;
  R.s = s;
  R.r = r;
  R.s_eff = s_eff;
  R.steps_min = smin;
  R.steps_max = smax;
  R.status_bits = status;
  return LOGDET_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 2 (OSA-IOP) with Algorithm 1 for every action of L
// ---------------------------------------------------------------------------
template <typename T>
int osaiop_impl(logdet_ctx* h, const SolveCfg& c, SolveOut& o, cudaStream_t st) {
  const int n = h->n, s = c.P / 3, r = c.P - 2 * (c.P / 3), b = s + r, m = c.m, k = c.k;
  const int V = Vec16<T>::N;
  const int ld = round_up(b, V), lds = round_up(s, V);
  double lo, hi;
  spectral_bounds(h, c, lo, hi);
  const double gamma = std::sqrt(lo * hi);  // Proposition 2.1
  const double alpha = lo;
  const double shift = std::log(gamma / alpha);
  uint32_t status = 0;
  DevBuf<T> qv(st);
  LD_TRY(qv.alloc(h->nnz));
  LD_TRY(scaled_values<T>(h, gamma, qv.p, st));
  const int kk = std::min(k, m);
  // Phase 1: Y = L S, one Algorithm 1 run per sketch column, basis kept.
  DevBuf<double> Y64(st);
  {
    DevBuf<T> Vst(st);
    LD_TRY(Vst.alloc((size_t)n * lds * m));
    LD_TRY(probe_fill<T>(probe_key(c.seed, 0), n, s, 0, Vst.p, lds, st));
    KState k1(st);
    LD_TRY(k1.alloc(1, s, lds, m, kk, c.tol, rescale_limit<T>()));
    LD_TRY(krylov_block<T>(h->rowptr, h->colind, qv.p, n, h->nnz, s, lds, m, kk, 1, false, Vst.p, Vst.p,
                           k1, st));
    DevBuf<double> cc(st), ws(st), w(st);
    LD_TRY(cc.alloc((size_t)lds * m));
    LD_TRY(ws.alloc(hesslog_workspace_doubles(m, lds)));
    LD_TRY(w.alloc((size_t)m * lds));
    LD_TRY(hessenberg_log_e1(k1.H.p, m + 1, k1.meff.p, m, lds, cc.p, m, ws.p, k1.status.p, st));
    prof_count();
    k_iop_weights<<<div_up(m * lds, 256), 256, 0, st>>>(cc.p, m, k1.sig.p, k1.edot.p, k1.meff.p, m,
                                                        lds, shift, w.p);
    LD_CHECK_LAUNCH();
    LD_TRY(Y64.alloc((size_t)n * lds));
    LD_TRY(sketch_assemble<T>(Vst.p, n, lds, m, w.p, Y64.p, lds, st));
    std::vector<uint32_t> st1(lds);
    LD_CUDA(cudaMemcpyAsync(st1.data(), k1.status.p, sizeof(uint32_t) * lds, cudaMemcpyDeviceToHost, st));
    LD_CUDA(cudaStreamSynchronize(st));
    for (int p = 0; p < s; ++p) status |= st1[p];
  }
  DevBuf<double> X64(st);
  int s_eff = 0;
  LD_TRY(hutchpp_split(n, s, r, Y64.p, lds, probe_key(c.seed, 1), X64, ld, &s_eff, &status, st));
  Y64.release();
  DevBuf<T> Xc(st);
  T* X0;
  if constexpr (std::is_same<T, double>::value) {
    X0 = X64.p;
  } else {
    LD_TRY(to_block<T>(X64.p, ld, n, Xc, st));
    X64.release();
    X0 = Xc.p;
  }
  // Phase 2: quadratic forms of L on [A | Z].
  KState k2(st);
  LD_TRY(k2.alloc(1, b, ld, m, kk, c.tol, rescale_limit<T>()));
  LD_TRY(krylov_block<T>(h->rowptr, h->colind, qv.p, n, h->nnz, b, ld, m, kk, 1, true, X0, nullptr, k2, st));
  DevBuf<double> cc(st), ws(st), qf(st);
  LD_TRY(cc.alloc((size_t)ld * m));
  LD_TRY(ws.alloc(hesslog_workspace_doubles(m, ld)));
  LD_TRY(qf.alloc(ld));
  LD_TRY(hessenberg_log_e1(k2.H.p, m + 1, k2.meff.p, m, ld, cc.p, m, ws.p, k2.status.p, st));
  prof_count();
  k_iop_qf<<<div_up(ld, 64), 64, 0, st>>>(cc.p, m, k2.sig.p, k2.edot.p, k2.meff.p, m, ld, shift, qf.p);
  LD_CHECK_LAUNCH();
  std::vector<double> qh, e1;
  int smin, smax;
  LD_TRY(collect<T>(k2, b, ld, m, qf.p, qh, e1, status, smin, smax, st));
  double tr_sub = 0.0, tr_res = 0.0;
  o.per_probe.assign(b, 0.0);
  o.zn2.assign(r, 0.0);
  for (int i = 0; i < s; ++i) {
    o.per_probe[i] = qh[i];
    tr_sub += qh[i];
  }
  for (int j = 0; j < r; ++j) {
    const double z2 = e1[s + j];
    o.zn2[j] = z2;
    o.per_probe[s + j] = z2 > 0.0 ? qh[s + j] / z2 : 0.0;
    tr_res += qh[s + j];
  }
  tr_res /= r;
  logdet_result& R = o.res;
  R.log_alpha = std::log(alpha);
  R.log_gamma = std::log(gamma);
  R.tr_sub = tr_sub;
  R.tr_res = tr_res;
  R.logdet = n * R.log_alpha + tr_sub + tr_res;
  R.s = s;
  R.r = r;
  R.s_eff = s_eff;
  R.steps_min = smin;
  R.steps_max = smax;
  R.status_bits = status;
  return LOGDET_OK;
}

int solve(logdet_ctx* h, const SolveCfg& c, cudaStream_t st, SolveOut& o) {
  memset(&o.res, 0, sizeof o.res);
  if (c.P < 3) { set_error("num_probes must be >= 3"); return LOGDET_EINVAL; }
  if (c.m < 1 || c.m > h->n || c.m > kMaxSteps) {
    set_error("krylov_steps=%d must be in [1, min(n, %d)]", c.m, kMaxSteps);
    return LOGDET_EINVAL;
  }
  const int s = c.P / 3, r = c.P - 2 * s;
  if (s > kMaxSketch || r > kMaxSketch) {
    set_error("num_probes=%d: s and r must be <= %d", c.P, kMaxSketch);
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
  if (c.precision != LOGDET_FP64 && c.precision != LOGDET_MIXED_FP32) {
    set_error("precision %d unknown", c.precision);
    return LOGDET_EINVAL;
  }
  double lo, hi;
  spectral_bounds(h, c, lo, hi);
  if (!(hi > 0.0) || !(lo > 0.0) || lo > hi) {
    set_error("spectral bounds [%g, %g] invalid", lo, hi);
    return LOGDET_ENOTSPD;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) { set_error("cudaSetDevice failed"); return LOGDET_ECUDA; }
  Events ev;
  LD_CUDA(cudaEventCreate(&ev.a));
  LD_CUDA(cudaEventCreate(&ev.b));
  LD_CUDA(cudaEventRecord(ev.a, st));
  int rc;
  if (c.method == 0)
    rc = c.precision == LOGDET_FP64 ? oslq_impl<double>(h, c, o, st) : oslq_impl<float>(h, c, o, st);
  else
    rc = c.precision == LOGDET_FP64 ? osaiop_impl<double>(h, c, o, st) : osaiop_impl<float>(h, c, o, st);
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

static SolveCfg make_cfg(int method, int32_t P, int32_t m, int32_t k, uint64_t seed,
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
  }
  return c;
}

static int run_estimator(int method, logdet_handle h, int32_t P, int32_t m, int32_t k, uint64_t seed,
                         const logdet_opts* opts, logdet_result* out) {
  if (!h || !out) { set_error("NULL handle or result"); return LOGDET_EINVAL; }
  SolveCfg c = make_cfg(method, P, m, k, seed, opts);
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

void logdet_destroy(logdet_handle h) { destroy_handle(h); }

int logdet_info(logdet_handle h, int32_t* n, int64_t* nnz, double* lo, double* hi) {
  if (!h) { set_error("NULL handle"); return LOGDET_EINVAL; }
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (lo) *lo = h->g_lo;
  if (hi) *hi = h->g_hi;
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

int logdet_spmm(logdet_handle h, const double* x, double* y, int32_t b, int32_t ld, void* cuda_stream) {
  if (!h || !x || !y || b < 1 || ld < b || (ld & 1) || ((uintptr_t)x & 15) || ((uintptr_t)y & 15)) {
    set_error("spmm: need b >= 1, even ld >= b and 16-byte aligned blocks");
    return LOGDET_EINVAL;
  }
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : h->stream;
  DevBuf<double> v(st);
  const double* vals = (const double*)h->vals;
  if (h->vals_dtype != LOGDET_VALS_F64) {
    LD_TRY(v.alloc(h->nnz));
    LD_TRY(scaled_values<double>(h, 1.0, v.p, st));
    vals = v.p;
  }
  LD_TRY(spmm_block<double>(h->rowptr, h->colind, vals, h->n, x, y, ld, st));
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

int logdet_hessenberg_log_e1(const double* H, int32_t ldh, const int32_t* msteps, int32_t m,
                             int32_t nprobe, double* c, uint32_t* status, void* cuda_stream) {
  if (!H || !c || m < 1 || nprobe < 1 || ldh < m) {
    set_error("hessenberg_log_e1: bad arguments");
    return LOGDET_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<double> ws(st);
  DevBuf<uint32_t> sd(st);
  LD_TRY(ws.alloc(hesslog_workspace_doubles(m, nprobe)));
  LD_TRY(sd.alloc(nprobe));
  LD_TRY(sd.zero());
  LD_TRY(hessenberg_log_e1(H, ldh, msteps, m, nprobe, c, m, ws.p, sd.p, st));
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

}  // extern "C"
