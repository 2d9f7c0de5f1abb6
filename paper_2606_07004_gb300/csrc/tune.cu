// Autotuner for the Krylov step kernels.
//
// The tunables are the probe-block width of a pass (the block's columns run
// as 1, 2 or 4 slices), the CTA size (hence rows per CTA iteration) and the
// tile depth (rows per partial sum).  For a matrix, block width and step
// shape (window dots of pass 1, basis vectors of pass 2, the extra u_1 dot)
// the tuner times every valid combination of one such step on scratch blocks
// with CUDA events, keeps the fastest and caches it per (element type, ld,
// n, nnz, SM count, step shape) in memory and, when LOGDET_TUNE_CACHE names
// a file, on disk (one line per shape).  A tuned layout changes the
// order of the fixed-order partial sums, so its results differ from the
// default layout's at rounding level only.  For FP32 blocks of a matrix with
// line structure the SpMM pass of each candidate is the line sweep (its own
// cache key), since that is the kernel the solve will run.
#include "dense.cuh"
#include "dia.cuh"
#include "krylov.cuh"
#include "solve.cuh"
#include "tune.cuh"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

namespace ld {

namespace {
using Key = std::tuple<int, int, int, long long, int, int, int, int>;
std::mutex g_mu;
std::map<Key, TuneCfg> g_cache;
bool g_loaded = false;

void load_file() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = std::getenv("LOGDET_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int f32, ld, n, sms, nd, nb, ex, split, threads, iters;
  long long nnz;
  while (std::fscanf(f, "%d %d %d %lld %d %d %d %d %d %d %d", &f32, &ld, &n, &nnz, &sms, &nd, &nb,
                     &ex, &split, &threads, &iters) == 11) {
    TuneCfg c;
    c.split = split;
    c.threads = threads;
    c.iters = iters;
    g_cache[Key(f32, ld, n, nnz, sms, nd, nb, ex)] = c;
  }
  std::fclose(f);
}

void save_entry(const Key& k, const TuneCfg& c) {
  const char* path = std::getenv("LOGDET_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %lld %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k),
               std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k),
               std::get<7>(k), c.split, c.threads, c.iters);
  std::fclose(f);
}

int gcd_i(int a, int b) { while (b) { int t = a % b; a = b; b = t; } return a; }
}  // namespace

template <typename T>
int autotune_krylov(logdet_ctx* h, const typename ValOf<T>::type* vals, int ld, int ndots,
                    int nbasis, int extra, cudaStream_t st, TuneCfg* out) {
  const int* rowptr = h->rowptr;
  const int* colind = h->colind;
  const int n = h->n;
  const long long nnz = h->nnz;
  constexpr int V = Vec16<T>::N;
  using Part = typename PartOf<T>::type;
  ndots = std::max(1, std::min(ndots, kMaxWin - 1));
  nbasis = std::max(1, std::min(nbasis, kMaxWin - 1));
  extra = extra ? 1 : 0;
  const bool sw_ok = std::is_same<T, float>::value && h->kind == 0 && h->dia.ndiag > 0 &&
                     h->dia_slot != nullptr;
  const int kind = std::is_same<T, double>::value ? 0
                   : std::is_same<T, float>::value ? (sw_ok ? 3 : 1)
                   : std::is_same<T, bf16>::value  ? 2
                                                   : 4;
  const Key key(kind, ld, n, nnz, sm_count(), ndots, nbasis, extra);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *out = it->second;
      return LOGDET_OK;
    }
  }
  // Candidates.
  std::vector<TuneCfg> cands;
  for (int split : {1, 2, 4}) {
    if (ld % split || (ld / split) % V) continue;
    const int G = ld / split / V;
    const int lcm = G / gcd_i(G, 32) * 32;
    for (int t = lcm; t <= 512 && t <= 3 * lcm; t += lcm)
      for (int iters : {8, 16, 32}) {
        TuneCfg c;
        c.split = split;
        c.threads = t;
        c.iters = iters;
        cands.push_back(c);
      }
  }
  if (cands.empty()) {
    *out = TuneCfg();
    return LOGDET_OK;
  }
  // Scratch: x (the pass-1 input), y (its output), z (the update's output),
  // partials for the deepest geometry, coefficients, and the other vectors of
  // the window as blocks of their own, so that the timed passes read as many
  // distinct blocks as a Krylov step does (with the window's vectors aliased
  // to x they hit in L2 where a real step streams them from HBM).  Where
  // free memory is short the window's vectors share x.
  const size_t blk = (size_t)n * ld;
  DevBuf<T> x(st), y(st), z(st);
  DevBuf<Part> part(st);
  DevBuf<double> coef(st), ycoef(st);
  LD_TRY(x.alloc(blk));
  LD_TRY(y.alloc(blk));
  LD_TRY(z.alloc(blk));
  const int nw = std::max(ndots, nbasis);  // window vectors, x the last
  std::vector<std::unique_ptr<DevBuf<T>>> win;
  {
    size_t free_b = 0, total_b = 0;
    LD_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t want = (size_t)(nw - 1) * blk * sizeof(T);
    if (2 * want <= free_b) {
      for (int i = 0; i + 1 < nw; ++i) {
        win.emplace_back(new DevBuf<T>(st));
        if (win.back()->alloc(blk) != LOGDET_OK) {
          win.pop_back();
          break;
        }
        LD_TRY(probe_fill<T>(probe_key(12345, 8 + i), n, ld, 0, win.back()->p, ld, st));
      }
    }
  }
  // Window vector i of nw (i = nw - 1 is x).
  auto wv = [&](int i) -> const T* {
    const int back = nw - 1 - i;
    return (back == 0 || back > (int)win.size()) ? x.p : win[back - 1]->p;
  };
  int max_slots = 1;
  for (auto& c : cands) {
    TileGeom g = tile_geom(ld / c.split, V, c.threads, c.iters);
    const int4* items = nullptr;
    int cnt = 0;
    LD_TRY(spmm_items(h, g.tile_rows, &items, &cnt));
    max_slots = std::max(max_slots, std::max(cnt, div_up(n, g.tile_rows)));
    SweepGeom sg;
    if (sw_ok && dia_sweep_geom(h, ld / c.split, g.threads, &sg))
      max_slots = std::max(max_slots, sg.units);
  }
  // Line sweep: FP32 values per row and diagonal (unscaled: only the time
  // counts) and the wait-failure flag.
  DevBuf<float> dvals(st);
  DevBuf<int> derr(st);
  if (sw_ok) {
    LD_TRY(dvals.alloc((size_t)dia_pad(h->dia.ndiag) * n));
    LD_TRY(dia_values_f32(h, 1.0, dvals.p, st));
    LD_TRY(derr.alloc(1));
    LD_TRY(derr.zero());
  }
  LD_TRY(part.alloc((size_t)std::max(ndots, 2) * ld * max_slots));
  LD_TRY(coef.alloc((size_t)kMaxWin * ld));
  LD_TRY(ycoef.alloc(ld));
  LD_TRY(probe_fill<T>(probe_key(12345, 7), n, ld, 0, x.p, ld, st));
  LD_TRY(fill_double(coef.p, (size_t)kMaxWin * ld, 0.25, st));
  LD_TRY(fill_double(ycoef.p, ld, 1.0, st));
  cudaEvent_t e0, e1;
  LD_CUDA(cudaEventCreate(&e0));
  LD_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  TuneCfg best_c = cands[0];
  for (auto& c : cands) {
    const int width = ld / c.split;
    TileGeom g = tile_geom(width, V, c.threads, c.iters);
    const int ntiles = div_up(n, g.tile_rows);
    const int4* items = nullptr;
    int nitems = 0;
    LD_TRY(spmm_items(h, g.tile_rows, &items, &nitems));
    SweepGeom sg;
    const bool use_sw = sw_ok && !items && dia_sweep_geom(h, width, g.threads, &sg);
    std::vector<SpmmJob<T>> sj;
    std::vector<UpdJob<T>> uj;
    for (int q = 0; q < c.split; ++q) {
      SpmmJob<T> J;
      memset(&J, 0, sizeof J);
      J.rowptr = rowptr;
      J.colind = colind;
      J.vals = vals;
      J.x = x.p;
      J.y = y.p;
      J.ndots = ndots;
      for (int d = 0; d < ndots; ++d) J.dotv[d] = wv(nw - ndots + d);
      J.part = part.p;
      J.n = n;
      J.ld = ld;
      J.col_off = q * width;
      J.width = width;
      J.b = width;
      J.nnz = nnz;
      J.tile_rows = g.tile_rows;
      J.ntiles = items ? nitems : ntiles;
      J.items = items;
      if constexpr (std::is_same<T, float>::value) {
        if (use_sw) {
          J.ntiles = sg.units;
          J.dia = dvals.p;
          J.err = derr.p;
          J.dia_T = sg.T;
          J.dia_kc = sg.kc;
          J.dia_nseg = sg.nseg;
          J.dia_nlines = sg.nlines;
          J.dia_tx = sg.tx;
          J.dia_ty = sg.ty;
          J.dia_txs = sg.txs;
          J.dinfo = h->dia;
          LD_TRY(dia_encode(J, x.p, n, ld, width));
        }
      }
      sj.push_back(J);
      UpdJob<T> U;
      memset(&U, 0, sizeof U);
      U.y = y.p;
      U.nbasis = nbasis;
      for (int i = 0; i < nbasis; ++i) U.basis[i] = wv(nw - nbasis + i);
      U.extra = extra ? wv(0) : nullptr;
      U.coef = coef.p;
      U.ycoef = ycoef.p;
      U.out = z.p;
      U.part = part.p;
      U.n = n;
      U.ld = ld;
      U.col_off = q * width;
      U.width = width;
      U.b = width;
      U.tile_rows = g.tile_rows;
      U.ntiles = ntiles;
      uj.push_back(U);
    }
    float tmin = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      LD_CUDA(cudaEventRecord(e0, st));
      LD_TRY(launch_spmm_jobs<T>(sj, g.threads, st));
      LD_TRY(launch_update_jobs<T>(uj, g.threads, st));
      LD_CUDA(cudaEventRecord(e1, st));
      LD_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      LD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) tmin = std::min(tmin, ms);  // first run warms caches
    }
    if (tmin < best) {
      best = tmin;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = best_c;
    save_entry(key, best_c);
  }
  *out = best_c;
  return LOGDET_OK;
}

template int autotune_krylov<double>(logdet_ctx*, const double*, int, int, int, int, cudaStream_t,
                                    TuneCfg*);
template int autotune_krylov<float>(logdet_ctx*, const float*, int, int, int, int, cudaStream_t,
                                    TuneCfg*);
template int autotune_krylov<bf16>(logdet_ctx*, const float*, int, int, int, int, cudaStream_t,
                                    TuneCfg*);
template int autotune_krylov<f32x2>(logdet_ctx*, const float*, int, int, int, int, cudaStream_t,
                                     TuneCfg*);

}  // namespace ld

extern "C" int logdet_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(ld::g_mu);
  ld::g_cache.clear();
  return LOGDET_OK;
}
