// Resumable solves.  A Solve is one OSLQ (Algorithm 3) or OSA-IOP
// (Algorithm 2 with Algorithm 1) log-determinant estimate, split into phases
// so that many solves can advance together:
//
//   SETUP   scaled values, probes, (OSLQ) sketch + Hutch++ split, first Krylov run set up
//   K1      Krylov steps (OSLQ: its only run; OSA-IOP: the sketch columns, basis kept)
//   MID     (OSA-IOP) log(H) e_1, Y = L S, Hutch++ split, second Krylov run set up
//   K2      (OSA-IOP) Krylov steps on [A | Z] with the u_1 dots
//   FINISH  Gauss rules / quadratic forms, results copied to pinned host memory
//
// Krylov phases advance one step at a time through job descriptors
// (KRun::spmm_job, coef_job, upd_job, norm_job) that a caller gathers from
// many solves into one batched launch per pass.  Everything else runs per
// solve on the solve's stream.  A solve's arithmetic depends only on its own
// data and its block geometry, never on the other jobs of a batch.
#pragma once

#include "dense.cuh"
#include "handle.cuh"
#include "krylov.cuh"

#include <memory>
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
  double shift = 0.0;  // solve for Q + shift I
  int precision = LOGDET_FP64;
  int autotune = 0;    // layout of the Krylov kernels from the autotuner
  int plain = 0;       // 1 = plain SLQ: no sketch, s = 0, r = P
  int gaussian = 0;    // 1 = Gaussian probes
  int block_width = 0; // > 0: columns per Krylov pass slice (logdet_opts.block_width)
};

struct SolveOut {
  logdet_result res;
  std::vector<double> per_probe;  // s + r
  std::vector<double> zn2;        // r
};

int validate_cfg(const logdet_ctx* h, const SolveCfg& c);
// Block entries per 16-byte vector for a precision (Vec16<T>::N of its
// block type): two for FP64 and double-float blocks, four for FP32 and BF16.
inline int precision_vec(int precision) {
  return (precision == LOGDET_FP64 || precision == LOGDET_MIXED_F32X2) ? 2 : 4;
}
void spectral_bounds(const logdet_ctx* h, const SolveCfg& c, double& lo, double& hi);

// Device arrays of one Krylov run (see KrylovState).
struct KState {
  DevBuf<double> alpha, beta, H, sig, edot, coef, ycoef, dbuf;
  DevBuf<int> meff, active;
  DevBuf<uint32_t> status, cnt;
  KrylovState st{};
  explicit KState(cudaStream_t s)
      : alpha(s), beta(s), H(s), sig(s), edot(s), coef(s), ycoef(s), dbuf(s), meff(s), active(s),
        status(s), cnt(s) {}
  int alloc(int method, int b, int ld, int m, int k, double tol, double rescale_lim);
};

template <typename T> constexpr double rescale_limit();
template <> constexpr double rescale_limit<double>() { return 200.0; }
template <> constexpr double rescale_limit<float>() { return 20.0; }
template <> constexpr double rescale_limit<bf16>() { return 20.0; }
template <> constexpr double rescale_limit<f32x2>() { return 20.0; }

// One Krylov run over a block X0 (n x ld, b live columns): method 0 is
// three-term Lanczos, method 1 IOP with window k.  With Vfull the basis is
// kept (u_j = Vfull + (j-1) n ld, X0 == Vfull); otherwise a ring of k+1
// blocks follows u_1 = X0.  track_e accumulates u_1^T u_j.
template <typename T>
struct KRun {
  using Part = typename PartOf<T>::type;
  const int* rowptr = nullptr;
  const int* colind = nullptr;
  const typename ValOf<T>::type* vals = nullptr;
  int n = 0;
  long long nnz = 0;
  int b = 0, ld = 0, m = 0, k = 2, method = 0;
  bool track_e = false;
  T* X0 = nullptr;
  T* Vfull = nullptr;
  const double* colshift = nullptr;  // optional [ld]: the scaled diagonal shift
  const double* colscale = nullptr;  // optional [ld]: a factor per column after the shift
  logdet_ctx* hctx = nullptr;        // matrix handle (work items of irregular matrices)
  const void* gtab = nullptr;        // gridded operator: scaled expanded table (compute type)
  TileGeom g{};
  TuneCfg tune{};
  int width = 0;  // columns per slice job (ld / tune.split)
  int ntiles = 0, nring = 0, ndmax = 0;
  const int4* items = nullptr;  // SpMM work items (nullptr: uniform tiles)
  int nslots = 0;               // SpMM partial slots per column (ntiles or the item count)
  size_t blk = 0;
  DevBuf<Part> part;
  DevBuf<T> y, ring;
  KState ks;
  const float* diavals = nullptr;  // FP32 values per row and diagonal: the line-sweep path
  DevBuf<int> dia_err;             // set if a staged copy's wait gave up
  bool sweep = false;              // pass 1 runs the line sweep
  int sw_T = 0, sw_kc = 0, sw_nseg = 0, sw_nlines = 0, sw_tx = 0, sw_ty = 0, sw_txs = 0;
  int done_steps = 0;  // steps whose pass 1 has been issued
  cudaStream_t st;

  explicit KRun(cudaStream_t s)
      : part(s), y(s), ring(s), ks(s), dia_err(s), st(s), krun_bar(s), krun_part2(s) {}

  // Allocate and queue the start-block norms and sigma_1 (one launch pair).
  int init(const int* rp, const int* ci, const typename ValOf<T>::type* v, int n_, long long nnz_,
           int b_, int ld_,
           int m_, int k_, int method_, bool track_e_, T* X0_, T* Vfull_, double tol,
           TuneCfg tc = TuneCfg());
  T* ptr(int i) const;
  int win_lo(int j) const { return method == 0 ? j : (j - k + 1 > 1 ? j - k + 1 : 1); }
  int next_step() const { return done_steps + 1; }
  bool finished() const { return done_steps >= m; }
  bool has_pass2(int j) const { return j < m; }
  int pass1_dots(int j) const { return method == 0 ? 1 : j - win_lo(j) + 1; }
  // Step j's jobs, one per column slice.
  int spmm_jobs(int j, std::vector<SpmmJob<T>>& out) const;
  // Gridded operator: step j's pass 1 (y = Q~ u_j and the window dots),
  // launched on the run's stream.
  int grid_pass1(int j);
  void upd_jobs(int j, std::vector<UpdJob<T>>& out) const;
  int slice_live(int q) const;
  // Scalar job over pass-1 partials (spmm_pass) or pass-2 / norm partials.
  ScalarJob scalar_job(int j, int ndots, bool spmm_pass = false) const;
  // Persistent run: whether the remaining steps qualify (LOGDET_KRYLOV_PERSISTENT=1,
  // uniform CSR tiles, one column slice, whole-warp CTAs, FP64 or FP32 blocks
  // of at most kPersistMaxBlock bytes and 128 columns, from the first step),
  // and the launch that issues them all.
  bool persistent_ok() const;
  int issue_rest_persistent();
  DevBuf<unsigned> krun_bar;
  DevBuf<Part> krun_part2;  // persistent run: pass-2 partials
};

// Blocks up to this size (bytes of one n x ld block) may run their Krylov
// steps as one persistent launch in the blocking and graph-plan paths.
constexpr size_t kPersistMaxBlock = (size_t)16 << 20;

// Batched launches of jobs that share element type and CTA size.
template <typename T>
int launch_spmm_jobs(const std::vector<SpmmJob<T>>& jobs, int threads, cudaStream_t s);
template <typename T>
int launch_update_jobs(const std::vector<UpdJob<T>>& jobs, int threads, cudaStream_t s);
int launch_scalar_jobs(const std::vector<ScalarJob>& jobs, const std::vector<int>& widths, int kind,
                       cudaStream_t s);

enum SolvePhase { PH_SETUP = 0, PH_K1, PH_MID, PH_K2, PH_FINISH, PH_WAIT, PH_DONE, PH_FAILED };

// Type-erased solve (FP64 or mixed FP32).
struct ISolve {
  virtual ~ISolve() {}
  virtual int phase() const = 0;
  virtual bool in_krylov() const = 0;
  virtual int krylov_threads() const = 0;
  virtual bool is_fp32() const = 0;
  virtual int elem_kind() const = 0;  // 0 FP64, 1 FP32, 2 BF16, 3 double-float vectors
  // Run the current non-Krylov phase (SETUP, MID, FINISH) and move on.
  virtual int run_phase() = 0;
  // Krylov step: append this solve's pass-1 job etc. for its next step.
  // (For a gridded operator the pass is launched here, on the solve's stream.)
  virtual int add_pass1(void* spmm_vec, std::vector<ScalarJob>& coef, std::vector<int>& widths) = 0;
  virtual bool add_pass2(void* upd_vec, std::vector<ScalarJob>& norm, std::vector<int>& widths) = 0;
  virtual void step_issued() = 0;
  // Issue every remaining step of the current Krylov phase as one persistent
  // launch: LOGDET_OK when issued, 1 when the run does not qualify (step by
  // step then), a negative code on error.
  virtual int issue_krylov_rest() = 0;
  // After FINISH's copies completed: assemble the host result.
  virtual int assemble(SolveOut& o) = 0;
  virtual cudaEvent_t done_event() const = 0;
  virtual size_t bytes_estimate() const = 0;
  // Graph plans: read the two probe keys (sketch, residual) from device
  // memory at run time, and take the pinned result buffer before capture.
  virtual void set_dev_keys(const uint64_t* keys) = 0;
  virtual int prepare_host() = 0;
  // Suspension between steps (the server's preemption): suspend() waits for
  // the stream, copies every device buffer of the solve to host memory and
  // frees it; resume() allocates the buffers again (new addresses), copies
  // the contents back and repoints the run at them.  The solve continues
  // exactly where it stopped: results are bit-identical.
  virtual int suspend() = 0;
  virtual int resume() = 0;
  virtual bool suspended() const = 0;
  // Shift groups hold several solves: member t's result.
  virtual int members() const { return 1; }
  virtual int assemble_member(int t, SolveOut& o) { return t == 0 ? assemble(o) : LOGDET_EINVAL; }
};

std::unique_ptr<ISolve> make_solve(logdet_ctx* h, const SolveCfg& c, cudaStream_t st, int* rc);
size_t estimate_solve_bytes(const logdet_ctx* h, const SolveCfg& c);

// Run one solve to completion on its stream (the blocking API).
int solve_blocking(logdet_ctx* h, const SolveCfg& c, cudaStream_t st, SolveOut& o);

// Solves that differ only in shift and seed (same method, probes, steps,
// window and precision), run in lockstep with their Krylov phases as one run
// over a block of all their columns; blocking.  Members go in balanced runs
// of at most kMaxGroupWidth block columns and 85 % of the device's memory.
constexpr int kMaxGroupWidth = 1024;
int solve_shifts(logdet_ctx* h, const std::vector<SolveCfg>& cfgs, cudaStream_t st,
                 std::vector<SolveOut>& outs);
// The consecutive runs [begin, end) those solves go through (validates them).
int shift_runs(logdet_ctx* h, const std::vector<SolveCfg>& cfgs,
               std::vector<std::pair<size_t, size_t>>& runs);
// One run as a resumable solve (the server steps it like any other).
std::unique_ptr<ISolve> make_group_solve(logdet_ctx* h, const std::vector<SolveCfg>& cfgs,
                                         cudaStream_t st, int* rc);

// Queue every phase of a solve on its stream, with batches of one, until it
// waits for its result copies; no host synchronisation (so the sequence can
// be captured into a CUDA graph).
int issue_solve(ISolve* sv, cudaStream_t st);

// Solver configuration from the C-ABI arguments.
SolveCfg make_solve_cfg(int method, int32_t P, int32_t m, int32_t k, uint64_t seed,
                        const logdet_opts* opts);

}  // namespace ld
