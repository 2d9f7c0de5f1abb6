/*
 * liblogdet: GB300 (sm_103a) log-determinant estimation for large sparse SPD
 * matrices by OSLQ and OSA-IOP (Mbingui, Tambue, Karambal, arXiv 2606.07004).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Return value: 0 (LOGDET_OK) on success, LOGDET_PENDING (> 0) for a
 *   request still in flight, a negative LOGDET_E* code on error.
 *   logdet_strerror() names a code; logdet_last_error() gives the detail of
 *   the calling thread's most recent failure.
 * - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *   global memory on the handle's device.  Sizes are element counts.
 * - Dense blocks are row-major: entry (row i, column p) of an n x b block
 *   with leading dimension ld (ld >= b) is at index i*ld + p.
 * - CSR input: rowptr[n+1] (int32, rowptr[0] = 0, non-decreasing),
 *   colind[nnz] (int32, strictly increasing within a row, in [0, n)),
 *   vals[nnz]; every row must store its diagonal entry.  The matrix must be
 *   symmetric; symmetry is the caller's promise and is not checked.
 * - Numerical events that do not stop a solve (Krylov breakdown, a
 *   non-positive Ritz value, a rank-deficient sketch) are reported in
 *   logdet_result.status_bits, not as errors.
 * - All entry points are thread-safe for distinct handles.  A handle must
 *   not be used by two threads at once.
 */
#ifndef LOGDET_H
#define LOGDET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define LOGDET_OK        0
#define LOGDET_PENDING   1
#define LOGDET_EINVAL   (-1)  /* bad argument or malformed CSR */
#define LOGDET_ENOMEM   (-2)  /* device allocation failed or over budget */
#define LOGDET_ENOTSPD  (-3)  /* spectral bounds show the matrix is not SPD */
#define LOGDET_ETIMEOUT (-4)  /* a bounded device wait or a host wait expired */
#define LOGDET_ECUDA    (-5)  /* a CUDA runtime call failed */
#define LOGDET_ENOENT   (-6)  /* unknown request id */
#define LOGDET_ECANCEL  (-7)  /* request cancelled */

/* ---- enums ------------------------------------------------------------- */
#define LOGDET_VALS_F64  0
#define LOGDET_VALS_F32  1

#define LOGDET_FP64        0  /* everything in IEEE binary64 */
#define LOGDET_MIXED_FP32  1  /* FP32 values and vectors, compensated FP32 dots,
                                 OSLQ's Hutch++ QR and projection in FP32 with
                                 compensated Gram sums (FP64 Cholesky factor),
                                 FP64 small solves */
#define LOGDET_MIXED_BF16VEC 2 /* as MIXED_FP32 but the Krylov vectors are stored in
                                 BF16 (FP32 arithmetic): a trial of the error budget */
#define LOGDET_MIXED_F32X2 3  /* FP32 matrix values; Krylov vectors stored as
                                 double-float pairs (hi + lo, two FP32 words, about
                                 48 significand bits) and computed on in double-float
                                 arithmetic on the FP32 pipe, compensated dots; the
                                 Hutch++ split and small solves in FP64.  For
                                 ill-conditioned matrices whose FP32-vector error
                                 exceeds the budget.  CSR operators only (EINVAL for
                                 gridded operators) */

#define LOGDET_METHOD_OSLQ    0
#define LOGDET_METHOD_OSAIOP  1

/* status_bits */
#define LOGDET_ST_BREAKDOWN      0x1u  /* a probe's Krylov run stopped at h < tol */
#define LOGDET_ST_NONPOS_RITZ    0x2u  /* a Ritz value <= 0 was clamped */
#define LOGDET_ST_RANK_DEFICIENT 0x4u  /* the sketch Y lost rank; columns dropped */
#define LOGDET_ST_LOG_FAILED     0x8u  /* log(H_m) did not converge for a probe */

typedef struct logdet_ctx* logdet_handle;

typedef struct {
  double logdet;     /* the estimate of log det Q */
  double tr_sub;     /* deterministic subspace term sum_i q_i^T f q_i */
  double tr_res;     /* residual term (1/r) sum_j z_j^T f z_j */
  double log_alpha;  /* log of the scale alpha: n*log_alpha + tr_sub + tr_res = logdet */
  double log_gamma;  /* OSA-IOP shift-scale log(gamma); 0 for OSLQ */
  int32_t s;         /* sketch columns floor(num_probes/3) */
  int32_t r;         /* residual probes num_probes - 2s */
  int32_t s_eff;     /* sketch rank kept after the QR */
  int32_t steps_min; /* smallest Krylov dimension reached over the probes */
  int32_t steps_max; /* largest */
  uint32_t status_bits;
  double device_ms;  /* device time of the solve (CUDA events; blocking calls) */
  double latency_ms; /* submit -> result on the host (server requests; blocking: wall time) */
  double queue_ms;   /* submit -> admission (server requests; blocking: 0) */
} logdet_result;

typedef struct {
  int32_t precision;   /* LOGDET_FP64 (default), LOGDET_MIXED_FP32, _BF16VEC or _F32X2 */
  double tol;          /* breakdown threshold on h_{m+1,m} / beta_j; 0 = 1e-12 */
  double lambda_lo;    /* spectral bounds; both 0 = clamped Gershgorin interval */
  double lambda_hi;
  int32_t autotune;    /* 1 = pick the Krylov kernels' layout (probe-block slices,
                          CTA size, tile depth) by timing candidates on this matrix,
                          cached per shape (and in the file LOGDET_TUNE_CACHE if set);
                          changes results at rounding level only.  0 = defaults */
  double* per_probe;   /* optional host out, length s+r: subspace forms q_i^T f q_i
                          (i < s) then normalised residual forms K(z_j/|z_j|) */
  double* z_norm2;     /* optional host out, length r: |z_j|^2 */
  void* stream;        /* optional cudaStream_t for this call; NULL = handle's */
  double shift;        /* solve for Q + shift*I (shift >= 0) without copying Q; the
                          Gershgorin interval moves by exactly shift.  0 = Q itself */
  int32_t plain_slq;   /* 1 = no Hutch++ split: all num_probes probes are residual
                          probes (s = 0), i.e. Hutchinson's estimator (Eq. TE) with
                          each form by the Gauss rule / Algorithm 1; num_probes >= 1 */
  int32_t gaussian_probes; /* 1 = N(0,1) probes by Box-Muller from the same counters:
                          u1 = ((z>>11)+1) 2^-53, u2 = (mix(z)>>11) 2^-53,
                          g = sqrt(-2 log u1) cos(2 pi u2); 0 = Rademacher */
  int32_t block_width; /* probe columns per Krylov pass: each block of probes
                          (the s + r probes, and OSA-IOP's s sketch columns; both
                          rounded up to a multiple of 2 columns for FP64 and
                          LOGDET_MIXED_F32X2, 4 for FP32 and BF16 vectors) runs
                          as slices of min(block_width, its columns) columns, one
                          job per slice, with the default CTA size and tile
                          depth.  0 = the default full-width block, or the
                          autotuner's choice when autotune = 1.  A width that is
                          not a multiple of 2 (FP64, F32X2) / 4 (FP32, BF16
                          vectors), or that does not
                          divide a block's rounded column count, is EINVAL.  Ignored
                          for gridded operators.  Changes results at rounding level
                          only (the order of the fixed-order partial sums). */
} logdet_opts;

/* Fill an opts struct with the defaults. */
void logdet_opts_default(logdet_opts* opts);

const char* logdet_strerror(int code);
const char* logdet_last_error(void);

/* ---- matrix handle -----------------------------------------------------
 * logdet_create: copies a host CSR matrix to the current CUDA device,
 * validates it (Sec. 2 takes Q symmetric positive definite; the checks here
 * are structural only) and computes its Gershgorin interval (Sec. 2.1, the
 * spectral interval used by both estimators).  vals_dtype is LOGDET_VALS_F64 or _F32.  The
 * caller may free its arrays on return.  Errors: EINVAL (n < 1, bad rowptr,
 * column out of range or unsorted or duplicated, missing diagonal, NaN),
 * ENOTSPD (Gershgorin upper bound <= 0), ENOMEM, ECUDA.
 */
int logdet_create(int32_t n, const int32_t* rowptr, const int32_t* colind,
                  const void* vals, int32_t vals_dtype, logdet_handle* out);

/* Same, but the three arrays are device pointers that the handle borrows:
 * they must stay valid and unchanged until logdet_destroy.  Validation runs
 * on the device. */
int logdet_create_device(int32_t n, const int32_t* rowptr_dev, const int32_t* colind_dev,
                         const void* vals_dev, int32_t vals_dtype, logdet_handle* out);

/* logdet_create_grid: a matrix-free operator on an nx x ny grid (field value
 * of point (x, y) at row y * nx + x):
 *   Q[(y, x), (y', x')] = w[|y - y'| * (radius + 1) + |x - x'|]
 * when |y - y'| <= radius and |x - x'| <= radius, else 0 — a compactly
 * supported stationary covariance restricted to the grid, such as the
 * Wendland covariance of the GRF maximum-likelihood study (Sec. 4), whose
 * support of tens of grid cells makes a stored CSR matrix impractical.
 * w: (radius + 1)^2 doubles on the host, copied; w[0] is the diagonal (add
 * a nugget there).  The caller guarantees that Q is SPD.  The handle works
 * with every estimator, the server, plans and logdet_spmm (applied by a
 * convolution kernel, nothing n x stencil is stored); FP64 and mixed FP32
 * only (EINVAL for LOGDET_MIXED_BF16VEC and LOGDET_MIXED_F32X2).  logdet_info reports n = nx * ny
 * and nnz = the entries of the implied matrix.  Errors: EINVAL (nx, ny < 1,
 * nx * ny >= 2^31, radius outside [0, 96], non-finite w), ENOTSPD
 * (Gershgorin upper bound <= 0), ENOMEM, ECUDA. */
int logdet_create_grid(int32_t nx, int32_t ny, int32_t radius, const double* w,
                       logdet_handle* out);

void logdet_destroy(logdet_handle h);

/* n, nnz and the Gershgorin interval [lo, hi] (unclamped) of the handle. */
int logdet_info(logdet_handle h, int32_t* n, int64_t* nnz, double* gersh_lo, double* gersh_hi);

/* Grid structure found at creation from host CSR arrays (n >= 4096), which
 * mixed-FP32 solves use to run the SpMM pass as a sweep over TMA-staged
 * windows of x instead of CSR gathers.  *dim = 2: every entry on one of at
 * most 16 diagonals with offsets l * L + c, |l| <= *reach <= 3, c within a
 * range of at most 16 (a 2D grid stencil, L the grid's row length): a line
 * sweep.  *dim = 3: a stencil on an L x ny x nz grid (row (z ny + y) L + x)
 * with offsets dz L ny + dy L + dx, |dz| <= *reach <= 2, |dy| <= 2,
 * |dx| <= 4, no entry wrapping across a line or plane edge, at most 16
 * diagonals: a plane sweep.  *line_stride = L.  All three are 0 when there
 * is no such structure (device-array handles, gridded operators, other
 * matrices).  Errors: EINVAL (null pointer). */
int logdet_grid_structure(logdet_handle h, int32_t* dim, int32_t* line_stride, int32_t* reach);

/* The same detection on host CSR arrays (n rows, rowptr[n + 1] and sorted
 * colind, int32, caller-owned), without a handle: host code only, no GPU
 * needed.  Outputs as for logdet_grid_structure.  Errors: EINVAL (null
 * pointer, n < 1). */
int logdet_grid_structure_csr(int32_t n, const int32_t* rowptr, const int32_t* colind,
                              int32_t* dim, int32_t* line_stride, int32_t* reach);

/* ---- estimators --------------------------------------------------------
 * logdet_oslq: Algorithm 3 (OSLQ, Sec. 3): J = Q/alpha with alpha the upper
 * spectral bound; s = floor(num_probes/3) Rademacher sketch columns give
 * Y = J S and A = orth(Y); each column of A and each projected residual probe
 * z_j = (I - A A^T) g_j (r = num_probes - 2s of them) runs krylov_steps
 * Lanczos steps and the Gauss quadrature sum_k tau_k^2 log(theta_k) of
 * Sec. 3.1.  log det = n log(alpha) + tr_sub + (1/r) sum_j |z_j|^2 K(z_j).
 * iop_window must be 0 or 2 (three-term Lanczos).  Probes are the
 * SplitMix64 Rademacher entries of (seed, stream 0 = S, 1 = G).
 * Blocks until the result is on the host.  Errors: EINVAL (num_probes < 3;
 * s = floor(num_probes/3) or r = num_probes - 2s above 64, the widest sketch
 * the Hutch++ QR kernels take; krylov_steps < 1, > n or > 256, the largest
 * tridiagonal the small-solve kernels take; bad window; a block_width that
 * does not fit the blocks; negative or non-finite shift), ENOTSPD (spectral
 * bounds not positive), ENOMEM, ECUDA.
 */
int logdet_oslq(logdet_handle h, int32_t num_probes, int32_t krylov_steps,
                int32_t iop_window, uint64_t seed, const logdet_opts* opts,
                logdet_result* out);

/* logdet_osaiop: Algorithm 2 (OSA-IOP, Sec. 2.2) with each action of
 * L = log(Q/gamma) + log(gamma/alpha) I computed by Algorithm 1
 * (Arnoldi-IOP-LOG, Sec. 2.1): gamma = sqrt(lambda_lo lambda_hi), alpha =
 * lambda_lo, incomplete orthogonalisation against the last iop_window basis
 * vectors (iop_window = 2 is the paper's length-2 IOP; iop_window >=
 * krylov_steps is full Arnoldi), log(H_m) e_1 of the small Hessenberg
 * matrix.  Y = L S, A = orth(Y), tr_sub = sum_i a_i^T L a_i,
 * tr_res = (1/r) sum_j z_j^T L z_j, log det = n log(alpha) + tr_sub + tr_res.
 * Errors as logdet_oslq (the same limits on s, r and krylov_steps); EINVAL
 * also for iop_window outside [1, 8].
 */
int logdet_osaiop(logdet_handle h, int32_t num_probes, int32_t krylov_steps,
                  int32_t iop_window, uint64_t seed, const logdet_opts* opts,
                  logdet_result* out);

/* logdet_oslq_shifts / logdet_osaiop_shifts: nshift solves of
 * log det(Q + shifts[t] I), t < nshift, each exactly the solve of
 * logdet_oslq / logdet_osaiop with opts->shift = shifts[t] and seed
 * seed0 + t (same probes, steps, window, precision and options otherwise),
 * run in lockstep: the Krylov phases of all of them go through one Krylov
 * run over a block of all their probe columns, so each SpMM gather fetches
 * the x row of every shift at once (the shifts scale the matrix differently,
 * Proposition 2.1; each column carries its own diagonal shift and scale).
 * The paper solves one operator at a time: this batches the shifted
 * log-determinants a likelihood scan over a diagonal parameter needs.
 * shifts: host array of nshift finite values >= 0 (caller-owned, read before
 * return); out: host array of nshift results.  out[t].device_ms is the whole
 * group's device time.  opts->shift, opts->per_probe and opts->z_norm2 are
 * not used.  Results agree with the separate solves to rounding (one SpMM
 * per step computes (Q/c_0 + shift_t/c_0) x c_0/c_t instead of
 * (Q + shift_t) x / c_t); a member that runs alone is bit-identical to its
 * separate solve.  The shifts go through in consecutive runs of equal size
 * (the last one possibly smaller), as few as allow at most floor(1024 / w)
 * members per run (w: one member's block width, num_probes -
 * floor(num_probes/3) rounded up to 2 for FP64 and double-float blocks, 4
 * for FP32/BF16) and an
 * estimated device memory (logdet_estimate_bytes per member) within 85 % of
 * the device's; the split depends only on the shapes and the device.
 * Blocks until the results are on the host.  Errors: EINVAL (nshift < 1;
 * NULL pointers; any member's configuration as logdet_oslq / logdet_osaiop;
 * a gridded operator), ENOTSPD, ENOMEM, ECUDA. */
int logdet_oslq_shifts(logdet_handle h, int32_t nshift, const double* shifts, int32_t num_probes,
                       int32_t krylov_steps, int32_t iop_window, uint64_t seed0,
                       const logdet_opts* opts, logdet_result* out);
int logdet_osaiop_shifts(logdet_handle h, int32_t nshift, const double* shifts,
                         int32_t num_probes, int32_t krylov_steps, int32_t iop_window,
                         uint64_t seed0, const logdet_opts* opts, logdet_result* out);

/* ---- step-level entry points (each one row of the hot path) ------------
 * logdet_probe_fill: the Rademacher probe entries of Algorithms 2/3
 * ("sample S with i.i.d. +-1 entries") by the SplitMix64 counter spec:
 *   key  = mix(seed + (stream+1)*0x9e3779b97f4a7c15)
 *   bits = mix(key + (col*2^32 + row + 1)*0x9e3779b97f4a7c15)
 *   out[row*ld + (col-col0)] = bits>>63 ? -1.0 : +1.0
 * for row in [0,n), col in [col0, col0+ncols).  out_dev: device, n*ld doubles.
 */
int logdet_probe_fill(uint64_t seed, int32_t stream, int32_t n, int32_t ncols, int32_t col0,
                      double* out_dev, int32_t ld, void* cuda_stream);

/* logdet_probe_fill_gaussian: the Gaussian alternative for the probes
 * (Algorithms 2/3 admit Gaussian entries besides +-1), entry formula as for
 * logdet_opts.gaussian_probes; layout as logdet_probe_fill. */
int logdet_probe_fill_gaussian(uint64_t seed, int32_t stream, int32_t n, int32_t ncols,
                               int32_t col0, double* out_dev, int32_t ld, void* cuda_stream);

/* logdet_spmm: Y = Q X for a device block X (n x b, leading dimension ld,
 * FP64), the matrix-vector products that are the estimators' only access to
 * Q (Sec. 1; the product of Q with a vector in Algorithm 1).  Sums run in
 * CSR order per row (a gridded operator: by stencil row dy, then dx). */
int logdet_spmm(logdet_handle h, const double* x_dev, double* y_dev, int32_t b, int32_t ld,
                void* cuda_stream);

/* logdet_orth: A = orth(Y) for a device block Y (n x s, ld) in FP64 by two
 * rounds of Cholesky QR (the QR step of Algorithms 2 and 3: an orthonormal
 * basis of span(Y)).  Column i of A equals column i of the thin QR factor
 * with positive diag(R).  A column whose |R_ii| <= 1e-6 max_j |y_j| is set to
 * zero and *s_eff counts the kept ones.  a_dev may alias y_dev. */
int logdet_orth(int32_t n, int32_t s, const double* y_dev, int32_t ldy, double* a_dev,
                int32_t lda, int32_t* s_eff, void* cuda_stream);

/* logdet_orth_f32: the same step for an FP32 block, as mixed-precision OSLQ
 * runs it (Algorithm 3's QR of Y = J S): two rounds of Cholesky QR whose Gram
 * sums are compensated FP32 dots (Dot2) accumulated per 256-row tile and
 * summed in FP64, an FP64 Cholesky factor, and FP32 applies of its inverse.
 * A (FP32, n x s in a block of leading dimension lda, a_dev may alias y_dev)
 * is orthonormal to FP32 rounding and spans the FP32 Y's columns; the column
 * drop rule and *s_eff are those of logdet_orth.  Products y_i y_j are formed
 * in FP32, so entries need magnitudes within about [1e-18, 1e18] (A does not
 * depend on the scale of Y: scale it first otherwise; the estimators' sketch
 * J S has entries of order 1).  Device pointers; blocks until done.  Errors:
 * EINVAL (NULL pointer, s outside [1, 64], ld < s), ENOMEM, ECUDA. */
int logdet_orth_f32(int32_t n, int32_t s, const float* y_dev, int32_t ldy, float* a_dev,
                    int32_t lda, int32_t* s_eff, void* cuda_stream);

/* logdet_quadform: *out = x^T (Q + shift I) x for the handle's operator
 * (CSR or gridded), x an n-vector of doubles on the device — the data term
 * of the Gaussian log-likelihood L(theta) of the GRF study (Sec. 4).  The
 * reduction runs on the device in a fixed order; blocks until *out (host) is
 * written.  Errors: EINVAL (NULL pointer, non-finite shift), ENOMEM, ECUDA. */
int logdet_quadform(logdet_handle h, const double* x_dev, double shift, double* out,
                    void* cuda_stream);

/* logdet_gauss_quadrature_log: for each of nprobe symmetric tridiagonals
 * (alpha[p*m .. +m_p), beta[p*m .. +m_p-1), m_p = msteps[p] or m if msteps
 * is NULL) the Gauss rule of Sec. 3.1: out[p] = sum_k tau_k^2 log(theta_k),
 * tau_k = e_1^T u_k.  Device pointers.  Evaluated as e_1^T log(T) e_1 by a
 * 200-node quadrature of the resolvent e_1^T (T + sI)^{-1} e_1 when T is
 * SPD (spectrum in [1e-9, 1] for error < 1e-15: the scaled operators have
 * lambda_max <= 1); otherwise by implicit QR, where a theta <= 0 is clamped
 * to clamp_lo and flagged in *status (host, optional). */
int logdet_gauss_quadrature_log(const double* alpha_dev, const double* beta_dev,
                                const int32_t* msteps_dev, int32_t m, int32_t nprobe,
                                double clamp_lo, double* out_dev, uint32_t* status,
                                void* cuda_stream);

/* logdet_hessenberg_log_e1: c_p = log(H_p) e_1 (principal logarithm,
 * the matrix logarithm of H_m in Algorithm 1) for nprobe upper Hessenberg matrices,
 * H_p column-major with leading dimension ldh at H_dev + p*ldh*m, order
 * m_p = msteps[p] (or m).  c_dev: nprobe x m (row p at c_dev + p*m).
 * Inverse scaling and squaring (Denman-Beavers square roots, Gauss-Legendre
 * partial-fraction Pade of degree 8).  status bit LOG_FAILED when a square
 * root does not converge.
 * logdet_hessenberg_log_e1_banded: the same for matrices that are zero above
 * upper bandwidth `band` >= 0 (Algorithm 1 with window k gives band = k - 1;
 * entries above the band are not read).  For band <= 8 and band + 1 < m it
 * uses a 241-node quadrature of the resolvent (H + sI)^{-1} e_1, one banded
 * solve per node (error < 1e-15 for spectra in [1e-9, 1e9] off the negative
 * real axis; LOG_FAILED on a zero pivot); otherwise the routine above.
 * LOGDET_EINVAL for band < 0. */
int logdet_hessenberg_log_e1(const double* H_dev, int32_t ldh, const int32_t* msteps_dev,
                             int32_t m, int32_t nprobe, double* c_dev, uint32_t* status,
                             void* cuda_stream);
int logdet_hessenberg_log_e1_banded(const double* H_dev, int32_t ldh, const int32_t* msteps_dev,
                                    int32_t m, int32_t nprobe, int32_t band, double* c_dev,
                                    uint32_t* status, void* cuda_stream);

/* ---- serving (continuous batching) --------------------------------------
 * The paper solves one log-determinant at a time; a GP hyper-parameter search
 * issues many.  A server admits requests of any size and method while slots
 * (max_slots) and an estimate of their device memory fit the budget, keeps
 * each one's Krylov state resident, and advances all requests that are in a
 * Krylov phase together: one batched launch per pass per tick.  Requests
 * join and leave the batch as they arrive and finish.  A request's result is
 * bit-identical to logdet_oslq / logdet_osaiop with the same arguments.
 *
 * logdet_server_create: budget in bytes (> 0), max_slots >= 1, optional
 *   cudaStream_t (NULL = a stream of its own).  Starts one scheduler thread.
 * logdet_server_destroy: cancels queued requests, finishes resident ones,
 *   joins the thread.
 * logdet_submit: non-blocking.  method LOGDET_METHOD_OSLQ / _OSAIOP; other
 *   arguments as logdet_oslq / logdet_osaiop.  The handle must stay alive
 *   until the request completes; opts->per_probe / z_norm2 (if set) are
 *   written when it completes and must stay valid until then.  Errors:
 *   EINVAL (bad arguments), ENOMEM (the request alone exceeds the budget).
 * logdet_poll: LOGDET_PENDING while queued or running, LOGDET_OK with *out
 *   filled (latency_ms, queue_ms set), or the request's error / ECANCEL.
 * logdet_wait: as poll but blocks up to timeout_us (< 0 = forever);
 *   ETIMEOUT when still pending.
 * logdet_cancel: queued requests never run; running ones leave at the next
 *   tick.  logdet_release forgets a finished request.  ENOENT: unknown id.
 */
/* logdet_estimate_bytes: the device memory (bytes, an upper estimate of the
 * peak) one solve with these arguments uses -- the amount a server reserves
 * against its budget when it admits the request.  Errors as logdet_submit. */
int logdet_estimate_bytes(logdet_handle h, int32_t method, int32_t num_probes,
                          int32_t krylov_steps, int32_t iop_window, const logdet_opts* opts,
                          size_t* bytes);

typedef struct logdet_server logdet_server;
typedef struct {
  int64_t submitted, admitted, completed, failed, cancelled;
  int64_t queued, resident, max_resident;
  int64_t ticks;          /* scheduler iterations */
  int64_t batched_steps;  /* request-steps advanced by batched launches */
  size_t bytes_in_use, bytes_budget;
  double busy_ms;         /* scheduler time spent issuing work */
  int64_t suspended;      /* requests held by logdet_suspend now */
  int64_t suspensions;    /* suspensions so far */
  int64_t suspended_in_krylov; /* of those, taken in the middle of a Krylov phase */
} logdet_stats;
int logdet_server_create(size_t device_mem_budget, int32_t max_slots, void* cuda_stream,
                         logdet_server** out);
void logdet_server_destroy(logdet_server* s);
int logdet_submit(logdet_server* s, logdet_handle h, int32_t method, int32_t num_probes,
                  int32_t krylov_steps, int32_t iop_window, uint64_t seed, const logdet_opts* opts,
                  uint64_t* req_id);
/* logdet_submit_shifts: the server form of logdet_oslq_shifts /
 *   logdet_osaiop_shifts (method LOGDET_METHOD_OSLQ / _OSAIOP): nshift
 *   requests, member t the solve with shift shifts[t] and seed seed0 + t,
 *   whose ids go to req_ids[0 .. nshift).  They are split into the same
 *   runs as the blocking call; each run is admitted as a whole (its members'
 *   estimates together against the budget, one slot) and advances in the
 *   batch as one Krylov run over all its members' columns, so the results
 *   are bit-identical to logdet_*_shifts with the same arguments.  Members
 *   are polled, waited for, logged and released one by one; cancelling one
 *   cancels its run; they cannot be suspended (EINVAL).  opts->per_probe /
 *   z_norm2 are not used.  Errors: as logdet_oslq_shifts, and ENOMEM when a
 *   run alone exceeds the budget (nothing is submitted then). */
int logdet_submit_shifts(logdet_server* s, logdet_handle h, int32_t method, int32_t nshift,
                         const double* shifts, int32_t num_probes, int32_t krylov_steps,
                         int32_t iop_window, uint64_t seed0, const logdet_opts* opts,
                         uint64_t* req_ids);
int logdet_poll(logdet_server* s, uint64_t req_id, logdet_result* out);
int logdet_wait(logdet_server* s, uint64_t req_id, int64_t timeout_us, logdet_result* out);
int logdet_cancel(logdet_server* s, uint64_t req_id);
int logdet_release(logdet_server* s, uint64_t req_id);
int logdet_server_stats(logdet_server* s, logdet_stats* out);
/* logdet_suspend: preemption.  A queued request leaves the queue; a running
 *   one leaves the batch at the next tick boundary (unless its result is
 *   already being copied out, in which case it just finishes): the scheduler
 *   waits for the server's stream, copies every device buffer of the solve
 *   (Krylov blocks, window ring, scalar state, sketch) to host memory and
 *   frees them, so its slot and budget go to other requests.  poll / wait
 *   report LOGDET_PENDING meanwhile.  Returns at once.  Errors: ENOENT,
 *   EINVAL (finished, failed or cancelled).
 * logdet_resume: puts a suspended request at the front of the queue; when
 *   admitted again its buffers are reallocated and filled from the host copy
 *   and it continues from the step where it stopped.  Its result is
 *   bit-identical to an uninterrupted run.  Resuming a running request whose
 *   suspension has not happened yet withdraws it.  Errors: ENOENT, EINVAL
 *   (not suspended).  logdet_cancel also ends a suspended request. */
int logdet_suspend(logdet_server* s, uint64_t req_id);
int logdet_resume(logdet_server* s, uint64_t req_id);
/* logdet_server_set_log: append one JSON line per request that leaves the
 *   server after admission (done, failed, or cancelled while resident) to
 *   the file `path` (opened for appending; NULL or
 *   "" stops logging): id, state, rc, n, nnz, method, precision, probes,
 *   steps, window, shift, seed, logdet, steps_min, steps_max, status_bits,
 *   latency_ms and queue_ms (submit -> result and submit -> admission, host
 *   clock).  Errors: EINVAL (NULL server, file not openable). */
int logdet_server_set_log(logdet_server* s, const char* path);

/* ---- checked builds (a substitute for the sanitizers in tests) ----------
 * The library built with -DLOGDET_CHECKED (liblogdet_checked.so) checks, in
 * the Krylov passes on the device, every index it takes from memory before
 * using it: work-item rows and partial slots, row ranges from rowptr,
 * column indices.  A violation sets a bit in the device word reported here
 * (1 work item, 2 row range, 4 column index, 8 partial slot) and the access
 * is redirected in range; nothing traps.  Every workspace buffer gets 256
 * guard bytes of 0xA5 on each side, read back when it is freed; changed
 * bytes are counted.  logdet_checked_report: *checked = 1 in a checked
 * build (0 otherwise, with both counts 0); *device_violations = the bits so
 * far (synchronises the device); *canary_bytes = changed guard bytes so far.
 * Errors: EINVAL (NULL pointer), ECUDA. */
int logdet_checked_report(int32_t* checked, uint32_t* device_violations, uint64_t* canary_bytes);

/* ---- graph plans (the paper has no counterpart: a deployment variant of
 * Algorithms 2 and 3 for repeated estimates of one shape) -------------------
 * A plan captures one complete OSLQ (method 0) or OSA-IOP (method 1) solve,
 * with the arguments of logdet_oslq / logdet_osaiop minus the seed, into a
 * CUDA graph; each logdet_plan_run replays it with a new seed as one graph
 * launch.  The result for a seed is bit-identical to logdet_oslq /
 * logdet_osaiop with that seed and the same options.
 *
 * logdet_plan_create: validates like logdet_oslq (LOGDET_EINVAL), runs one
 *   ordinary solve (kernel loading, autotuned layout) and captures the next
 *   on a stream of its own.  opts->stream (optional) is the stream runs are
 *   launched on; opts->per_probe / z_norm2 are ignored (see run).  The plan
 *   borrows the handle: destroy the plan first.  LOGDET_ECUDA if the capture
 *   or the instantiation fails (logdet_last_error says why).
 * logdet_plan_run: one estimate for `seed`; blocks until its result is on
 *   the host.  per_probe (s + r doubles) and z_norm2 (r doubles) are optional
 *   outputs as in logdet_opts.  result.device_ms times the seed copy and the
 *   graph launch with CUDA events.  A plan runs one estimate at a time: calls
 *   on one plan from several threads must be serialised by the caller.
 * logdet_plan_kernels: kernel launches one run replays.
 * Memory: between runs a plan holds the graph's device allocations (about
 *   logdet_estimate_bytes of its shape) and a pinned result buffer. */
typedef struct logdet_plan_s* logdet_plan;
int logdet_plan_create(logdet_handle h, int32_t method, int32_t num_probes, int32_t krylov_steps,
                       int32_t iop_window, const logdet_opts* opts, logdet_plan* out);
int logdet_plan_run(logdet_plan p, uint64_t seed, logdet_result* out, double* per_probe,
                    double* z_norm2);
int logdet_plan_kernels(logdet_plan p, int64_t* kernels);
void logdet_plan_destroy(logdet_plan p);

/* logdet_hessenberg_log_e1_noalloc: the same computation as
 * logdet_hessenberg_log_e1, for callers that cannot allocate device memory
 * while they run: hosts whose device memory is handed out once at start-up
 * under a fixed budget, callers under an external allocator that owns all
 * device memory and forbids cudaMalloc/cudaFree, and loops that must not pay
 * for cudaFree, which synchronises the whole device.  The paper has no
 * counterpart; this is a deployment variant.  It allocates nothing: its
 * scratch is a statically sized device array of 8 MiB + 16 KiB inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  The first call on each device looks up that array's device address
 * and keeps it for the life of the process: make that first call before any
 * stream capture, and do not use this entry point after a reset of the
 * device (cudaDeviceReset) in the same process.  Limits: nprobe <= 4096 and,
 * for m >= 81 (work matrices beyond shared memory), 4 m^2 nprobe <= 1048576;
 * larger requests return LOGDET_EINVAL without running.  All calls share the
 * one array, so calls whose kernels may overlap on the GPU (different streams
 * with no ordering between them) race; order them on one stream.  Each call
 * clears the status words it uses and blocks until they are read back.
 * Arguments, layouts and status bits as logdet_hessenberg_log_e1. */
int logdet_hessenberg_log_e1_noalloc(const double* H_dev, int32_t ldh, const int32_t* msteps_dev,
                                     int32_t m, int32_t nprobe, double* c_dev, uint32_t* status,
                                     void* cuda_stream);

/* ---- instrumentation (the paper has no counterpart: it reports only
 * wall-clock seconds per solve) -------------------------------------------
 * logdet_launch_count: kernels this process has launched through the library.
 * logdet_profile_enable(1): from then on every launch is bracketed by CUDA
 * events on its own stream and tagged with a class and its algorithmic work
 * (FLOPs and the bytes it must move once: CSR once, each vector once).
 * logdet_profile_read sums, for one class, the launches recorded since the
 * last logdet_profile_reset: count, device milliseconds, FLOPs, bytes.  It
 * waits for the recorded events.  Classes: 0 SpMM pass, 1 update pass,
 * 2 per-probe scalar kernels, 3 Cholesky QR, 4 residual projection,
 * 5 small solves (Gauss rules, Hessenberg logs), 6 other, 7 gridded-operator
 * applications, 8 persistent Krylov runs (all passes and scalar steps of a
 * small run in one launch).
 */
#define LOGDET_KC_SPMM    0
#define LOGDET_KC_UPDATE  1
#define LOGDET_KC_SCALAR  2
#define LOGDET_KC_QR      3
#define LOGDET_KC_PROJECT 4
#define LOGDET_KC_SMALL   5
#define LOGDET_KC_OTHER   6
#define LOGDET_KC_GRID    7
#define LOGDET_KC_KRUN    8
#define LOGDET_KC_COUNT   9
int64_t logdet_launch_count(void);
/* Forget the autotuner's in-memory cache (the file, if any, is kept). */
int logdet_autotune_clear(void);
int logdet_profile_enable(int on);
int logdet_profile_reset(void);
int logdet_profile_read(int32_t kclass, int64_t* launches, double* device_ms, double* flops,
                        double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* LOGDET_H */
