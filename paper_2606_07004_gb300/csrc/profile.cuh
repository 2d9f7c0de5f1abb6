// Per-kernel-class instrumentation: a launch counter (always on) and, when
// enabled, CUDA events around every launch on the launching stream together
// with the launch's algorithmic FLOPs and bytes.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace ld {

enum KClass {
  KC_SPMM = 0,    // pass 1: SpMM with fused dots
  KC_UPDATE = 1,  // pass 2: window update with fused norms
  KC_SCALAR = 2,  // per-probe scalar recurrences and norm seeds
  KC_QR = 3,      // Cholesky QR2 of the sketch
  KC_PROJECT = 4, // Hutch++ residual projection
  KC_SMALL = 5,   // tridiagonal Gauss rules, Hessenberg logarithms
  KC_OTHER = 6,   // probe fill, conversions, sketch assembly, Gershgorin, scaling
  KC_GRID = 7,    // gridded-operator application (the pass-1 SpMM of a grid handle)
  KC_KRUN = 8,    // persistent Krylov run: every step of a small run in one launch
  KC_COUNT = 9
};

void prof_count();  // one kernel launch
void prof_add_launches(long long n);  // n kernel launches (a graph replay)
bool prof_enabled();
// Bracket a launch: begin() records a start event when profiling is on and
// returns a token; end() records the stop event with the launch's work.
int prof_begin(cudaStream_t s);
void prof_end(int token, KClass c, cudaStream_t s, double flops, double bytes);

struct ProfScope {
  int tok;
  KClass c;
  cudaStream_t s;
  double flops, bytes;
  ProfScope(KClass c_, cudaStream_t s_, double f = 0, double b = 0)
      : tok(prof_begin(s_)), c(c_), s(s_), flops(f), bytes(b) { prof_count(); }
  ~ProfScope() { prof_end(tok, c, s, flops, bytes); }
};

// NVTX range around host-side issue work (solve phases, Krylov steps, server
// ticks, plan replays): visible in Nsight timelines, free without a tool.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace ld
