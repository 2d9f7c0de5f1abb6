// Graph plans: one OSLQ / OSA-IOP solve of fixed shape captured once into a
// CUDA graph and replayed, one graph launch per estimate, with a new seed per
// run.  The replay issues exactly the kernels and copies of the blocking
// path in the same order with the same launch geometry, so a plan's result
// for a seed is bit-identical to logdet_oslq / logdet_osaiop with that seed.
//
// What varies between runs is the seed only: the two probe keys (sketch and
// residual streams) live in a 16-byte device array that the probe kernels
// read at run time, written by one host-to-device copy before each launch.
// Every other input (matrix, spectral interval, shift, precision, sizes) is
// fixed when the plan is made.  The device buffers of the solve are graph
// allocations (allocated and freed inside the graph), so between runs the
// plan holds the graph's reserved memory and one pinned result buffer.
#include "handle.cuh"
#include "profile.cuh"
#include "solve.cuh"

#include <cstring>
#include <memory>
#include <vector>

struct logdet_plan_s {
  logdet_ctx* h = nullptr;
  ld::SolveCfg cfg;
  cudaStream_t own = nullptr;   // capture stream (and replay stream by default)
  cudaStream_t st = nullptr;    // replay stream
  std::unique_ptr<ld::ISolve> sv;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t* d_keys = nullptr;
  uint64_t* h_keys = nullptr;   // pinned
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  long long kernels = 0;        // kernel nodes per replay

  ~logdet_plan_s() {
    if (st) cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    sv.reset();
    if (d_keys) cudaFree(d_keys);
    if (h_keys) cudaFreeHost(h_keys);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (own) {
      cudaStreamSynchronize(own);
      cudaStreamDestroy(own);
    }
  }
};

namespace ld {

static int plan_build(logdet_plan_s* p, const logdet_opts* opts) {
  logdet_ctx* h = p->h;
  LD_CUDA(cudaStreamCreateWithFlags(&p->own, cudaStreamNonBlocking));
  p->st = (opts && opts->stream) ? (cudaStream_t)opts->stream : p->own;
  // One ordinary solve first: loads the kernels and fills the layout cache
  // (the autotuner times candidates with host synchronisation, which a
  // capture cannot contain).
  {
    SolveOut warm;
    LD_TRY(solve_blocking(h, p->cfg, p->own, warm));
  }
  LD_CUDA(cudaMalloc(reinterpret_cast<void**>(&p->d_keys), 2 * sizeof(uint64_t)));
  LD_CUDA(cudaMallocHost(reinterpret_cast<void**>(&p->h_keys), 2 * sizeof(uint64_t)));
  int rc = LOGDET_OK;
  p->sv = make_solve(h, p->cfg, p->own, &rc);
  if (!p->sv) return rc ? rc : LOGDET_EINVAL;
  p->sv->set_dev_keys(p->d_keys);
  LD_TRY(p->sv->prepare_host());
  LD_CUDA(cudaStreamSynchronize(p->own));

  LD_CUDA(cudaStreamBeginCapture(p->own, cudaStreamCaptureModeThreadLocal));
  const long long before = logdet_launch_count();
  rc = issue_solve(p->sv.get(), p->own);
  const long long issued = logdet_launch_count() - before;
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(p->own, &g);
  if (rc || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (!rc) {
      set_error("graph capture failed: %s", cudaGetErrorString(ec));
      rc = LOGDET_ECUDA;
    }
    return rc;
  }
  // The launches counted during capture did not run; replays count them.
  prof_add_launches(-issued);
  p->graph = g;
  size_t nn = 0;
  LD_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) LD_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType t;
    LD_CUDA(cudaGraphNodeGetType(nodes[i], &t));
    if (t == cudaGraphNodeTypeKernel) ++p->kernels;
  }
  LD_CUDA(cudaGraphInstantiate(&p->exec, g, 0));
  LD_CUDA(cudaGraphUpload(p->exec, p->st));
  LD_CUDA(cudaEventCreate(&p->e0));
  LD_CUDA(cudaEventCreate(&p->e1));
  LD_CUDA(cudaStreamSynchronize(p->st));
  return LOGDET_OK;
}

}  // namespace ld

using namespace ld;

extern "C" {

int logdet_plan_create(logdet_handle h, int32_t method, int32_t num_probes, int32_t krylov_steps,
                       int32_t iop_window, const logdet_opts* opts, logdet_plan* out) {
  if (!h || !out) { set_error("plan_create: NULL handle or output"); return LOGDET_EINVAL; }
  *out = nullptr;
  if (method != 0 && method != 1) { set_error("plan_create: method must be 0 or 1"); return LOGDET_EINVAL; }
  SolveCfg c = make_solve_cfg(method, num_probes, krylov_steps, iop_window, 0, opts);
  LD_TRY(validate_cfg(h, c));
  if (cudaSetDevice(h->device) != cudaSuccess) { set_error("cudaSetDevice failed"); return LOGDET_ECUDA; }
  std::unique_ptr<logdet_plan_s> p(new logdet_plan_s);
  p->h = h;
  p->cfg = c;
  LD_TRY(plan_build(p.get(), opts));
  *out = p.release();
  return LOGDET_OK;
}

int logdet_plan_run(logdet_plan p, uint64_t seed, logdet_result* out, double* per_probe,
                    double* z_norm2) {
  if (!p || !out) { set_error("plan_run: NULL plan or result"); return LOGDET_EINVAL; }
  NvtxRange nv("logdet plan run");
  if (cudaSetDevice(p->h->device) != cudaSuccess) { set_error("cudaSetDevice failed"); return LOGDET_ECUDA; }
  p->h_keys[0] = probe_key(seed, 0);
  p->h_keys[1] = probe_key(seed, 1);
  LD_CUDA(cudaEventRecord(p->e0, p->st));
  LD_CUDA(cudaMemcpyAsync(p->d_keys, p->h_keys, 2 * sizeof(uint64_t), cudaMemcpyHostToDevice, p->st));
  LD_CUDA(cudaGraphLaunch(p->exec, p->st));
  LD_CUDA(cudaEventRecord(p->e1, p->st));
  LD_CUDA(cudaEventSynchronize(p->e1));
  prof_add_launches(p->kernels);
  SolveOut o;
  LD_TRY(p->sv->assemble(o));
  float ms = 0.f;
  LD_CUDA(cudaEventElapsedTime(&ms, p->e0, p->e1));
  *out = o.res;
  out->device_ms = ms;
  if (per_probe)
    for (size_t i = 0; i < o.per_probe.size(); ++i) per_probe[i] = o.per_probe[i];
  if (z_norm2)
    for (size_t i = 0; i < o.zn2.size(); ++i) z_norm2[i] = o.zn2[i];
  return LOGDET_OK;
}

int logdet_plan_kernels(logdet_plan p, int64_t* kernels) {
  if (!p || !kernels) { set_error("plan_kernels: NULL argument"); return LOGDET_EINVAL; }
  *kernels = p->kernels;
  return LOGDET_OK;
}

void logdet_plan_destroy(logdet_plan p) { delete p; }

}  // extern "C"
