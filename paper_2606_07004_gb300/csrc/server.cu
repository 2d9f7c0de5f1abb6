// Continuous-batching log-determinant server.
//
// Requests (a matrix handle plus OSLQ / OSA-IOP parameters) are queued by
// logdet_submit from any thread.  One scheduler thread owns the device work:
// every tick it admits queued requests while slots and the device-memory
// budget allow, runs the pending non-Krylov phase of each resident request
// (set-up, OSA-IOP mid-phase, finish), and then advances every request that
// is in a Krylov phase by one step with ONE batched launch per pass (SpMM +
// dots, scalar coefficients, update + norms, scalar norms) over all of them.
// Requests therefore enter and leave the batch as they arrive and finish.
// Because each job keeps its own block geometry and fixed-order reductions,
// a request's result is bit-identical whether it runs alone, in any mix, or
// through the blocking logdet_oslq / logdet_osaiop calls.
#include "handle.cuh"
#include "solve.cuh"
#include "profile.cuh"

#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

struct logdet_server;

namespace ld {

static double now_us() {
  using namespace std::chrono;
  return duration_cast<duration<double, std::micro>>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING, RQ_DONE, RQ_FAILED, RQ_CANCELLED, RQ_SUSPENDED };

struct Request {
  uint64_t id = 0;
  logdet_ctx* h = nullptr;
  SolveCfg cfg;
  double* user_per_probe = nullptr;
  double* user_zn2 = nullptr;
  std::unique_ptr<ISolve> solve;
  int state = RQ_QUEUED;
  int rc = LOGDET_OK;
  size_t bytes = 0;
  bool cancel = false;
  bool suspend = false;   // logdet_suspend asked; the scheduler acts at a tick boundary
  double t_submit = 0, t_admit = 0, t_done = 0;
  SolveOut out;
  // Shift groups (logdet_submit_shifts): a run of members goes through the
  // queue and the batch as one internal request (the run's GroupSolve) whose
  // members are the requests the caller sees.
  std::vector<SolveCfg> group_cfgs;               // run: its members' configurations
  std::vector<std::shared_ptr<Request>> members;  // run: its member requests
  std::weak_ptr<Request> run;                     // member: its run
};

}  // namespace ld

using namespace ld;

struct logdet_server {
  size_t budget = 0;
  int max_slots = 1;
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<std::shared_ptr<Request>> active;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_id = 1;
  size_t used = 0;
  bool stop = false;
  std::thread worker;
  std::deque<cudaEvent_t> ticks;  // run-ahead limiter
  // statistics
  int64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_failed = 0, n_cancelled = 0;
  int64_t n_ticks = 0, n_batched_steps = 0, max_resident = 0;
  int64_t n_suspensions = 0, n_suspended_in_krylov = 0;
  std::vector<std::shared_ptr<Request>> held;  // suspended requests
  FILE* log = nullptr;  // per-request records (logdet_server_set_log), one JSON line each
  double busy_us = 0.0;

  void loop();
  int tick(std::vector<std::shared_ptr<Request>>& act);
  void complete(const std::shared_ptr<Request>& r, int state, int rc);
};

void logdet_server::complete(const std::shared_ptr<Request>& r, int state_, int rc_) {
  // Called with mu held.
  if (!r->members.empty()) {
    // A shift-group run: every member finishes with it (the run itself is
    // internal: it is not counted, logged or visible).
    for (size_t t = 0; t < r->members.size(); ++t) {
      auto& mb = r->members[t];
      int st_m = state_, rc_m = rc_;
      if (state_ == RQ_DONE) {
        rc_m = r->solve->assemble_member((int)t, mb->out);
        if (rc_m) st_m = RQ_FAILED;
      }
      mb->t_admit = r->t_admit;
      complete(mb, st_m, rc_m);
    }
    r->state = state_;
    r->t_done = now_us();
    r->solve.reset();
    used -= r->bytes;
    cv_done.notify_all();
    return;
  }
  r->state = state_;
  r->rc = rc_;
  r->t_done = now_us();
  if (state_ == RQ_DONE) {
    r->out.res.latency_ms = (r->t_done - r->t_submit) / 1e3;
    r->out.res.queue_ms = (r->t_admit - r->t_submit) / 1e3;
    if (r->user_per_probe)
      for (size_t i = 0; i < r->out.per_probe.size(); ++i) r->user_per_probe[i] = r->out.per_probe[i];
    if (r->user_zn2)
      for (size_t i = 0; i < r->out.zn2.size(); ++i) r->user_zn2[i] = r->out.zn2[i];
    ++n_completed;
  } else if (state_ == RQ_FAILED) {
    ++n_failed;
  } else if (state_ == RQ_CANCELLED) {
    ++n_cancelled;
  }
  if (log) {
    const SolveCfg& c = r->cfg;
    const logdet_result& o = r->out.res;
    const char* sname = state_ == RQ_DONE ? "done" : state_ == RQ_FAILED ? "failed" : "cancelled";
    fprintf(log,
            "{\"id\": %llu, \"state\": \"%s\", \"rc\": %d, \"n\": %d, \"nnz\": %lld, "
            "\"method\": \"%s\", \"precision\": %d, \"probes\": %d, \"steps\": %d, "
            "\"window\": %d, \"shift\": %.17g, \"seed\": %llu, \"logdet\": %.17g, "
            "\"steps_min\": %d, \"steps_max\": %d, \"status_bits\": %u, "
            "\"latency_ms\": %.3f, \"queue_ms\": %.3f}\n",
            (unsigned long long)r->id, sname, rc_, r->h ? r->h->n : 0, r->h ? r->h->nnz : 0LL,
            c.method == 0 ? "oslq" : "osaiop", c.precision, c.P, c.m, c.k, c.shift,
            (unsigned long long)c.seed, state_ == RQ_DONE ? o.logdet : 0.0,
            state_ == RQ_DONE ? o.steps_min : 0, state_ == RQ_DONE ? o.steps_max : 0,
            state_ == RQ_DONE ? o.status_bits : 0u, (r->t_done - r->t_submit) / 1e3,
            r->t_admit > 0 ? (r->t_admit - r->t_submit) / 1e3 : 0.0);
    fflush(log);
  }
  // Device buffers are freed in stream order, after any work still queued.
  r->solve.reset();
  used -= r->bytes;
  cv_done.notify_all();
}

// Kernel variant of a job (the template width it launches with).
static int width_class(int k) { return k <= 0 ? 0 : k == 1 ? 1 : k == 2 ? 2 : k <= 4 ? 4 : 9; }
template <typename T> static int job_class(const SpmmJob<T>& j) { return width_class(j.ndots); }
// Update jobs with the extra dot (OSA-IOP) run in their own instance.
template <typename T> static int job_class(const UpdJob<T>& j) {
  return width_class(j.nbasis) + (j.extra ? 16 : 0);
}

int logdet_server::tick(std::vector<std::shared_ptr<Request>>& act) {
  NvtxRange nv("logdet server tick");
  // 1. non-Krylov phases, per request
  for (auto& r : act) {
    ISolve* sv = r->solve.get();
    if (!sv || sv->in_krylov()) continue;
    const int ph = sv->phase();
    if (ph == PH_SETUP || ph == PH_MID || ph == PH_FINISH) {
      int rc = sv->run_phase();
      if (rc) r->rc = rc;
    }
  }
  // 2. one batched Krylov step over every request in a Krylov phase, grouped
  //    by element type, CTA size and kernel variant (dots / basis vectors
  //    class): a job never runs in a wider variant than its own, which would
  //    cost registers and occupancy.  Group key: threads * 32 + class.
  auto put = [&](auto& groups, auto& tmp, int th) {
    if (tmp.empty()) return;
    auto& dst = groups[th * 32 + job_class(tmp[0])];
    dst.insert(dst.end(), tmp.begin(), tmp.end());
  };
  std::map<int, std::vector<SpmmJob<double>>> sd;
  std::map<int, std::vector<SpmmJob<float>>> sf;
  std::map<int, std::vector<SpmmJob<bf16>>> sb;
  std::map<int, std::vector<UpdJob<double>>> ud;
  std::map<int, std::vector<UpdJob<float>>> uf;
  std::map<int, std::vector<UpdJob<bf16>>> ub;
  std::map<int, std::vector<SpmmJob<f32x2>>> sx;
  std::map<int, std::vector<UpdJob<f32x2>>> ux;
  std::vector<ScalarJob> coef, norm;
  std::vector<int> wc, wn;
  std::vector<ISolve*> stepping;
  // A solve's jobs of one pass into the groups of its element type.
  auto pass1 = [&](auto& groups, ISolve* sv, int th) {
    typename std::decay_t<decltype(groups)>::mapped_type tmp;
    const int rc = sv->add_pass1(&tmp, coef, wc);
    if (!rc) put(groups, tmp, th);
    return rc;
  };
  auto pass2 = [&](auto& groups, ISolve* sv, int th) {
    typename std::decay_t<decltype(groups)>::mapped_type tmp;
    sv->add_pass2(&tmp, norm, wn);
    put(groups, tmp, th);
  };
  for (auto& r : act) {
    ISolve* sv = r->solve.get();
    if (!sv || !sv->in_krylov() || r->rc) continue;
    const int th = sv->krylov_threads();
    const int ek = sv->elem_kind();
    const int rc = ek == 0   ? pass1(sd, sv, th)
                   : ek == 1 ? pass1(sf, sv, th)
                   : ek == 2 ? pass1(sb, sv, th)
                             : pass1(sx, sv, th);
    if (rc) {
      r->rc = rc;  // this request fails; the others step on
      continue;
    }
    stepping.push_back(sv);
  }
  if (stepping.empty()) return 0;
  for (auto& kv : sd) LD_TRY(launch_spmm_jobs<double>(kv.second, kv.first / 32, st));
  for (auto& kv : sf) LD_TRY(launch_spmm_jobs<float>(kv.second, kv.first / 32, st));
  for (auto& kv : sb) LD_TRY(launch_spmm_jobs<bf16>(kv.second, kv.first / 32, st));
  for (auto& kv : sx) LD_TRY(launch_spmm_jobs<f32x2>(kv.second, kv.first / 32, st));
  LD_TRY(launch_scalar_jobs(coef, wc, SK_COEF, st));
  for (ISolve* sv : stepping) {
    const int th = sv->krylov_threads();
    const int ek = sv->elem_kind();
    if (ek == 0) pass2(ud, sv, th);
    else if (ek == 1) pass2(uf, sv, th);
    else if (ek == 2) pass2(ub, sv, th);
    else pass2(ux, sv, th);
  }
  for (auto& kv : ud) LD_TRY(launch_update_jobs<double>(kv.second, kv.first / 32, st));
  for (auto& kv : uf) LD_TRY(launch_update_jobs<float>(kv.second, kv.first / 32, st));
  for (auto& kv : ub) LD_TRY(launch_update_jobs<bf16>(kv.second, kv.first / 32, st));
  for (auto& kv : ux) LD_TRY(launch_update_jobs<f32x2>(kv.second, kv.first / 32, st));
  if (!norm.empty()) LD_TRY(launch_scalar_jobs(norm, wn, SK_NORM, st));
  for (ISolve* sv : stepping) sv->step_issued();
  n_batched_steps += (int64_t)stepping.size();
  return (int)stepping.size();
}

void logdet_server::loop() {
  cudaSetDevice(device);
  std::vector<std::shared_ptr<Request>> act;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(mu);
      // Admission: FIFO while a slot is free and the budget allows.
      while (!queue.empty() && (int)active.size() < max_slots) {
        auto r = queue.front();
        if (r->cancel) {
          queue.pop_front();
          r->state = RQ_CANCELLED;
          ++n_cancelled;
          for (auto& mb : r->members) {
            mb->state = RQ_CANCELLED;
            ++n_cancelled;
          }
          if (!r->members.empty()) --n_cancelled;  // (a run counts through its members)
          cv_done.notify_all();
          continue;
        }
        if (used + r->bytes > budget) break;
        queue.pop_front();
        used += r->bytes;
        r->state = RQ_RUNNING;
        r->t_admit = now_us();
        active.push_back(r);
        if (r->members.empty()) {
          ++n_admitted;
        } else {
          for (auto& mb : r->members) {
            mb->state = RQ_RUNNING;
            mb->t_admit = r->t_admit;
          }
          n_admitted += (int64_t)r->members.size();
        }
      }
      max_resident = std::max<int64_t>(max_resident, (int64_t)active.size());
      if (active.empty()) {
        if (stop) break;
        cv_work.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      // Running requests that were cancelled leave at the tick boundary;
      // suspended ones leave with their state copied to host memory (a
      // request whose result copies are in flight finishes instead).
      for (size_t i = 0; i < active.size();) {
        auto& r = active[i];
        if (r->cancel) {
          complete(r, RQ_CANCELLED, LOGDET_ECANCEL);
          active.erase(active.begin() + i);
          continue;
        }
        if (r->suspend && !r->rc && (!r->solve || r->solve->phase() != PH_WAIT)) {
          r->suspend = false;
          const bool mid_krylov = r->solve && r->solve->in_krylov();
          const int src = r->solve ? r->solve->suspend() : LOGDET_OK;
          if (src) {
            r->rc = src;
            ++i;
            continue;
          }
          used -= r->bytes;
          r->state = RQ_SUSPENDED;
          held.push_back(r);
          ++n_suspensions;
          if (mid_krylov) ++n_suspended_in_krylov;
          active.erase(active.begin() + i);
          cv_done.notify_all();
          continue;
        }
        r->suspend = false;
        ++i;
      }
      if (active.empty()) continue;
      act = active;
    }
    const double t0 = now_us();
    // Solves for newly admitted requests (allocation happens in their SETUP
    // phase); resumed requests get their device state back.
    for (auto& r : act) {
      if (!r->solve && !r->rc) {
        int rc = LOGDET_OK;
        r->solve = r->group_cfgs.empty() ? make_solve(r->h, r->cfg, st, &rc)
                                         : make_group_solve(r->h, r->group_cfgs, st, &rc);
        if (!r->solve) r->rc = rc ? rc : LOGDET_EINVAL;
      } else if (r->solve && r->solve->suspended() && !r->rc) {
        const int rc = r->solve->resume();
        if (rc) r->rc = rc;
      }
    }
    int rc = tick(act);
    bool issued = rc > 0;
    if (rc < 0) {
      // A launch failed: fail every resident request.
      std::lock_guard<std::mutex> lk(mu);
      for (auto& r : act) r->rc = rc;
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(ev, st);
      ticks.push_back(ev);
    }
    // Keep at most two ticks in flight ahead of the device.  With no Krylov
    // step issued, wait for the oldest tick (or a finishing request) instead
    // of spinning.
    while (ticks.size() > 2 || (!issued && !ticks.empty())) {
      cudaEventSynchronize(ticks.front());
      cudaEventDestroy(ticks.front());
      ticks.pop_front();
      if (!issued) break;
    }
    if (!issued) {
      for (auto& r : act)
        if (r->solve && r->solve->phase() == PH_WAIT) {
          cudaEventSynchronize(r->solve->done_event());
          break;
        }
    }
    ++n_ticks;
    busy_us += now_us() - t0;
    // Completions.
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < active.size();) {
      auto& r = active[i];
      bool gone = false;
      if (r->rc) {
        cudaStreamSynchronize(st);
        complete(r, RQ_FAILED, r->rc);
        gone = true;
      } else if (r->solve && r->solve->phase() == PH_WAIT &&
                 cudaEventQuery(r->solve->done_event()) == cudaSuccess) {
        const int arc = r->members.empty() ? r->solve->assemble(r->out) : LOGDET_OK;
        complete(r, arc ? RQ_FAILED : RQ_DONE, arc);
        gone = true;
      }
      if (gone) active.erase(active.begin() + i);
      else ++i;
    }
  }
  while (!ticks.empty()) {
    cudaEventSynchronize(ticks.front());
    cudaEventDestroy(ticks.front());
    ticks.pop_front();
  }
}

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

int logdet_server_create(size_t budget, int32_t max_slots, void* cuda_stream, logdet_server** out) {
  if (!out || budget == 0 || max_slots < 1) {
    set_error("server: need out != NULL, budget > 0, max_slots >= 1");
    return LOGDET_EINVAL;
  }
  *out = nullptr;
  auto* s = new logdet_server();
  s->budget = budget;
  s->max_slots = max_slots;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    set_error("server: no CUDA device");
    return LOGDET_ECUDA;
  }
  int rc = ensure_pool(s->device);
  if (rc) { delete s; return rc; }
  if (cuda_stream) {
    s->st = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      set_error("server: cudaStreamCreate failed");
      return LOGDET_ECUDA;
    }
    s->own_stream = true;
  }
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return LOGDET_OK;
}

void logdet_server_destroy(logdet_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& r : s->queue) {
      r->state = RQ_CANCELLED;
      ++s->n_cancelled;
      for (auto& mb : r->members) mb->state = RQ_CANCELLED;
      if (!r->members.empty()) s->n_cancelled += (int64_t)r->members.size() - 1;
    }
    s->queue.clear();
    for (auto& r : s->held) {
      r->state = RQ_CANCELLED;
      r->solve.reset();
      ++s->n_cancelled;
    }
    s->held.clear();
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaStreamSynchronize(s->st);
  if (s->own_stream) cudaStreamDestroy(s->st);
  if (s->log) fclose(s->log);
  delete s;
}

int logdet_submit(logdet_server* s, logdet_handle h, int32_t method, int32_t num_probes,
                  int32_t krylov_steps, int32_t iop_window, uint64_t seed, const logdet_opts* opts,
                  uint64_t* req_id) {
  if (!s || !h || !req_id) {
    set_error("submit: NULL server, handle or req_id");
    return LOGDET_EINVAL;
  }
  auto r = std::make_shared<Request>();
  r->h = h;
  SolveCfg& c = r->cfg;
  c = make_solve_cfg(method, num_probes, krylov_steps, iop_window, seed, opts);
  if (opts) {
    r->user_per_probe = opts->per_probe;
    r->user_zn2 = opts->z_norm2;
  }
  LD_TRY(validate_cfg(h, c));
  r->bytes = estimate_solve_bytes(h, c);
  if (r->bytes > s->budget) {
    set_error("submit: request needs ~%zu bytes, more than the server budget %zu", r->bytes, s->budget);
    return LOGDET_ENOMEM;
  }
  r->t_submit = now_us();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      set_error("submit: server is shutting down");
      return LOGDET_ECANCEL;
    }
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->queue.push_back(r);
    ++s->n_submitted;
    *req_id = r->id;
  }
  s->cv_work.notify_all();
  return LOGDET_OK;
}

int logdet_submit_shifts(logdet_server* s, logdet_handle h, int32_t method, int32_t nshift,
                         const double* shifts, int32_t num_probes, int32_t krylov_steps,
                         int32_t iop_window, uint64_t seed0, const logdet_opts* opts,
                         uint64_t* req_ids) {
  if (!s || !h || !shifts || !req_ids) {
    set_error("submit_shifts: NULL server, handle, shifts or req_ids");
    return LOGDET_EINVAL;
  }
  if (nshift < 1) {
    set_error("submit_shifts: nshift=%d must be >= 1", nshift);
    return LOGDET_EINVAL;
  }
  std::vector<SolveCfg> cfgs;
  for (int t = 0; t < nshift; ++t) {
    SolveCfg c = make_solve_cfg(method, num_probes, krylov_steps, iop_window, seed0 + (uint64_t)t,
                                opts);
    c.shift = shifts[t];
    cfgs.push_back(c);
  }
  std::vector<std::pair<size_t, size_t>> runs;
  LD_TRY(shift_runs(h, cfgs, runs));
  std::vector<std::shared_ptr<Request>> rs;
  const double now = now_us();
  for (const auto& rg : runs) {
    auto run = std::make_shared<Request>();
    run->h = h;
    run->group_cfgs.assign(cfgs.begin() + rg.first, cfgs.begin() + rg.second);
    run->cfg = run->group_cfgs[0];
    run->t_submit = now;
    for (const SolveCfg& c : run->group_cfgs) run->bytes += estimate_solve_bytes(h, c);
    if (run->bytes > s->budget) {
      set_error("submit_shifts: a run of %zu shifts needs ~%zu bytes, more than the budget %zu",
                run->group_cfgs.size(), run->bytes, s->budget);
      return LOGDET_ENOMEM;
    }
    for (const SolveCfg& c : run->group_cfgs) {
      auto mb = std::make_shared<Request>();
      mb->h = h;
      mb->cfg = c;
      mb->t_submit = now;
      mb->run = run;
      run->members.push_back(mb);
    }
    rs.push_back(run);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      set_error("submit_shifts: server is shutting down");
      return LOGDET_ECANCEL;
    }
    size_t t = 0;
    for (auto& run : rs) {
      run->id = 0;  // internal
      for (auto& mb : run->members) {
        mb->id = s->next_id++;
        s->all[mb->id] = mb;
        req_ids[t++] = mb->id;
        ++s->n_submitted;
      }
      s->queue.push_back(run);
    }
  }
  s->cv_work.notify_all();
  return LOGDET_OK;
}

int logdet_estimate_bytes(logdet_handle h, int32_t method, int32_t num_probes, int32_t krylov_steps,
                          int32_t iop_window, const logdet_opts* opts, size_t* bytes) {
  if (!h || !bytes) { set_error("estimate_bytes: NULL argument"); return LOGDET_EINVAL; }
  const SolveCfg c = make_solve_cfg(method, num_probes, krylov_steps, iop_window, 0, opts);
  LD_TRY(validate_cfg(h, c));
  *bytes = estimate_solve_bytes(h, c);
  return LOGDET_OK;
}

static int result_of(const std::shared_ptr<Request>& r, logdet_result* out) {
  switch (r->state) {
    case RQ_QUEUED:
    case RQ_RUNNING:
    case RQ_SUSPENDED: return LOGDET_PENDING;
    case RQ_DONE:
      if (out) *out = r->out.res;
      return LOGDET_OK;
    case RQ_CANCELLED: return LOGDET_ECANCEL;
    default: return r->rc ? r->rc : LOGDET_ECUDA;
  }
}

int logdet_poll(logdet_server* s, uint64_t id, logdet_result* out) {
  if (!s) { set_error("poll: NULL server"); return LOGDET_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) { set_error("poll: unknown request %llu", (unsigned long long)id); return LOGDET_ENOENT; }
  return result_of(it->second, out);
}

int logdet_wait(logdet_server* s, uint64_t id, int64_t timeout_us, logdet_result* out) {
  if (!s) { set_error("wait: NULL server"); return LOGDET_EINVAL; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) { set_error("wait: unknown request %llu", (unsigned long long)id); return LOGDET_ENOENT; }
  auto r = it->second;
  auto pending = [&] {
    return r->state == RQ_QUEUED || r->state == RQ_RUNNING || r->state == RQ_SUSPENDED;
  };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, [&] { return !pending() || s->stop; });
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !pending(); })) {
    set_error("wait: request %llu still pending after %lld us", (unsigned long long)id, (long long)timeout_us);
    return LOGDET_ETIMEOUT;
  }
  return result_of(r, out);
}

int logdet_cancel(logdet_server* s, uint64_t id) {
  if (!s) { set_error("cancel: NULL server"); return LOGDET_EINVAL; }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) { set_error("cancel: unknown request"); return LOGDET_ENOENT; }
    auto r = it->second;
    if (auto run = r->run.lock()) {  // a shift-group member: its whole run stops
      run->cancel = true;
      r = run;
    }
    r->cancel = true;
    if (r->state == RQ_SUSPENDED) {  // held: no slot and no budget to give back
      for (size_t i = 0; i < s->held.size(); ++i)
        if (s->held[i] == r) {
          s->held.erase(s->held.begin() + i);
          break;
        }
      r->state = RQ_CANCELLED;
      r->solve.reset();
      ++s->n_cancelled;
      s->cv_done.notify_all();
    }
  }
  s->cv_work.notify_all();
  return LOGDET_OK;
}

int logdet_release(logdet_server* s, uint64_t id) {
  if (!s) { set_error("release: NULL server"); return LOGDET_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) { set_error("release: unknown request"); return LOGDET_ENOENT; }
  const int st = it->second->state;
  if (st == RQ_QUEUED || st == RQ_RUNNING || st == RQ_SUSPENDED) {
    set_error("release: request still pending");
    return LOGDET_PENDING;
  }
  s->all.erase(it);
  return LOGDET_OK;
}

int logdet_server_set_log(logdet_server* s, const char* path) {
  if (!s) { set_error("set_log: NULL server"); return LOGDET_EINVAL; }
  FILE* f = nullptr;
  if (path && path[0]) {
    f = fopen(path, "a");
    if (!f) { set_error("set_log: cannot open %s", path); return LOGDET_EINVAL; }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->log) fclose(s->log);
  s->log = f;
  return LOGDET_OK;
}

int logdet_suspend(logdet_server* s, uint64_t id) {
  if (!s) { set_error("suspend: NULL server"); return LOGDET_EINVAL; }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) { set_error("suspend: unknown request"); return LOGDET_ENOENT; }
    auto r = it->second;
    if (!r->run.expired()) {
      set_error("suspend: request %llu is a shift-group member", (unsigned long long)id);
      return LOGDET_EINVAL;
    }
    if (r->state == RQ_QUEUED) {  // not admitted yet: leaves the queue, holds nothing
      for (size_t i = 0; i < s->queue.size(); ++i)
        if (s->queue[i] == r) {
          s->queue.erase(s->queue.begin() + i);
          break;
        }
      r->state = RQ_SUSPENDED;
      s->held.push_back(r);
      ++s->n_suspensions;
      return LOGDET_OK;
    }
    if (r->state != RQ_RUNNING) {
      set_error("suspend: request %llu is not queued or running", (unsigned long long)id);
      return LOGDET_EINVAL;
    }
    r->suspend = true;
  }
  s->cv_work.notify_all();
  return LOGDET_OK;
}

int logdet_resume(logdet_server* s, uint64_t id) {
  if (!s) { set_error("resume: NULL server"); return LOGDET_EINVAL; }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) { set_error("resume: unknown request"); return LOGDET_ENOENT; }
    auto r = it->second;
    if (r->state == RQ_RUNNING && r->suspend) {  // not acted on yet: withdrawn
      r->suspend = false;
      return LOGDET_OK;
    }
    if (r->state != RQ_SUSPENDED) {
      set_error("resume: request %llu is not suspended", (unsigned long long)id);
      return LOGDET_EINVAL;
    }
    for (size_t i = 0; i < s->held.size(); ++i)
      if (s->held[i] == r) {
        s->held.erase(s->held.begin() + i);
        break;
      }
    r->state = RQ_QUEUED;
    s->queue.push_front(r);
  }
  s->cv_work.notify_all();
  return LOGDET_OK;
}

int logdet_server_stats(logdet_server* s, logdet_stats* out) {
  if (!s || !out) { set_error("stats: NULL argument"); return LOGDET_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->n_submitted;
  out->admitted = s->n_admitted;
  out->completed = s->n_completed;
  out->failed = s->n_failed;
  out->cancelled = s->n_cancelled;
  out->queued = (int64_t)s->queue.size();
  out->resident = (int64_t)s->active.size();
  out->max_resident = s->max_resident;
  out->ticks = s->n_ticks;
  out->batched_steps = s->n_batched_steps;
  out->bytes_in_use = s->used;
  out->bytes_budget = s->budget;
  out->busy_ms = s->busy_us / 1e3;
  out->suspended = (int64_t)s->held.size();
  out->suspensions = s->n_suspensions;
  out->suspended_in_krylov = s->n_suspended_in_krylov;
  return LOGDET_OK;
}

}  // extern "C"
