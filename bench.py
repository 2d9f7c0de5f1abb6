#!/usr/bin/env python3
"""Throughput benchmark of the OSLQ / OSA-IOP hot path on one or more GPUs.

Workload (one "step"): the 3D 7-point Dirichlet Laplacian on a 128^3 grid plus
0.01 I (n = 2,097,152, nnz = 14,581,760, FP64 values), 60 Rademacher probes,
50 Krylov steps; OSLQ once and OSA-IOP with windows k = 2, 4 and 8 -- four
log-determinant solves that together run every step of the hot path (sketch,
Hutch++ QR and projection, SpMM + window dots, window update + norms,
tridiagonal Gauss rules, Hessenberg logarithms, assembly).

  python bench.py [--gpus N --steps K --warmup W]           # CUDA path
  python bench.py --impl reference [...]                    # FP64 CPU oracle

At N = 1 the line also carries three bounded objects, each with its own clock
record: matern_mixed (the mixed-precision configuration: Matern 1024^2, FP32
vectors, OSLQ m = 80, 120 probes; solves/s, error against the FP64 CUDA path,
HBM roofline of the Krylov passes), serving (the continuous-batching
configuration at a reduced request count: mixed batched server against plain
FP64 one at a time, solves/s and p50/p99 latency) and irregular_batch (8
shifts of a 2M-row power-law graph Laplacian, OSA-IOP m = 100, k = 4, FP32
vectors: as one shift group, through the server and one after the other;
error of the extreme shifts against FP64; then the forms within the 1e-4
budget, the same group with FP64 vectors and with double-float vectors).

Under torchrun every rank solves its own copy of the workload (independent
problems, no data-path collective: weak scaling); the barrier and the max over
ranks of the timed region use torch.distributed.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "logdet solves/s, p50/p99 at rel err ≤1e-4 vs FP64; SpMM+Krylov HBM GB/s"
UNIT = "solves/s"
GRID, SHIFT, PROBES, STEPS_M, WINDOWS = 128, 0.01, 60, 50, (2, 4, 8)
SOLVES_PER_STEP = 1 + len(WINDOWS)
# FP64 FMA peak of this GPU: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.070 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # FP32 FMA lanes x clock
PROFILE_MD = os.path.join(ROOT, "profiles", "k_spmm_fp64_laplacian3d_100.md")  # noqa
CSRC = os.path.join(ROOT, "paper_2606_07004_gb300", "csrc")
KRYLOV_SRC = os.path.join(CSRC, "krylov.cu")


def workload_config():
    return {
        "workload": f"3D 7-point Dirichlet Laplacian {GRID}^3 + {SHIFT} I (n=2097152, "
                    "nnz=14581760), FP64; per step OSLQ + OSA-IOP k=2,4,8, m=50, 60 probes",
        "matrix": "laplacian_3d", "grid": GRID, "shift": SHIFT, "n": GRID ** 3, "nnz": 14581760,
        "num_probes": PROBES, "krylov_steps": STEPS_M, "iop_windows": list(WINDOWS),
        "solves_per_step": SOLVES_PER_STEP, "seed": "1000 + step index",
        "l2": "inputs larger than L2 (CSR 183 MB, 40-probe FP64 block 671 MB per vector)",
        "parallelism": "replicas (one independent workload per GPU)",
    }


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# distributed helpers
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws, backend):
    if ws <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def aggregate_value(solves_per_rank: int, world_size: int, t_max: float) -> float:
    """Whole-job throughput: every rank solves its own copy of the workload, so
    the job completes world_size * solves_per_rank solves in the slowest rank's time."""
    return solves_per_rank * world_size / t_max


def max_over_ranks(dist, x, device=None):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of one GPU while a region runs, kept in
    a temporary file (or under --clock-dir when given) and summarised at stop."""
    clock_dir = None

    def __init__(self, gpu_index, tag="main"):
        import tempfile
        self.proc = None
        self.gpu = gpu_index
        if self.clock_dir:
            os.makedirs(self.clock_dir, exist_ok=True)
            self.path = os.path.join(self.clock_dir, f"clocks_{tag}_gpu{gpu_index}.csv")
            self.keep = True
        else:
            fd, self.path = tempfile.mkstemp(prefix=f"logdet_clocks_{tag}_", suffix=".csv")
            os.close(fd)
            self.keep = False

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_FIELDS}", "--format=csv",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, names = [], [], set()
        keys = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit():
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for k, v in zip(keys, parts[5:9]):
                if v.lower() == "active":
                    names.add(k)
        if not self.keep:
            try:
                os.remove(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(names)}


# ---------------------------------------------------------------------------
# CPU oracle sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(seed: int) -> dict:
    """Time the FP64 oracle on a bounded sample of one step and extrapolate.

    OSLQ: the full Hutch++ split (Y = J S, orth, projection) plus the Lanczos
    quadrature of one range probe and one residual probe; a full solve is
    split + 20 x (range probe) + 20 x (residual probe).  OSA-IOP (each k): one
    L-action by Algorithm 1 (a residual probe) plus an orth + projection of a
    same-size sketch; a full solve is 60 L-actions + that split.
    """
    import numpy as np
    import oracle as O
    from oracle import estimators as E
    import workloads as W

    A = W.laplacian_3d(GRID, shift=SHIFT)
    Q = A.to_scipy()
    n = A.n
    s = PROBES // 3
    r = PROBES - 2 * s
    lo, hi = O.spectral_interval(Q)
    out = {}
    t0 = time.perf_counter()
    J = Q / hi
    S = O.rademacher_block(seed, 0, n, s)
    G = O.rademacher_block(seed, 1, n, r)
    Y = J @ S
    Aq = O.orth(Y)
    Z = G - Aq @ (Aq.T @ G)
    t_split = time.perf_counter() - t0
    t0 = time.perf_counter()
    al, be = O.lanczos(J, Aq[:, 0], STEPS_M)
    O.gauss_quadrature_log(al, be)
    t_q = time.perf_counter() - t0
    t0 = time.perf_counter()
    al, be = O.lanczos(J, Z[:, 0], STEPS_M)
    O.gauss_quadrature_log(al, be)
    t_z = time.perf_counter() - t0
    out["oslq"] = t_split + s * t_q + r * t_z
    gamma = math.sqrt(lo * hi)
    Qt = Q / gamma
    shift = math.log(gamma / lo)
    t0 = time.perf_counter()
    Aq2 = O.orth(Y)
    Aq2 @ (Aq2.T @ G)
    t_sp = time.perf_counter() - t0          # the OSA-IOP split (orth + projection)
    for k in WINDOWS:
        t0 = time.perf_counter()
        y = E.iop_log_action(Qt, Z[:, 0], STEPS_M, k, shift)
        float(np.dot(Z[:, 0], y))
        t_act = time.perf_counter() - t0
        out[f"osaiop_k{k}"] = (2 * s + r) * t_act + t_sp
    total = sum(out.values())
    return {"est_solve_s": out, "est_step_s": total, "solves_per_s": SOLVES_PER_STEP / total,
            "split_s": {"oslq": t_split, "osaiop": t_sp}}


def run_oracle_sample_child(seed: int, all_cores: bool = False) -> dict:
    """Run oracle_sample in a fresh single-threaded interpreter (BLAS threads = 1),
    and with all_cores also the all-cores sample (processes spawned there)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    t0 = time.perf_counter()
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample-child", str(seed)]
    if all_cores:
        cmd.append("--oracle-all-cores")
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {r.stderr[-2000:]}")
    res = json.loads(r.stdout.strip().splitlines()[-1])
    res["wall_s"] = time.perf_counter() - t0
    return res


def _pool_probe_worker(seed, idx, kind, k, grid, barrier, out):
    """One worker of the all-cores sample: builds the operator and its probe
    (untimed), waits for the others, then times one Lanczos quadrature
    (kind 'q') or one Algorithm-1 L-action with window k (kind 'a')."""
    import numpy as np
    import oracle as O
    from oracle import estimators as E
    import workloads as W
    Q = W.laplacian_3d(grid, shift=SHIFT).to_scipy()
    lo, hi = O.spectral_interval(Q)
    v = O.rademacher_block(seed, 1, Q.shape[0], idx + 1, 0)[:, idx].copy()
    if kind == "q":
        J = Q / hi
        v /= np.linalg.norm(v)
    else:
        gamma = math.sqrt(lo * hi)
        Qt = Q / gamma
        shift = math.log(gamma / lo)
    barrier.wait()
    t0 = time.perf_counter()
    if kind == "q":
        al, be = O.lanczos(J, v, STEPS_M)
        O.gauss_quadrature_log(al, be)
    else:
        y = E.iop_log_action(Qt, v, STEPS_M, k, shift)
        float(np.dot(v, y))
    out[idx] = time.perf_counter() - t0


def oracle_sample_all_cores(seed: int, one_thread: dict, grid: int = GRID) -> dict:
    """The oracle with its independent probes spread over all host cores: C
    processes (spawn, BLAS threads = 1 each) run C probes at once; a solve
    takes ceil(probes / C) such rounds plus the single-threaded Hutch++ split
    measured by the one-thread sample."""
    import multiprocessing as mp
    C = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    s = PROBES // 3
    r = PROBES - 2 * s

    def rounds(kind, k=0):
        barrier = ctx.Barrier(C)
        out = ctx.Array("d", C)
        ps = [ctx.Process(target=_pool_probe_worker, args=(seed, i, kind, k, grid, barrier, out))
              for i in range(C)]
        for p_ in ps:
            p_.start()
        for p_ in ps:
            p_.join()
        if any(p_.exitcode != 0 for p_ in ps):
            raise RuntimeError("an oracle worker failed")
        return max(out[:])

    split = one_thread["split_s"]
    est = {"oslq": split["oslq"] + math.ceil((s + r) / C) * rounds("q")}
    for k in WINDOWS:
        est[f"osaiop_k{k}"] = split["osaiop"] + math.ceil((2 * s + r) / C) * rounds("a", k)
    total = sum(est.values())
    return {"est_solve_s": est, "est_step_s": total, "solves_per_s": SOLVES_PER_STEP / total,
            "cores": C}


SAMPLE_DESC = ("FP64 NumPy/SciPy oracle, 1 thread: full Hutch++ split + 2 Lanczos probes for OSLQ, "
               "1 Algorithm-1 L-action + orth/projection per OSA-IOP window; per-solve time "
               "extrapolated to 40 Lanczos probes (OSLQ) and 60 L-actions (OSA-IOP)")


def reference_arm(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    vals, steps = [], []
    for i in range(args.warmup + args.steps):
        res = run_oracle_sample_child(1000 + i)
        if i >= args.warmup:
            vals.append(res["solves_per_s"])
            steps.append(res["est_step_s"])
    v = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": SAMPLE_DESC},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# CUDA arm
# ---------------------------------------------------------------------------
def spmm_kernel_digest():
    """SHA-256 of the CSR SpMM kernel's source: krylov.cu from its gather
    batch constant (the vector-load helper, the launch-bound helper and the
    tile loop follow) through the kernel's closing brace, then krylov.cuh and
    common.cuh (the headers it includes).  Edits elsewhere in krylov.cu leave
    it alone."""
    text = open(KRYLOV_SRC).read()
    i0 = text.index("constexpr int kGather = 4;")
    i1 = text.index("k_spmm(const __grid_constant__ SpmmBatch<T> B) {", i0)
    depth, j = 0, text.index("{", i1)
    while True:
        c = text[j]
        depth += (c == "{") - (c == "}")
        j += 1
        if depth == 0:
            break
    h = hashlib.sha256(text[i0:j].encode())
    for name in ("krylov.cuh", "common.cuh"):
        h.update(open(os.path.join(CSRC, name), "rb").read())
    return h.hexdigest()


def traffic_ratio_from_profile():
    """DRAM bytes / algorithmic bytes of the SpMM kernel from the committed ncu
    summary (a smaller grid of the same operator), if it was taken on the
    current kernel source; the bench scales it by its own per-launch bytes."""
    try:
        text = open(PROFILE_MD).read()
        src = spmm_kernel_digest()
        m_src = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
        m_tr = re.search(r"traffic_over_algorithmic:\s*([0-9.eE+]+)", text)
        if m_src and m_tr and m_src.group(1) == src:
            return float(m_tr.group(1))
    except Exception:
        pass
    return None


def d2h_bytes_per_step(n_blocks_gersh: int) -> int:
    """Device-to-host bytes the library copies per step (counted from its copies)."""
    s = PROBES // 3
    b = PROBES
    ld = b + (b % 2)
    lds = s + (s % 2)
    total = 2 * 8 * n_blocks_gersh + 4          # Gershgorin partials + flags (handle creation)
    per_collect = ld * (8 + 4 + 4) + ld * (STEPS_M + 2) * 8
    total += per_collect + 4 * s                  # OSLQ: results + kept-column flags
    for _ in WINDOWS:
        total += per_collect + 4 * s + 4 * lds    # OSA-IOP: + phase-1 status
    return total


def cuda_arm(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(ws, "nccl")
    dev = torch.device("cuda", local)
    from paper_2606_07004_gb300 import binding as B
    import workloads as W

    A = W.laplacian_3d(GRID, shift=SHIFT)
    stream = torch.cuda.Stream(device=dev)
    h = B.Handle.from_csr(A)

    at = 1 if args.autotune else 0

    def run_step(handle, seed, lat):
        rs = [("oslq", handle.oslq(PROBES, STEPS_M, seed=seed, stream=stream, autotune=at))]
        for k in WINDOWS:
            rs.append((f"osaiop_k{k}", handle.osaiop(PROBES, STEPS_M, iop_window=k, seed=seed,
                                                     stream=stream, autotune=at)))
        for name, r in rs:
            lat.setdefault(name, []).append(r.device_ms)
        return rs

    for i in range(args.warmup):
        run_step(h, 1000 + i, {})
    torch.cuda.synchronize()

    # ---- device-timed region ----
    lat = {}
    clocks = ClockSampler(local)
    B.logdet_profile_reset()
    B.logdet_profile_enable(True)
    launches0 = B.logdet_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        run_step(h, 1000 + args.warmup + i, lat)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    launches = B.logdet_launch_count() - launches0
    B.logdet_profile_enable(False)
    prof = B.profile_snapshot()
    t_dev = e0.elapsed_time(e1) / 1e3
    t_dev_max = max_over_ranks(dist, t_dev, dev)
    value = aggregate_value(SOLVES_PER_STEP * args.steps, ws, t_dev_max)

    # ---- end-to-end through the public API from pinned host buffers ----
    rp = torch.from_numpy(A.rowptr).pin_memory().numpy()
    ci = torch.from_numpy(A.colind).pin_memory().numpy()
    vv = torch.from_numpy(A.vals).pin_memory().numpy()
    h2d = rp.nbytes + ci.nbytes + vv.nbytes
    e2e_steps = max(1, min(args.steps, 3))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        with B.Handle(A.n, rp, ci, vv) as he:
            rs = run_step(he, 5000 + i, {})
            _ = [float(r.logdet) for _, r in rs]
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(dist, time.perf_counter() - t0, dev)
    e2e_value = aggregate_value(SOLVES_PER_STEP * e2e_steps, ws, t_e2e)
    h.close()

    pk, pk_kind = peaks()
    sp = prof["spmm"]
    achieved = sp["flops"] / (sp["ms"] / 1e3) / 1e12 if sp["ms"] > 0 else 0.0
    kr_bytes = prof["spmm"]["bytes"] + prof["update"]["bytes"]
    kr_ms = prof["spmm"]["ms"] + prof["update"]["ms"]
    kr_gbs = kr_bytes / (kr_ms / 1e3) / 1e9 if kr_ms > 0 else 0.0
    ratio = traffic_ratio_from_profile()
    traffic = ratio * sp["bytes"] / max(1, sp["launches"]) if ratio else None

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(workload_config(), autotune=bool(args.autotune)),
        "roofline": {
            "kernel": "k_spmm<double> (SpMM + fused window dots)",
            "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": traffic,
            "peak_source": "FP64 FMA peak from unit counts and clock: 152 SMs x 2 DFMA/clk x "
                           "2 flop x 2.070 GHz (a DFMA loop measured 1.20 TFLOP/s)",
            "launches": sp["launches"], "avg_launch_ms": sp["ms"] / max(1, sp["launches"]),
            "flops_per_launch": sp["flops"] / max(1, sp["launches"]),
            "bytes_per_launch": sp["bytes"] / max(1, sp["launches"]),
            "algorithmic_gbs": sp["bytes"] / (sp["ms"] / 1e3) / 1e9 if sp["ms"] > 0 else 0.0,
        },
        "krylov_hbm": {"algorithmic_gbs": kr_gbs, "peak_gbs": pk.get("hbm_gbs"),
                       "frac": kr_gbs / pk.get("hbm_gbs", 6776.6),
                       "peak_source": pk_kind,
                       "note": "SpMM + update passes; FP64 here is ALU-bound, see roofline"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": d2h_bytes_per_step(min((A.n + 255) // 256, 4 * 152)),
                "steps": e2e_steps,
                "includes": "logdet_create from pinned host CSR (validation, H2D, Gershgorin), "
                            "4 solves, results to host, logdet_destroy"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "latency_ms": {k: {"p50": pct(v, 0.5), "p99": pct(v, 0.99), "mean": statistics.mean(v)}
                       for k, v in lat.items()},
        "latency_note": "device time per blocking solve of each kind (CUDA events); serving "
                        "latencies (submit to result) are in the serving object",
        "kernel_ms": {k: v["ms"] / args.steps for k, v in prof.items()},
    }
    if rank == 0 and ws == 1 and not args.no_extras:
        # The mixed-precision, serving and batched irregular configurations,
        # bounded, each with its own clock record (one GPU only: at N > 1
        # every rank would repeat them).
        for key, fn in (("matern_mixed", lambda: matern_measure(args.extra_solves, 2, at)),
                        ("serving", lambda: serving_measure(args.serving_requests, args.slots,
                                                            args.budget_gb)),
                        ("irregular_batch", lambda: multishift_measure(args.budget_gb, at,
                                                                       fp64_all=False))):
            try:
                line[key] = fn()
            except Exception as e:  # reported, not hidden
                line[key] = {"error": f"{type(e).__name__}: {str(e)[:300]}"}
        if "serving" in line and "requests" in line["serving"]:
            line["serving"]["note"] = ("the configured stream has 2000 requests; this line runs "
                                       "%d of the same law to bound the benchmark's run time"
                                       % args.serving_requests)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            res = run_oracle_sample_child(1000, all_cores=True)
            line["cpu_baseline"] = {"value": res["solves_per_s"], "unit": UNIT, "cores": 1,
                                    "kind": "oracle", "sample": SAMPLE_DESC,
                                    "est_solve_s": res["est_solve_s"], "wall_s": res["wall_s"]}
            ac = res.get("all_cores")
            if ac:
                line["cpu_baseline"]["all_cores"] = {
                    "value": ac["solves_per_s"], "unit": UNIT, "cores": ac["cores"],
                    "kind": "oracle", "est_solve_s": ac["est_solve_s"],
                    "sample": "the same oracle with its independent probes on all host cores "
                              "(one spawned process per core, BLAS threads = 1; C probes per "
                              "round, the Hutch++ split single-threaded)"}
        except Exception as e:  # reported, not hidden
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": SAMPLE_DESC, "error": str(e)[:300]}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


MATERN_N, MATERN_K2, MATERN_P, MATERN_M = 1024, 0.05, 120, 80


def matern_measure(solves: int, warmup: int, autotune: int, bf16_trial: bool = False) -> dict:
    """Mixed-precision workload: SPDE Matern precision (0.05 I + L_2D)^2 on a
    1024^2 grid (n = 1,048,576, 13-point stencil), FP32 values and vectors,
    compensated FP32 dots and Hutch++ split, FP64 small solves; OSLQ m = 80
    with 120 probes.  Solves/s (CUDA events on the solve stream, inputs
    resident), the HBM roofline of the Krylov passes, per-solve device
    latency, and the relative error against the FP64 CUDA path on the same
    (FP32-valued) matrix and seed.  With bf16_trial, the same solves with the
    Krylov vectors stored in BF16."""
    import numpy as np
    import torch
    from paper_2606_07004_gb300 import binding as B
    import workloads as W

    A = W.matern_2d(MATERN_N, MATERN_K2, dtype=np.float32)
    h = B.Handle.from_csr(A)
    P, m = MATERN_P, MATERN_M
    stream = torch.cuda.Stream()
    for i in range(warmup):
        h.oslq(P, m, seed=i, precision=B.MIXED_FP32, stream=stream, autotune=autotune)
    torch.cuda.synchronize()
    B.logdet_profile_reset()
    B.logdet_profile_enable(True)
    clocks = ClockSampler(torch.cuda.current_device(), "matern")
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = [h.oslq(P, m, seed=100 + i, precision=B.MIXED_FP32, stream=stream, autotune=autotune)
           for i in range(solves)]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    B.logdet_profile_enable(False)
    prof = B.profile_snapshot()
    t = e0.elapsed_time(e1) / 1e3
    ref = h.oslq(P, m, seed=100, precision=B.FP64, stream=stream)
    err = abs(res[0].logdet - ref.logdet) / abs(ref.logdet)
    pk, kind = peaks()
    kb = prof["spmm"]["bytes"] + prof["update"]["bytes"]
    kms = prof["spmm"]["ms"] + prof["update"]["ms"]
    gbs = kb / (kms / 1e3) / 1e9
    sp_ = prof["spmm"]
    lat = [r.device_ms for r in res]
    out = {
        "workload": "Matern (0.05 I + L)^2 on 1024^2 (n=1048576, nnz=%d), mixed FP32, OSLQ m=80, "
                    "120 probes, seed 100 + solve index" % A.nnz,
        "value": solves / t, "unit": UNIT, "solves": solves, "warmup": warmup,
        "dtype": "f32 (compensated dots and Hutch++ Gram sums; FP64 small solves)",
        "rel_err_vs_fp64": err, "within_1e-4": err <= 1e-4, "logdet": res[0].logdet,
        "logdet_fp64": ref.logdet, "fp64_solve_ms": ref.device_ms,
        "latency_ms": {"p50": _pct(lat, 0.5), "p99": _pct(lat, 0.99),
                       "what": "device time per blocking solve (CUDA events)"},
        "roofline": {"kernels": "k_spmm_sweep<float> + k_update<float> (SpMM + Krylov passes)",
                     "bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / pk["hbm_gbs"], "peak_source": kind,
                     "spmm_gbs": sp_["bytes"] / (sp_["ms"] / 1e3) / 1e9,
                     "update_gbs": prof["update"]["bytes"] / (prof["update"]["ms"] / 1e3) / 1e9},
        "kernel_ms_per_solve": {k: v["ms"] / solves for k, v in prof.items()},
        "clocks": clk,
    }
    if bf16_trial:
        h.oslq(P, m, seed=0, precision=B.MIXED_BF16VEC)
        B.logdet_profile_reset()
        B.logdet_profile_enable(True)
        e0.record(stream)
        rb = [h.oslq(P, m, seed=100 + i, precision=B.MIXED_BF16VEC, stream=stream)
              for i in range(solves)]
        e1.record(stream)
        torch.cuda.synchronize()
        B.logdet_profile_enable(False)
        pb = B.profile_snapshot()
        tb = e0.elapsed_time(e1) / 1e3
        errb = abs(rb[0].logdet - ref.logdet) / abs(ref.logdet)
        kbb = pb["spmm"]["bytes"] + pb["update"]["bytes"]
        kmb = pb["spmm"]["ms"] + pb["update"]["ms"]
        out["bf16_vector_trial"] = {
            "value": solves / tb, "unit": UNIT, "rel_err_vs_fp64": errb, "within_1e-4": errb <= 1e-4,
            "krylov_gbs": kbb / (kmb / 1e3) / 1e9,
            "kernel_ms_per_solve": {k: v["ms"] / solves for k, v in pb.items()}}
    h.close()
    return out


def matern_case(args):
    """--workload matern: the mixed-precision line on its own, with the BF16
    vector-storage trial."""
    out = matern_measure(args.steps, args.warmup, args.autotune, bf16_trial=True)
    print(json.dumps(dict(out, metric=METRIC)))
    return 0


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(math.ceil(q * len(xs))) - 1))]


SERVING_P, SERVING_M = 30, 50


def serving_requests(N: int, seed: int = 2024):
    """The request stream of the serving workload: request i has type uniform
    over {2D 5-point Laplacian, 3D 7-point Laplacian, Matern}, a size n drawn
    log-uniformly from [1e4, 4e6] and rounded to a grid side (sqrt n for the 2D
    grids, cbrt n for the 3D grid), and a value t drawn log-uniformly from
    [1e-3, 1]: the diagonal shift of a Laplacian (Q + t I, applied
    matrix-free), the kappa^2 of a Matern operator (k^2 I + L)^2.  Seed =
    request index.  Returns [(type, side, t)]."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(N):
        typ = ("l2d", "l3d", "mat")[int(rng.integers(3))]
        n = math.exp(rng.uniform(math.log(1e4), math.log(4e6)))
        t = math.exp(rng.uniform(math.log(1e-3), 0.0))
        side = int(round(n ** (1 / 3))) if typ == "l3d" else int(round(n ** 0.5))
        out.append((typ, side, t))
    return out


def serving_measure(N: int, slots: int, budget_gb: float) -> dict:
    """Continuous-batching serving workload (a GP hyper-parameter search's
    stream of log-determinants; request law in serving_requests), OSLQ m = 50
    with 30 probes per request.  The mixed-precision batched server is timed on
    a burst (all requests at t = 0: capacity) and on a Poisson stream at 0.8 x
    that capacity; the plain FP64 form is timed one blocking solve at a time
    and its FIFO queue replayed on the same arrival times.  Latencies are host
    wall clock, submit to result."""
    import threading
    from concurrent.futures import ThreadPoolExecutor
    import numpy as np
    import torch
    from paper_2606_07004_gb300 import binding as B
    import workloads as W

    reqs = serving_requests(N)
    t_build = time.perf_counter()
    keys = sorted({(typ, side, t if typ == "mat" else 0.0) for typ, side, t in reqs})

    def make(key):
        typ, side, k2 = key
        if typ == "l3d":
            return W.laplacian_3d(side)
        if typ == "l2d":
            return W.laplacian_2d(side)
        return W.matern_2d(side, k2)

    handles, rows = {}, 0
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        for key, A in zip(keys, ex.map(make, keys)):
            handles[key] = B.Handle.from_csr(A)
            rows += A.n
    t_build = time.perf_counter() - t_build
    jobs = []
    for i, (typ, side, t) in enumerate(reqs):
        key = (typ, side, t if typ == "mat" else 0.0)
        jobs.append((handles[key], 0.0 if typ == "mat" else t, i))
    P, m = SERVING_P, SERVING_M
    budget = int(budget_gb * (1 << 30))
    clocks = ClockSampler(torch.cuda.current_device(), "serving")
    clocks.start()
    # 1. burst through the server (mixed FP32): capacity
    with B.Server(budget, max_slots=slots) as srv:
        srv.wait(srv.submit(jobs[0][0], B.METHOD_OSLQ, P, m, seed=0, precision=B.MIXED_FP32,
                            shift=jobs[0][1]))  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = [srv.submit(h, B.METHOD_OSLQ, P, m, seed=s, precision=B.MIXED_FP32, shift=sh)
               for h, sh, s in jobs]
        burst = [srv.wait(i) for i in ids]
        t_burst = time.perf_counter() - t0
        st_burst = srv.stats()
    cap = N / t_burst
    lam = 0.8 * cap
    arrivals = np.cumsum(np.random.default_rng(7).exponential(1.0 / lam, N))
    # 2. Poisson stream through the server
    with B.Server(budget, max_slots=slots) as srv:
        ids = [None] * N
        t0 = time.perf_counter()

        def feeder():
            for i, (h, sh, s) in enumerate(jobs):
                dt = arrivals[i] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                ids[i] = srv.submit(h, B.METHOD_OSLQ, P, m, seed=s, precision=B.MIXED_FP32, shift=sh)

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        stream = [srv.wait(i) for i in ids]
        t_stream = time.perf_counter() - t0
        st_stream = srv.stats()
    lat_srv = [r.latency_ms for r in stream]
    # 3. plain FP64 one at a time (blocking), FIFO replay on the same arrivals
    jobs[0][0].oslq(P, m, seed=0, shift=jobs[0][1])  # warm-up
    svc, r64 = [], []
    for h, sh, s in jobs:
        t1 = time.perf_counter()
        r64.append(h.oslq(P, m, seed=s, shift=sh))
        svc.append(time.perf_counter() - t1)
    clk = clocks.stop()
    done, lat64 = 0.0, []
    for a, sv in zip(arrivals, svc):
        done = max(done, a) + sv
        lat64.append(1e3 * (done - a))
    errs = [abs(a.logdet - b.logdet) / abs(b.logdet) for a, b in zip(stream, r64)]
    same = all(a.logdet == b.logdet for a, b in zip(stream, burst))
    for h in handles.values():
        h.close()
    ns = sorted(side ** (3 if typ == "l3d" else 2) for typ, side, _ in reqs)
    fp64_rate = N / sum(svc)
    return {
        "workload": "serving: %d OSLQ requests (m=50, 30 probes), type uniform over {2D Laplacian, "
                    "3D Laplacian, Matern}, n log-uniform [1e4, 4e6] rounded to a grid side, "
                    "shift (Laplacians) / kappa^2 (Matern) log-uniform [1e-3, 1]" % N,
        "requests": N, "distinct_matrices": len(handles),
        "n": {"min": ns[0], "median": ns[len(ns) // 2], "max": ns[-1], "total_rows": rows},
        "unit": UNIT,
        "mixed_batched": {"burst_solves_per_s": cap, "stream_rate": lam,
                          "stream_solves_per_s": N / t_stream,
                          "p50_ms": _pct(lat_srv, 0.5), "p99_ms": _pct(lat_srv, 0.99),
                          "max_resident": st_stream["max_resident"], "slots": slots,
                          "batched_steps_per_tick": st_burst["batched_steps"] / max(1, st_burst["ticks"])},
        "fp64_one_at_a_time": {"solves_per_s": fp64_rate, "p50_ms": _pct(lat64, 0.5),
                               "p99_ms": _pct(lat64, 0.99)},
        "speedup_solves_per_s": cap / fp64_rate,
        "max_rel_err_mixed_vs_fp64": max(errs), "within_1e-4": max(errs) <= 1e-4,
        "burst_equals_stream_bitwise": same,
        "latency": "host wall clock, submit to result; FP64 latencies from a FIFO replay of "
                   "the measured service times on the same Poisson arrivals",
        "matrix_build_s": t_build, "clocks": clk}


def serving_case(args):
    """--workload serving: the serving line on its own (--requests N)."""
    out = serving_measure(args.requests, args.slots, args.budget_gb)
    print(json.dumps(dict(out, metric=METRIC)))
    return 0


def multishift_measure(budget_gb: float, autotune: int, fp64_all: bool = True) -> dict:
    """Batched irregular workload: the Laplacian of a Chung-Lu power-law graph
    (n = 2,097,152, exponent 2.3, mean degree 8) with 8 diagonal shifts drawn
    uniformly from [1e-3, 1e-1]; OSA-IOP m = 100, k = 4, 64 probes per shift,
    FP32 values and vectors.  The 8 shifted operators share the CSR and run
    three ways: as one shift group (logdet_osaiop_shifts: one Krylov run over
    all 8 x 64 probe columns), through the server (8 solves advancing
    together, one launch per pass) and one after the other.  The server
    results are bitwise those of the serial solves; the group's agree to
    rounding.  Each mixed estimate is compared with the FP64 CUDA path (same
    seed): every shift, or with fp64_all False the smallest and the
    largest.  The forms within the 1e-4 budget follow: the same group with
    FP64 vectors and with double-float vectors (FP32 values)."""
    import numpy as np
    import torch
    from paper_2606_07004_gb300 import binding as B
    import workloads as W

    t0 = time.perf_counter()
    A = W.powerlaw_graph_laplacian(2 ** 21, exponent=2.3, mean_degree=8.0, seed=7,
                                   dtype=np.float32)
    t_build = time.perf_counter() - t0
    shifts = np.random.default_rng(11).uniform(1e-3, 1e-1, 8)
    P, m, k = 64, 100, 4
    h = B.Handle.from_csr(A)
    need = h.estimate_bytes(B.METHOD_OSAIOP, P, m, k, precision=B.MIXED_FP32)
    budget = int(min(budget_gb * (1 << 30), 8 * need * 1.05))
    clocks = ClockSampler(torch.cuda.current_device(), "irregular")
    clocks.start()
    # The same 8 solves as one shift group: one Krylov run over all 8 x 64
    # probe columns, so each gather fetches the x row of every shift.  Timed
    # first, after one untimed group of the same size: it tunes the block
    # widths and grows the memory pool to the group's working set (a short
    # warm-up group left the timed one paying for the pool's growth), which
    # the server and the serial solves then reuse.
    h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, precision=B.MIXED_FP32,
                    autotune=autotune)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    group = h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, precision=B.MIXED_FP32,
                            autotune=autotune)
    t_group = time.perf_counter() - t1
    with B.Server(budget, max_slots=8) as srv:
        srv.wait(srv.submit(h, B.METHOD_OSAIOP, P, 10, k, seed=0, precision=B.MIXED_FP32,
                            shift=float(shifts[0]), autotune=autotune))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ids = [srv.submit(h, B.METHOD_OSAIOP, P, m, k, seed=t, precision=B.MIXED_FP32,
                          shift=float(sh), autotune=autotune) for t, sh in enumerate(shifts)]
        batched = [srv.wait(i) for i in ids]
        t_batched = time.perf_counter() - t1
        st = srv.stats()
        # the same 8 as one shift group through the server (logdet_submit_shifts)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        gids = srv.submit_shifts(h, B.METHOD_OSAIOP, shifts, P, m, k, seed0=0,
                                 precision=B.MIXED_FP32, autotune=autotune)
        sgroup = [srv.wait(i) for i in gids]
        t_sgroup = time.perf_counter() - t1
    t1 = time.perf_counter()
    serial = [h.osaiop(P, m, iop_window=k, seed=t, precision=B.MIXED_FP32, shift=float(sh),
                       autotune=autotune) for t, sh in enumerate(shifts)]
    t_serial = time.perf_counter() - t1
    clk = clocks.stop()
    # Error of the mixed estimates against the FP64 CUDA path (same seed).
    which = list(range(8)) if fp64_all else sorted({int(np.argmin(shifts)), int(np.argmax(shifts))})
    r64 = {t: h.osaiop(P, m, iop_window=k, seed=t, shift=float(shifts[t])) for t in which}
    errs = {t: abs(batched[t].logdet - r64[t].logdet) / abs(r64[t].logdet) for t in which}
    gerrs = {t: abs(group[t].logdet - r64[t].logdet) / abs(r64[t].logdet) for t in which}
    # The configuration at the 1e-4 budget: FP64 vectors as a shift group
    # (two runs of 4: eight FP64 phase-1 bases do not fit the device).  The
    # warm-up is the full group: a short one (m = 10) fits in one run of 8,
    # so the layouts of the runs of 4 would be tuned inside the timed call.
    h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, autotune=autotune)
    clocks64 = ClockSampler(torch.cuda.current_device(), "irregular_fp64")
    clocks64.start()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    group64 = h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, autotune=autotune)
    t_group64 = time.perf_counter() - t1
    clk64 = clocks64.stop()
    g64errs = {t: abs(group64[t].logdet - r64[t].logdet) / abs(r64[t].logdet) for t in which}
    # Double-float vectors (FP32 values, vectors as hi + lo float pairs):
    # the same group, for the 1e-4 budget at FP32-pipe arithmetic.
    h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, precision=B.MIXED_F32X2,
                    autotune=autotune)  # the full group as warm-up, as for FP64
    clocksdf = ClockSampler(torch.cuda.current_device(), "irregular_f32x2")
    clocksdf.start()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    groupdf = h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, precision=B.MIXED_F32X2,
                              autotune=autotune)
    t_groupdf = time.perf_counter() - t1
    clkdf = clocksdf.stop()
    gdferrs = {t: abs(groupdf[t].logdet - r64[t].logdet) / abs(r64[t].logdet) for t in which}
    B.logdet_profile_reset()
    B.logdet_profile_enable(True)
    h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, precision=B.MIXED_F32X2,
                    autotune=autotune)
    B.logdet_profile_enable(False)
    dfprof = B.profile_snapshot()
    B.logdet_profile_reset()
    B.logdet_profile_enable(True)
    h.osaiop_shifts(shifts, P, m, iop_window=k, seed0=0, precision=B.MIXED_FP32,
                    autotune=autotune)
    B.logdet_profile_enable(False)
    gprof = B.profile_snapshot()
    # Device time per kernel class of one of the solves run alone.
    B.logdet_profile_reset()
    B.logdet_profile_enable(True)
    h.osaiop(P, m, iop_window=k, seed=0, precision=B.MIXED_FP32, shift=float(shifts[0]),
             autotune=autotune)
    B.logdet_profile_enable(False)
    prof = B.profile_snapshot()
    h.close()
    return {
        "workload": "power-law graph Laplacian n=%d nnz=%d, 8 shifts U[1e-3,1e-1], OSA-IOP m=100 "
                    "k=4, 64 probes each, mixed FP32" % (A.n, A.nnz),
        "unit": UNIT,
        "group_solves_per_s": 8 / t_group, "batched_solves_per_s": 8 / t_batched,
        "server_group_solves_per_s": 8 / t_sgroup,
        "server_group_equals_group_bitwise": all(a.logdet == b.logdet
                                                 for a, b in zip(sgroup, group)),
        "serial_solves_per_s": 8 / t_serial,
        "group_s": t_group, "batched_s": t_batched, "serial_s": t_serial,
        "rel_err_group_mixed_vs_fp64": {f"shift_{t}": gerrs[t] for t in which},
        "fp64_group": {"solves_per_s": 8 / t_group64, "s": t_group64,
                       "rel_diff_vs_fp64_solves": {f"shift_{t}": g64errs[t] for t in which},
                       "note": "FP64 vectors, the same 8 shifts as a shift group: the batched "
                               "configuration within the 1e-4 budget",
                       "clocks": clk64},
        "f32x2_group": {"solves_per_s": 8 / t_groupdf, "s": t_groupdf,
                        "rel_err_vs_fp64": {f"shift_{t}": gdferrs[t] for t in which},
                        "within_1e-4": all(e <= 1e-4 for e in gdferrs.values()),
                        "kernel_ms_8_solves": {k_: v["ms"] for k_, v in dfprof.items()},
                        "note": "FP32 values, double-float vectors (LOGDET_MIXED_F32X2), the "
                                "same 8 shifts as a shift group",
                        "clocks": clkdf},
        "max_rel_diff_group_vs_serial": max(abs(a.logdet - b.logdet) / abs(b.logdet)
                                            for a, b in zip(group, serial)),
        "kernel_ms_group_8_solves": {k_: v["ms"] for k_, v in gprof.items()},
        "bitwise_equal_batched_vs_serial": all(a.logdet == b.logdet for a, b in zip(batched, serial)),
        "logdets": [r.logdet for r in batched], "shifts": list(map(float, shifts)),
        "rel_err_mixed_vs_fp64": {f"shift_{t}": errs[t] for t in which},
        "within_1e-4": all(e <= 1e-4 for e in errs.values()),
        "within_1e-3": all(e <= 1e-3 for e in errs.values()),
        "error_note": "at m = 100 the IOP recurrence amplifies the rounding of stored FP32 "
                      "vectors on this graph (about 7e3 x 2^-24); double-float vectors "
                      "(f32x2_group) stay within 1e-8 of FP64",
        "fp64_solve_ms": {f"shift_{t}": r64[t].device_ms for t in which},
        "bytes_per_solve_estimate": need, "max_resident": st["max_resident"],
        "kernel_ms_one_solve": {k_: v["ms"] for k_, v in prof.items()},
        "krylov_algorithmic_gbs_one_solve": (prof["spmm"]["bytes"] + prof["update"]["bytes"]) /
        ((prof["spmm"]["ms"] + prof["update"]["ms"]) / 1e3) / 1e9,
        "graph_build_s": t_build, "clocks": clk}


def multishift_case(args):
    """--workload multishift: the batched irregular line on its own."""
    out = multishift_measure(args.budget_gb, args.autotune, fp64_all=True)
    print(json.dumps(dict(out, metric=METRIC)))
    return 0


def small2d_case(args):
    """Latency-bound workload: 2D 5-point Dirichlet Laplacian 64^2 + 0.1 I
    (n = 4096, nnz = 20,224; the whole working set sits in L2), OSLQ m = 30
    with 30 probes, FP64, one seed per solve.  Three ways to run the same
    solves: the blocking call (about 135 launches issued from the host per
    solve; also timed with the Krylov phase as one persistent launch, 18
    launches), a graph plan (the solve captured once, one graph launch per
    seed; bit-identical results) and the batched server (many solves per
    launch).
    Reports solves/s and per-solve latency of each."""
    import numpy as np
    import torch
    from paper_2606_07004_gb300 import binding as B
    import workloads as W

    A = W.laplacian_2d(64, shift=0.1)
    P, m = 30, 30
    N = max(args.steps, 50)
    with B.Handle.from_csr(A) as h:
        for i in range(args.warmup):
            h.oslq(P, m, seed=i)
        torch.cuda.synchronize()
        c0 = B.logdet_launch_count()
        t0 = time.perf_counter()
        lat_b = []
        blocking = []
        for i in range(N):
            t1 = time.perf_counter()
            blocking.append(h.oslq(P, m, seed=1000 + i))
            lat_b.append((time.perf_counter() - t1) * 1e3)
        t_b = time.perf_counter() - t0
        launches_b = (B.logdet_launch_count() - c0) / N
        # the same blocking solves with the Krylov phase as one persistent
        # launch (opt-in) instead of four launches per step
        os.environ["LOGDET_KRYLOV_PERSISTENT"] = "1"
        h.oslq(P, m, seed=0)
        c0 = B.logdet_launch_count()
        t0 = time.perf_counter()
        lat_s = []
        stepwise = []
        for i in range(N):
            t1 = time.perf_counter()
            stepwise.append(h.oslq(P, m, seed=1000 + i))
            lat_s.append((time.perf_counter() - t1) * 1e3)
        t_s_b = time.perf_counter() - t0
        launches_s = (B.logdet_launch_count() - c0) / N
        del os.environ["LOGDET_KRYLOV_PERSISTENT"]
        same_steps = all(a.logdet == b.logdet and np.array_equal(a.per_probe, b.per_probe)
                         for a, b in zip(blocking, stepwise))
        t0 = time.perf_counter()
        plan = B.Plan(h, B.METHOD_OSLQ, P, m)
        t_plan_make = time.perf_counter() - t0
        for i in range(args.warmup):
            plan.run(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat_p = []
        replay = []
        for i in range(N):
            t1 = time.perf_counter()
            replay.append(plan.run(1000 + i))
            lat_p.append((time.perf_counter() - t1) * 1e3)
        t_p = time.perf_counter() - t0
        same = all(a.logdet == b.logdet and np.array_equal(a.per_probe, b.per_probe)
                   for a, b in zip(blocking, replay))
        # Device time per kernel class of one blocking solve (CUDA events per launch).
        B.logdet_profile_reset()
        B.logdet_profile_enable(True)
        for i in range(10):
            h.oslq(P, m, seed=2000 + i)
        B.logdet_profile_enable(False)
        prof = {k: {"ms": v["ms"] / 10, "launches": v["launches"] / 10}
                for k, v in B.profile_snapshot().items()}
        kernels = plan.kernels()
        plan.close()
        with B.Server(8 << 30) as srv:
            srv.wait(srv.submit(h, B.METHOD_OSLQ, P, m, seed=0))
            M = 4 * N
            t0 = time.perf_counter()
            ids = [srv.submit(h, B.METHOD_OSLQ, P, m, seed=1000 + i) for i in range(M)]
            served = [srv.wait(i) for i in ids]
            t_s = time.perf_counter() - t0
        same_srv = all(a.logdet == b.logdet for a, b in zip(blocking, served[:N]))
    exact = W.closed_form_logdet_laplacian_2d(64, shift=0.1)
    print(json.dumps({
        "workload": "2D Laplacian 64^2 + 0.1 I (n=4096, nnz=%d), OSLQ m=30, 30 probes, FP64" % A.nnz,
        "metric": METRIC, "unit": UNIT, "dtype": "f64",
        "blocking": {"value": N / t_b, "latency_ms": {"p50": _pct(lat_b, 0.5), "p99": _pct(lat_b, 0.99)},
                     "launches_per_solve": launches_b, "krylov": "four launches per step"},
        "blocking_persistent": {"value": N / t_s_b,
                                "latency_ms": {"p50": _pct(lat_s, 0.5), "p99": _pct(lat_s, 0.99)},
                                "launches_per_solve": launches_s,
                                "krylov": "one persistent launch per Krylov phase "
                                          "(LOGDET_KRYLOV_PERSISTENT=1)",
                                "bitwise_equal_to_step_path": same_steps},
        "graph_plan": {"value": N / t_p, "latency_ms": {"p50": _pct(lat_p, 0.5), "p99": _pct(lat_p, 0.99)},
                       "kernels_per_replay": kernels, "capture_s": t_plan_make,
                       "bitwise_equal_to_blocking": same},
        "server_batched": {"value": M / t_s, "requests": M, "bitwise_equal_to_blocking": same_srv},
        "kernel_ms_per_solve": prof,
        "mean_rel_err_vs_exact": float(np.mean([abs(r.logdet - exact) / exact for r in blocking])),
        "timing": "host wall clock per solve (submit to result on host), inputs resident"}))
    return 0


def grf_case(args):
    """GRF maximum-likelihood sweep (Sec. 4, GRF study): a 900 x 1200 field
    (n = 1,080,000) drawn with precision Q(50) by circulant embedding, Q(theta)
    the Wendland C^2 covariance with support theta grid cells plus a 0.1
    nugget, applied matrix-free (up to 19,600 stencil entries per row at
    theta = 80: 21.7e9 implied nonzeros); theta in {20, ..., 80}.  OSA-IOP
    m = 20, m_vec = 21, tol = 1e-6 and OSLQ m = 60, m_vec = 30 (the paper's
    settings), mixed FP32, all seven thetas through one server.  Reports the
    sweep times, L(theta), the argmax, the relative error of the mixed
    log-determinant against FP64 at theta = 20, and the FP32 roofline of the
    stencil kernel (bound: FP32 FMA issue)."""
    import numpy as np
    import torch
    from paper_2606_07004_gb300 import binding as B, grf
    import workloads as W

    nx, ny = 1200, 900
    thetas = [20.0, 30.0, 40.0, 50.0, 60.0, 70.0, 80.0]
    t0 = time.perf_counter()
    x = W.grf_sample(nx, ny, W.wendland_table(50.0, 0.1), seed=7)
    t_field = time.perf_counter() - t0
    xd = torch.as_tensor(x, device="cuda")
    # warm-up (kernel loading) on a small sweep
    grf.loglik_sweep(xd, nx, ny, [20.0], num_probes=21, krylov_steps=4)
    out = {}
    B.logdet_profile_reset()
    B.logdet_profile_enable(True)
    clocks = ClockSampler(0)
    clocks.start()
    for name, kw in (("osaiop", dict(method=B.METHOD_OSAIOP, num_probes=21, krylov_steps=20,
                                     iop_window=2, tol=1e-6)),
                     ("oslq", dict(method=B.METHOD_OSLQ, num_probes=30, krylov_steps=60,
                                   iop_window=0, tol=None))):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sw = grf.loglik_sweep(xd, nx, ny, thetas, precision=B.MIXED_FP32, seed=11, **kw)
        dt = time.perf_counter() - t1
        out[name] = {"sweep_s": dt, "logdets_per_s": len(thetas) / dt, "theta_hat": sw.theta_hat,
                     "logdet": sw.logdet, "loglik": sw.loglik,
                     "steps": [[r.steps_min, r.steps_max] for r in sw.results]}
    clk = clocks.stop()
    B.logdet_profile_enable(False)
    prof = B.profile_snapshot()
    # mixed against FP64 at theta = 20 (same seed and probes)
    with B.Handle.grid(nx, ny, grf.wendland_table(20.0, 0.1)) as h:
        r64 = h.osaiop(21, 20, iop_window=2, seed=11, tol=1e-6)
        r32 = h.osaiop(21, 20, iop_window=2, seed=11, tol=1e-6, precision=B.MIXED_FP32)
    g = prof["grid"]
    achieved = g["flops"] / (g["ms"] / 1e3) / 1e12
    print(json.dumps({
        "workload": "GRF MLE sweep: Wendland C2 on 900 x 1200 (n=1080000), theta 20..80 cells, "
                    "nugget 0.1, field drawn with theta=50, mixed FP32, matrix-free",
        "metric": METRIC, "unit": "logdets/s", "osaiop": out["osaiop"], "oslq": out["oslq"],
        "rel_err_mixed_vs_fp64_theta20": abs(r32.logdet - r64.logdet) / abs(r64.logdet),
        "roofline": {"kernel": "k_grid_apply<float> (+ FP64 at theta 20 excluded)", "bound": "alu",
                     "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS,
                     "peak_source": "FP32 FMA peak from unit counts and clock: 152 SMs x 128 "
                                    "lanes x 2 flop x 2.070 GHz"},
        "kernel_ms": {k: v["ms"] for k, v in prof.items()},
        "field_build_s": t_field, "clocks": clk}))
    return 0


def small_case(args):
    """One OSLQ (m=12) and one OSA-IOP (k=4, m=12) solve with 60 probes on the 3D
    Laplacian 100^3 + 0.01 I: the capture target for ncu (blocks larger than
    L2, about 3 GB on the device).  With --workload matern: one mixed-FP32
    OSLQ solve (m=12, 120 probes) on the Matern 1024^2 operator instead; with
    --workload grf: one mixed-FP32 OSLQ solve (m=4, 30 probes) on the
    Wendland theta=50 gridded operator, 900 x 1200; with --workload
    multishift: one mixed-FP32 OSA-IOP solve (k=4, m=4, 64 probes, shift
    0.01) on the 2M-row power-law graph Laplacian, then a shift group of 8
    such solves (m=4) on the 512k-row graph of the same law (the group's
    block is 8 x 44 columns wide; about 3 GB on the device), in mixed FP32
    and with double-float vectors."""
    import torch
    from paper_2606_07004_gb300 import binding as B
    import workloads as W
    if args.workload == "multishift":
        import numpy as np
        A = W.powerlaw_graph_laplacian(2 ** 21, exponent=2.3, mean_degree=8.0, seed=7,
                                       dtype=np.float32)
        with B.Handle.from_csr(A) as h:
            r = h.osaiop(64, 4, iop_window=4, seed=1, precision=B.MIXED_FP32, shift=0.01)
        del A
        A = W.powerlaw_graph_laplacian(2 ** 19, exponent=2.3, mean_degree=8.0, seed=7,
                                       dtype=np.float32)
        shifts = np.random.default_rng(11).uniform(1e-3, 1e-1, 8)
        with B.Handle.from_csr(A) as h:
            g = h.osaiop_shifts(shifts, 64, 4, iop_window=4, seed0=0, precision=B.MIXED_FP32)
            gdf = h.osaiop_shifts(shifts, 64, 4, iop_window=4, seed0=0, precision=B.MIXED_F32X2)
        torch.cuda.synchronize()
        print(json.dumps({"small_case": "multishift", "osaiop": r.logdet, "ms": r.device_ms,
                          "group_512k": [x.logdet for x in g], "group_ms": g[0].device_ms,
                          "group_512k_f32x2": [x.logdet for x in gdf],
                          "group_f32x2_ms": gdf[0].device_ms}))
        return 0
    if args.workload == "grf":
        from paper_2606_07004_gb300 import grf
        with B.Handle.grid(1200, 900, grf.wendland_table(50.0, 0.1)) as h:
            r = h.oslq(30, 4, seed=1, precision=B.MIXED_FP32)
        torch.cuda.synchronize()
        print(json.dumps({"small_case": "grf", "oslq": r.logdet, "oslq_ms": r.device_ms}))
        return 0
    if args.workload == "matern":
        import numpy as np
        A = W.matern_2d(1024, 0.05, dtype=np.float32)
        with B.Handle.from_csr(A) as h:
            r = h.oslq(120, 12, seed=1, precision=B.MIXED_FP32, autotune=args.autotune)
        torch.cuda.synchronize()
        print(json.dumps({"small_case": "matern", "oslq": r.logdet, "oslq_ms": r.device_ms}))
        return 0
    A = W.laplacian_3d(100, shift=SHIFT, dtype=__import__("numpy").float32 if args.small_case_fp32
                       else __import__("numpy").float64)
    prec = B.MIXED_FP32 if args.small_case_fp32 else B.FP64
    with B.Handle.from_csr(A) as h:
        r1 = h.oslq(PROBES, 12, seed=1, precision=prec, autotune=args.autotune)
        r2 = h.osaiop(PROBES, 12, iop_window=4, seed=1, precision=prec, autotune=args.autotune)
    torch.cuda.synchronize()
    print(json.dumps({"small_case": True, "oslq": r1.logdet, "osaiop_k4": r2.logdet,
                      "oslq_ms": r1.device_ms, "osaiop_ms": r2.device_ms}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1 = autotuned Krylov kernel layout (tuned during warm-up); 0 = defaults")
    ap.add_argument("--workload", choices=["laplacian3d", "matern", "serving", "multishift",
                                           "small2d", "grf"],
                    default="laplacian3d",
                    help="extra measurement lines (not the default bench): matern = mixed "
                         "precision; serving = continuous batching; multishift = 8 shifts; "
                         "small2d = latency-bound 64^2 case (blocking, graph plan, server)")
    ap.add_argument("--requests", type=int, default=200, help="serving: number of requests")
    ap.add_argument("--slots", type=int, default=64, help="serving: server slots")
    ap.add_argument("--budget-gb", type=float, default=200.0, help="server memory budget")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without the matern_mixed and serving objects")
    ap.add_argument("--extra-solves", type=int, default=10,
                    help="timed solves of the matern_mixed object of the default line")
    ap.add_argument("--serving-requests", type=int, default=120,
                    help="requests of the serving object of the default line")
    ap.add_argument("--clock-dir", default=None,
                    help="keep the nvidia-smi clock samples as CSV files in this directory")
    ap.add_argument("--small-case", action="store_true",
                    help="one OSLQ + one OSA-IOP solve on a 100^3 Laplacian (profiling target)")
    ap.add_argument("--small-case-fp32", action="store_true", help="the small case in mixed FP32")
    ap.add_argument("--oracle-sample-child", type=int, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-all-cores", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    ClockSampler.clock_dir = args.clock_dir
    if args.small_case or args.small_case_fp32:
        return small_case(args)
    if args.workload == "matern":
        return matern_case(args)
    if args.workload == "serving":
        return serving_case(args)
    if args.workload == "multishift":
        return multishift_case(args)
    if args.workload == "small2d":
        return small2d_case(args)
    if args.workload == "grf":
        return grf_case(args)
    if args.oracle_sample_child is not None:
        res = oracle_sample(args.oracle_sample_child)
        if args.oracle_all_cores:
            res["all_cores"] = oracle_sample_all_cores(args.oracle_sample_child, res)
        print(json.dumps(res))
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    return cuda_arm(args)


if __name__ == "__main__":
    sys.exit(main())
