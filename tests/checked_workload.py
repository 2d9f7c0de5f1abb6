"""Workload run by test_gpu_checked.py in a subprocess, once against the
library named by LOGDET_LIB (the checked build) and once against the normal
build: every kind of solve on small inputs (FP64, mixed FP32 and double-float
vectors, OSLQ and OSA-IOP, uniform tiles and work items of an irregular
graph, the line and plane sweeps, shift groups, graph plans, the server with
a suspension).
Prints one JSON line: the results (repr of each estimate, so that the two
builds can be compared bit for bit) and the checked build's report."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from paper_2606_07004_gb300 import binding as B  # noqa: E402


def main():
    out = {}
    lap3 = W.laplacian_3d(20, 18, 16, shift=0.01)
    mat = W.matern_2d(80, 0.05, dtype=np.float32)          # line sweep (n >= 4096)
    lap3f = W.laplacian_3d(24, 21, 19, shift=0.02, dtype=np.float32)   # plane sweep
    graph = W.powerlaw_graph_laplacian(30011, seed=4).with_diagonal_shift(0.02)  # work items
    with B.Handle.from_csr(lap3) as h:
        out["lap3_oslq"] = repr(h.oslq(30, 20, seed=1).logdet)
        out["lap3_iop4"] = repr(h.osaiop(30, 16, iop_window=4, seed=1).logdet)
        out["lap3_iop8_mixed"] = repr(h.osaiop(30, 16, iop_window=8, seed=1,
                                               precision=B.MIXED_FP32).logdet)
        out["lap3_group"] = [repr(r.logdet) for r in h.osaiop_shifts([0.0, 0.3], 24, 12,
                                                                     iop_window=2, seed0=3)]
        with B.Plan(h, B.METHOD_OSLQ, 30, 20) as p:
            out["lap3_plan"] = repr(p.run(1).logdet)
        out["lap3_oslq_df"] = repr(h.oslq(30, 20, seed=1, precision=B.MIXED_F32X2).logdet)
        out["lap3_group_df"] = [repr(r.logdet) for r in h.oslq_shifts([0.0, 0.3], 24, 12, seed0=3,
                                                                      precision=B.MIXED_F32X2)]
    with B.Handle.from_csr(mat) as h:
        out["matern_oslq_mixed"] = repr(h.oslq(36, 20, seed=2, precision=B.MIXED_FP32).logdet)
    with B.Handle.from_csr(lap3f) as h:
        out["lap3f_iop2_mixed"] = repr(h.osaiop(36, 16, iop_window=2, seed=2,
                                                precision=B.MIXED_FP32).logdet)
    with B.Handle.from_csr(graph) as h:
        out["graph_iop4"] = repr(h.osaiop(24, 20, iop_window=4, seed=5).logdet)
        out["graph_oslq_mixed"] = repr(h.oslq(24, 20, seed=5, precision=B.MIXED_FP32).logdet)
        out["graph_iop4_df"] = repr(h.osaiop(24, 20, iop_window=4, seed=5,
                                             precision=B.MIXED_F32X2).logdet)
        with B.Server(8 << 30, max_slots=4) as srv:
            a = srv.submit(h, B.METHOD_OSAIOP, 24, 120, 4, seed=6)
            b = srv.submit(h, B.METHOD_OSLQ, 24, 60, seed=7, precision=B.MIXED_FP32)
            time.sleep(0.02)
            try:
                srv.suspend(a)
                t0 = time.time()
                while srv.stats()["suspended"] != 1 and srv.poll(a) is None and time.time() - t0 < 30:
                    time.sleep(0.002)
                if srv.stats()["suspended"] == 1:
                    srv.resume(a)
            except B.LogdetError:
                pass   # already finished
            out["server_a"] = repr(srv.wait(a).logdet)
            out["server_b"] = repr(srv.wait(b).logdet)
    out["report"] = B.checked_report()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
