"""The benchmark's multi-rank path on CPU ranks (gloo, world size 2).

Each rank solves its own copy of the workload (replicas; no data-path
collective).  The only collectives are the barrier and the max of the timed
region over ranks, and the whole-job value is world_size * solves / max time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    d = bench.dist_init(ws, "gloo")
    t_rank = 1.0 + 0.5 * rank                      # rank 1 is the slow one
    d.barrier()
    t = bench.max_over_ranks(d, t_rank)
    out[rank] = (t, bench.aggregate_value(8, ws, t))
    d.barrier()
    d.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ws = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    t, v = res[0]
    assert t == 1.5
    assert v == pytest.approx(8 * 2 / 1.5)


def test_reference_arm_on_nonzero_rank_exits_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        gpus, steps, warmup = 2, 1, 0
    assert bench.reference_arm(A()) == 0
    assert capsys.readouterr().out == ""


def test_single_rank_needs_no_process_group():
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.25) == 3.25
