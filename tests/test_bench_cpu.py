"""Host logic of bench.py that needs no GPU: the staleness key of the committed
SpMM counters (the roofline `traffic` field is reported only while the kernel
they were taken on is unchanged)."""
import os
import shutil

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402


@pytest.fixture
def csrc_copy(tmp_path, monkeypatch):
    dst = tmp_path / "csrc"
    shutil.copytree(bench.CSRC, dst)
    monkeypatch.setattr(bench, "CSRC", str(dst))
    monkeypatch.setattr(bench, "KRYLOV_SRC", str(dst / "krylov.cu"))
    return dst


def _edit(path, old, new):
    text = path.read_text()
    assert old in text
    path.write_text(text.replace(old, new, 1))


def test_digest_ignores_edits_outside_the_spmm_kernel(csrc_copy):
    before = bench.spmm_kernel_digest()
    _edit(csrc_copy / "krylov.cu", "k_update(const __grid_constant__ UpdBatch<T> B) {",
          "k_update(const __grid_constant__ UpdBatch<T> B) {  // edited")
    assert bench.spmm_kernel_digest() == before


def test_digest_follows_the_spmm_kernel_and_its_headers(csrc_copy):
    before = bench.spmm_kernel_digest()
    _edit(csrc_copy / "krylov.cu", "k_spmm(const __grid_constant__ SpmmBatch<T> B) {",
          "k_spmm(const __grid_constant__ SpmmBatch<T> B) {  // edited")
    inside = bench.spmm_kernel_digest()
    assert inside != before
    with open(os.path.join(csrc_copy, "common.cuh"), "a") as f:
        f.write("\n// edited\n")
    assert bench.spmm_kernel_digest() not in (before, inside)
    # A stale digest turns the traffic figure off.
    assert bench.traffic_ratio_from_profile() is None


def test_serving_request_law():
    # Type uniform over the three operators, n log-uniform in [1e4, 4e6]
    # rounded to a grid side, shift / kappa^2 log-uniform in [1e-3, 1].
    import math
    import numpy as np
    reqs = bench.serving_requests(3000, seed=5)
    assert bench.serving_requests(3000, seed=5) == reqs          # seeded
    types = [r[0] for r in reqs]
    for t in ("l2d", "l3d", "mat"):
        assert abs(types.count(t) / len(reqs) - 1 / 3) < 0.04
    n = np.array([side ** (3 if typ == "l3d" else 2) for typ, side, _ in reqs], dtype=float)
    assert n.min() >= 0.9e4 and n.max() <= 4.1e6
    u = (np.log(n) - math.log(1e4)) / (math.log(4e6) - math.log(1e4))
    assert abs(u.mean() - 0.5) < 0.03 and abs(np.median(u) - 0.5) < 0.05
    t = np.array([r[2] for r in reqs])
    assert t.min() >= 1e-3 and t.max() <= 1.0
    assert abs(np.mean(np.log10(t)) + 1.5) < 0.05
    # no pool of sizes: most requests get a grid of their own size
    assert len({(typ, side) for typ, side, _ in reqs}) > 1000
