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
