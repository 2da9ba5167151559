"""Host-side logic of bench.py that needs no GPU: the DRAM traffic it reports
is taken from the committed ncu summary only while the step kernel's sources
are the ones that summary was captured on, and is scaled by the cells of the
launch; the CPU-baseline crop is bounded."""
import json
import os
import shutil

import pytest

import bench

REPO = bench.ROOT


def _tree(tmp_path, traffic):
    """A copy of the step kernel's sources and a traffic summary under tmp_path."""
    for rel in bench.KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copyfile(os.path.join(REPO, rel), dst)
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "step_kernel_traffic.json").write_text(json.dumps(traffic))


def test_committed_traffic_summary_names_its_kernel_source():
    with open(os.path.join(REPO, "profiles", "step_kernel_traffic.json")) as fh:
        d = json.load(fh)
    assert len(d["source_sha"]) == 16
    # the per-node figure is ncu's DRAM bytes of a full launch: at least the
    # 144 algorithmic bytes, and not far above them
    assert bench.BYTES_PER_CELL <= d["dram_bytes_per_cell"] <= 1.1 * bench.BYTES_PER_CELL
    assert os.path.exists(os.path.join(REPO, d["summary"]))


def test_traffic_is_reported_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, {"source_sha": "0" * 16, "dram_bytes_per_cell": 145.0})
    sha = bench.kernel_source_sha()
    assert bench.recorded_traffic(1000) is None  # captured on another source
    _tree(tmp_path, {"source_sha": sha, "dram_bytes_per_cell": 145.0})
    assert bench.recorded_traffic(1000) == pytest.approx(145000.0)
    # any edit of a kernel source, comments included, retires the figure
    src = tmp_path / bench.KERNEL_SOURCES[0]
    src.write_text(src.read_text() + "\n")
    assert bench.kernel_source_sha() != sha
    assert bench.recorded_traffic(1000) is None


def test_missing_traffic_summary_gives_none(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _tree(tmp_path, {})
    os.remove(tmp_path / "profiles" / "step_kernel_traffic.json")
    assert bench.recorded_traffic(1000) is None


def test_cpu_baseline_crop_is_bounded():
    for steps, warmup in ((10, 2), (200, 10), (1, 0)):
        side = bench.crop_side(steps, warmup)
        assert 64 <= side <= 1024 and side % 8 == 0
        assert side * side * (steps + warmup) <= 2.0e7
