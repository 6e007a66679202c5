"""The bench line's roofline bookkeeping (bench.py).

The executed-flop and DRAM-byte counts the roofline divides by come from ncu
captures of particular kernel sources. Each count is stored beside a sha256
of the files that define its kernel, and the line marks its roofline stale
(traffic null) when those files change.
"""
import os
import shutil

import bench


def test_every_captured_count_names_its_sources():
    for key in bench.TRAFFIC_PER_LAUNCH:
        assert key in bench.PROFILED_SHA256, key
        assert key[1] in bench.KERNEL_FILES, key
    for (kind, path) in bench.FLOPS_PER_POINT_STAGE:
        assert path in bench.KERNEL_FILES, (kind, path)


def test_the_committed_counts_are_from_the_current_sources():
    """The stamped hashes are those of the sources in the tree, so the
    default bench line reports its roofline as current."""
    for key, sha in bench.PROFILED_SHA256.items():
        assert bench.sources_sha256(key[1]) == sha, key


def test_a_changed_kernel_file_changes_the_hash(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2204_01133_gb300", "csrc")
    dst = tmp_path / "paper_2204_01133_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    before = {p: bench.sources_sha256(p) for p in bench.KERNEL_FILES}
    with open(dst / "at_stage.cu", "a") as f:
        f.write("\n")
    after = {p: bench.sources_sha256(p) for p in bench.KERNEL_FILES}
    assert after["stage"] != before["stage"]
    assert after["persistent"] == before["persistent"]
    assert after["fused"] == before["fused"]
    # the shared device header belongs to every path
    with open(dst / "at_device.cuh", "a") as f:
        f.write("\n")
    again = {p: bench.sources_sha256(p) for p in bench.KERNEL_FILES}
    assert all(again[p] != after[p] for p in bench.KERNEL_FILES)
