"""The benchmark reports `roofline.traffic` from the committed ncu record only while the recorded batched
sweep kernel, its argument struct, the kernel that orders the batch's rows and the device helpers the
sweep calls are unchanged since the capture, and only for the launch configuration and chain count that
were captured."""
import json
import os
import shutil

import bench


def record():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        return json.load(f)


def test_record_matches_the_sources_and_launch():
    t = record()
    assert t["source_digest"] == bench.kernel_source_digest(t["kernel"])
    got = bench.load_traffic(t["kernel"], t["config"], t["launches_per_sweep"])
    assert got == t["dram_bytes_per_sweep"]
    # another launch configuration or chain count: no traffic figure
    other = dict(t["config"], chunk=t["config"]["chunk"] + 1)
    assert bench.load_traffic(t["kernel"], other, t["launches_per_sweep"]) is None
    assert bench.load_traffic(t["kernel"], t["config"], t["launches_per_sweep"] + 1) is None
    assert bench.load_traffic("k_batch_sweep<99>", t["config"], t["launches_per_sweep"]) is None


def copy_tree(tmp_path):
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1606_00803_gb300", "csrc"),
                    root / "paper_1606_00803_gb300" / "csrc")
    shutil.copytree(os.path.join(bench.ROOT, "profiles"), root / "profiles")
    return root


def digest_of(root, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(root))
    return bench.kernel_source_digest(record()["kernel"])


def edit(path, old, new):
    s = path.read_text()
    assert old in s
    path.write_text(s.replace(old, new, 1))


def test_digest_follows_the_kernel_and_its_helpers_only(tmp_path, monkeypatch):
    root = copy_tree(tmp_path)
    csrc = root / "paper_1606_00803_gb300" / "csrc"
    base = digest_of(root, monkeypatch)
    assert base == record()["source_digest"]
    # unrelated code: the FP64 sweep and the quality kernels do not enter the digest
    edit(csrc / "lms_kernels.cu", "k_quality_partials_f64(int32_t ntri", "k_quality_partials_f64(int32_t  ntri")
    assert digest_of(root, monkeypatch) == base
    # the batched kernel's body, its argument struct, a helper it calls: each changes the digest
    for path, old, new in ((csrc / "lms_kernels.cu", "if (w < 0) continue;  // boundary vertex",
                            "if (w < 0) { continue; }  // boundary vertex"),
                           (csrc / "lms_internal.h", "const int32_t* items_pbase;", "const int32_t*  items_pbase;"),
                           (csrc / "lms_kernels.cu", "while (j >= e0 && abs(col_idx[j] - v) < dx) {",
                            "while (j >= e0 && abs(col_idx[j] - v) < dx)  {"),
                           (csrc / "lms_device.cuh", "c = __fsub_rn(__fsub_rn(t, s), y);",
                            "c = __fsub_rn(__fsub_rn(t, s), y);  // compensation")):
        saved = path.read_text()
        edit(path, old, new)
        assert digest_of(root, monkeypatch) != base
        t = record()
        assert bench.load_traffic(t["kernel"], t["config"], t["launches_per_sweep"]) is None
        path.write_text(saved)
    assert digest_of(root, monkeypatch) == base
