"""bench.py's DRAM-traffic record of the sweep (CPU only): the committed ncu figures are used only
while the sweep's source is the one they were taken on, and that source hash covers the sweep and
the device code before it, not the kernels after it."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _copy_tree(tmp_path, kernel_text):
    csrc = tmp_path / "paper_1608_04601_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "pic_kernels.cu").write_text(kernel_text)
    for f in ("pic_device.cuh", "pic_internal.h"):
        (csrc / f).write_bytes(open(os.path.join(ROOT, "paper_1608_04601_gb300", "csrc", f), "rb").read())
    (tmp_path / "profiles").mkdir()
    return tmp_path


def test_hash_ignores_kernels_after_the_sweep_and_sees_changes_before(tmp_path, monkeypatch):
    src = open(os.path.join(ROOT, "paper_1608_04601_gb300", "csrc", "pic_kernels.cu")).read()
    cut = src.index("struct PSum")
    monkeypatch.setattr(bench, "ROOT", str(_copy_tree(tmp_path / "a", src)))
    h0 = bench.sweep_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(_copy_tree(tmp_path / "b", src + "\n// a later kernel\n")))
    assert bench.sweep_source_hash() == h0
    changed = src[:cut - 1] + " " + src[cut - 1:]
    monkeypatch.setattr(bench, "ROOT", str(_copy_tree(tmp_path / "c", changed)))
    assert bench.sweep_source_hash() != h0


def test_record_used_only_for_the_same_source_and_kernel(tmp_path, monkeypatch):
    src = open(os.path.join(ROOT, "paper_1608_04601_gb300", "csrc", "pic_kernels.cu")).read()
    root = _copy_tree(tmp_path, src)
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = {"fp32": {"kernel": "k_sweep<float,256,2>", "dram_bytes_per_particle": 22.0,
                    "source_hash": bench.sweep_source_hash()}}
    (root / "profiles" / "sweep_traffic.json").write_text(json.dumps(rec))
    c2, c3 = "C2 ar-like", "C3 he-like"
    assert bench.recorded_traffic("fp32", "k_sweep<float,256,2>", c2)["dram_bytes_per_particle"] == 22.0
    assert bench.recorded_traffic("fp32", "k_sweep<float,256,4>", c2) is None
    assert bench.recorded_traffic("fp64", "k_sweep<float,256,2>", c2) is None
    # the large discharge has its own record (a capture of the same physics at fewer particles)
    assert bench.recorded_traffic("fp32", "k_sweep<float,256,2>", c3) is None
    rec["fp32_c3"] = dict(rec["fp32"], dram_bytes_per_particle=41.0)
    (root / "profiles" / "sweep_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("fp32", "k_sweep<float,256,2>", c3)["dram_bytes_per_particle"] == 41.0
    rec["fp32"]["source_hash"] = "0" * 16
    (root / "profiles" / "sweep_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("fp32", "k_sweep<float,256,2>", c2) is None


def test_committed_record_names_its_command_and_kernel():
    rec = json.load(open(os.path.join(ROOT, "profiles", "sweep_traffic.json")))["fp32"]
    assert rec["kernel"].startswith("k_sweep<float,")
    assert rec["command"].startswith("ncu ") and "--clock-control none" in rec["command"]
    assert 0 < rec["dram_bytes_per_particle"] < 200
