"""Host helpers of the benchmark: the algorithmic bytes charged per launch, the gate that
drops the ncu traffic figure once the kernel source has changed, and the parsing of the
clock samples taken while the timed region runs."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_per_cell():
    # every population read once and written once; f has 19 directions, g has 7
    assert bench.kernel_alg_bytes("phaseC", 4) == 152 and bench.kernel_alg_bytes("phaseC", 2) == 76
    assert bench.kernel_alg_bytes("phaseC7", 4) == 56
    assert bench.kernel_alg_bytes("phaseA", 4) == 104
    assert bench.kernel_alg_bytes("fused", 4) == bench.BYTES_PER_LU == 208
    assert bench.kernel_alg_bytes("phaseC", 4) + bench.kernel_alg_bytes("phaseC7", 4) == bench.BYTES_PER_LU
    assert bench.kernel_alg_bytes("no_such_kernel", 4) is None


def test_traffic_figure_only_for_the_profiled_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_phaseC.json").write_text(json.dumps(
        {"kernel": "phaseC", "kernel_src_sha": "abc", "dram_bytes_per_cell": 142.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("phaseC", "abc", 1000) == 142500.0
    assert bench.ncu_traffic("phaseC", "changed", 1000) is None  # kernel changed since the capture
    assert bench.ncu_traffic("phaseC_f16", "abc", 1000) is None   # no capture for this form


def test_source_digest_covers_the_kernel_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2206_00946_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("kernel a")
    (csrc / "b.cuh").write_text("header b")
    (csrc / "notes.txt").write_text("not source")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.src_digest()
    assert len(d0) == 16
    (csrc / "notes.txt").write_text("edited")
    assert bench.src_digest() == d0
    (csrc / "b.cuh").write_text("header b, edited")
    assert bench.src_digest() != d0


def test_kernel_digest_follows_the_kernel_code_only(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2206_00946_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_HEADERS:
        (csrc / f).write_text(f"header {f}")
    api = ("host code before\n" + bench.KERNEL_BLOCK[0] + "\nKBODY\n" + bench.KERNEL_BLOCK[1] +
           "\nreductions and host code after\n")
    (csrc / "lbm_api.cu").write_text(api)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.kernel_digest()
    (csrc / "lbm_api.cu").write_text(api.replace("host code after", "host code edited"))
    assert bench.kernel_digest() == d0
    (csrc / "lbm_api.cu").write_text(api.replace("KBODY", "KBODY edited"))
    assert bench.kernel_digest() != d0
    (csrc / "lbm_api.cu").write_text(api.replace("KBODY", "KBODY // a comment"))
    assert bench.kernel_digest() == d0  # comments and layout do not count
    (csrc / "lbm_api.cu").write_text(api)
    (csrc / bench.KERNEL_HEADERS[2]).write_text("edited")
    assert bench.kernel_digest() != d0


def test_clock_summary_reads_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
        "0, [N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active",
    ]
    d = s.summary()
    assert d["sm_mhz"] == 2055 and d["sm_max_mhz"] == 2070 and d["samples"] == 3
    assert d["reasons"] == ["sw_power_cap"]
    s.lines.append("0, 1500, 2070, 1200, 0x48, Active, Not Active, Active, Not Active")
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    d = bench.ClockSampler(0).summary()
    assert d["sm_mhz"] is None and d["samples"] == 0 and d["reasons"] == []
