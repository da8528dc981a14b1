"""Host logic of bench.py that the reported roofline rests on: the DRAM
traffic table is used only for the source it was captured on, the FP64 peak
follows the unit count and the sampled clock, and the launch-list summary
adds the per-launch durations of an ncu CSV (in any of the time units ncu
writes)."""
import json
import os

import bench


def test_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2602_23778_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "k.cu"
    src.write_text("__global__ void k() {}\n")
    table = {"bf16": {"source_sha256_16": bench.source_hash(str(src)), "dram_bytes_per_launch": 123.0}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(table))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("k.cu", "bf16") == 123.0
    assert bench.traffic_for("k.cu", "fp64") is None          # no entry
    src.write_text("__global__ void k() { }\n")                 # the kernel changed since the capture
    assert bench.traffic_for("k.cu", "bf16") is None


def test_committed_traffic_entries_name_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        table = json.load(f)
    files = {"bf16": "sliced.cu", "csr": "spmm.cu", "fp64": "fp64.cu"}
    for key, ent in table.items():
        assert key in files, key
        assert ent["dram_bytes_per_launch"] > 0
        assert len(ent["source_sha256_16"]) == 16


def test_fp64_peak_from_units_and_clock():
    # 152 SMs x 2 DFMA a clock x 2 flops
    assert abs(bench.fp64_peak({"sm_mhz": 2070.0}) - 152 * 2 * 2 * 2.07e9 / 1e12) < 1e-12
    assert abs(bench.fp64_peak({"sm_mhz": 1000.0}) - 0.608) < 1e-12
    assert bench.fp64_peak({"sm_mhz": None}) == bench.fp64_peak({"sm_mhz": 2070.0})   # unsampled: max clock
    assert bench.fp64_peak(None) == bench.fp64_peak({"sm_mhz": 2070.0})


def test_summarize_launches(tmp_path):
    head = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = [
        ("0", "void a_kernel<8>(int)", "gpu__time_duration.sum", "usecond", "10"),
        ("0", "void a_kernel<8>(int)", "dram__bytes_read.sum", "byte", "999"),
        ("1", "b_kernel(int)", "gpu__time_duration.sum", "nsecond", "5000"),
        ("2", "void a_kernel<8>(int)", "gpu__time_duration.sum", "msecond", "0.02"),
    ]
    path = tmp_path / "l.csv"
    path.write_text("==PROF== Connected\n" + head + "".join(",".join('"%s"' % v for v in r) + "\n" for r in rows))
    out = bench.summarize_launches(str(path))
    lines = {ln.split()[0]: ln.split() for ln in out.splitlines()[1:]}
    assert lines["a_kernel"][1] == "2" and abs(float(lines["a_kernel"][2]) - 30.0) < 1e-9
    assert lines["b_kernel"][1] == "1" and abs(float(lines["b_kernel"][2]) - 5.0) < 1e-9
    assert lines["TOTAL"][1] == "3" and abs(float(lines["TOTAL"][2]) - 35.0) < 1e-9
