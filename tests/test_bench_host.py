"""Host-side logic of bench.py (no GPU): the DRAM traffic of the sweep kernel
is reported only for the kernel source, variant and launch form its ncu
record was taken on; the peak from the measured-peaks file falls back when
the file is missing; the default arguments give the timing rules (warm-up
steps >= 3) on the 256^3 clumpy 4-bin workload."""
import json
import os
import shutil

import pytest

import bench


def test_recorded_traffic_matches_only_its_source_and_variant(tmp_path, monkeypatch):
    rec = dict(line.split(": ", 1) for line in
               open(os.path.join(bench.HERE, "profiles", "traffic_sweep_grf64.txt")).read().splitlines()
               if ": " in line)
    v, pers = int(rec["variant"]), int(rec["persistent"])
    assert bench.recorded_traffic("grf64", v, pers) == int(rec["dram_bytes_per_launch"])
    assert bench.recorded_traffic("grf64", v + 1, pers) is None
    assert bench.recorded_traffic("grf64", v, 1 - pers) is None
    assert bench.recorded_traffic("grf128", v, pers) is None            # no record for that workload
    # a changed kernel source invalidates the record
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_1410_0763_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(os.path.join(bench.HERE, "profiles", "traffic_sweep_grf64.txt"), root / "profiles")
    src = root / "paper_1410_0763_gb300" / "csrc" / "art_kernels.cuh"
    shutil.copy(os.path.join(bench.HERE, "paper_1410_0763_gb300", "csrc", "art_kernels.cuh"), src)
    monkeypatch.setattr(bench, "HERE", str(root))
    assert bench.recorded_traffic("grf64", v, pers) == int(rec["dram_bytes_per_launch"])
    src.write_text(src.read_text() + "\n// changed\n")
    assert bench.recorded_traffic("grf64", v, pers) is None


def test_bf16_peak_falls_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "HERE", str(tmp_path))
    assert bench.measured_bf16_peak() == 1700.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"bf16_tflops_sustained": 1711.0}))
    assert bench.measured_bf16_peak() == pytest.approx(1711.0)


def test_default_arguments(monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps > 0 and a.workload == "clumpy4" and a.impl == "ours"
    assert not a.paper_tests and a.profile_case is None


def test_kernel_source_follows_the_variant():
    assert bench.kernel_source(15).endswith("art_kernels.cuh")
    assert bench.kernel_source(16).endswith("art_wave.cuh")
