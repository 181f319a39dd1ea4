"""Host-side arithmetic of bench.py's roofline fields (no GPU): the
double-float peak of the maxvol kernel and the rule that a captured DRAM
traffic figure is reported only while every source it lists is unchanged."""
import hashlib

import pytest

import bench


def test_maxvol_peak_from_instruction_counts():
    # all warm start: 11 FP32 instructions per multiply-add (2 flops)
    sms, lanes, mhz = bench.SMS, bench.FP32_PER_SM_CLK, 2000.0
    rate = sms * lanes * mhz * 1e6                        # FP32 instructions / s
    warm = 1e9                                            # multiply-adds
    peak = bench.maxvol_dd_peak_tflops(2 * warm, warm, mhz)
    assert peak == pytest.approx(2 * rate / bench.DD_OPS_WARM / 1e12)
    # all updates: 15 instructions per multiply-add
    peak = bench.maxvol_dd_peak_tflops(2e9, 0.0, mhz)
    assert peak == pytest.approx(2 * rate / bench.DD_OPS_UPDATE / 1e12)
    # a mix lies between the two
    mix = bench.maxvol_dd_peak_tflops(4e9, 1e9, mhz)
    assert 2 * rate / bench.DD_OPS_UPDATE / 1e12 < mix < 2 * rate / bench.DD_OPS_WARM / 1e12
    assert bench.maxvol_dd_peak_tflops(0.0, 0.0, mhz) == 0.0


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)


def test_captured_traffic_follows_the_listed_sources(tmp_path, monkeypatch):
    root = tmp_path
    csrc = root / "paper_1611_01391_gb300" / "csrc"
    prof = root / "profiles"
    csrc.mkdir(parents=True)
    prof.mkdir()
    _write(csrc / "a.cu", "kernel a\n")
    _write(csrc / "b.cuh", "header b\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = hashlib.sha256(b"kernel a\nheader b\n").hexdigest()
    assert bench.sources_sha256(["a.cu", "b.cuh"]) == h
    _write(prof / "p.md", f"sources: a.cu, b.cuh\nsources_sha256: {h}\ntraffic_bytes_per_launch: 1234\n")
    assert bench.captured_traffic("a.cu", "p.md") == 1234.0
    # a listed header changes: the figure no longer describes the kernel
    _write(csrc / "b.cuh", "header b, edited\n")
    assert bench.captured_traffic("a.cu", "p.md") is None
    # single-file form: the kernel file's own hash
    ha = hashlib.sha256(b"kernel a\n").hexdigest()
    _write(prof / "q.md", f"source_sha256: {ha}\ntraffic_bytes_per_launch: 99\n")
    assert bench.captured_traffic("a.cu", "q.md") == 99.0
    _write(csrc / "a.cu", "kernel a, edited\n")
    assert bench.captured_traffic("a.cu", "q.md") is None
    # a missing summary or a missing figure gives None
    assert bench.captured_traffic("a.cu", "absent.md") is None
    _write(prof / "r.md", f"sources: b.cuh\nsources_sha256: {bench.sources_sha256(['b.cuh'])}\n")
    assert bench.captured_traffic("a.cu", "r.md") is None

