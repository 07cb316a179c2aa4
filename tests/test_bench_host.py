"""Host-side arithmetic of bench.py's measurement keys, on synthetic inputs (no GPU):
the roofline of a kernel class (bound, achieved, fraction, implementation bytes), the
DRAM traffic taken from a committed ncu summary only while the kernel's source is
unchanged, the peaks fallback, and the parsing of the nvidia-smi clock samples."""
import json
import os

import pytest

import bench

PEAKS = {"hbm_gbs": 6795.1, "bf16_tflops": 1918.9, "bf16_tflops_sustained": 1706.4, "source": "measured"}
FP64, FP32 = 1.2e12, 38e12


def _cls(ms, count, bytes_, flops, impl=None):
    d = {"ms": ms, "count": count, "bytes": bytes_, "flops": flops}
    if impl is not None:
        d["impl_bytes"] = impl
    return d


def test_roofline_of_the_dominant_hbm_class(monkeypatch):
    monkeypatch.setattr(bench, "ncu_traffic", lambda cls, impl=None: None)
    # 4 launches of 2.5 ms, 10 GB algorithmic and 25 GB implementation bytes each
    report = {"orth.f32": _cls(10.0, 4, 4e10, 4e10, impl=1e11),
              "D2.f32": _cls(6.0, 3, 1e9, 1e12)}
    r = bench.roofline(report, PEAKS, FP64, FP32)
    assert r["kernel"] == "orth.f32" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(1e10 / 2.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])
    assert r["implementation_bytes_per_launch"] == pytest.approx(2.5e10)
    assert r["implementation_GB_per_s"] == pytest.approx(2.5e10 / 2.5e-3 / 1e9)
    assert r["share_of_profiled_time"] == pytest.approx(10.0 / 16.0)
    assert r["traffic"] is None


def test_roofline_bounds_follow_the_arithmetic_intensity(monkeypatch):
    monkeypatch.setattr(bench, "ncu_traffic", lambda cls, impl=None: None)
    # FP64 with 10 flop/B: above the FP64 ridge (1.2e12 / 6.8e12 B/s) -> ALU bound
    r = bench.roofline({"D1.f64": _cls(2.0, 2, 1e9, 1e10)}, PEAKS, FP64, FP32)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(FP64 / 1e12)
    assert r["achieved"] == pytest.approx(5e9 / 1e-3 / 1e12)
    # FP32 with 1 flop/B: below the FP32 ridge -> HBM bound
    r = bench.roofline({"D1.f32": _cls(2.0, 2, 1e9, 1e9)}, PEAKS, FP64, FP32)
    assert r["bound"] == "hbm"
    # BF16 with 500 flop/B: above the tensor ridge -> measured sustained BF16 peak
    r = bench.roofline({"Dinv.bf16": _cls(1.0, 1, 1e9, 5e11)}, PEAKS, FP64, FP32)
    assert r["bound"] == "tensor" and r["peak"] == PEAKS["bf16_tflops_sustained"]
    assert r["frac"] == pytest.approx(5e11 / 1e-3 / 1e12 / PEAKS["bf16_tflops_sustained"])
    # BF16 with 75 flop/B: HBM bound
    r = bench.roofline({"D2.bf16": _cls(1.0, 1, 1e9, 7.5e10)}, PEAKS, FP64, FP32)
    assert r["bound"] == "hbm"


def _fake_tree(tmp_path, src_text, entry):
    csrc = tmp_path / "paper_2211_15383_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src_text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"classes": {"orth.f32": entry}}))


def test_traffic_only_while_the_source_is_unchanged(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    _fake_tree(tmp_path, "kernel v1", {"source": "k.cu", "source_sha": None, "dram_bytes_per_launch": 7e9,
                                       "per_implementation_byte": 0.998})
    sha = bench.source_sha("k.cu")
    assert sha is not None and len(sha) == 16
    p = tmp_path / "profiles" / "ncu_traffic.json"
    d = json.loads(p.read_text())
    d["classes"]["orth.f32"]["source_sha"] = sha
    p.write_text(json.dumps(d))
    # scaled per implementation byte to this run's launches, else the stored figure
    assert bench.ncu_traffic("orth.f32", 1e10) == pytest.approx(0.998e10)
    assert bench.ncu_traffic("orth.f32") == pytest.approx(7e9)
    assert bench.ncu_traffic("mr1.bf16", 1e10) is None
    # the kernel changed since the counters were taken: no traffic figure
    (tmp_path / "paper_2211_15383_gb300" / "csrc" / "k.cu").write_text("kernel v2")
    assert bench.ncu_traffic("orth.f32", 1e10) is None


def test_committed_traffic_entries_are_well_formed():
    p = os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")
    d = json.load(open(p))
    for cls, e in d["classes"].items():
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2211_15383_gb300", "csrc", e["source"])), cls
        assert len(e["source_sha"]) == 16
        assert e.get("per_implementation_byte") or e.get("dram_bytes_per_launch"), cls
        if e.get("per_implementation_byte"):
            # traffic below the implementation bytes is impossible beyond the counters' noise
            assert 0.9 < e["per_implementation_byte"] < 3.0, cls


def test_peaks_fallback_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p = bench.measured_peaks()
    assert p["source"] == "fallback" and p["hbm_gbs"] == 6800.0 and p["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6795.1, "bf16_tflops": 1918.9,
                                                              "bf16_tflops_sustained": 1706.4}))
    p = bench.measured_peaks()
    assert p["source"] == "measured" and p["hbm_gbs"] == 6795.1 and p["bf16_tflops_sustained"] == 1706.4


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_parsed(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1396.9, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
                    "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n")
    c = bench.Clocks(0)
    c.proc, c.path = _Proc(), str(path)
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["power_w_max"] == pytest.approx(1396.9)
    assert out["reasons"] == ["sw_power_cap"]
    assert not path.exists()
