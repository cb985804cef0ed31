"""Host logic of bench.py (no GPU): the algorithmic work of the sketch (32 real flops per
quaternion multiply-add, 24 when A is pure; 16 bytes per FP32 quaternion, 12 when pure, 32
in FP64), the DRAM-traffic pin (reported only for the captured kernel and workload), and the
peak denominators' fallback."""
import json
import os

import pytest

import bench


def test_algorithmic_flops_and_bytes():
    cfg = dict(m=8192, n=8192, s=101, l=203, prec="bf16x3")
    flops, abytes = bench.algorithmic(cfg)
    assert flops == 32 * 8192 * 8192 * (101 + 203)          # 653 GFLOP on c2
    assert abytes == 4 * 8192 * 8192 * 4                    # 1.074 GB on c2
    flops_p, abytes_p = bench.algorithmic(dict(cfg, pure=True))
    assert flops_p == 24 * 8192 * 8192 * 304 and abytes_p == 3 * 8192 * 8192 * 4
    _, abytes64 = bench.algorithmic(dict(cfg, prec="fp64"))
    assert abytes64 == 2 * abytes


def _sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in bench.SKETCH_TRAFFIC["sources"]:
        with open(os.path.join(bench.ROOT, "paper_2404_14783_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def test_traffic_pin_only_for_the_captured_kernel_and_workload(monkeypatch):
    captured = _sources_hash() == bench.SKETCH_TRAFFIC["sha256"]
    assert bench.sketch_traffic("bf16x3", "c2") == (bench.SKETCH_TRAFFIC["bytes"] if captured else None)
    assert bench.sketch_traffic("bf16", "c2") is None
    assert bench.sketch_traffic("bf16x3", "c1") is None
    monkeypatch.setitem(bench.SKETCH_TRAFFIC, "sha256", "0" * 64)   # the kernel changed
    assert bench.sketch_traffic("bf16x3", "c2") is None


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    p = bench.load_peaks()
    assert p["_source"] == "fallback" and p["hbm_gbs"] > 0 and p["bf16_tflops"] > 0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1.0, "bf16_tflops": 2.0}))
    p = bench.load_peaks()
    assert p["_source"] == "measured" and p["bf16_tflops"] == 2.0
