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


def test_json_line_assembly_with_a_stubbed_run(monkeypatch, capsys):
    """The JSON line of the default (c2) arm from a stubbed device run: the contract's keys,
    value = A bytes / step time, and gpu_launches = the launches of the K timed steps."""
    steps, ms, per_step = 4, 10.0, 102
    cfg = dict(m=8192, n=8192, s=101, l=203, prec="bf16x3", emb="gaussian", pure=False)
    flops, abytes = bench.algorithmic(cfg)
    res = dict(ms=ms, gbs=abytes / (ms * 1e-3) / 1e9, launches=per_step * steps,
               stage_ms={"draw": 0.1, "sketch": 2.75, "rangefinder": 4.5, "core": 1.1, "error": 0.8},
               clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}, final_err=1.6e-3,
               status=0, e2e_ms=11.0, flops=flops, abytes=abytes, cfg=cfg, w={}, e2e_gbs=97.6,
               h2d=abytes, d2h=8, truncate_ms=33.0, trunc_rank=50,
               e2e_modes={"pipelined": 11.0, "streamed": 12.0, "copy": 15.0}, e2e_err=1.6e-3,
               e2e_status=0)
    monkeypatch.setattr(bench, "run_ours", lambda args, rank, world, local_rank: res)
    monkeypatch.setattr("sys.argv", ["bench.py", "--steps", str(steps), "--no-cpu"])
    bench.main()
    line = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")][-1]
    out = json.loads(line)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in out, key
    assert out["steps"] == steps and out["warmup"] >= 3 and out["n_gpus"] == 1
    assert out["value"] == pytest.approx(abytes / (ms * 1e-3) / 1e9)
    assert out["gpu_launches"] == per_step * steps and out["gpu_launches_per_step"] == per_step
    roof = out["roofline"]
    assert roof["achieved"] == pytest.approx(flops / 2.75e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert set(out["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
