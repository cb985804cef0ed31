"""Benchmark of the one-pass randomized quaternion low-rank approximation on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec P]

Workload c2 (quaternion A 8192 x 8192, FP32 planes, sigma_i = i^-2, k=50, s=101, l=203,
Gaussian test matrices).  One step is one pass of the whole path: draw Omega and Psi,
sketch Y = A Omega and W = Psi A from one read of A (Sec. 4.1), pseudo-QR rangefinder with
three corrections (Alg. 1), QB stage X = (Psi H)^dagger W (Alg. 3) and the relative error
||A - HX||_F / ||A||_F (Sec. 5, a second read of A).  The metric is A bytes per second
through that step ("A GB/s"), with TFLOP/s and the FP32 SIMT path at equal error beside it.

Under torchrun each rank runs its own independent replica (weak scaling, no collective on
the data path); rank 0 prints one JSON line with the max time over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
N_SMS = 152
FP32_LANES_PER_SM = 128

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the fused
# sketch kernel on the c2 workload, from one ncu capture of the bench command.  It
# is reported only while the kernel's sources hash to what was captured.
SKETCH_TRAFFIC = {"bytes": 1233799680 + 27543040,
                  "sources": ["qs_sketch_tc.cu", "qs_tc_ptx.cuh"],
                  "sha256": "cfa3389d4917fd06e5d955c292f6644c1cdcb4f2beddaf503f0740ba6169935b"}


def sketch_traffic(prec, workload_name):
    """Captured per-launch DRAM bytes of the fused sketch, or None when not applicable."""
    import hashlib
    if prec != "bf16x3" or workload_name != "c2":
        return None
    h = hashlib.sha256()
    for f in SKETCH_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_2404_14783_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return SKETCH_TRAFFIC["bytes"] if h.hexdigest() == SKETCH_TRAFFIC["sha256"] else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


def max_over_ranks(value, world):
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name):
    import workloads as WL
    w = dict(WL.WORKLOADS[name])
    w["name"] = name
    return w


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def algorithmic(cfg):
    """Useful flops of the sketch (32 real flops per quaternion MAC, 24 if A is pure) and
    A bytes as stored."""
    m, n, s, l = cfg["m"], cfg["n"], cfg["s"], cfg["l"]
    per = 24 if cfg.get("pure") else 32
    esz = 8 if cfg["prec"] == "fp64" else 4
    planes = 3 if cfg.get("pure") else 4
    return per * m * n * (s + l), planes * m * n * esz


def make_A(w, device, prec):
    """The workload's matrix on the device: a (4, m, n) tensor, or for a pure quaternion
    workload the list [None, A_x, A_y, A_z] of its three stored planes."""
    import numpy as np
    import torch
    import workloads as WL
    dt = np.float64 if prec == "fp64" else np.float32
    if w["name"] == "c1":
        return torch.as_tensor(WL.make_c1(seed=w["seed"]).astype(dt), device=device).contiguous()
    if w["name"] == "c3":
        P = WL.make_c3(device)
        return [None, P[0], P[1], P[2]]
    if w["name"] == "c5":
        P = WL.make_c5(device)
        return [None, P[0], P[1], P[2]]
    if w["name"] == "lorenz":
        import paper_2404_14783_gb300 as pkg
        u0 = torch.as_tensor(WL.lorenz_initial_states(w["n"], seed=w["seed"], radius=w["radius"]),
                             device=device)
        return pkg.lorenz4d(u0, w["m"], w["dt"], w["a"], w["b"], w["c"], dtype=torch.float32)
    return WL.make_decay(w["m"], w["n"], seed=w["seed"], rank_cap=w.get("rank_cap", 1024),
                         device=device, dtype=dt).contiguous()


def planes_of(A):
    """The stored planes of a (4, m, n) tensor or a plane list (None for a zero plane)."""
    return [A[p] for p in range(4)] if not isinstance(A, list) else A


def a_nbytes(A):
    return sum(p.numel() * p.element_size() for p in planes_of(A) if p is not None)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2404_14783_gb300 as pkg
    pkg.load_library()     # fails loudly when the CUDA library is not built
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = workload(args.workload)
    pure = bool(w.get("pure", False))
    cfg = dict(m=w["m"], n=w["n"], s=w["s"], l=w["l"], prec=args.prec, emb=w["emb"],
               pure=pure)
    A = make_A(w, dev, args.prec)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    qs = pkg.QSketch(cfg["m"], cfg["n"], cfg["s"], cfg["l"], emb=cfg["emb"], prec=args.prec,
                     seed=w["seed"] + rank, rf_prec=args.rf_prec, pure=pure)
    err_out = torch.zeros(1, dtype=torch.float64, device=dev)
    E = [torch.cuda.Event(enable_timing=True) for _ in range(6)]

    def step(ev=None, A_in=A):
        if ev: ev[0].record(stream)
        qs.reset(seed=w["seed"] + rank)                    # draw Omega, Psi; zero Y, W
        if ev: ev[1].record(stream)
        qs.update(A_in, theta=0.0)                         # fused one-read sketch
        if ev: ev[2].record(stream)
        qs.rangefinder(args.rangefinder, 3)
        if ev: ev[3].record(stream)
        qs.core()
        if ev: ev[4].record(stream)
        qs.error(A_in, out=err_out)
        if ev: ev[5].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    launches0 = pkg.launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    stage_ms = {k: 0.0 for k in ("draw", "sketch", "rangefinder", "core", "error")}
    per_step_events = []
    t0.record(stream)
    for _ in range(args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        step(ev)
        per_step_events.append(ev)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = pkg.launch_count() - launches0
    clocks = sampler.stop()
    total_ms = t0.elapsed_time(t1)
    for ev in per_step_events:
        for i, k in enumerate(stage_ms):
            stage_ms[k] += ev[i].elapsed_time(ev[i + 1]) / args.steps
    total_ms = max_over_ranks(total_ms, world)
    final_err = float(err_out.item())
    status = qs.device_status()
    # truncation stage (Alg. 4, rank k) after the step: informational, not in the step time
    k = int(w.get("k", min(w["s"], 50)))
    tr0 = torch.cuda.Event(enable_timing=True)
    tr1 = torch.cuda.Event(enable_timing=True)
    qs.truncate(k)
    tr0.record(stream)
    for _ in range(3):
        qs.truncate(k)
    tr1.record(stream)
    torch.cuda.synchronize()
    truncate_ms = tr0.elapsed_time(tr1) / 3

    # end to end through the public API, every step: pinned host A streamed in by row blocks
    # (qsketch_update_host, resident staging: the copy of block b+1 overlaps the sketch of
    # block b and A stays on the device for the error pass), the step, the error read back to
    # the host.  Reported: two staging buffers taken in turn, each with an event after the
    # error pass that last read it, so one step's copies overlap the previous step's
    # rangefinder, core and error pass.  One staging buffer (copies wait for the previous
    # step) and the plain copy-then-step loop are timed beside it.
    A_host = [None if p is None else p.cpu().pin_memory() for p in planes_of(A)]
    n = cfg["n"]
    a_dtype = next(p for p in A_host if p is not None).dtype
    staging = [torch.empty(qs.staging_shape(), dtype=a_dtype, device=dev) for _ in range(2)]

    def stg_planes(stg):
        return [None if A_host[p] is None else stg[p, :, :n] for p in range(4)]
    freed = [torch.cuda.Event(), torch.cuda.Event()]
    err_host = torch.zeros(1, dtype=torch.float64).pin_memory()

    def e2e_loop(mode, steps, used):
        for i in range(steps):
            j = i & 1 if mode == "pipelined" else 0
            stg = staging[j]
            qs.reset(seed=w["seed"] + rank)
            if mode == "copy":
                for p in range(4):
                    if A_host[p] is not None:
                        stg[p, :, :n].copy_(A_host[p], non_blocking=True)
                qs.update(stg_planes(stg), theta=0.0)
            else:
                qs.update_host(A_host, stg, block_rows=args.stream_rows, theta=0.0,
                               staging_free=freed[j] if mode == "pipelined" and used[j] else None)
            qs.rangefinder(args.rangefinder, 3)
            qs.core()
            qs.error(stg_planes(stg), out=err_out)
            freed[j].record(stream)
            used[j] = True
            err_host.copy_(err_out, non_blocking=True)

    e2e = {}
    for mode in ("pipelined", "streamed", "copy"):
        used = [False, False]          # both staging buffers have an event once warmed up
        e2e_loop(mode, max(2, args.warmup), used)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_loop(mode, args.steps, used)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e[mode] = e0.elapsed_time(e1) / args.steps
        if mode == "pipelined":
            e2e_err = float(err_host.item())
    e2e_ms = e2e["pipelined"]
    e2e_status = qs.device_status()
    del staging, A_host

    flops, abytes = algorithmic(cfg)
    ms = total_ms / args.steps
    gbs = world * abytes / (ms * 1e-3) / 1e9
    result = dict(ms=ms, gbs=gbs, stage_ms=stage_ms, clocks=clocks, launches=launches,
                  final_err=final_err, status=status, e2e_ms=e2e_ms, flops=flops, abytes=abytes,
                  cfg=cfg, w=w, e2e_gbs=world * abytes / (e2e_ms * 1e-3) / 1e9,
                  h2d=a_nbytes(A), d2h=8, truncate_ms=truncate_ms, trunc_rank=k,
                  e2e_modes=e2e, e2e_err=e2e_err, e2e_status=e2e_status)
    # the stages after the sketch in the other arithmetics, on this step's Y and W (rank 0,
    # informational): native FP64, and the mixed mode with its device-chosen FP32 steps
    if rank == 0 and args.prec != "fp64" and not args.no_compare:
        result["rf_variants"] = {}
        for rf in ("fp64", "mixed"):
            if rf == args.rf_prec:
                continue
            qv = pkg.QSketch(cfg["m"], cfg["n"], cfg["s"], cfg["l"], emb=cfg["emb"], prec=args.prec,
                             seed=w["seed"], rf_prec=rf, pure=pure)
            qv.get("Y").copy_(qs.get("Y"))
            qv.get("W").copy_(qs.get("W"))
            for _ in range(2):
                qv.rangefinder(args.rangefinder, 3)
                qv.core()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            reps = 3
            ev[0].record(stream)
            for _ in range(reps):
                qv.rangefinder(args.rangefinder, 3)
            ev[1].record(stream)
            for _ in range(reps):
                qv.core()
            ev[2].record(stream)
            err_v = float(qv.error(A).item())
            torch.cuda.synchronize()
            result["rf_variants"][rf] = dict(
                rangefinder_ms=ev[0].elapsed_time(ev[1]) / reps,
                core_ms=ev[1].elapsed_time(ev[2]) / reps,
                final_rel_error=err_v, device_status=int(qv.device_status()))
            qv.close()
    # FP32 SIMT comparison path at equal error (rank 0 only, device resident): the sketch
    # timed over 20 repetitions after warm-up, the whole path once for its final error
    if rank == 0 and args.prec != "fp32" and not args.no_compare:
        qs32 = pkg.QSketch(cfg["m"], cfg["n"], cfg["s"], cfg["l"], emb=cfg["emb"], prec="fp32",
                           seed=w["seed"], rf_prec=args.rf_prec, pure=pure)
        for _ in range(args.warmup):
            qs32.update(A, theta=0.0)
        reps32 = 20 if cfg["m"] * cfg["n"] <= 8192 * 8192 else 5
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(reps32):
            qs32.update(A, theta=0.0)
        s1.record(stream)
        qs32.reset(seed=w["seed"])
        qs32.update(A, theta=0.0)
        qs32.rangefinder(args.rangefinder, 3)
        qs32.core()
        e32 = float(qs32.error(A).item())
        torch.cuda.synchronize()
        result["fp32"] = dict(sketch_ms=s0.elapsed_time(s1) / reps32, reps=reps32, err=e32)
        qs32.close()
    qs.close()
    return result


def run_batch(args):
    """c4: 256 matrices sketched by qsketch_update_batched (one persistent launch over all
    matrices after the launches that write their descriptors, in the plan the autotuner
    qsketch_tune_batched chose; the call replayed from a CUDA graph) against a loop of
    per-matrix qsketch_update calls; inputs resident in HBM (21 GB, larger than L2)."""
    import torch
    import paper_2404_14783_gb300 as pkg
    import workloads as WL
    pkg.load_library()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    spec = dict(WL.WORKLOADS["c4"])
    batch = WL.make_c4_batch(dev)
    sk, mats, flops, abytes = [], [], 0, 0
    for i, (m, n, k, A) in enumerate(batch):
        s = 2 * k + 1
        l = min(2 * s + 1, m, n)          # l <= min(m, n) (Sec. 4.1): clamps k = 64 at m = 256
        sk.append(pkg.QSketch(m, n, s, l, emb=spec["emb"], prec=args.prec, seed=spec["seed"] + i))
        mats.append(A)
        flops += 32 * m * n * (s + l)
        abytes += 16 * m * n
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def loop():
        for q, A in zip(sk, mats):
            q.update(A, theta=0.0)

    pkg.tune_batched(sk, mats, reps=2)     # the autotuner's plan for this batch signature
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        pkg.update_batched(sk, mats)
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        pkg.update_batched(sk, mats)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    sampler = ClockSampler(0)
    sampler.start()
    t_batched = timed(graph.replay, args.steps)
    t_loop = timed(loop, args.steps)
    clocks = sampler.stop()
    status = max(int(q.device_status()) for q in sk)
    peaks = load_peaks()
    products = 2 if spec["emb"] == "rademacher" and args.prec == "bf16x3" else (
        3 if args.prec == "bf16x3" else 1)
    out = {"metric": "one-pass quaternion approx: A GB/s & TFLOPS, split-BF16 vs FP32 at equal error",
           "value": abytes / (t_batched * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batched,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"bf16x3": "bf16x3", "bf16": "bf16"}.get(args.prec, args.prec),
           "data": "synthetic",
           "config": {"workload": f"c4: batch of {len(sk)} quaternion matrices, m, n ~ "
                                  f"U[{spec['lo']}, {spec['hi']}], k ~ U{{{spec['k_lo']}..{spec['k_hi']}}}, "
                                  "s = 2k+1, l = min(2s+1, m, n), Rademacher, sketch only",
                      "A_bytes": abytes, "useful_flops": flops,
                      "l2": "inputs larger than L2 (A is %.1f GB)" % (abytes / 1e9)},
           "roofline": {"bound": "tensor", "achieved": flops / (t_batched * 1e-3) / 1e12,
                        "peak": peaks.get("bf16_tflops"), "unit": "TFLOP/s",
                        "frac": flops / (t_batched * 1e-3) / 1e12 / peaks.get("bf16_tflops"),
                        "traffic": None, "issued_products": products,
                        "peak_source": peaks["_source"] + " bf16 burst"},
           "batched": {"persistent_graph_ms": t_batched, "per_matrix_loop_ms": t_loop,
                       "speedup": t_loop / t_batched,
                       "launches_per_call": {"batched": None, "loop": None}},
           "device_status": status, "clocks": clocks}
    # launches per call, counted by the library (the graph replays count nothing)
    c0 = pkg.launch_count()
    pkg.update_batched(sk, mats)
    c1 = pkg.launch_count()
    loop()
    c2 = pkg.launch_count()
    torch.cuda.synchronize()
    out["batched"]["launches_per_call"] = {"batched": c1 - c0, "loop": c2 - c1}
    out["gpu_launches"] = (c1 - c0) * args.steps      # the timed batched calls (graph replays)
    out["gpu_launches_per_call"] = c1 - c0
    print(json.dumps(out), flush=True)


def run_rf_curve(args):
    """Rangefinder time against the sketch height m with m = 20 s (the paper's timing of its
    rangefinders, Sec. 3.4): Y (m x s, quaternion Gaussian, FP32 values in a split-BF16
    handle, double-float stages) written into a handle; each kind timed with CUDA events over
    `steps` calls after `warmup` calls."""
    import numpy as np
    import torch
    import paper_2404_14783_gb300 as pkg
    pkg.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    kinds = ("pseudo_qr", "pseudo_svd", "pseudo_qr_householder", "pseudo_svd_householder")
    curve = []
    sampler = ClockSampler(0)
    sampler.start()
    for m in (500, 1000, 2000, 3000, 4000, 5000):
        s = m // 20
        l = min(2 * s + 1, m)
        qs = pkg.QSketch(m, l, s, l, emb="gaussian", prec="bf16x3", seed=1)
        gen = torch.Generator(device=dev)
        gen.manual_seed(m)
        qs.get("Y").copy_(torch.randn((4, m, s), generator=gen, device=dev))
        row = {"m": m, "s": s}
        for kind in kinds:
            for _ in range(args.warmup):
                qs.rangefinder(kind, 3)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                qs.rangefinder(kind, 3)
            e1.record(stream)
            torch.cuda.synchronize()
            row[kind + "_ms"] = e0.elapsed_time(e1) / args.steps
        row["device_status"] = int(qs.device_status())
        curve.append(row)
        qs.close()
    clocks = sampler.stop()
    last = curve[-1]
    out = {"metric": "rangefinder time vs m (m = 20 s): pseudo-QR with 3 corrections",
           "value": last["pseudo_qr_ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": last["pseudo_qr_ms"], "higher_is_better": False,
           "scaling": "none", "vs_baseline": None, "dtype": "df64", "data": "synthetic",
           "config": {"workload": "rangefinders on quaternion Gaussian Y, m in 500..5000, s = m/20",
                      "l2": "Y is at most 5000 x 250 quaternion (L2-resident): small-matrix latency"},
           "curve": curve, "clocks": clocks}
    print(json.dumps(out), flush=True)


def batch_reference(args):
    """The oracle's sketch (Sec. 4.1, FP64 on the host cores) on a bounded sample of the c4
    batch: its first two matrices (same sizes and spectra as the GPU run's; the host's torch
    generator draws other factor values), the metric scaled to A GB/s."""
    import numpy as np
    import oracle as O
    import workloads as WL
    spec = dict(WL.WORKLOADS["c4"])
    sample = WL.make_c4_batch("cpu", dict(count=2))
    vals = []
    for it in range(args.warmup + args.steps):
        t, abytes = 0.0, 0
        for i, (m, n, k, A) in enumerate(sample):
            s = 2 * k + 1
            l = min(2 * s + 1, m, n)
            A64 = A.double().numpy()
            Om = O.draw_embedding(n, s, O.EMB_RADEMACHER, O.STREAM_OMEGA, spec["seed"] + i)
            Psi = O.draw_embedding(l, m, O.EMB_RADEMACHER, O.STREAM_PSI, spec["seed"] + i)
            t0 = time.perf_counter()
            O.sketch(A64, Om, Psi)
            t += time.perf_counter() - t0
            abytes += 16 * m * n
        if it >= args.warmup:
            vals.append((abytes / t / 1e9, t))
    v = statistics.median([g for g, _ in vals])
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample_desc = "first 2 matrices of the c4 batch: " + ", ".join(
        f"{m}x{n} k={k}" for m, n, k, _ in sample)
    out = {"impl": "reference", "metric": "one-pass quaternion approx: A GB/s & TFLOPS, split-BF16 vs FP32 at equal error",
           "value": v, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": statistics.median([t for _, t in vals]) * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "c4: batch of quaternion matrices, sketch only (oracle sample)"},
           "cpu_baseline": {"value": v, "unit": "GB/s", "cores": threads, "kind": "oracle",
                            "sample": sample_desc},
           "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_sample(w, rows):
    """A bounded sample of the workload for the oracle on the host cores, as FP64 numpy
    (4, rows', n') planes, and its description: c1/c2 the first rows of the matrix; c3 the
    first rows and columns of the same image (same generator); c5 a 32^3 grid with the same
    time steps.  The oracle's rate on the sample is reported as A GB/s of the sample."""
    import numpy as np
    import workloads as WL
    if w["name"] == "c1":
        A = WL.make_c1(seed=w["seed"])[:, :rows]
        return A, f"first {A.shape[1]} rows x {A.shape[2]} cols of c1"
    if w["name"] == "c3":
        cols = 8192      # the oracle's least-squares solve costs ~2.5 ms per column of A
        P = WL.make_c3("cpu", m=w["m"], n=w["n"], rows=rows)[:, :, :cols].double().numpy()
        A = np.concatenate([np.zeros((1,) + P.shape[1:]), P])
        return A, f"first {rows} rows x first {cols} cols of the c3 image (pure)"
    if w["name"] == "c5":
        P = WL.make_c5("cpu", grid=32).double().numpy()
        A = np.concatenate([np.zeros((1,) + P.shape[1:]), P])
        return A, f"32^3-grid c5 snapshots ({A.shape[1]} rows x {A.shape[2]} cols, pure)"
    if w["name"] == "lorenz":
        import oracle as O
        u0 = WL.lorenz_initial_states(w["n"], seed=w["seed"], radius=w["radius"])
        A = O.lorenz4d_snapshots(u0, rows, w["dt"], w["a"], w["b"], w["c"])
        return A, f"first {rows} time instances x {w['n']} trajectories (the oracle's own RK4)"
    A = WL.make_decay(w["m"], w["n"], seed=w["seed"], rank_cap=w.get("rank_cap", 1024),
                      dtype=np.float64)[:, :rows]
    return A, f"first {A.shape[1]} rows x {A.shape[2]} cols of {w['name']}"


def cpu_baseline(w, rows, reps=1, sample=None):
    """The FP64 oracle's whole one-pass path on the host cores on a bounded sample of the
    workload (cpu_sample).  Returns (A GB/s, seconds, threads, description); the bytes are
    those of the sample as the GPU workload stores it (FP32, 3 planes when pure)."""
    import oracle as O
    A, desc = sample if sample is not None else cpu_sample(w, rows)
    m, n = A.shape[1], A.shape[2]
    kind = O.EMB_GAUSSIAN if w["emb"] == "gaussian" else O.EMB_RADEMACHER
    l = min(w["l"], m, n)
    Om = O.draw_embedding(n, w["s"], kind, O.STREAM_OMEGA, w["seed"])
    Psi = O.draw_embedding(l, m, kind, O.STREAM_PSI, w["seed"])
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        O.onepass(A, Om, Psi, "pseudo_qr", 3)
        times.append(time.perf_counter() - t)
    sec = min(times)
    abytes = (3 if w.get("pure") else 4) * m * n * 4      # A bytes as stored in the FP32 workload
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return abytes / sec / 1e9, sec, threads, desc


WORKLOAD_TEXT = {
    "c1": "quaternion A 512x384 FP64 planes, U diag(0.5^i) V* + 1e-6 noise, k=10, s=21, l=43, Gaussian Omega/Psi",
    "c2": "quaternion A 8192x8192 FP32 planes, sigma_i=i^-2, k=50, s=101, l=203, Gaussian Omega/Psi",
    "c3": "pure-quaternion image-like A 31365x27125 FP32 (3 channels of 64 random Fourier modes in [0,0.98] "
          "+ U(0,0.02)), k=100, s=201, l=403, Rademacher Omega/Psi (exact in BF16)",
    "c5": "pure-quaternion flow snapshots A 2097152x256 FP32 (128^3 grid x 256 steps, 32 divergence-free "
          "Taylor-Green-type modes + 1e-4 noise), k=20, s=41, l=83, Gaussian Omega/Psi",
    "lorenz": "4D Lorenz-type system snapshots A 20000x10000 FP32 (x + yi + zj + wk after each of 20000 "
              "RK4 steps of 1e-3 from 10000 states on the radius-20 sphere, a=15, b=2, c=28), k=100, "
              "s=201, l=403, Gaussian Omega/Psi",
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp64", "fp32", "bf16", "bf16x3"])
    ap.add_argument("--workload", default="c2",
                    help="c2 (default: the one-pass step), c1, c3, c5, lorenz (the same step on those "
                         "workloads), c4 (the batched sketch), rf_curve (rangefinder time vs m)")
    ap.add_argument("--rangefinder", default="pseudo_qr")
    ap.add_argument("--rf-prec", default="df64", choices=["df64", "fp64", "mixed"],
                    help="arithmetic of the rangefinder, core and truncation stages")
    ap.add_argument("--cpu-rows", type=int, default=None,
                    help="rows of the oracle's sample (default: 4096 for c2, 256 for c3)")
    ap.add_argument("--stream-rows", type=int, default=1024,
                    help="row-block height of the streamed host update in the e2e loop")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.cpu_rows is None:
        args.cpu_rows = {"c3": 256, "lorenz": 1024}.get(args.workload, 4096)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.workload == "c4":
        if rank == 0:      # the batch workload runs on one GPU / on the host cores
            run_batch(args) if args.impl == "ours" else batch_reference(args)
        return
    if args.workload == "rf_curve":
        if rank == 0 and args.impl == "ours":
            run_rf_curve(args)
        elif rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the rangefinder timing curve "
                              "has no oracle arm (the oracle's timing is in the c2 line)"}))
        return
    w = workload(args.workload)
    metric = "one-pass quaternion approx: A GB/s & TFLOPS, split-BF16 vs FP32 at equal error"
    abytes_w = (3 if w.get("pure") else 4) * w["m"] * w["n"] * (8 if args.prec == "fp64" else 4)
    config = {"workload": f"{w['name']}: {WORKLOAD_TEXT[w['name']]}",
              "m": w["m"], "n": w["n"], "s": w["s"], "l": w["l"], "prec": args.prec,
              "rangefinder": args.rangefinder, "n_correction": 3, "rf_prec": args.rf_prec,
              "l2": "inputs larger than L2 (A is %.2f GB per step)" % (abytes_w / 1e9),
              "parallelism": "replicas"}

    if args.impl == "reference":
        if rank != 0:
            return
        vals = []
        smp = cpu_sample(w, args.cpu_rows)
        for i in range(args.warmup + args.steps):
            gbs, sec, thr, sample = cpu_baseline(w, args.cpu_rows, sample=smp)
            if i >= args.warmup:
                vals.append((gbs, sec))
        v = statistics.median([g for g, _ in vals])
        out = {"impl": "reference", "metric": metric, "value": v, "unit": "GB/s",
               "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": statistics.median([s for _, s in vals]) * 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": config,
               "cpu_baseline": {"value": v, "unit": "GB/s", "cores": thr, "kind": "oracle",
                                "sample": sample},
               "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    peaks = load_peaks()
    flops, abytes = res["flops"], res["abytes"]
    sk_ms = res["stage_ms"]["sketch"]
    tc = args.prec in ("bf16", "bf16x3")
    products = {"bf16x3": 3 if w["emb"] == "gaussian" else 2, "bf16": 1}.get(args.prec, 1)
    if tc:
        peak = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": flops / (sk_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s"}
    else:
        clk = peaks.get("sm_max_mhz", 2070.0)
        per_sm = FP32_LANES_PER_SM * 2 if args.prec == "fp32" else 4.0
        peak = N_SMS * per_sm * clk * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / (sk_ms * 1e-3) / 1e12, "peak": peak,
                "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = sketch_traffic(args.prec, w["name"])
    roof["kernel"] = "fused sketch (qsketch_update)"
    roof["peak_source"] = peaks["_source"] + (" bf16 burst" if tc else " derived FP32 ALU")
    out = {"metric": metric, "value": res["gbs"], "unit": "GB/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.prec == "fp64" else args.prec.replace("fp32", "f32") + "+" + {
               "df64": "df64", "fp64": "f64", "mixed": "df64/f32"}[args.rf_prec],
           "data": "synthetic", "config": config, "roofline": roof,
           "tflops": {"useful_step": world * flops / (res["ms"] * 1e-3) / 1e12,
                      "useful_sketch": flops / (sk_ms * 1e-3) / 1e12,
                      "issued_sketch": products * flops / (sk_ms * 1e-3) / 1e12 if tc else None},
           "sketch_gbs": abytes / (sk_ms * 1e-3) / 1e9,
           "stages_ms": res["stage_ms"], "final_rel_error": res["final_err"],
           "truncation_stage_ms": {"rank": res["trunc_rank"], "ms": res["truncate_ms"],
                                   "note": "Alg. 4 after the step, not in ms_per_step"},
           "device_status": res["status"],
           "e2e": {"value": res["e2e_gbs"], "unit": "GB/s", "h2d_bytes_per_step": res["h2d"],
                   "d2h_bytes_per_step": res["d2h"], "ms_per_step": res["e2e_ms"],
                   "mode": f"qsketch_update_host, row blocks of {args.stream_rows}, two resident "
                           "staging buffers in turn (next step's copies overlap this step)",
                   "one_staging_ms": res["e2e_modes"]["streamed"],
                   "copy_then_step_ms": res["e2e_modes"]["copy"],
                   "final_err": res["e2e_err"], "device_status": res["e2e_status"]},
           "gpu_launches": res["launches"], "gpu_launches_per_step": res["launches"] / args.steps,
           "clocks": res["clocks"]}
    if "rf_variants" in res:
        out["stages_after_sketch_variants"] = res["rf_variants"]
    if "fp32" in res:
        clk = (res["clocks"] or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        fp32_peak = N_SMS * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
        # the SIMT sketch runs on 64 x 64 quaternion tiles: Y = A Omega pads s, W = Psi A pads l
        pad = lambda v: -(-v // 64) * 64
        m_, n_, s_, l_ = w["m"], w["n"], w["s"], w["l"]
        issued32 = flops * (pad(m_) * pad(s_) * n_ + pad(l_) * pad(n_) * m_) / (m_ * n_ * (s_ + l_))
        out["fp32_path"] = {"sketch_ms": res["fp32"]["sketch_ms"], "reps": res["fp32"]["reps"],
                            "sketch_tflops": flops / (res["fp32"]["sketch_ms"] * 1e-3) / 1e12,
                            "issued_tflops": issued32 / (res["fp32"]["sketch_ms"] * 1e-3) / 1e12,
                            "frac_issued_of_fp32_peak": issued32 / (res["fp32"]["sketch_ms"] * 1e-3) / 1e12 / fp32_peak,
                            "fp32_alu_peak_tflops": fp32_peak,
                            "frac_of_fp32_peak": flops / (res["fp32"]["sketch_ms"] * 1e-3) / 1e12 / fp32_peak,
                            "final_rel_error": res["fp32"]["err"],
                            "sketch_speedup_vs_fp32": res["fp32"]["sketch_ms"] / sk_ms,
                            "error_ratio": res["final_err"] / res["fp32"]["err"]}
    if not args.no_cpu:
        gbs, sec, thr, sample = cpu_baseline(w, args.cpu_rows)
        out["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": thr, "kind": "oracle",
                               "sample": sample, "seconds": sec}
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
