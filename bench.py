#!/usr/bin/env python3
"""Benchmark: WMC denoising throughput on GB300 (gigapixel-iterations per second).

One step = the whole hot path on one 4096 x 4096 FP32 synthetic image (64 bumps, 32 shapes,
sigma 0.02, seed 1): one H^w evaluation pass (wmc_eval), 500 Jacobi iterations of the
L2-denoising flow (wmc_denoise: lambda 1, step 0.25, replicate boundary) and the FP64
energies (wmc_energy).  value = H*W*500 / step time (the evaluation pass and the energies
are inside the timed step but not counted as work).  L2 is flushed before every timed step,
outside the events (a 256 MiB write, then a 256 MiB read of another buffer, which leaves L2 clean).

The same JSON line carries, under "secondary", compact measurements of the other workloads
(each a few seconds of GPU time; --no-secondary skips them): the 4096^2 sigma 0.1 image, the
256^2 PR1 run (plain launches and a CUDA graph replay), the 16384^2 FP32/BF16/FP16 rates, the
512-image batch against looping the single-image path, and the 32 x 512^2 unrolled
forward + backward.  The CPU-baseline leg times the FP64 oracle on the host cores and compares
its result with the GPU's on the same crop ("parity").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload scale|pr1|precision|batch|diff|l1|fd]

--impl reference times the FP64 CPU oracle on the host cores on a bounded crop of the same
workload.  Under torchrun (N > 1) every rank denoises its own image (independent replicas:
weak scaling, no communication) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gigapixel-iterations/s of WMC denoising (1 GB300) and % of HBM roofline"
UNIT = "Gpix-iter/s"
H = W = 4096
ITERS = 500
LAM = 1.0
STEP = 0.25
SIGMA = 0.02
WORKLOAD = (f"{H}x{W} f32 synthetic image (64 bumps + 32 shapes, sigma {SIGMA}, seed 1): "
            f"1 WMC eval pass + {ITERS} L2-denoising iterations (lambda {LAM}, step {STEP}, "
            f"replicate) + FP64 energies")
BYTES_PER_PX_LAUNCH = 12  # read U, read f, write U (FP32): algorithmic bytes of one pass
# Algorithmic FP32 operations on the FMA pipe per output pixel-iteration: the stencil in the
# L +- a_j form evaluated cell by cell (L and the four odd parts: 20, |L|-|a_j|: 4, sign guard: 1)
# and the update (2); compare/select/sign logic (7 more) runs on the separate ALU pipe and is not
# counted.  The kernels share four per-row values between the three cells that read a row, so
# they execute fewer: FMA_OPS_EXECUTED_PER_PX_ITER (14 for the linear part instead of 20).
FMA_OPS_PER_PX_ITER = 27
FMA_OPS_EXECUTED_PER_PX_ITER = 21
DEFAULT_T = 4
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one 4-step flow launch on this
# image, from the ncu capture of one warm-L2 launch of the current kernel summarised in
# profiles/flow_tile_t4_4096x4096_full.md; reported as roofline.traffic for the default 4 steps
# per launch and the full 500 iterations only
TILE_T4_DRAM_BYTES = 89.02e6  # 67.19 MB read + 21.83 MB written
# GB300 HBM3e nominal bandwidth (GB/s); fractions are reported against it and against the
# measured copy bandwidth
NOMINAL_HBM_GBS = 8000.0
# The paper's one throughput figure (the abstract and Sec. IV-D, support region and complexity):
# WMC computed at 33.2 gigapixels/s on an NVIDIA TITAN X (Pascal); image size, precision and pass
# not stated.  Another machine: context for the eval pass, not a target.
PAPER_EVAL_CONTEXT = {"value": 33.2, "unit": "Gpix/s", "hardware": "NVIDIA TITAN X (Pascal)",
                      "note": "paper figure; size, precision and pass not stated"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--steps-per-launch", type=int, default=0)
    ap.add_argument("--iters", type=int, default=ITERS, help="override (profiling runs only)")
    ap.add_argument("--workload", default="scale", choices=["scale", "pr1", "precision", "batch", "diff", "l1", "fd"],
                    help="scale: the headline 4096^2 run; pr1 / precision / batch / diff: the 256^2, "
                         "reduced-storage, uneven-batch and reverse-mode measurements (one JSON line "
                         "each, not the headline)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the secondary workloads")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(rank: int) -> int:
    """Input seed of a replica: rank 0 times the workload image (seed 1); other ranks get their
    own image of the same recipe (replicas share nothing)."""
    return 1 + 1000 * rank


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values (all-reduce MAX; the identity for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, slowest_ms: float) -> float:
    """Whole-job throughput in G units/s: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (slowest_ms * 1e-3) / 1e9


class L2Flush:
    """Evicts the workload's data from the 126 MB L2 before a timed run: writes a 256 MiB buffer,
    then reads a second 256 MiB buffer so that the write's dirty lines are written back here and
    not inside the timed run."""

    def __init__(self, device):
        import torch
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        self.r = torch.ones(64 << 20, dtype=torch.float32, device=device)

    def __call__(self):
        self.w.zero_()
        self.r.sum()


L2_NOTE = "flushed before each timed step (256 MiB write, then 256 MiB read of a second buffer)"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        rows = []
        with open(self.file.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_rate(u, crop: int, iters: int, threads: int):
    """Oracle throughput (Gpix-iter/s) on a crop x crop corner of the image, `iters` steps, on
    `threads` host threads (its OpenMP loops; the result does not depend on the count)."""
    import oracle
    f = np.ascontiguousarray(u[:crop, :crop], dtype=np.float64)
    oracle.build()
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.denoise(f, LAM, STEP, iters)
    dt = time.perf_counter() - t0
    return crop * crop * iters / dt / 1e9, dt


def oracle_parity(u, gpu_result, crop: int, iters: int, threads: int):
    """The CPU-baseline leg's comparison of the GPU with the FP64 oracle: `iters` oracle steps on
    the crop x crop corner of the input (run step by step, counting the opposite-sign near-ties of
    Eq. act that each step meets), against `gpu_result` (the GPU's U^iters of the whole image, on
    the host).  The oracle's crop has a false edge, whose influence travels one pixel per step,
    so the two are compared on the top-left (crop - iters)^2 window, where the crop's result is
    the whole image's."""
    import oracle
    F = np.ascontiguousarray(u[:crop, :crop], dtype=np.float64)
    R = float(u.max() - u.min())
    tau = 2.0 ** -18 * R  # the tie band of the parity protocol
    oracle.set_threads(threads)
    U, ties = F.copy(), 0
    for _ in range(iters):
        ties += oracle.count_ties(U[:crop - iters + 1, :crop - iters + 1], tau)
        U = oracle.denoise(F, LAM, STEP, 1, u0=U)
    n = crop - iters
    d = np.abs(np.asarray(gpu_result[:n, :n], dtype=np.float64) - U[:n, :n])
    mse = float((d ** 2).mean())
    return {"window": f"top-left {n}x{n} of the image (oracle on the {crop}x{crop} crop, {iters} iterations)",
            "max_abs_err_over_range": float(d.max()) / R, "tol_over_range": 1e-5,
            "pixels_beyond_tol": int((d > 1e-5 * R).sum()), "pixels": n * n,
            "tie_events": ties, "tie_band_over_range": 2.0 ** -18,
            "psnr_db_vs_oracle": 10 * math.log10(R * R / mse) if mse > 0 else None,
            "note": "tie events: opposite-sign near-ties of Eq. act met by the oracle's trajectory "
                    "(each step, on the region that reaches the window); a different choice there "
                    "is valid and moves the pixel by about 2 step lambda |H^w|"}


def energy_parity(wmc, f, out, ws, ews, iters: int, T: int, u_host):
    """The CPU-baseline leg's check of the step's energies (Eq. wmcr with q = 1 and the data term
    of Eq. 1): the GPU's sum |H^w| and 1/2 sum (U - f)^2 of its U^iters over the whole image
    against the FP64 oracle's sums of the same U (read back) and f.  The GPU sums FP32 per-pixel
    terms in 16-cell FP32 partials and double-float accumulators; the relative errors say what
    that leaves of FP64."""
    import oracle
    uf = wmc.denoise(f, LAM, STEP, iters, out=out, steps_per_launch=T, workspace=ws)
    eg = wmc.energy(uf, f, None, workspace=ews).cpu().tolist()
    eo = oracle.energies(uf.double().cpu().numpy(), np.asarray(u_host, dtype=np.float64))
    return {"image": f"{H}x{W}, U after {iters} iterations", "gpu": eg[:2], "oracle": list(eo[:2]),
            "rel_err": [abs(eg[k] - eo[k]) / abs(eo[k]) if eo[k] else abs(eg[k]) for k in range(2)],
            "terms": ["sum |H^w|", "1/2 sum (U - f)^2"]}


def host_threads() -> int:
    return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1903_07189_gb300 import synth
    u = synth.make_image(H, W, seed=1, n_bumps=64, n_shapes=32, sigma=SIGMA)
    crop, iters, threads = 2048, 8, host_threads()
    for _ in range(args.warmup):
        cpu_oracle_rate(u, 128, 2, threads)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = cpu_oracle_rate(u, crop, iters, threads)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    sample = (f"{crop}x{crop} top-left crop of the workload image, {iters} iterations per step "
              f"(oracle, FP64, {threads} threads)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def fma_peak(wmc, dev):
    """The compute roofline's denominator: FP32 FMA lane-operations per second of this GPU,
    measured by the library's probe (8 independent packed FP32x2 FMA chains per thread, 8 CTAs
    per SM, best of 5 launches of about 20 ms), with the device's SM count beside it."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    rate = wmc.measure_fma_rate(dev, iters=200_000, reps=5)
    return {"tops": rate / 1e12, "sms": props.multi_processor_count,
            "how": "wmc_probe_fma: 8 packed FP32x2 FMA chains per thread, 8 CTAs per SM, best of 5 "
                   "(an FMA counts as one lane-operation)"}


def event_ms(fn, reps, flush=None):
    """Median device time (CUDA events on the current stream) of fn() over `reps` runs."""
    import torch
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def measure_scale_image(wmc, dev, u_host, iters, T, reps, flush):
    """The headline step (eval + `iters` flow iterations + energies) on another image of the
    4096^2 recipe: Gpix-iter/s over the median step time, L2 flushed before each step."""
    import torch
    f = torch.from_numpy(u_host).to(dev)
    hw, out = torch.empty_like(f), torch.empty_like(f)
    h, w = f.shape
    ws = torch.empty(wmc.load().wmc_denoise_workspace_size(h, w, w, 0), dtype=torch.uint8, device=dev)
    ews = torch.empty(wmc.load().wmc_energy_workspace_size(h, w), dtype=torch.uint8, device=dev)
    en = torch.empty(3, dtype=torch.float64, device=dev)

    def step():
        wmc.eval(f, out=hw)
        wmc.denoise(f, LAM, STEP, iters, out=out, steps_per_launch=T, workspace=ws)
        wmc.energy(out, f, None, out=en, workspace=ews)
    for _ in range(3):
        step()
    ms = event_ms(step, reps, flush)
    return {"gpix_iter_s": h * w * iters / (ms * 1e-3) / 1e9, "ms_per_step": ms, "steps": reps}


def measure_pr1(wmc, dev, reps=50):
    """256 x 256 PR1 image (seed 0, 8 bumps + 4 shapes, sigma 0.05): one evaluation plus 100
    iterations (lambda 1, step 0.25, replicate), the input resident on the device; timed as plain
    launches and as one replay of a CUDA graph of the same calls, for the default and the largest
    steps per launch.  The image (786 KB per iteration) lives in L2: the run is launch and latency
    bound."""
    import torch
    from paper_1903_07189_gb300 import synth
    f = torch.from_numpy(synth.pr1_image()).to(dev)
    hw, out = torch.empty_like(f), torch.empty_like(f)
    n = f.numel()
    ws = torch.empty(wmc.load().wmc_denoise_workspace_size(256, 256, 256, 0), dtype=torch.uint8, device=dev)
    res = {}
    ctas = wmc.cluster_size(256, 256, 100, dev)
    for T in (DEFAULT_T, 8, 0):
        def run():
            wmc.eval(f, out=hw)
            wmc.denoise(f, 1.0, 0.25, 100, out=out, steps_per_launch=T, workspace=ws)
        for _ in range(3):
            run()
        t_plain = event_ms(run, reps)
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            run()
        torch.cuda.current_stream(dev).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            run()
        g.replay()
        t_graph = event_ms(g.replay, reps)
        # the default configuration runs the 100 iterations as one cluster launch (when the
        # device schedules a cluster of `ctas` CTAs)
        launches = 1 + (1 if (T == 0 and ctas) else math.ceil(100 / (T or DEFAULT_T)))
        key = f"T{T}" if T else "default"
        res[key] = {"plain_us": 1e3 * t_plain, "graph_us": 1e3 * t_graph, "launches": launches,
                    "plain_gpix_iter_s": n * 100 / (t_plain * 1e-3) / 1e9,
                    "graph_gpix_iter_s": n * 100 / (t_graph * 1e-3) / 1e9}
        if T == 0:
            res[key]["cluster_ctas"] = ctas
    # The evaluation and the iterations both read only f: with the evaluation on a second stream
    # (forked from and joined to the first) the two kernels run side by side on separate SMs.
    main, side = torch.cuda.current_stream(dev), torch.cuda.Stream(dev)

    def run_forked():
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            wmc.eval(f, out=hw)
        wmc.denoise(f, 1.0, 0.25, 100, out=out, workspace=ws)
        torch.cuda.current_stream(dev).wait_stream(side)
    for _ in range(3):
        run_forked()
    t_plain = event_ms(run_forked, reps)
    s = torch.cuda.Stream(dev)
    s.wait_stream(main)
    with torch.cuda.stream(s):
        run_forked()
    main.wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run_forked()
    g.replay()
    t_graph = event_ms(g.replay, reps)
    res["default_eval_on_second_stream"] = {"plain_us": 1e3 * t_plain, "graph_us": 1e3 * t_graph,
                                            "graph_gpix_iter_s": n * 100 / (t_graph * 1e-3) / 1e9}
    return {"workload": "256x256 f32 (seed 0, 8 bumps + 4 shapes, sigma 0.05): 1 eval + 100 iterations, "
                        "lambda 1, step 0.25, replicate", "runs": reps, **res}


def measure_precision_rates(wmc, dev, img, iters, T, reps=2):
    """The 16384^2 image stored as FP32, BF16 and FP16 (FP32 arithmetic, every step rounded to
    the storage type): `iters` iterations per storage type, Gpix-iter/s of the best of `reps`
    runs.  Returns the rates and the results (host, FP64) for the error against the oracle."""
    import torch
    n = img.shape[0]
    rates, outs = {}, {}
    for name, dt in [("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float16)]:
        f = torch.from_numpy(img).to(dev).to(dt)
        out = torch.empty_like(f)
        ws = torch.empty(wmc.load().wmc_denoise_workspace_size(n, n, n, wmc.DTYPES[dt]), dtype=torch.uint8,
                         device=dev)
        run = lambda: wmc.denoise(f, LAM, STEP, iters, out=out, steps_per_launch=T, workspace=ws)
        run()
        ms = min(event_ms(run, 1) for _ in range(reps))
        rates[name] = {"gpix_iter_s": n * n * iters / (ms * 1e-3) / 1e9, "ms": ms}
        outs[name] = out
        del f, ws
    return rates, outs


def measure_batch(wmc, dev, fs, lams, steps, iters, reps, world=1, T=0, tile=0):
    """Many uneven images advanced together: (a) one plan's run captured in a CUDA graph and
    replayed, (b) the same run launched directly, (c) looping the single-image path (its default
    configuration); the batch's steps per launch and tile shape are picked by the library's
    autotuner unless given."""
    import torch
    tune = {}
    if not T:
        (T, tile), tune = wmc.batch_autotune(fs, lams, steps)
    b = wmc.Batch(fs, lams, steps, steps_per_launch=T, tile=tile)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        b.run(iters)
    torch.cuda.current_stream(dev).wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run(iters)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(fn, k):
        barrier()
        return max_over_ranks(min(event_ms(fn, 1) for _ in range(k)), world, dev)

    graph.replay()
    t_graph = timed(graph.replay, max(1, reps))
    t_direct = timed(lambda: b.run(iters), max(1, min(reps, 3)))
    b.check_status()
    outs = [torch.empty_like(f) for f in fs]
    ws = torch.empty(max([wmc.load().wmc_denoise_workspace_size(f.shape[0], f.shape[1], f.shape[1], 0)
                          for f in fs] or [256]), dtype=torch.uint8, device=dev)

    def loop():  # the single-image path in its default configuration
        for f, l, st, o in zip(fs, lams, steps, outs):
            wmc.denoise(f, l, st, iters, out=o, workspace=ws)

    loop()
    t_loop = timed(loop, 1)
    same = all(torch.equal(a, c) for a, c in zip(b.outs, outs))
    same = max_over_ranks(0.0 if same else 1.0, world, dev) == 0.0
    px = sum(f.numel() for f in fs) * world  # the ranks' shares are balanced within 1 %
    return {"steps_per_launch": T, "tile": tile,
            "autotune_ms_per_iter": {f"T{k[0]}_tile{k[1]}": v for k, v in tune.items()},
            "batched_graph": px * iters / (t_graph * 1e-3) / 1e9,
            "batched_direct": px * iters / (t_direct * 1e-3) / 1e9,
            "single_image_loop": px * iters / (t_loop * 1e-3) / 1e9,
            "ms": {"graph": t_graph, "direct": t_direct, "loop": t_loop},
            "batched_equals_loop_bitwise": same}


def batch_inputs(dev, n=512, mine=None):
    """The 512-image batch: sides uniform in [64, 1536] (seed 999), image i seed 1000+i, 8 bumps +
    4 shapes, sigma_i ~ U[0.01, 0.15], lambda_i ~ U[0.5, 2] (seed 998), step_i = 0.5/(1+lambda_i)."""
    import torch
    from paper_1903_07189_gb300 import synth
    sizes = synth.batch_sizes(n)
    params = synth.batch_params(n)
    mine = list(range(n)) if mine is None else mine
    fs = [torch.from_numpy(synth.make_image(sizes[i][0], sizes[i][1], seed=1000 + i, n_bumps=8,
                                            n_shapes=4, sigma=params[i][0])).to(dev) for i in mine]
    lams = [params[i][1] for i in mine]
    return fs, lams, [0.5 / (1 + l) for l in lams], sizes


def measure_diff(wmc, dev, reps=5):
    """32 images of 512 x 512 (seed 2000+i, 8 bumps + 4 shapes, sigma 0.05), K = 50 unrolled steps
    (step 0.25), checkpoints every 7, loss MSE(U^K, clean), one learnable lambda per image:
    forward, backward and forward + backward pixel-steps/s (n h w K per call) and the extra
    device memory the call holds."""
    import torch
    from paper_1903_07189_gb300 import synth
    n, h, w, K, c, step = 32, 512, 512, 50, 7, 0.25
    pairs = [synth.make_image(h, w, seed=2000 + i, n_bumps=8, n_shapes=4, sigma=0.05, return_clean=True)
             for i in range(n)]
    f = torch.from_numpy(np.stack([p[0] for p in pairs]).astype(np.float32)).to(dev)
    clean = torch.from_numpy(np.stack([p[1] for p in pairs]).astype(np.float32)).to(dev)
    lam = torch.full((n,), 1.0, device=dev, requires_grad=True)

    def fwd_bwd():
        u = wmc.unrolled_denoise(f, lam, step, K, ckpt_every=c)
        loss = ((u - clean) ** 2).mean()
        lam.grad = None
        loss.backward()
        return loss

    for _ in range(3):
        fwd_bwd()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.reset_peak_memory_stats(dev)
    base_mem = torch.cuda.memory_allocated(dev)
    for a, m, e in ev:
        a.record()
        u = wmc.unrolled_denoise(f, lam, step, K, ckpt_every=c)
        loss = ((u - clean) ** 2).mean()
        m.record()
        lam.grad = None
        loss.backward()
        e.record()
    torch.cuda.synchronize()
    peak = torch.cuda.max_memory_allocated(dev) - base_mem
    t_f = min(a.elapsed_time(m) for a, m, _ in ev)
    t_b = min(m.elapsed_time(e) for _, m, e in ev)
    t_fb = min(a.elapsed_time(e) for a, _, e in ev)
    units = n * h * w * K
    return {"fwd_bwd": units / (t_fb * 1e-3) / 1e9, "fwd": units / (t_f * 1e-3) / 1e9,
            "bwd": units / (t_b * 1e-3) / 1e9, "unit": "Gpix-step/s", "ms": {"fwd": t_f, "bwd": t_b, "fwd_bwd": t_fb},
            "peak_extra_mib": peak / 2**20, "no_checkpoint_mib": n * h * w * 4 * (K + 1) / 2**20,
            "workload": "32 x 512^2 f32, K = 50, step 0.25, checkpoints every 7, loss MSE(U^K, clean)"}, (f, clean, lam, fwd_bwd)


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1903_07189_gb300 import synth, wmc
    wmc.load()

    u_host = synth.make_image(H, W, seed=replica_seed(rank), n_bumps=64, n_shapes=32, sigma=SIGMA)
    f = torch.from_numpy(u_host).to(dev)
    hw = torch.empty_like(f)
    out = torch.empty_like(f)
    lib = wmc.load()
    ws = torch.empty(lib.wmc_denoise_workspace_size(H, W, W, 0), dtype=torch.uint8, device=dev)
    ews = torch.empty(lib.wmc_energy_workspace_size(H, W), dtype=torch.uint8, device=dev)
    energies = torch.empty(3, dtype=torch.float64, device=dev)
    flush = L2Flush(dev)
    iters = args.iters
    T = args.steps_per_launch or DEFAULT_T
    n_launch = math.ceil(iters / T)
    peak_fma = fma_peak(wmc, dev)

    def step():
        v0.record()
        wmc.eval(f, out=hw)
        v1.record()
        e0.record()
        wmc.denoise(f, LAM, STEP, iters, out=out, steps_per_launch=T, workspace=ws)
        e1.record()
        wmc.energy(out, f, None, out=energies, workspace=ews)
        n1.record()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n1 = torch.cuda.Event(enable_timing=True)
    for _ in range(max(args.warmup, 3)):
        flush()
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    d0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    d1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    nv1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with Clocks(local) as clk:
        barrier()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush()
            e0, e1, v0, v1, n1 = d0[k], d1[k], ev0[k], ev1[k], nv1[k]
            starts[k].record()
            step()
            ends[k].record()
        barrier()
        wall = time.perf_counter() - wall0
    clocks = clk.summary()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    den_ms = [a.elapsed_time(b) for a, b in zip(d0, d1)]
    eval_ms = statistics.median(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    energy_ms = statistics.median(a.elapsed_time(b) for a, b in zip(d1, nv1))
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(H * W * iters * args.steps, world, total_ms)

    # dominant kernel: the flow kernel, n_launch launches per denoise call (T steps each)
    launch_ms = statistics.mean(den_ms) / n_launch
    peak, peak_kind = peaks()
    hbm_achieved = BYTES_PER_PX_LAUNCH * H * W / (launch_ms * 1e-3) / 1e9
    fp32_achieved = FMA_OPS_PER_PX_ITER * H * W * T / (launch_ms * 1e-3) / 1e12
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    nominal_fma = peak_fma["sms"] * 128 * sm_mhz * 1e6 / 1e12
    if T > 1:
        full = T == DEFAULT_T and iters == ITERS
        roofline = {"bound": "alu", "achieved": fp32_achieved, "peak": peak_fma["tops"], "unit": "TFLOP/s",
                    "frac": fp32_achieved / peak_fma["tops"],
                    "traffic": TILE_T4_DRAM_BYTES if full else None,
                    "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one warm-L2 4-step "
                                      "launch on this image (profiles/flow_tile_t4_4096x4096_full.md)"
                                      if full and TILE_T4_DRAM_BYTES else "not captured for this configuration",
                    "kernel": f"wmc::tile_flow_kernel<T={T}> (flow, {T} Jacobi steps per launch, 128 x 64 regions)",
                    "peak_kind": "measured: FP32 FMA pipe lane-operations per second (an FMA counts once), " + peak_fma["how"],
                    "peak_nominal": {"value": nominal_fma, "how": f"{peak_fma['sms']} SMs (queried) x 128 lanes x "
                                                                   f"{sm_mhz:.0f} MHz (sampled)",
                                     "frac": fp32_achieved / nominal_fma},
                    "algorithmic_ops_per_px_iter": FMA_OPS_PER_PX_ITER,
                    "executed_ops_per_px_iter": FMA_OPS_EXECUTED_PER_PX_ITER,
                    "executed_frac": fp32_achieved * FMA_OPS_EXECUTED_PER_PX_ITER / FMA_OPS_PER_PX_ITER / peak_fma["tops"],
                    "launch_ms": launch_ms,
                    # the same iterations unblocked would move 12 B per pixel-iteration
                    "unblocked_equivalent": {"gbs": value * BYTES_PER_PX_LAUNCH,
                                             "frac": value * BYTES_PER_PX_LAUNCH / peak,
                                             "frac_of_nominal": value * BYTES_PER_PX_LAUNCH / NOMINAL_HBM_GBS},
                    "hbm": {"achieved": hbm_achieved, "peak": peak, "unit": "GB/s", "frac": hbm_achieved / peak,
                            "peak_kind": peak_kind, "frac_of_nominal": hbm_achieved / NOMINAL_HBM_GBS}}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": peak, "unit": "GB/s",
                    "frac": hbm_achieved / peak, "traffic": None, "kernel": "wmc::stream4_kernel (flow step)",
                    "peak_kind": peak_kind, "launch_ms": launch_ms}

    e2e = None
    if not args.no_e2e:
        fh = torch.from_numpy(u_host).pin_memory()
        oh = torch.empty_like(fh).pin_memory()
        hws = torch.empty(wmc.denoise_host_workspace_size(H, W), dtype=torch.uint8, device=dev)
        st = torch.cuda.current_stream(dev)
        for _ in range(2):
            wmc.denoise_host(fh, LAM, STEP, iters, out=oh, workspace=hws, device=dev)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ne = max(1, min(args.steps, 10))
        for _ in range(ne):
            wmc.denoise_host(fh, LAM, STEP, iters, out=oh, workspace=hws, device=dev)
            st.synchronize()
        barrier()
        dt = max_over_ranks((time.perf_counter() - t0) / ne, world, dev)
        e2e = {"value": job_rate(H * W * iters, world, dt * 1e3), "unit": UNIT, "h2d_bytes_per_step": H * W * 4,
               "d2h_bytes_per_step": H * W * 4, "call": "wmc_denoise_host (pinned host f in, U out)"}

    secondary = None
    if rank == 0 and world == 1 and not args.no_secondary:
        secondary = {}
        u2 = synth.make_image(H, W, seed=2, n_bumps=64, n_shapes=32, sigma=0.1)
        secondary["scale_sigma_0p1"] = {"image": f"{H}x{W}, 64 bumps + 32 shapes, sigma 0.1, seed 2",
                                        **measure_scale_image(wmc, dev, u2, iters, T, 3, flush)}
        secondary["pr1"] = measure_pr1(wmc, dev)
        del flush
        torch.cuda.empty_cache()
        prec_img = synth.make_image(16384, 16384, seed=3, n_bumps=64, n_shapes=32, sigma=0.05)
        rates, outs = measure_precision_rates(wmc, dev, prec_img, 200, T)
        del outs, prec_img
        torch.cuda.empty_cache()
        secondary["precision_16384"] = {"iters": 200, **{k: v["gpix_iter_s"] for k, v in rates.items()},
                                        "unit": UNIT, "note": "FP32 arithmetic; every step rounded to the storage type"}
        fs, lams, steps_b, _ = batch_inputs(dev)
        bres = measure_batch(wmc, dev, fs, lams, steps_b, 300, 3)
        secondary["batch_512"] = {k: bres[k] for k in ("batched_graph", "single_image_loop", "steps_per_launch", "tile",
                                                         "batched_equals_loop_bitwise")}
        secondary["batch_512"]["vs_single_image_headline"] = bres["batched_graph"] / value
        del fs, bres
        torch.cuda.empty_cache()
        dres, _ = measure_diff(wmc, dev)
        secondary["diff_32x512"] = {k: dres[k] for k in ("fwd_bwd", "fwd", "bwd", "unit", "peak_extra_mib")}
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = host_threads()
        rate, dt = cpu_oracle_rate(u_host, 2048, 32, threads)
        rate1, dt1 = cpu_oracle_rate(u_host, 512, 32, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": f"512x512 top-left crop, 32 iterations ({dt1:.1f} s)"},
               "sample": f"2048x2048 top-left crop, 32 iterations (FP64 oracle, {threads} threads, {dt:.1f} s wall, "
                         f"{dt * threads:.0f} core-s)"}
        # the step's FP64 energies (of U^iters and f, whole image) against the oracle's on the same U
        cpu["energy_parity"] = energy_parity(wmc, f, out, ws, ews, iters, T, u_host)
        # the same crop and iterations on the GPU, in the bench's launch configuration, against it
        g32 = wmc.denoise(f, LAM, STEP, 32, out=out, steps_per_launch=T, workspace=ws)
        cpu["parity"] = oracle_parity(u_host, g32[:2048, :2048].double().cpu().numpy(), 2048, 32, threads)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "l2": L2_NOTE,
                           "steps_per_launch": T, "iters": iters, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "eval": {"ms": eval_ms, "gpix_s": H * W / (eval_ms * 1e-3) / 1e9,
                         "hbm_gbs": 8 * H * W / (eval_ms * 1e-3) / 1e9,
                         "hbm_frac": 8 * H * W / (eval_ms * 1e-3) / 1e9 / peak,
                         "hbm_frac_of_nominal": 8 * H * W / (eval_ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS,
                         "kernel": "wmc::eval_tma_kernel (persistent, double-buffered TMA windows), 8 B per pixel",
                         "paper_context": PAPER_EVAL_CONTEXT},
                # U was written by the last flow launch, so part of it is still in L2
                "energy": {"ms": energy_ms, "hbm_gbs": 8 * H * W / (energy_ms * 1e-3) / 1e9,
                           "hbm_frac": 8 * H * W / (energy_ms * 1e-3) / 1e9 / peak,
                           "kernel": "wmc::energy_tma_kernel (FP64 energies of U and f; persistent, TMA windows), 8 B per pixel"},
                "secondary": secondary,
                "gpu_launches": args.steps * (2 + n_launch), "clocks": clocks,
                "wall_s_timed_region": wall}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_pr1(args):
    import torch
    from paper_1903_07189_gb300 import wmc
    dev = torch.device("cuda", 0)
    res = measure_pr1(wmc, dev, reps=max(10, args.steps))
    print(json.dumps({"workload": "pr1", "metric": METRIC, "unit": UNIT, "results": res}), flush=True)
    return 0


def run_precision(args):
    """16384 x 16384 image (64 bumps, 32 shapes, sigma 0.05, seed 3) stored as FP32, BF16 and FP16,
    200 iterations each: throughput per storage type, the single-pass kernels at this size, and a
    CPU-baseline leg that times the FP64 oracle on the top-left 2248 x 2248 crop (200 px of light
    cone) and, from that run, gives each result's error on the 2048 x 2048 crop."""
    import torch
    from paper_1903_07189_gb300 import synth, wmc
    dev = torch.device("cuda", 0)
    n, iters, crop, margin = 16384, 200, 2048, 200
    T = args.steps_per_launch or DEFAULT_T
    img = synth.make_image(n, n, seed=3, n_bumps=64, n_shapes=32, sigma=0.05)
    rates, outs = measure_precision_rates(wmc, dev, img, iters, T, reps=max(1, min(args.steps, 3)))
    got = {k: o[:crop, :crop].float().cpu().numpy().astype(np.float64) for k, o in outs.items()}
    # the single-pass kernels at this size: one evaluation (8 B per pixel) and one-step launches
    # (12 B per pixel-iteration), against the measured copy bandwidth
    peak, _ = peaks()
    f = torch.from_numpy(img).to(dev)
    hw, out = torch.empty_like(f), torch.empty_like(f)
    ws = torch.empty(wmc.load().wmc_denoise_workspace_size(n, n, n, 0), dtype=torch.uint8, device=dev)
    te = min(event_ms(lambda: wmc.eval(f, out=hw), 1) for _ in range(5))
    t1 = min(event_ms(lambda: wmc.denoise(f, LAM, STEP, 10, out=out, steps_per_launch=1, workspace=ws), 1)
             for _ in range(3)) / 10
    single = {"eval_ms": te, "eval_hbm_frac": 8 * n * n / (te * 1e-3) / 1e9 / peak,
              "step_ms": t1, "step_hbm_frac": 12 * n * n / (t1 * 1e-3) / 1e9 / peak,
              "kernel": {"eval": "wmc::eval_tma_kernel (persistent, double-buffered TMA windows)",
                         "step": "wmc::stream4_kernel (4 cells per lane)"}}
    del f, hw, out, ws, outs
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        threads = host_threads()
        oracle.set_threads(threads)
        sub = img[:crop + margin, :crop + margin].astype(np.float64)
        t0 = time.perf_counter()
        ref = oracle.denoise(sub, LAM, STEP, iters)[:crop, :crop]
        oracle_s = time.perf_counter() - t0
        errs = {}
        for name in ("f32", "bf16", "f16"):
            err = np.abs(got[name] - ref)
            mse = float((err ** 2).mean())
            e = {"max_abs_err_vs_fp64": float(err.max()),
                 "psnr_vs_fp64_db": 10 * np.log10(1.0 / mse) if mse > 0 else float("inf")}
            if name != "f32":
                emu = oracle.denoise(sub, LAM, STEP, iters, storage=name)[:crop, :crop]
                e2 = np.abs(got[name] - emu)
                e["max_abs_err_vs_emulated_storage"] = float(e2.max())
                e["frac_beyond_1ulp_vs_emulated"] = float(
                    (e2 > np.abs(emu) * (2.0 ** -7 if name == "bf16" else 2.0 ** -10)).mean())
            errs[name] = e
        px = (crop + margin) ** 2 * iters
        cpu = {"value": px / oracle_s / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"top-left {crop + margin}x{crop + margin} crop, {iters} iterations (FP64, {oracle_s:.1f} s)",
               "errors_on_top_left_2048": errs}
    line = {"workload": "precision", "metric": METRIC, "unit": UNIT, "config": {
        "image": f"{n}x{n} synthetic (64 bumps + 32 shapes, sigma 0.05, seed 3)", "iters": iters,
        "lambda": LAM, "step": STEP, "boundary": "replicate", "steps_per_launch": T,
        "arithmetic": "FP32 for every storage type; every step rounds to the storage type"},
        "results": rates, "single_pass_f32": single, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """512 images, sides uniform in [64, 1536] (seeded), image i: seed 1000+i, 8 bumps + 4 shapes,
    sigma_i ~ U[0.01, 0.15], lambda_i ~ U[0.5, 2], step_i = 0.5/(1+lambda_i); 300 iterations.
    Aggregate pixel-iterations/s of (a) one batch plan run captured in a CUDA graph and replayed,
    (b) the same run launched directly, (c) looping the single-image path over the images.
    Under torchrun the images are partitioned over the ranks by pixel count (wmc.shard_lpt; no
    communication on the data path) and each rate is all ranks' pixel-iterations over the
    slowest rank's time (strong scaling: the batch is fixed)."""
    import torch
    from paper_1903_07189_gb300 import synth, wmc
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n, iters = 512, 300
    sizes = synth.batch_sizes(n)
    costs = [h * w for h, w in sizes]
    owner, loads = wmc.shard_lpt(costs, world)
    mine = [i for i in range(n) if owner[i] == rank]
    fs, lams, steps, _ = batch_inputs(dev, n, mine)
    res = measure_batch(wmc, dev, fs, lams, steps, iters, max(1, min(args.steps, 5)), world,
                        T=args.steps_per_launch, tile=0)
    if rank == 0:
        line = {"workload": "batch", "metric": METRIC, "unit": UNIT, "n_gpus": world,
                "scaling": "strong", "config": {
                    "images": n, "pixels": sum(costs), "sides": "uniform [64, 1536] (seed 999)", "iters": iters,
                    "sigma": "U[0.01, 0.15]", "lambda": "U[0.5, 2]", "step": "0.5/(1+lambda)", "dtype": "f32",
                    "shard": {"rule": "longest first to the least-loaded rank, by pixel count",
                              "pixels_per_rank": loads}},
                "results": res}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_l1(args):
    """L1-fidelity primal-dual iteration (Sec. V-C, A = I) on the 4096^2 workload image: lambda 50,
    step 0.01, alpha 0.05 (step/alpha inside the stable range of the (U, d) update), 200
    iterations, one streaming launch per iteration.  Algorithmic bytes per pixel-iteration: read
    U, f, d and write U, d (20 B in FP32)."""
    import torch
    from paper_1903_07189_gb300 import synth, wmc
    dev = torch.device("cuda", 0)
    iters = 200 if args.iters == ITERS else args.iters
    lam, step, alpha = 50.0, 0.01, 0.05
    f_np, clean_np = synth.scale_image(SIGMA, return_clean=True)
    f = torch.from_numpy(f_np).to(dev)
    clean = torch.from_numpy(clean_np).to(dev)
    out = torch.empty_like(f)
    d = torch.empty_like(f)
    ws = torch.empty(wmc.load().wmc_denoise_l1_workspace_size(H, W, W), dtype=torch.uint8, device=dev)
    flush = L2Flush(dev)

    def run():
        d.zero_()
        wmc.denoise_l1(f, lam, step, alpha, iters, d=d, out=out, workspace=ws)

    for _ in range(max(3, args.warmup)):
        run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(3, min(args.steps, 10))):
        flush()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        e.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(e))
    ms = statistics.median(ts)
    launch_ms = ms / iters
    peak, peak_kind = peaks()
    gbs = 20 * H * W / (launch_ms * 1e-3) / 1e9
    en = wmc.energy(out, None, clean).cpu()
    line = {"workload": "l1", "metric": METRIC, "unit": UNIT, "config": {
                "image": WORKLOAD.split(":")[0], "iters": iters, "lambda": lam, "step": step,
                "alpha": alpha, "dtype": "f32", "l2": L2_NOTE},
            "results": {"value": H * W * iters / (ms * 1e-3) / 1e9, "ms": ms,
                        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                     "frac": gbs / peak, "peak_kind": peak_kind,
                                     "bytes_per_px_iter": 20, "launch_ms": launch_ms},
                        "psnr_vs_clean_db": wmc.psnr(float(en[2]), H * W),
                        "psnr_input_db": wmc.psnr(float(((f.double() - clean.double()) ** 2).sum()), H * W)}}
    print(json.dumps(line), flush=True)
    return 0


def run_fd(args):
    """The conventional finite-difference WMC of Eq. rhs (the comparator of Sec. V-D) on the
    4096^2 workload image: one evaluation pass (8 B per pixel) and 100 denoising iterations with
    lambda 1, step 0.1 (one streaming launch each, 12 B per pixel-iteration)."""
    import torch
    from paper_1903_07189_gb300 import synth, wmc
    dev = torch.device("cuda", 0)
    iters = 100 if args.iters == ITERS else args.iters
    f = torch.from_numpy(synth.scale_image(SIGMA)).to(dev)
    hw, out = torch.empty_like(f), torch.empty_like(f)
    ws = torch.empty(wmc.load().wmc_denoise_workspace_size(H, W, W, 0), dtype=torch.uint8, device=dev)
    flush = L2Flush(dev)
    for _ in range(max(3, args.warmup)):
        wmc.eval_fd(f, out=hw)
        wmc.denoise_fd(f, 1.0, 0.1, iters, out=out, workspace=ws)
    torch.cuda.synchronize()
    te, tf = [], []
    for _ in range(max(3, min(args.steps, 10))):
        flush()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        wmc.eval_fd(f, out=hw)
        b.record()
        wmc.denoise_fd(f, 1.0, 0.1, iters, out=out, workspace=ws)
        c.record()
        torch.cuda.synchronize()
        te.append(a.elapsed_time(b))
        tf.append(b.elapsed_time(c))
    peak, peak_kind = peaks()
    me, mf = statistics.median(te), statistics.median(tf)
    line = {"workload": "fd", "metric": METRIC, "unit": UNIT, "config": {
                "image": WORKLOAD.split(":")[0], "iters": iters, "lambda": 1.0, "step": 0.1, "dtype": "f32",
                "l2": L2_NOTE},
            "results": {"eval_gpix_s": H * W / (me * 1e-3) / 1e9, "eval_ms": me,
                        "eval_hbm_frac": 8 * H * W / (me * 1e-3) / 1e9 / peak,
                        "flow_gpix_iter_s": H * W * iters / (mf * 1e-3) / 1e9, "flow_ms": mf,
                        "flow_hbm_frac": 12 * H * W * iters / (mf * 1e-3) / 1e9 / peak,
                        "peak_gbs": peak, "peak_kind": peak_kind}}
    print(json.dumps(line), flush=True)
    return 0


def run_diff(args):
    """Training through the unrolled flow (measure_diff), plus the loss over a few Adam steps on
    the 32 lambdas (it must go down)."""
    import torch
    from paper_1903_07189_gb300 import wmc
    dev = torch.device("cuda", 0)
    res, (f, clean, lam, fwd_bwd) = measure_diff(wmc, dev, reps=max(3, min(args.steps, 20)))
    opt = torch.optim.Adam([lam], lr=0.1)
    losses = []
    for _ in range(5):
        opt.zero_grad()
        losses.append(float(fwd_bwd()))
        opt.step()
    res.update({"adam_losses": losses, "lambda_mean_after": float(lam.mean())})
    line = {"workload": "diff", "metric": "gigapixel-steps/s of unrolled denoising, forward + backward",
            "unit": "Gpix-step/s", "config": {"lambda_init": 1.0, "dtype": "f32",
                                              "inputs": "synthetic, seed 2000+i, 8 bumps + 4 shapes, sigma 0.05"},
            "results": res}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "pr1":
        return run_pr1(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "diff":
        return run_diff(args)
    if args.workload == "l1":
        return run_l1(args)
    if args.workload == "fd":
        return run_fd(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
