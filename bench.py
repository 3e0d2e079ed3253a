#!/usr/bin/env python3
"""Benchmark: WMC denoising throughput on GB300 (gigapixel-iterations per second).

One step = the whole hot path on one 4096 x 4096 FP32 synthetic image (64 bumps, 32 shapes,
sigma 0.02, seed 1): one H^w evaluation pass (wmc_eval), 500 Jacobi iterations of the
L2-denoising flow (wmc_denoise: lambda 1, step 0.25, replicate boundary) and the FP64
energies (wmc_energy).  value = H*W*500 / step time (the evaluation pass and the energies
are inside the timed step but not counted as work).  L2 is flushed before every timed step,
outside the events (a 256 MiB write, then a 256 MiB read of another buffer, which leaves L2 clean).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

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
# FP32 operations on the FMA pipe per output pixel-iteration of the stencil + update as the
# kernels compute it (L and the four odd parts: 20, |L|-|a_j|: 4, sign guard: 1, update: 2);
# compare/select/sign logic (7 more) runs on the separate ALU pipe and is not counted.
FMA_OPS_PER_PX_ITER = 27
SMS, FP32_LANES_PER_SM = 152, 128
DEFAULT_T = 4
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one 4-step tile-kernel launch on
# this image, from an ncu capture of a warm-L2 launch (67.15 MB read + 20.98 MB written); valid
# for the default 4 steps per launch only.
TILE_T4_DRAM_BYTES = 88.13e6
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
    ap.add_argument("--workload", default="scale", choices=["scale", "precision", "batch", "diff", "l1", "fd"],
                    help="scale: the headline 4096^2 run; precision / batch / diff: the reduced-"
                         "storage, uneven-batch and reverse-mode measurements (one JSON line "
                         "each, not the headline)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp32_peak = SMS * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12  # TFLOP-lane-ops/s on the FMA pipe
    fp32_achieved = FMA_OPS_PER_PX_ITER * H * W * T / (launch_ms * 1e-3) / 1e12
    if T > 1:
        roofline = {"bound": "alu", "achieved": fp32_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": fp32_achieved / fp32_peak,
                    "traffic": TILE_T4_DRAM_BYTES if (T == 4 and iters == ITERS) else None,
                    "kernel": f"wmc::tile_flow_kernel<T={T}> (flow, {T} Jacobi steps per launch, 128 x 64 regions)",
                    "peak_kind": f"FP32 FMA pipe lane-operations (an FMA counts once): {SMS} SMs x {FP32_LANES_PER_SM} lanes x {sm_mhz:.0f} MHz "
                                 "(unit counts and the sampled clock)",
                    "algorithmic_ops_per_px_iter": FMA_OPS_PER_PX_ITER, "launch_ms": launch_ms,
                    # the same iterations unblocked would move 12 B per pixel-iteration
                    "unblocked_equivalent": {"gbs": value * BYTES_PER_PX_LAUNCH,
                                             "frac": value * BYTES_PER_PX_LAUNCH / peak,
                                             "frac_of_nominal": value * BYTES_PER_PX_LAUNCH / NOMINAL_HBM_GBS},
                    "hbm": {"achieved": hbm_achieved, "peak": peak, "unit": "GB/s", "frac": hbm_achieved / peak,
                            "peak_kind": peak_kind, "frac_of_nominal": hbm_achieved / NOMINAL_HBM_GBS}}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": peak, "unit": "GB/s",
                    "frac": hbm_achieved / peak, "traffic": None, "kernel": "wmc::stream_kernel (flow step)",
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
        ne = max(1, min(args.steps, 3))
        for _ in range(ne):
            wmc.denoise_host(fh, LAM, STEP, iters, out=oh, workspace=hws, device=dev)
            st.synchronize()
        barrier()
        dt = max_over_ranks((time.perf_counter() - t0) / ne, world, dev)
        e2e = {"value": job_rate(H * W * iters, world, dt * 1e3), "unit": UNIT, "h2d_bytes_per_step": H * W * 4,
               "d2h_bytes_per_step": H * W * 4, "call": "wmc_denoise_host (pinned host f in, U out)"}

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
                "gpu_launches": args.steps * (2 + n_launch), "clocks": clocks,
                "wall_s_timed_region": wall}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_precision(args):
    """16384 x 16384 image (64 bumps, 32 shapes, sigma 0.05, seed 3) stored as FP32, BF16 and FP16,
    200 iterations each; throughput per storage type and error against the FP64 oracle on the
    top-left 2048 x 2048 crop (the oracle runs on a 2248 x 2248 crop: 200 px of light cone)."""
    import torch
    import oracle
    from paper_1903_07189_gb300 import synth, wmc
    dev = torch.device("cuda", 0)
    n, iters, crop, margin = 16384, 200, 2048, 200
    img = synth.make_image(n, n, seed=3, n_bumps=64, n_shapes=32, sigma=0.05)
    oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    ref = oracle.denoise(img[:crop + margin, :crop + margin].astype(np.float64), LAM, STEP, iters)[:crop, :crop]
    oracle_s = time.perf_counter() - t0
    ref_bf = {}
    for st in ("bf16", "f16"):
        sub = img[:crop + margin, :crop + margin].astype(np.float64)
        ref_bf[st] = oracle.denoise(sub, LAM, STEP, iters, storage=st)[:crop, :crop]
    results = {}
    for name, dt in [("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float16)]:
        f = torch.from_numpy(img).to(dev).to(dt)
        out = torch.empty_like(f)
        ws = torch.empty(wmc.load().wmc_denoise_workspace_size(n, n, n, wmc.DTYPES[dt]), dtype=torch.uint8,
                         device=dev)
        T = args.steps_per_launch or DEFAULT_T
        wmc.denoise(f, LAM, STEP, iters, out=out, steps_per_launch=T, workspace=ws)
        torch.cuda.synchronize()
        times = []
        for _ in range(max(1, min(args.steps, 3))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            wmc.denoise(f, LAM, STEP, iters, out=out, steps_per_launch=T, workspace=ws)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        got = out[:crop, :crop].float().cpu().numpy().astype(np.float64)
        err = np.abs(got - ref)
        mse = float((err ** 2).mean())
        r = {"gpix_iter_s": n * n * iters / (min(times) * 1e-3) / 1e9, "ms": min(times),
             "max_abs_err_vs_fp64": float(err.max()),
             "psnr_vs_fp64_db": 10 * np.log10(1.0 / mse) if mse > 0 else float("inf")}
        if name == "f32":
            # the single-pass kernels at this size: one evaluation (8 B per pixel) and one-step
            # launches (12 B per pixel-iteration), against the measured copy bandwidth
            peak, _ = peaks()
            hw = torch.empty_like(f)

            def best(fn, reps=5):
                fn()
                ts = []
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    fn()
                    b.record()
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b))
                return min(ts)
            te = best(lambda: wmc.eval(f, out=hw))
            t1 = best(lambda: wmc.denoise(f, LAM, STEP, 10, out=out, steps_per_launch=1, workspace=ws)) / 10
            r["single_pass"] = {"eval_ms": te, "eval_hbm_frac": 8 * n * n / (te * 1e-3) / 1e9 / peak,
                                "step_ms": t1, "step_hbm_frac": 12 * n * n / (t1 * 1e-3) / 1e9 / peak,
                                "kernel": {"eval": "wmc::eval_tma_kernel (persistent, double-buffered TMA windows)",
                                           "step": "wmc::stream4_kernel (4 cells per lane)"}}
            del hw
        if name in ref_bf:
            e2 = np.abs(got - ref_bf[name])
            r["max_abs_err_vs_emulated_storage"] = float(e2.max())
            r["frac_beyond_1ulp_vs_emulated"] = float((e2 > np.abs(ref_bf[name]) * (2.0 ** -7 if name == "bf16" else 2.0 ** -10)).mean())
        results[name] = r
        del f, out, ws
        torch.cuda.empty_cache()
    line = {"workload": "precision", "metric": METRIC, "unit": UNIT, "config": {
        "image": f"{n}x{n} synthetic (64 bumps + 32 shapes, sigma 0.05, seed 3)", "iters": iters,
        "lambda": LAM, "step": STEP, "boundary": "replicate",
        "error_crop": f"top-left {crop}x{crop} (oracle on {crop + margin}x{crop + margin}, FP64, "
                      f"{oracle.get_threads()} threads, {oracle_s:.1f} s)",
        "arithmetic": "FP32 for every storage type; every step rounds to the storage type"},
        "results": results}
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
    params = synth.batch_params(n)
    costs = [h * w for h, w in sizes]
    owner, loads = wmc.shard_lpt(costs, world)
    mine = [i for i in range(n) if owner[i] == rank]
    fs = [torch.from_numpy(synth.make_image(sizes[i][0], sizes[i][1], seed=1000 + i, n_bumps=8,
                                            n_shapes=4, sigma=params[i][0])).to(dev) for i in mine]
    lams = [params[i][1] for i in mine]
    steps = [0.5 / (1 + l) for l in lams]
    px = sum(costs)
    # steps per launch and tile shape picked by the library's autotuner (times each candidate on
    # this batch)
    if args.steps_per_launch:
        (T, tile), tune = (args.steps_per_launch, 0), {}
    else:
        (T, tile), tune = wmc.batch_autotune(fs, lams, steps)
    b = wmc.Batch(fs, lams, steps, steps_per_launch=T, tile=tile)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(iters)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run(iters)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            barrier()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            e.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(e))
        return max_over_ranks(min(ts), world, dev)

    graph.replay()
    t_graph = timed(graph.replay, max(1, min(args.steps, 5)))
    t_direct = timed(lambda: b.run(iters), max(1, min(args.steps, 3)))
    b.check_status()
    outs = [torch.empty_like(f) for f in fs]
    ws = torch.empty(max([wmc.load().wmc_denoise_workspace_size(sizes[i][0], sizes[i][1], sizes[i][1], 0)
                          for i in mine] or [256]), dtype=torch.uint8, device=dev)

    def loop():
        for f, l, st, o in zip(fs, lams, steps, outs):
            wmc.denoise(f, l, st, iters, out=o, steps_per_launch=T, workspace=ws, tile=tile)

    loop()
    t_loop = timed(loop, 1)
    same = all(torch.equal(a, c) for a, c in zip(b.outs, outs))
    same = max_over_ranks(0.0 if same else 1.0, world, dev) == 0.0
    if rank == 0:
        line = {"workload": "batch", "metric": METRIC, "unit": UNIT, "n_gpus": world,
                "scaling": "strong", "config": {
                    "images": n, "pixels": px, "sides": "uniform [64, 1536] (seed 999)", "iters": iters,
                    "sigma": "U[0.01, 0.15]", "lambda": "U[0.5, 2]", "step": "0.5/(1+lambda)", "dtype": "f32",
                    "steps_per_launch": T, "tile": tile,
                    "autotune_ms_per_iter": {f"T{k[0]}_tile{k[1]}": v for k, v in tune.items()},
                    "shard": {"rule": "longest first to the least-loaded rank, by pixel count",
                              "pixels_per_rank": loads}},
                "results": {"batched_graph": px * iters / (t_graph * 1e-3) / 1e9,
                            "batched_direct": px * iters / (t_direct * 1e-3) / 1e9,
                            "single_image_loop": px * iters / (t_loop * 1e-3) / 1e9,
                            "ms": {"graph": t_graph, "direct": t_direct, "loop": t_loop},
                            "batched_equals_loop_bitwise": same}}
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
    """Training through the unrolled flow: 32 images of 512 x 512 (seed 2000+i, 8 bumps + 4
    shapes, sigma 0.05), one learnable lambda per image (init 1.0), K = 50 denoising steps with
    step 0.25, checkpoints every 7 steps, loss = mean squared error of U^K against the clean
    image.  Reports forward, backward and forward+backward pixel-steps/s (n*h*w*K per call), the
    device memory the checkpoints save, and the loss over a few gradient steps on lambda."""
    import torch
    from paper_1903_07189_gb300 import synth, wmc
    dev = torch.device("cuda", 0)
    n, h, w, K, c, step = 32, 512, 512, 50, 7, 0.25
    pairs = [synth.make_image(h, w, seed=2000 + i, n_bumps=8, n_shapes=4, sigma=0.05,
                              return_clean=True) for i in range(n)]
    f = torch.from_numpy(np.stack([p[0] for p in pairs]).astype(np.float32)).to(dev)
    clean = torch.from_numpy(np.stack([p[1] for p in pairs]).astype(np.float32)).to(dev)
    lam = torch.full((n,), 1.0, device=dev, requires_grad=True)

    def fwd_bwd():
        u = wmc.unrolled_denoise(f, lam, step, K, ckpt_every=c)
        loss = ((u - clean) ** 2).mean()
        lam.grad = None
        loss.backward()
        return loss

    for _ in range(max(3, args.warmup)):
        fwd_bwd()
    torch.cuda.synchronize()
    reps = max(3, min(args.steps, 20))
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
    # a few Adam steps on lambda: the loss must go down
    opt = torch.optim.Adam([lam], lr=0.1)
    losses = []
    for _ in range(5):
        opt.zero_grad()
        losses.append(float(fwd_bwd()))
        opt.step()
    line = {"workload": "diff", "metric": "gigapixel-steps/s of unrolled denoising, forward + backward",
            "unit": "Gpix-step/s", "config": {
                "images": n, "h": h, "w": w, "K": K, "ckpt_every": c, "step": step, "lambda_init": 1.0,
                "loss": "MSE(U^K, clean)", "dtype": "f32", "inputs": "synthetic, seed 2000+i, 8 bumps + "
                "4 shapes, sigma 0.05"},
            "results": {"fwd_bwd": units / (t_fb * 1e-3) / 1e9, "fwd": units / (t_f * 1e-3) / 1e9,
                        "bwd": units / (t_b * 1e-3) / 1e9,
                        "ms": {"fwd": t_f, "bwd": t_b, "fwd_bwd": t_fb},
                        "peak_extra_mib": peak / 2**20,
                        "no_checkpoint_mib": n * h * w * 4 * (K + 1) / 2**20,
                        "adam_losses": losses, "lambda_mean_after": float(lam.mean())}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
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
