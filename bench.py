"""Benchmark of the SPA sweep on GB300 (one JSON line on stdout).

A step is one whole SPA sweep (every row of the hot path: init, T x [reweight,
log-sum-exp/ESS, resampling, proposal scales, M x (propose, likelihood, accept),
summaries]) over one synthetic hit region, with the inputs resident in HBM. The
metric is particle-log-likelihood throughput: algorithmic multiply-adds N*n*p per
likelihood evaluation (the split-BF16 doubling is not counted) over the sweep's
T*M + 1 evaluations, divided by the sweep wall time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload hit-region|batched|...]
                  [--precision split_bf16|fp32] [--impl reference]

--impl reference times the FP64 CPU oracle (the reference arm of this build) on a
bounded sample of the same workload. Under torchrun each rank runs its own sweep
(independent replicas: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20  # larger than the 129 MB L2


def _rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def replica_seed_base(rank: int) -> int:
    """Seeds of rank r's sweeps start at 1000 (r + 1): the replicas are independent runs."""
    return 1000 * (rank + 1)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (all-reduce MAX; gloo on CPU tensors, NCCL on device ones)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(gmac_per_step: float, steps: int, world: int, total_ms: float) -> float:
    """Whole-job throughput: every rank did `steps` sweeps in at most total_ms (weak scaling)."""
    return world * gmac_per_step * steps / (total_ms / 1e3)


def workload_desc(w):
    return (f"{w['name']}: n={w['n']} p={w['p']} N={w['N']} T={w['T']} M={w['M']} "
            f"{w['move'].upper()} nu={w['nu']:g}")


def algorithmic_gmac(w):
    return w["N"] * w["n"] * w["p"] * (w["T"] * w["M"] + 1) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def code_digest(sources) -> str:
    """Hash of C++/CUDA source texts with comments and blank lines left out and each line's
    whitespace runs collapsed to one space."""
    import re

    h = hashlib.sha256()
    for src in sources:
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(" ".join(line.split()) for line in src.splitlines() if line.strip()).encode())
    return h.hexdigest()[:16]


def kernel_source_sha() -> str:
    """code_digest of the likelihood kernel's source (its file and the device header): the
    recorded DRAM counters belong to the code, so a comment edit keeps them while any code
    change drops them."""
    csrc = os.path.join(ROOT, "paper_1106_0322_gb300", "csrc")
    return code_digest(open(os.path.join(csrc, f), encoding="utf-8").read() for f in ("k_loglik_tc.cu", "spa_device.cuh"))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def profile_traffic(workload: str):
    """DRAM bytes per launch of the likelihood kernel from the committed ncu summary, if it
    was captured from the current kernel source."""
    path = os.path.join(ROOT, "profiles", "roofline_counters.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = d.get(workload)
    if not e or e.get("kernel_sha") != kernel_source_sha():
        return None
    return e.get("dram_bytes_per_launch")


def oracle_sample_shape(w, region, sched, cfg, seconds_target):
    """(particles, steps) of a bounded oracle sample of about seconds_target: calibrated on one
    step with at most 512 particles, then full N if one step fits, else fewer particles."""
    import oracle

    n0 = min(w["N"], 512)
    t0 = time.perf_counter()
    oracle.run(region.G, region.y, w["nu"], sched[:1], n0, w["M"], seed=1, cfg=cfg)
    per_particle_step = (time.perf_counter() - t0) / n0
    full_step = per_particle_step * w["N"]
    if full_step <= seconds_target:
        return w["N"], max(1, min(w["T"], int(seconds_target / max(full_step, 1e-4))))
    return max(64, int(seconds_target / max(per_particle_step, 1e-9))), 1


def oracle_gmac(w, Ns, steps):
    return Ns * w["n"] * w["p"] * (steps * w["M"] + 1) / 1e9


def cpu_oracle_sample(w, region, sched, seconds_target=15.0, seed=1):
    """Time the FP64 oracle on a bounded prefix of the sweep (init + the first steps; fewer
    particles when one step at full N would take longer than the target)."""
    import oracle

    threads = oracle.max_threads()
    cfg = oracle.make_config(move=w["move"])
    Ns, steps = oracle_sample_shape(w, region, sched, cfg, seconds_target)
    t0 = time.perf_counter()
    oracle.run(region.G, region.y, w["nu"], sched[:steps], Ns, w["M"], seed=seed, cfg=cfg)
    dt = time.perf_counter() - t0
    return {"value": oracle_gmac(w, Ns, steps) / dt, "unit": "GMAC/s", "cores": threads, "kind": "oracle",
            "sample": f"first {steps} of {w['T']} scale steps (init + {steps * w['M']} moves) of the same "
                      f"workload with {Ns} of {w['N']} particles, {dt:.1f} s on {threads} threads"}


def reference_arm(args, w):
    """--impl reference: the FP64 oracle timed on the host cores, bounded samples."""
    rank, world, _ = _rank_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1106_0322_gb300 import synth

    oracle.build()
    region = synth.workload_region(w["name"])
    sched = synth.workload_schedule(w["name"])
    cfg = oracle.make_config(move=w["move"])
    budget = 150.0 / max(1, args.steps + args.warmup)
    Ns, steps_per = oracle_sample_shape(w, region, sched, cfg, budget)
    gmac = oracle_gmac(w, Ns, steps_per)
    for k in range(args.warmup):
        oracle.run(region.G, region.y, w["nu"], sched[:steps_per], Ns, w["M"], seed=100 + k, cfg=cfg)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(region.G, region.y, w["nu"], sched[:steps_per], Ns, w["M"], seed=200 + k, cfg=cfg)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = gmac * args.steps / tot
    threads = oracle.max_threads()
    sample = (f"each step: first {steps_per} of {w['T']} scale steps (init + {steps_per * w['M']} moves) of the "
              f"workload with {Ns} of {w['N']} particles, FP64, {threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GMAC/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(w), "sample": sample, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "GMAC/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GMAC/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


METRIC = "SPA sweep particle-loglik throughput (algorithmic GMAC/s = N*n*p*(T*M+1) / sweep wall time)"
METRIC_BATCHED = ("batched SPA sweeps: particle-loglik throughput over all regions (algorithmic GMAC/s = "
                  "sum_r N n_r p_r (T M + 1) x 2 for MALA's likelihood + adjoint / batch wall time)")

BATCHED = dict(R=64, N=4096, T=100, M=5, move="mala", seed=1004)


def batched_bench(args, emit=True):
    """The batched workload: 64 uneven regions (n ~ U[1000, 5000], p ~ U[20, 500]), each its
    own MALA sweep (N = 4096, T = 100, M = 5, split-BF16), all captured into one CUDA graph
    (spa_batch) and launched once per step. Timed on the host around spa_batch_run, which
    uploads the seeds, launches the graph, copies the results back and synchronises."""
    import numpy as np
    import torch

    rank, world, _ = _rank_env()
    if emit:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__

    __graft_entry__.build()
    import paper_1106_0322_gb300 as spa
    from paper_1106_0322_gb300 import synth

    b = BATCHED
    pairs = synth.batched_regions(b["R"], seed=b["seed"])
    sched = synth.geometric_schedule(b["T"])
    cfg = spa.make_config(move=b["move"], precision=args.precision)
    regs = [spa.Region(g.G, g.y, nu, config=cfg) for g, nu in pairs]
    gmac = sum(b["N"] * g.G.shape[0] * g.G.shape[1] * (b["T"] * b["M"] + 1) * 2 for g, _ in pairs) / 1e9
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    batch = spa.Batch(regs, [sched] * b["R"], [b["N"]] * b["R"], [b["M"]] * b["R"], list(range(1, b["R"] + 1)))
    build_s = time.perf_counter() - t0
    for k in range(args.warmup):
        batch.run(seeds=[100 * k + r for r in range(b["R"])])
    sampler = ClockSampler(0)
    torch.cuda.synchronize()
    sampler.start()
    times = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = batch.run(seeds=[10000 + 100 * k + r for r in range(b["R"])])
        times.append(time.perf_counter() - t0)
    clocks = sampler.stop()
    assert all(np.all(np.isfinite(o["mean"])) for o in outs)
    ms = 1e3 * sum(times) / len(times)
    # the same regions one after another (one spa_run graph each, each waited for)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, g in enumerate(regs):
        g.run(sched, b["N"], b["M"], 7 + r)
    seq_ms = 1e3 * (time.perf_counter() - t0)
    line = {
        "metric": METRIC_BATCHED, "value": gmac / (ms / 1e3), "unit": "GMAC/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if args.precision == "split_bf16" else "f32", "data": "synthetic",
        "config": {"workload": f"batched: R={b['R']} regions, n~U[1000,5000], p~U[20,500], N={b['N']} T={b['T']} "
                               f"M={b['M']} {b['move'].upper()}, nu in {{1,2,4,16}}",
                   "precision": args.precision, "l2": "flushed (512 MB write) before each timed batch",
                   "timing": "host wall clock around spa_batch_run (graph launch + result copies + sync)"},
        "gpu_launches": batch.launch_count() * args.steps,
        "graph_build_s": build_s,
        "sequential_regions_ms": seq_ms,
        "speedup_vs_sequential": seq_ms / ms,
        "clocks": clocks,
        "roofline": {"bound": "tensor", "achieved": 2 * 1e9 * gmac / (ms / 1e3) / 1e12,
                     "peak": tensor_peak_burst()[0], "unit": "TFLOP/s",
                     "frac": 2 * 1e9 * gmac / (ms / 1e3) / 1e12 / tensor_peak_burst()[0], "traffic": None,
                     "kernel": "whole batch (all regions' likelihood and adjoint contractions over the batch time)",
                     "peak_source": tensor_peak_burst()[1]},
    }
    batch.close()
    for g in regs:
        g.close()
    if not emit:
        return line
    print(json.dumps(line), flush=True)
    return 0


def loglik_roofline(reg, w, args, stream):
    """The likelihood kernel timed alone with CUDA events (200 launches on the sweep's
    stream, in the sweep's launch configuration), against the measured BF16 peak."""
    import torch

    reps = 200
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reg.loglik_repeat(w["N"], 5, stream.cuda_stream)
    e0.record(stream)
    reg.loglik_repeat(w["N"], reps, stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    reg.sync()
    kern_ms = e0.elapsed_time(e1) / reps
    flop = 2.0 * w["N"] * w["n"] * w["p"]
    achieved = flop / (kern_ms / 1e3) / 1e12
    if args.precision == "split_bf16":
        peak, peak_src = tensor_peak_burst()
        bound = "tensor"
        kernel = "k_loglik_tc"
    else:
        peak, peak_src = fp32_simt_peak()
        bound = "alu"
        kernel = "k_eta_tile"
    cfg, src = reg.tile_config()
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": profile_traffic(args.workload) if bound == "tensor" else None,
                "kernel": kernel, "tile_bn": reg.loglik_tile_width(),
                "tile_config": cfg, "tile_source": {0: "fixed", 1: "table", 2: "timed"}.get(src),
                "launch_ms": kern_ms, "peak_source": peak_src,
                "algorithmic_flop_per_launch": flop}
    return roofline


def tensor_peak_burst():
    """The BF16 tensor peak for a kernel timed alone in a short burst of launches: the
    measured burst figure (the sustained one was taken at the power-capped clock of a
    seconds-long GEMM loop)."""
    peaks, src = measured_peaks()
    return peaks["bf16_tflops"], f"{src}: bf16 burst (kernel timed alone, 200 back-to-back launches)"


FFMA_PER_CLK_PER_SM = 128  # FP32 fused multiply-adds per clock per SM


def fp32_simt_peak():
    """Derived FP32 FFMA peak of the CUDA cores: SMs x 128 FFMA/clk x 2 FLOP x the maximum SM
    clock (the measured peaks cover copies and GEMMs only)."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peaks, _ = measured_peaks()
    mhz = peaks.get("sm_max_mhz") or 2070.0
    peak = sms * FFMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12
    return peak, f"derived: {sms} SMs x {FFMA_PER_CLK_PER_SM} FFMA/clk x 2 FLOP x {mhz:.0f} MHz"


SFU_OPS_PER_CLK_PER_SM = 16  # MUFU (ex2, lg2, rcp, ...) results per clock per SM


def site_roofline(w, ms_per_step, clocks):
    """The single-coordinate cycle is bound by the SFU: every trial update needs one ex2 per
    individual. Achieved = N M p n T ex2 / sweep time, against SMs x 16 per clock x the
    maximum SM clock (a derived peak: the measured peaks cover copies and GEMMs only)."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * SFU_OPS_PER_CLK_PER_SM * mhz * 1e6 / 1e9
    ops = w["N"] * w["M"] * w["p"] * w["n"] * w["T"]
    achieved = ops / (ms_per_step / 1e3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s (SFU ex2)", "frac": achieved / peak,
            "traffic": None, "kernel": "k_move_site",
            "peak_source": f"derived: {sms} SMs x {SFU_OPS_PER_CLK_PER_SM} SFU results/clk x {mhz:.0f} MHz",
            "algorithmic_ops_per_sweep": ops, "note": "whole-sweep rate (the cycle kernel dominates the sweep)"}


def matched_error(args):
    """Split-BF16 against plain FP32 at matched posterior-mean error on one workload.

    Gold: the mean over 16 seeds of the FP32 path at 4N. For each path and particle count
    N' in {N/4, N/2, N, 2N}: 8 seeds, the RMSE over (t, j) of each seed's posterior means
    against the gold, averaged over seeds, and the sweep's device time. The split path's
    time at the FP32 path's error at N is interpolated in log-log (error ~ N'^-1/2)."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1106_0322_gb300 as spa
    from paper_1106_0322_gb300 import synth

    w = dict(synth.WORKLOADS[args.workload])
    region = synth.workload_region(args.workload)
    sched = synth.workload_schedule(args.workload)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    T, p = w["T"], w["p"]

    def runs(precision, N, seeds):
        cfg = spa.make_config(move=w["move"], precision=precision, stream=stream.cuda_stream)
        reg = spa.Region(region.G, region.y, w["nu"], config=cfg)
        out = {"mean": torch.empty((T, p), dtype=torch.float64, device=dev)}
        means, ms = [], []
        reg.run_device(torch.tensor(sched, device=dev), N, w["M"], 1, out)  # graph + workspace
        for s in seeds:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reg.run_device(torch.tensor(sched, device=dev), N, w["M"], s, out)
            e1.record(stream)
            e1.synchronize()
            reg.sync()
            ms.append(e0.elapsed_time(e1))
            means.append(out["mean"].cpu().numpy().copy())
        reg.close()
        return np.array(means), float(np.median(ms))

    N = w["N"]
    gold_means, _ = runs("fp32", 4 * N, list(range(9000, 9016)))
    gold = gold_means.mean(axis=0)
    table = {}
    for prec in ("split_bf16", "fp32"):
        rows = []
        for f in (0.25, 0.5, 1.0, 2.0):
            Nf = int(N * f)
            m, ms = runs(prec, Nf, list(range(100, 108)))
            rmse = float(np.mean([np.sqrt(np.mean((mi - gold) ** 2)) for mi in m]))
            rows.append({"N": Nf, "rmse": rmse, "ms": ms})
        table[prec] = rows
    target = next(r for r in table["fp32"] if r["N"] == N)
    sp = table["split_bf16"]
    le = np.log([r["rmse"] for r in sp])
    lt = np.log([r["ms"] for r in sp])
    order = np.argsort(le)
    t_at = float(np.exp(np.interp(np.log(target["rmse"]), le[order], lt[order])))
    line = {"metric": "SPA sweep wall time at matched posterior-mean error (split-BF16 vs plain FP32)",
            "workload": workload_desc(dict(w, name=args.workload)),
            "gold": "mean of 16 seeds of the FP32 path at 4N",
            "fp32_at_N": target, "split_bf16_ms_at_matched_error": t_at,
            "speedup_at_matched_error": target["ms"] / t_at, "table": table}
    print(json.dumps(line), flush=True)
    return 0


def out_buffers(dev, T, p):
    """Device-resident per-scale outputs of one sweep (the spa_result arrays)."""
    import torch

    return {
        "mean": torch.empty((T, p), dtype=torch.float64, device=dev),
        "quantile": torch.empty((T, p, 3), dtype=torch.float64, device=dev),
        "conc": torch.empty((T, p, 2), dtype=torch.float64, device=dev),
        "ess": torch.empty(T, dtype=torch.float64, device=dev),
        "log_z_inc": torch.empty(T, dtype=torch.float64, device=dev),
        "accept_rate": torch.empty(T, dtype=torch.float64, device=dev),
        "resampled": torch.empty(T, dtype=torch.uint8, device=dev),
    }


def time_sweeps(reg, sched_d, w, steps, warmup, stream, flush, out_d, seed0):
    """Device time (CUDA events on the sweep's stream) of `steps` sweeps after `warmup`
    untimed ones, with L2 flushed before each timed sweep (outside the events)."""
    import torch

    for k in range(warmup):
        reg.run_device(sched_d, w["N"], w["M"], seed0 + k, out_d)
    reg.sync()
    torch.cuda.synchronize()
    times = []
    for k in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reg.run_device(sched_d, w["N"], w["M"], seed0 + warmup + k, out_d)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    reg.sync()
    return times


def grad_roofline(reg, w, stream):
    """MALA's per-move tensor-core kernels (residual likelihood pass, adjoint GEMM, gradient
    finish) timed alone with CUDA events, 100 back-to-back groups, against the burst BF16
    peak: 2 N n p multiply-adds per group (the forward contraction and the adjoint)."""
    import torch

    reps = 100
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reg.grad_repeat(w["N"], 5, stream.cuda_stream)
    e0.record(stream)
    reg.grad_repeat(w["N"], reps, stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    reg.sync()
    ms = e0.elapsed_time(e1) / reps
    flop = 2.0 * 2.0 * w["N"] * w["n"] * w["p"]
    achieved = flop / (ms / 1e3) / 1e12
    peak, src = tensor_peak_burst()
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_loglik_tc<resid> + k_adjoint_tc + k_grad_finish", "launch_ms": ms,
            "peak_source": src, "algorithmic_flop_per_launch": flop}


def workload_line(name, args, stream, flush, dev, steps=3, warmup=2):
    """A compact line for another workload (its own sweep time, throughput and roofline)."""
    import paper_1106_0322_gb300 as spa
    import torch
    from paper_1106_0322_gb300 import synth

    w = dict(synth.WORKLOADS[name], name=name)
    region = synth.workload_region(name)
    sched_d = torch.tensor(synth.workload_schedule(name), dtype=torch.float64, device=dev)
    cfg = spa.make_config(move=w["move"], precision="split_bf16", stream=stream.cuda_stream)
    reg = spa.Region(region.G, region.y, w["nu"], config=cfg)
    out_d = out_buffers(dev, w["T"], w["p"])
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    times = time_sweeps(reg, sched_d, w, steps, warmup, stream, flush, out_d, 300)
    clocks = sampler.stop()
    ms = sum(times) / len(times)
    # MALA's per-move work counts the adjoint's N n p multiply-adds as well
    mult = 2 if w["move"] == "mala" else 1
    gmac = mult * algorithmic_gmac(w)
    if w["move"] == "mala":
        roof = grad_roofline(reg, w, stream)
    else:
        roof = loglik_roofline(reg, w, argparse.Namespace(precision="split_bf16", workload=name), stream)
    line = {"workload": workload_desc(w), "precision": "split_bf16", "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "value": gmac / (ms / 1e3), "unit": "GMAC/s",
            "metric_note": "N n p (T M + 1) algorithmic multiply-adds" + (" x 2 (likelihood + adjoint)" if mult == 2
                                                                            else "") + " / sweep time",
            "roofline": roof, "gpu_launches": int(reg.last_launch_count() * steps), "clocks": clocks}
    reg.close()
    return line


def matched_error_compact(w, region, sched_d, stream, flush, dev, seeds=4, gold_seeds=8):
    """Split-BF16 against plain FP32 at matched posterior-mean error, compact: gold = the mean
    of gold_seeds FP32 sweeps at 4N; each path's error = RMSE over (t, j) of one sweep's
    posterior means against the gold, averaged over `seeds` sweeps; the split path at N/2,
    N and 2N, its sweep time interpolated (log-log) at the FP32 path's error at N."""
    import numpy as np
    import paper_1106_0322_gb300 as spa
    import torch

    T, p = w["T"], w["p"]

    def runs(precision, N, seed_list):
        cfg = spa.make_config(move=w["move"], precision=precision, stream=stream.cuda_stream)
        reg = spa.Region(region.G, region.y, w["nu"], config=cfg)
        out = out_buffers(dev, T, p)
        reg.run_device(sched_d, N, w["M"], 1, out)
        means, ms = [], []
        for s in seed_list:
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reg.run_device(sched_d, N, w["M"], s, out)
            e1.record(stream)
            e1.synchronize()
            reg.sync()
            ms.append(e0.elapsed_time(e1))
            means.append(out["mean"].cpu().numpy().copy())
        reg.close()
        return np.array(means), float(np.median(ms))

    N = w["N"]
    gold = runs("fp32", 4 * N, list(range(9000, 9000 + gold_seeds)))[0].mean(axis=0)

    def rmse(m):
        return float(np.mean([np.sqrt(np.mean((mi - gold) ** 2)) for mi in m]))

    m32, ms32 = runs("fp32", N, list(range(100, 100 + seeds)))
    e32 = rmse(m32)
    table = []
    for f in (0.5, 1.0, 2.0):
        m, ms = runs("split_bf16", int(N * f), list(range(100, 100 + seeds)))
        table.append({"N": int(N * f), "rmse": rmse(m), "ms": ms})
    le = np.log([r["rmse"] for r in table])
    lt = np.log([r["ms"] for r in table])
    order = np.argsort(le)
    t_at = float(np.exp(np.interp(np.log(e32), le[order], lt[order])))
    split_at_N = next(r for r in table if r["N"] == N)
    return {"gold": f"mean of {gold_seeds} FP32 sweeps at 4N", "seeds": seeds,
            "fp32": {"N": N, "rmse": e32, "ms": ms32}, "split_bf16_at_N": split_at_N, "split_bf16_table": table,
            "split_bf16_ms_at_fp32_error": t_at, "speedup_at_matched_error": ms32 / t_at,
            "note": "errors flatten at the gold's own Monte Carlo error above N = 4096"}


def batched_line(args, stream, dev, warmup=1, steps=2):
    """The batched workload, compact (see batched_bench): one spa_batch of 64 regions."""
    ns = argparse.Namespace(precision="split_bf16", warmup=warmup, steps=steps)
    return batched_bench(ns, emit=False)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="hit-region")
    ap.add_argument("--precision", default="split_bf16", choices=["split_bf16", "fp32"])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ess-frac", type=float, default=0.75,
                    help="resample when ESS < ess_frac * N (1.0 resamples at every step; for profiling the resampling kernels)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the compact split-large / mala / batched / matched-error keys of the default line")
    ap.add_argument("--matched-error", action="store_true",
                    help="split-BF16 vs plain FP32 wall time at matched posterior-mean error (one JSON line)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3

    from paper_1106_0322_gb300 import synth

    if args.matched_error:
        return matched_error(args)
    if args.workload == "batched":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no reference-arm sample; "
                                                                  "run the reference arm on hit-region"}))
            return 0
        return batched_bench(args)
    w = dict(synth.WORKLOADS[args.workload])
    w["name"] = args.workload
    if args.impl == "reference":
        return reference_arm(args, w)

    import numpy as np
    import torch

    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__

    __graft_entry__.build()
    import paper_1106_0322_gb300 as spa

    region = synth.workload_region(args.workload)
    sched_h = synth.workload_schedule(args.workload)
    sched_d = torch.tensor(sched_h, dtype=torch.float64, device=dev)
    # A dedicated stream: the library runs on it and the events are recorded on it (the
    # legacy default stream has handle 0, which the library reads as "its own stream").
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    assert stream.cuda_stream != 0
    init = dict(init="resample_move", burn_in_steps=w["burn_in"]) if w.get("burn_in") else {}
    cfg = spa.make_config(move=w["move"], precision=args.precision, stream=stream.cuda_stream,
                          ess_frac=args.ess_frac, **init)
    reg = spa.Region(region.G, region.y, w["nu"], config=cfg)
    T, p = w["T"], w["p"]
    out_d = out_buffers(dev, T, p)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    seed_base = replica_seed_base(rank)

    def one_sweep(k):
        reg.run_device(sched_d, w["N"], w["M"], seed_base + k, out_d)

    for k in range(args.warmup):
        one_sweep(k)
    reg.sync()
    torch.cuda.synchronize()

    # ---------------------------------------------------------------- timed region
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    total_ms = 0.0
    for k in range(args.steps):
        flush.zero_()  # L2 flushed between timed sweeps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if k == 0:  # marks the first timed sweep for kernel profilers (ncu --nvtx-include)
            torch.cuda.nvtx.range_push("spa_timed_sweep")
        e0.record(stream)
        one_sweep(args.warmup + k)
        e1.record(stream)
        if k == 0:
            torch.cuda.nvtx.range_pop()
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    reg.sync()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    launches = reg.last_launch_count() * args.steps
    total_ms = max_over_ranks(total_ms, world, dev)
    ms_per_step = total_ms / args.steps
    gmac = algorithmic_gmac(w)
    value = whole_job_value(gmac, args.steps, world, total_ms)
    assert np.all(np.isfinite(out_d["mean"].cpu().numpy()))

    # ----------------------------------- dominant kernel: the likelihood GEMM + epilogue
    if w["move"] == "site":
        roofline = site_roofline(w, ms_per_step, clocks)
    elif w["move"] == "mala" and args.precision == "split_bf16":
        roofline = grad_roofline(reg, w, stream)
    else:
        roofline = loglik_roofline(reg, w, args, stream)

    # --------------------------------- plain FP32 comparator sweep on the same workload
    # (the same K timed sweeps and warm-up rule as the split path, with its own clock record)
    plain = None
    if args.precision == "split_bf16" and rank == 0 and w["move"] != "site":
        reg32 = spa.Region(region.G, region.y, w["nu"],
                           config=spa.make_config(move=w["move"], precision="fp32", stream=stream.cuda_stream, **init))
        s32 = ClockSampler(torch.cuda.current_device())
        s32.start()
        t32 = time_sweeps(reg32, sched_d, w, args.steps, args.warmup, stream, flush, out_d, 7000)
        c32 = s32.stop()
        pms = sum(t32) / len(t32)
        plain = {"ms_per_step": pms, "steps": args.steps, "warmup": args.warmup, "value": gmac / (pms / 1e3),
                 "unit": "GMAC/s", "speedup_of_split_bf16": pms / ms_per_step, "clocks": c32,
                 "roofline": loglik_roofline(reg32, w, argparse.Namespace(precision="fp32", workload=args.workload),
                                             stream)}
        reg32.close()

    # ---------------- the other configurations of the chosen form, compact (rank 0, N = 1)
    extras = None
    if rank == 0 and world == 1 and not args.no_extras and args.precision == "split_bf16" and \
            args.workload == "hit-region":
        extras = {"split-large": workload_line("split-large", args, stream, flush, dev),
                  "mala": workload_line("mala", args, stream, flush, dev),
                  "batched": batched_line(args, stream, dev)}
        extras["matched_error"] = matched_error_compact(w, region, sched_d, stream, flush, dev)
        torch.cuda.set_stream(stream)

    # ------------------------------------------ end to end through the C ABI, host buffers
    e2e = None
    if not args.no_e2e:
        G_pin = torch.from_numpy(region.G).pin_memory()
        y_pin = torch.from_numpy(region.y).pin_memory()
        ereg = spa.Region(region.G, region.y, w["nu"],
                          config=spa.make_config(move=w["move"], precision=args.precision, **init))
        ereg.run(sched_h, w["N"], w["M"], 1)  # builds the graph once, as a long-lived context does
        t_e2e = 0.0
        ksteps = max(2, min(args.steps, 5))
        for k in range(ksteps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ereg.set_data(G_pin.numpy(), y_pin.numpy())
            res = ereg.run(sched_h, w["N"], w["M"], 50 + k)
            t_e2e += time.perf_counter() - t0
        bi = region.G.nbytes + region.y.nbytes + sched_h.nbytes + 8
        bo = sum(v.nbytes for v in res.values())
        e2e = {"value": gmac * ksteps / t_e2e, "unit": "GMAC/s", "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(bo), "ms_per_step": 1e3 * t_e2e / ksteps,
               "path": "spa_set_data (pinned host G, y) + spa_run (host schedule -> host results)"}
        ereg.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w, region, sched_h)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "GMAC/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "bf16" if args.precision == "split_bf16" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(w), "precision": args.precision,
                       "l2": "flushed (512 MB write) between timed sweeps",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "accumulate": "fp32 (tcgen05 TMEM)" if args.precision == "split_bf16" else "fp32 FFMA",
                       "weights": "fp64"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "plain_fp32": plain,
            "workloads": extras,
        }
        print(json.dumps(line), flush=True)
    reg.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
