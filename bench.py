"""Benchmark of the DE phase-tracking hot path (arxiv 1906.10598) on B300.

A step is one full DE fit (DE/rand/1/bin, Table 3-1-1 controls) of the
paper-size block: N = 400,000 int16 samples at 10 kHz (40 s), population 64,
1250 generations = 64 x 1251 = 80,064 objective evaluations (the paper's
400K-sample / ~80,000-evaluation experiment, Sec. 1.3), default precision tier
(FP64-anchored phase, FP32 cosine and residuals).

Metric: objective sample-evaluations per second = N * pop * (gens + 1) / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

``--impl reference`` times the FP64 CPU oracle (the only reference this paper
has) on a bounded sample of the same workload. Under torchrun (N > 1) each
rank fits its own block (independent blocks: weak scaling, no collective on the
data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "paper400k_int16_pop64_g1250"
WORKLOAD_FULL = "perigee400k_int16_pop64_g1250_full_model"
METRIC = "objective sample-evals/s"
UNIT = "sample-evals/s"
# paper: 400K-sample block, ~80,000 objective evaluations, 6.5 s on a GTX580 (Sec. 1.3)
PAPER_SAMPLE_EVALS_PER_S = 400_000 * 80_000 / 6.5
# SFU-bound roofline: one cosine per sample-eval at the pure __cosf rate that
# pt_pipe_rate measures on this GPU (per SM clock), times the SMs and the
# maximum SM clock the fits run at (no throttle reason: checked by the clocks)
SM_MAX_MHZ = 2032.0
# ncu summary of the DE kernel: its DRAM bytes per launch and the sources it was taken on
PROFILE = os.path.join(ROOT, "profiles", "k_de_paper400k_full.md")
PROFILE_FULL_MODEL = os.path.join(ROOT, "profiles", "k_de_perigee400k_full_model.md")
KERNEL_SOURCES = ("pt_kernels.cuh", "pt_device.cuh")


def _code_only(src: str) -> str:
    """C/C++ source without comments, one space per whitespace run: the hash of
    the kernel sources follows their code, not their comments."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1906_10598_b300", "csrc", name)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()


def _profile_fields(path: str):
    fields = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.startswith(("traffic_bytes_per_launch", "kernel_sources_sha256",
                                                "fp64_pipe_pct_of_peak", "warp_inst_per_32_evals")):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
    return fields


def profiled_traffic(path: str = PROFILE):
    """(DRAM bytes per launch, note) from the committed ncu summary, or (None,
    why) when the kernel sources changed since that capture."""
    try:
        fields = _profile_fields(path)
        if fields.get("kernel_sources_sha256") != kernel_sources_sha256():
            return None, "kernel sources changed since the ncu capture"
        return int(fields["traffic_bytes_per_launch"]), "ncu dram__bytes_read + write, one launch (" + \
            os.path.basename(path) + ")"
    except (OSError, KeyError, ValueError):
        return None, "no ncu summary"


def profiled_inst_per_32(path: str = PROFILE):
    """Warp instructions per warp of 32 sample-evaluations of the DE kernel
    (ncu, all opcodes) from the committed summary, or None once the kernel
    sources changed since."""
    try:
        fields = _profile_fields(path)
        if fields.get("kernel_sources_sha256") != kernel_sources_sha256():
            return None
        return float(fields["warp_inst_per_32_evals"])
    except (OSError, KeyError, ValueError):
        return None


def profiled_fp64_share(path: str = PROFILE):
    """The FP64 pipe's share of its peak over one launch (the DE's trial
    generation and phase set-up, counted apart from the SFU roofline) from the
    committed ncu summary, or None when the kernel sources changed since."""
    try:
        fields = _profile_fields(path)
        if fields.get("kernel_sources_sha256") != kernel_sources_sha256():
            return None
        return float(fields["fp64_pipe_pct_of_peak"]) / 100.0
    except (OSError, KeyError, ValueError):
        return None


def measure_pipes(device: int, full: bool = True) -> dict:
    """The pipe microbenchmarks (pt_pipe_rate) on `device`: the pure __cosf
    rate (the objective's roofline denominator), __cosf with 2, 4, 6 and 8 FP32
    FMAs each, FP32 FMAs alone (the issue rate) and FP64 FMAs alone. Per SM
    clock per SM and per second."""
    import paper_1906_10598_b300 as pt
    out = {"cos": pt.pipe_rate(device, pt.PIPE_COS, 0), "ffma": pt.pipe_rate(device, pt.PIPE_FFMA)}
    if full:
        for nf in (2, 4, 6, 8):
            out[f"cos_{nf}ffma"] = pt.pipe_rate(device, pt.PIPE_COS, nf)
        out["dfma"] = pt.pipe_rate(device, pt.PIPE_DFMA)
        out["ex2"] = pt.pipe_rate(device, pt.PIPE_EX2)
    return out


def sfu_peak(rates: dict) -> dict:
    """The objective's roofline denominator from the measured pipe rates: one
    SFU cosine per sample-evaluation at the pure __cosf rate (per SM clock,
    clock64), times the SM count and the maximum SM clock."""
    sms = _sm_count()
    per_clk = rates["cos"]["per_clk_sm"]
    return {"peak": per_clk * sms * SM_MAX_MHZ * 1e6, "per_clk_sm": per_clk,
            "measured_per_s": rates["cos"]["per_s"], "measured_mhz": rates["cos"]["sm_mhz"],
            "basis": f"measured pure __cosf rate {per_clk:.2f}/clk/SM (pt_pipe_rate) x {sms} SMs x "
                     f"{SM_MAX_MHZ:.0f} MHz, one cosine per sample-eval"}


def issue_peak(rates: dict, inst_per_32) -> dict:
    """The issue-rate ceiling of the kernel: the measured warp instructions per
    SM clock (FFMA alone) over the kernel's warp instructions per warp of 32
    sample-evaluations (ncu, all opcodes), or None without a current capture."""
    if not inst_per_32:
        return None
    ipc = rates["ffma"]["per_clk_sm"] / 32.0
    return {"peak": ipc * 32.0 / inst_per_32 * _sm_count() * SM_MAX_MHZ * 1e6, "warp_inst_per_clk_sm": ipc,
            "warp_inst_per_32_evals": inst_per_32}


def run_peaks(args):
    """The pipe rates of this GPU (pt_pipe_rate) with the clocks sampled while
    they run: the denominators of the objective's roofline."""
    from paper_1906_10598_b300 import build
    build.build()
    sampler = ClockSampler(0)
    sampler.start()
    rates = measure_pipes(0, full=True)
    clocks = sampler.stop()
    sms = _sm_count()
    line = {"metric": "pipe rates", "sms": sms, "rates": rates, "clocks": clocks,
            "cos_per_clk_sm": rates["cos"]["per_clk_sm"],
            "warp_inst_per_clk_sm": rates["ffma"]["per_clk_sm"] / 32.0,
            "dfma_per_clk_sm": rates["dfma"]["per_clk_sm"],
            "sfu_peak_sample_evals_per_s_at_max_clock": rates["cos"]["per_clk_sm"] * sms * SM_MAX_MHZ * 1e6}
    print(json.dumps(line))
    return 0


def _sm_count() -> int:
    import torch
    return int(torch.cuda.get_device_properties(0).multi_processor_count)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "sm_mhz_min": float(min(sm))}


def cpu_baseline(blk: synth.Block, gens: int = 240, full: bool = False, one_core: bool = True):
    """The oracle (FP64, libm cos, OpenMP over candidates) timed on this host's
    cores on a bounded sample of the workload: the same block and population
    for `gens` generations instead of 1250 (the full model's fit with full)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    s = blk.values()
    t = time.perf_counter()
    solve = oracle.de_solve_full if full else oracle.de_solve
    solve(s, blk.fs, blk.t0, blk.bounds, blk.pop, gens, blk.F, blk.CR, blk.de_seed, nthreads=cores)
    dt = time.perf_counter() - t
    evals = blk.n * blk.pop * (gens + 1)
    out = {"value": evals / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"oracle DE{' (full model)' if full else ''} on the 400K int16 block, pop {blk.pop}, "
                     f"{gens} generations ({evals:.3g} sample-evals, {dt:.1f} s)"}
    if not one_core:
        return out
    # and on one core, on a shorter sample (the paper's single-thread baseline)
    g1 = max(1, gens // 15)
    t = time.perf_counter()
    solve(s, blk.fs, blk.t0, blk.bounds, blk.pop, g1, blk.F, blk.CR, blk.de_seed, nthreads=1)
    dt1 = time.perf_counter() - t
    evals1 = blk.n * blk.pop * (g1 + 1)
    out["one_core"] = {"value": evals1 / dt1, "unit": UNIT, "cores": 1,
                       "sample": f"the same DE for {g1} generations on one thread ({evals1:.3g} sample-evals, "
                                 f"{dt1:.1f} s)"}
    return out


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    blk = synth.paper400k(0)
    gens = 4
    vals = []
    for i in range(args.warmup + args.steps):
        # the one-core figure once, with the last step
        vals.append(cpu_baseline(blk, gens=gens, one_core=i == args.warmup + args.steps - 1))
    timed = vals[args.warmup:]
    v = float(np.mean([x["value"] for x in timed]))
    base = dict(timed[-1])
    base["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": blk.n * blk.pop * (gens + 1) / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": v / PAPER_SAMPLE_EVALS_PER_S, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": blk.n, "fs": blk.fs, "pop": blk.pop, "gens_timed": gens,
                       "sample": "each step: oracle DE with 4 generations on the full block"},
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build, replicas
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    # one paper-size block per rank (equal costs: the router gives rank r block r)
    (unit,) = replicas.my_units([1.0] * world, world, rank)
    full = args.model == "full"
    blk = synth.perigee400k(unit, gens=args.gens) if full else synth.paper400k(unit, gens=args.gens)
    ctx = pt.Context(local)
    # a dedicated stream: the library launches on it and the CUDA events below
    # are recorded on it, so they bracket exactly the library's work
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx.set_stream(stream.cuda_stream)
    ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
    # the roofline's denominators, measured on this GPU before the timed region
    rates = measure_pipes(local, full=False)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 126 MB L2
    bounds = blk.bounds.copy()
    if args.objective == "cor":
        # Eq. 2-2-5 / 2-2-6: the amplitude is the constant average amplitude
        ctx.set_objective("cor")
        bounds[0] = (blk.truth[0], blk.truth[0])
    evals = blk.sample_evals()

    def step():
        if full:
            return ctx.de_solve_full(bounds, blk.pop, blk.gens, blk.F, blk.CR, blk.de_seed)
        return ctx.de_solve(bounds, blk.pop, blk.gens, blk.F, blk.CR, blk.de_seed, pt.TIER_F64)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, kern_ms = [], []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()  # L2 flush outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        params, sse = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(ctx.last_kernel_ms())
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    total_ms = float(np.sum(step_ms))
    total_ms = replicas.max_over_ranks(total_ms, device="cuda")

    # end to end through the C ABI with host buffers: H2D of the step's samples
    # (pt_load_block, from pinned host memory) + the fit + D2H of the result,
    # every step
    host_samples = torch.from_numpy(blk.samples).pin_memory().numpy()
    e2e_s = []
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.load_block(host_samples, blk.fs, blk.t0, blk.scale)
        step()
        e2e_s.append(time.perf_counter() - t)
    e2e_v = evals * world / replicas.max_over_ranks(float(np.mean(e2e_s)), device="cuda")

    value = evals * args.steps * world / (total_ms * 1e-3)
    k_avg = float(np.mean(kern_ms)) * 1e-3
    achieved = evals / k_avg
    sfu = sfu_peak(rates)
    peak = sfu["peak"]
    prof = PROFILE_FULL_MODEL if full else PROFILE
    traffic, traffic_note = profiled_traffic(prof)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": UNIT, "frac": achieved / peak,
            "traffic": traffic, "traffic_note": traffic_note,
            "kernel": "k_de<TIER_F64, OBJ_CHI2, MODEL_FULL>" if full else "k_de<TIER_F64>",
            "peak_basis": sfu["basis"], "peak_measured_per_s": sfu["measured_per_s"],
            "cos_per_clk_sm_measured": sfu["per_clk_sm"]}
    if clocks.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (peak * clocks["sm_mhz"] / SM_MAX_MHZ)
    ip = issue_peak(rates, profiled_inst_per_32(prof))
    roof["issue_peak"] = ip["peak"] if ip else None
    roof["frac_of_issue_peak"] = achieved / ip["peak"] if ip else None
    roof["issue_peak_basis"] = (f"measured {ip['warp_inst_per_clk_sm']:.2f} warp instructions/clk/SM (FFMA alone) / "
                                f"{ip['warp_inst_per_32_evals']:.2f} warp instructions per 32 sample-evals (ncu)"
                                if ip else "no ncu capture of the current kernel sources")
    roof["fp64_pipe_share"] = profiled_fp64_share(prof)
    roof["fp64_pipe_note"] = "ncu sm__inst_executed_pipe_fp64 % of peak over one launch (trial generation, set-up)"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / world / PAPER_SAMPLE_EVALS_PER_S, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_FULL if full else WORKLOAD, "n": blk.n, "fs": blk.fs,
                       "storage": "int16", "pop": blk.pop, "gens": blk.gens,
                       "model": "full (A, phi0, f0, f1, f2, A1, f3)" if full else "cubic (A, phi0, f0, f1, f2)",
                       "tier": "f64-anchored phase, f32 cos", "l2": "flushed between steps",
                       "objective": "chi-square (Eq. 2-2-4)" if args.objective == "chi2" else
                       "correlation (Eq. 2-2-5, constant A)",
                       "de_seconds": total_ms / args.steps * 1e-3, "wall_s": wall},
            "roofline": roof, "clocks": clocks, "gpu_launches": args.steps,
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(blk.samples.nbytes),
                    "d2h_bytes_per_step": (len(params) + 1) * 8 + 8}}
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(blk, full=full) if world == 1 else None
    if world == 1 and not args.no_extras and not full:
        # the other metrics the workload names, on the same GPU in the same run:
        # the batched form (256 uneven blocks, one launch under a CUDA graph),
        # the all-FP64 single-block form on a sample of its blocks, and the
        # serving loop's latency (4 station streams, compressed replay)
        ctx.close()
        ctx = None
        torch.cuda.set_stream(torch.cuda.default_stream())
        mb = measure_batch(256, steps=1, warmup=1, e2e_steps=1)
        ms_ = measure_serve(args.serve_seconds, args.speedup, args.inflight)
        mo = measure_objective(4096, steps=5, warmup=3)
        line["batch_blocks_per_s"] = mb["blocks_per_s"]
        line["plain_f64_blocks_per_s"] = mb["plain_blocks_per_s"]
        line["batch_over_plain_f64"] = mb["blocks_per_s"] / mb["plain_blocks_per_s"]
        line["batch_sample_evals_per_s"] = mb["evals"] / mb["mean_s"]
        line["batch_frac_of_sfu_peak"] = mb["evals"] / mb["mean_s"] / peak
        line["batch_fit_sse_rel_err_vs_oracle_max"] = float(max(mb["rel"]))
        line["serve_p50_ms"] = float(np.percentile(ms_["lat"], 50) * 1e3)
        line["serve_p99_ms"] = float(np.percentile(ms_["lat"], 99) * 1e3)
        line["serve_p99_over_block_duration"] = float(np.percentile(ms_["lat_rel"], 99))
        line["serve_p99_over_real_block_duration"] = float(np.percentile(ms_["lat_real_rel"], 99))
        line["serve_blocks"] = ms_["n"]
        line["serve_status_ok"] = ms_["status_ok"]
        line["objective_sample_evals_per_s"] = mo["achieved"]
        line["objective_frac_of_sfu_peak"] = mo["achieved"] / peak
        line["objective_sse_rel_err_vs_oracle_max"] = mo["sse_rel_err_max"]
        line["objective_clocks"] = mo["clocks"]
        line["extras_config"] = {
            "batch": "256 blocks, N log-uniform 50K-1M int16, fs 1-50 kHz, pop 32-128, G = ceil(80000/pop); "
                     "one timed run after one warm-up, CUDA events, L2 flushed",
            "plain_f64": "all-FP64 tier, one pt_de_solve per block on the batch's quartile- and median-length "
                         "blocks, blocks/s extrapolated to the batch's sample-evals",
            "objective": "pt_objective alone (k_objective<TIER_F64, 16>, Eq. 2-2-4): the 400K int16 block x 4096 "
                         "candidates inside its bounds, device pointers, L2 flushed, 5 timed calls after 3 "
                         "warm-up calls, by the library's kernel events; SSE of 8 of them against the oracle",
            "serve": f"4 streams (10/20/35/50 kHz, 1-10 s blocks), {args.serve_seconds:.0f} simulated s replayed "
                     f"{args.speedup:.0f}x faster than real time, pop 64, 1250 generations, warm-started; "
                     "latency from arrival to result; serve_p99_over_block_duration is against the compressed "
                     "duration"}
    if rank == 0:
        line["fit"] = {"params": [float(v) for v in params], "sse": float(sse), "truth": [float(v) for v in blk.truth]}
        print(json.dumps(line))
    if ctx is not None:
        ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure_batch(nblocks: int, steps: int, warmup: int, full: bool = False, e2e_steps: int = 1,
                  check_fits: bool = True) -> dict:
    """256 independent blocks of uneven length (N log-uniform 50K-1M int16, fs 1-50
    kHz, pop 32-128, G = ceil(80000/pop)) in one persistent launch under a CUDA
    graph, launch shape chosen by the autotuner, timed with CUDA events over
    `steps` runs (L2 flushed between them). Compared with the all-FP64
    single-block form on a sample of the same blocks. With full: the same
    shapes for the full model (synth.batch_full)."""
    import torch
    import oracle
    import paper_1906_10598_b300 as pt
    blocks = synth.batch_full(0, nblocks=nblocks) if full else synth.batch(0, nblocks=nblocks)
    ctx = pt.Context(0)
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    t = time.perf_counter()
    batch = pt.Batch(ctx, blocks, pt.TIER_F64)
    create_s = time.perf_counter() - t
    info = batch.info()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        batch.run()
    sampler = ClockSampler(0)
    sampler.start()
    ms = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        ms.append(batch.run())
    clocks = sampler.stop()
    params, sse = batch.results()
    mean_s = float(np.mean(ms)) * 1e-3
    evals = info["sample_evals"]
    rel = []
    if check_fits:
        # fit check on a few blocks against the oracle objective
        for i in range(0, len(blocks), max(1, len(blocks) // 4)):
            b = blocks[i]
            want = (oracle.sse_full if full else oracle.sse)(b.values(), b.fs, b.t0, params[i])
            rel.append(abs(sse[i] - want) / want)
    # all-FP64 single-block form on a sample of the blocks (one pt_de_solve each)
    order = np.argsort([b.n for b in blocks])
    sample_ids = [int(order[len(order) // 4]), int(order[len(order) // 2])]
    plain_s, plain_evals, fast_s = 0.0, 0.0, 0.0
    for i in sample_ids:
        b = blocks[i]
        ctx.load_block(b.samples, b.fs, b.t0, b.scale)
        solve = ctx.de_solve_full if full else ctx.de_solve
        solve(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, block_id=b.block_id, tier=pt.TIER_PLAIN)
        plain_s += ctx.last_kernel_ms() * 1e-3
        solve(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, block_id=b.block_id, tier=pt.TIER_F64)
        fast_s += ctx.last_kernel_ms() * 1e-3
        plain_evals += b.sample_evals()
    plain_rate = plain_evals / plain_s
    # end to end: fresh batch every step (H2D of every block's samples from
    # pinned host memory, launch, results)
    for b in blocks:
        b.samples = torch.from_numpy(b.samples).pin_memory().numpy()
    e2e = []
    for _ in range(max(1, e2e_steps)):
        torch.cuda.synchronize()
        t = time.perf_counter()
        bb = pt.Batch(ctx, blocks, pt.TIER_F64)
        bb.run()
        bb.results()
        bb.close()
        e2e.append(time.perf_counter() - t)
    batch.close()
    ctx.close()
    return {"blocks": blocks, "info": info, "create_s": create_s, "mean_s": mean_s, "evals": evals,
            "clocks": clocks, "rel": rel, "plain_rate": plain_rate, "sample_ids": sample_ids, "fast_s": fast_s,
            "plain_s": plain_s, "e2e_s": float(np.mean(e2e)),
            "plain_blocks_per_s": len(blocks) / (evals / plain_rate), "blocks_per_s": len(blocks) / mean_s}


def run_batch(args):
    """The batched workload alone (see measure_batch), one JSON line."""
    from paper_1906_10598_b300 import build
    build.build()
    full = args.model == "full"
    m = measure_batch(args.nblocks, args.steps, args.warmup, full=full, e2e_steps=max(1, args.steps // 3))
    blocks, info, evals, mean_s = m["blocks"], m["info"], m["evals"], m["mean_s"]
    sfu = sfu_peak(measure_pipes(0, full=False))
    nbytes = int(sum(b.samples.nbytes for b in blocks))
    line = {"metric": "batched objective sample-evals/s", "value": evals / mean_s, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch{len(blocks)}_int16_n50k-1m_pop32-128" + ("_full_model" if full else ""),
                       "model": "full" if full else "cubic", "blocks": len(blocks),
                       "total_samples": int(sum(b.n for b in blocks)), "l2": "flushed between steps",
                       "group_ctas": info["group_ctas"], "groups": info["ngroups"],
                       "uses_graph": info["uses_graph"], "autotune_predicted_ms": info["predicted_ms"],
                       "tune_rate_per_cta": info["tune_rate"], "tune_gen_us": info["tune_gen_us"],
                       "tune_rate_stream_per_cta": info["tune_rate_stream"], "create_s": m["create_s"]},
            "blocks_per_s": m["blocks_per_s"],
            "roofline": {"bound": "alu", "achieved": evals / mean_s, "peak": sfu["peak"], "unit": UNIT,
                         "frac": evals / mean_s / sfu["peak"], "traffic": None, "peak_basis": sfu["basis"],
                         "kernel": "k_de<TIER_F64, OBJ_CHI2, MODEL_FULL> (grouped)" if full else
                         "k_de<TIER_F64> (grouped)"},
            "plain_f64_single_block": {"sample_evals_per_s": m["plain_rate"],
                                       "blocks_per_s_est": m["plain_blocks_per_s"],
                                       "sampled_blocks": m["sample_ids"],
                                       "default_tier_single_block_s": m["fast_s"],
                                       "plain_tier_single_block_s": m["plain_s"]},
            "fit_sse_rel_err_vs_oracle_max": float(max(m["rel"])),
            "clocks": m["clocks"], "gpu_launches": args.steps,
            "e2e": {"value": evals / m["e2e_s"], "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": len(blocks) * 64}}
    print(json.dumps(line))
    return 0


def measure_serve(sim_seconds: float, speedup: float, inflight: int) -> dict:
    """Four simulated station streams (10/20/35/50 kHz, 1-10 s blocks, drifting
    Doppler) deliver blocks as they fill, in real time compressed by
    `speedup`; each block is submitted on arrival (pt_submit), warm-started
    from the stream's latest fit (Sec. 3.1.1 running-time ranges), and
    collected with pt_poll. Latency = completion - arrival."""
    import paper_1906_10598_b300 as pt
    specs = synth.make_streams(0)
    X = speedup
    plan = []  # (arrival_sim_s, stream, index, block)
    for sp in specs:
        nb = max(2, int(sim_seconds // sp.block_s))
        for k in range(nb):
            b = synth.stream_block(sp, k)
            plan.append(((k + 1) * sp.block_s, sp.stream_id, k, b))
    plan.sort(key=lambda x: x[0])
    ctx = pt.Context(0)
    server = pt.Server(ctx, max_inflight=inflight, ctas_per_request=0, max_queued=256)
    # warm up the kernels once
    w = plan[0][3]
    ctx.load_block(w.samples, w.fs, w.t0, w.scale)
    ctx.de_solve(w.bounds, w.pop, 5, w.F, w.CR, 0)
    latest = {}  # stream -> (index, params)
    tickets, meta, results = {}, {}, {}
    t0 = server.clock()
    i = 0
    while len(results) < len(plan):
        now = server.clock() - t0
        while i < len(plan) and plan[i][0] / X <= now:
            arr, sid, k, b = plan[i]
            bounds = b.bounds
            if sid in latest:
                kp, prev = latest[sid]
                T = b.T
                bounds = pt.warm_bounds(prev, (k - kp) * T, T)
                # A: the previous fit's +-10 % range, widened like the first block's if it drifted
                bounds[0] = (min(bounds[0, 0], 0.8 * prev[0]), max(bounds[0, 1], 1.2 * prev[0]))
            t = server.submit(b, pt.TIER_F64, stream_id=sid, bounds=bounds)
            if t is None:
                break  # queue full: retry on the next pass
            tickets[t] = i
            meta[i] = (arr / X + t0, bounds)
            i += 1
        for t in list(tickets):
            r = server.poll(t)
            if r is not None:
                j = tickets.pop(t)
                results[j] = r
                _, sid, k, b = plan[j]
                if sid not in latest or latest[sid][0] < k:
                    latest[sid] = (k, r["params"])
        time.sleep(0.0005)
    wall = max(r["t_done"] for r in results.values()) - (plan[0][0] / X + t0)
    lat, lat_rel, f0err, inb = [], [], [], 0
    for j, r in results.items():
        arr_wall, bounds = meta[j]
        _, sid, k, b = plan[j]
        L_ = r["t_done"] - arr_wall
        lat.append(L_)
        lat_rel.append(L_ / (b.T / X))
        f0err.append(abs(r["params"][2] - b.truth[2]))
        inb += int(np.all(b.truth >= bounds[:, 0] - 1e-12) and np.all(b.truth <= bounds[:, 1] + 1e-12)
                   if np.ndim(bounds) == 2 else 1)
    # continuity of consecutive fits of each stream (Eq. 3-1-2)
    cont, ncont = 0, 0
    for sp in specs:
        idx = sorted(j for j in results if plan[j][1] == sp.stream_id)
        for a, b_ in zip(idx, idx[1:]):
            ok, _, _ = pt.continuity(results[a]["params"], sp.block_s, results[b_]["params"], sp.block_s, 0.3, 10.0)
            cont += int(ok)
            ncont += 1
    evals = sum(plan[j][3].sample_evals() for j in results)
    ctx.close()
    return {"specs": specs, "X": X, "n": len(results), "wall": wall, "lat": lat, "lat_rel": lat_rel,
            "lat_real_rel": [v / X for v in lat_rel], "f0err": f0err, "inb": inb, "cont": cont, "ncont": ncont,
            "evals": evals, "status_ok": sum(r["status"] == 0 for r in results.values()) / len(results)}


def run_serve(args):
    """The serving replay alone (see measure_serve), one JSON line."""
    from paper_1906_10598_b300 import build
    build.build()
    m = measure_serve(args.sim_seconds, args.speedup, args.inflight)
    specs, lat, lat_rel = m["specs"], m["lat"], m["lat_rel"]
    line = {"metric": "served blocks/s", "value": m["n"] / m["wall"], "unit": "blocks/s", "n_gpus": 1,
            "steps": m["n"], "warmup": 1, "ms_per_step": m["wall"] / m["n"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve4_streams_10-50khz_1-10s", "streams": len(specs),
                       "block_s": [sp.block_s for sp in specs], "fs": [sp.fs for sp in specs],
                       "time_compression": m["X"], "sim_seconds": args.sim_seconds, "max_inflight": args.inflight,
                       "pop": 64, "gens": 1250},
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                           "max": float(np.max(lat) * 1e3)},
            "latency_over_block_duration": {"p50": float(np.percentile(lat_rel, 50)),
                                            "p99": float(np.percentile(lat_rel, 99)),
                                            "note": "block duration compressed by time_compression"},
            "sample_evals_per_s": m["evals"] / m["wall"],
            "warm_start_truth_in_bounds": m["inb"] / m["n"],
            "continuity_pass": m["cont"] / max(1, m["ncont"]),
            "f0_abs_err_hz": {"median": float(np.median(m["f0err"])), "max": float(np.max(m["f0err"]))},
            "status_ok": m["status_ok"]}
    print(json.dumps(line))
    return 0


def measure_objective(ncand: int, steps: int, warmup: int) -> dict:
    """The objective kernel alone (pt_objective, Eq. 2-2-4): the paper-size
    400K int16 block against `ncand` candidates drawn inside its bounds,
    candidates and results resident on the device (device pointers), L2
    flushed between steps. Per-call CUDA-event times on the library's stream
    and the library's own kernel times, the clocks during the timed calls,
    and the SSE of sampled candidates against the oracle (after timing)."""
    import torch
    import paper_1906_10598_b300 as pt
    blk = synth.paper400k(0)
    ctx = pt.Context(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx.set_stream(stream.cuda_stream)
    try:
        ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
        rng = np.random.default_rng(0)
        lo, hi = blk.bounds[:, 0], blk.bounds[:, 1]
        cands = torch.tensor(lo + rng.random((ncand, 5)) * (hi - lo), dtype=torch.float64, device="cuda")
        out = torch.empty(ncand, dtype=torch.float64, device="cuda")
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        for _ in range(warmup):
            ctx.objective(cands, pt.TIER_F64, out=out)
        sampler = ClockSampler(0)
        sampler.start()
        ms, kms = [], []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.objective(cands, pt.TIER_F64, out=out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            kms.append(ctx.last_kernel_ms())
        clocks = sampler.stop()
        got = out.cpu().numpy()
        idx = np.arange(0, ncand, max(1, ncand // 8))
        host_cands = cands.cpu().numpy()[idx]
    finally:
        ctx.close()
        torch.cuda.set_stream(torch.cuda.default_stream())
    import oracle
    want = oracle.sse_many(blk.values(), blk.fs, blk.t0, host_cands)
    evals = float(blk.n) * ncand
    return {"n": blk.n, "evals": evals, "ms": ms, "kernel_ms": kms, "clocks": clocks,
            "value": evals * steps / (float(np.sum(ms)) * 1e-3), "achieved": evals / (float(np.mean(kms)) * 1e-3),
            "sse_rel_err_max": float(np.max(np.abs(got[idx] - want) / want))}


def run_objective(args):
    """The objective kernel alone (measure_objective) as its own JSON line,
    against the SFU roofline."""
    from paper_1906_10598_b300 import build
    build.build()
    mo = measure_objective(args.ncand, args.steps, args.warmup)
    sfu = sfu_peak(measure_pipes(0, full=False))
    peak = sfu["peak"]
    line = {"metric": "objective kernel sample-evals/s", "value": mo["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(mo["ms"])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper400k_int16_objective", "n": mo["n"], "candidates": args.ncand,
                       "tier": "f64-anchored phase, f32 cos", "l2": "flushed between steps"},
            "roofline": {"bound": "alu", "achieved": mo["achieved"], "peak": peak, "unit": UNIT,
                         "frac": mo["achieved"] / peak, "traffic": None, "kernel": "k_objective<TIER_F64, 16>",
                         "peak_basis": sfu["basis"]},
            "clocks": mo["clocks"], "gpu_launches": 2 * args.steps,
            "sse_rel_err_vs_oracle_max": mo["sse_rel_err_max"]}
    print(json.dumps(line))
    return 0


def run_track(args):
    """One station stream (20 kHz, 2 s blocks, quartic phase plus Doppler
    sinusoid, 25 dB) tracked block by block with pt_track (Sec. 3.1.4): warm
    ranges, Eq. 3-1-2 acceptance, enlarge-and-retry, integration Doppler over
    10 s count intervals (Eq. 4-1-2). Reports blocks/s, the real-time factor,
    the quality histogram and the integration-Doppler error against the
    stream's true phase change.

    With --model full: a perigee-like stream (2 kHz, 10 s blocks, quartic
    phase with F3 ~ 1.6e-3 cycles/s^4 and an amplitude slope) tracked with
    the full model (pt_track_create_full), 0.05 rad / 0.05 rad/s continuity
    thresholds, 30 s count intervals."""
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    full = args.model == "full"
    if full:
        sp = synth.perigee_stream(0)
        nblk, per_int = min(args.track_blocks, 30), 3
    else:
        sp = synth.make_streams(seed=11)[1]
        sp.block_s, sp.snr_db = 2.0, 25.0
        nblk, per_int = args.track_blocks, 5
    blocks = [synth.stream_block(sp, k) for k in range(nblk)]
    if full:
        b0 = blocks[0]
        T = b0.T
        t0 = synth.stream_taylor_truth_full(sp, (b0.n - 1) / 2 / sp.fs)
        rng = np.random.default_rng(0)

        def win(v, h):
            c = v + rng.uniform(-0.5, 0.5) * h
            return (c - h, c + h)

        bounds0 = np.array([(0.8 * t0[0], 1.2 * t0[0]), (-math.pi, math.pi), win(t0[2], 2 / T),
                            win(t0[3], 4 / T ** 2), win(t0[4], 24 / T ** 3), (-0.24 * t0[0] / T, 0.24 * t0[0] / T),
                            win(t0[6], 192 / T ** 4)])
        thr = dict(max_dphi=0.05, max_dfreq=0.05)
    else:
        bounds0 = blocks[0].bounds
        thr = dict(max_dphi=0.3, max_dfreq=2 * math.pi * 1.0)
    ctx = pt.Context(0)
    tr = pt.Tracker(ctx, bounds0, pop=64, gens=1250, seed=0, enlarge=2.0, max_attempts=3,
                    count_interval=per_int * sp.block_s, **thr)
    w = pt.Tracker(ctx, bounds0, pop=64, gens=20)
    w.block(blocks[0].samples, blocks[0].fs, blocks[0].scale)  # load the kernels
    w.close()
    t = time.perf_counter()
    res = [tr.block(b.samples, b.fs, b.scale) for b in blocks]
    wall = time.perf_counter() - t
    q = [r["quality"] for r in res]
    n = blocks[0].n
    idop_err, dphi = [], [r["dphi"] for r in res if not math.isnan(r["dphi"])]
    for k, r in enumerate(res):
        if not math.isnan(r["int_doppler"]):
            t_s = (k + 1 - per_int) * n / sp.fs - 0.5 / sp.fs
            t_e = (k + 1) * n / sp.fs - 0.5 / sp.fs
            true = 2 * math.pi * float(synth.stream_phase_cycles(sp, np.array([t_e]))[0]
                                       - synth.stream_phase_cycles(sp, np.array([t_s]))[0]) / (t_e - t_s)
            idop_err.append(abs(r["int_doppler"] - true))
    f0err = [abs(r["params"][2] - b.truth[2]) for r, b in zip(res, blocks) if r["quality"] > 0]
    dfreq = [r["dfreq"] for r in res if not math.isnan(r["dfreq"])]
    line = {"metric": "tracked blocks/s", "value": nblk / wall, "unit": "blocks/s", "n_gpus": 1, "steps": nblk,
            "warmup": 1, "ms_per_step": wall / nblk * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "track1_perigee_2khz_10s_full_model" if full else "track1_stream_20khz_2s",
                       "model": "full" if full else "cubic", "fs": sp.fs, "block_s": sp.block_s, "blocks": nblk,
                       "pop": 64, "gens": 1250, "count_interval_s": per_int * sp.block_s, "max_attempts": 3,
                       "max_dphi_rad": thr["max_dphi"], "max_dfreq_rad_s": thr["max_dfreq"]},
            "real_time_factor": sp.block_s * nblk / wall,
            "quality_histogram": {str(v): q.count(v) for v in sorted(set(q))},
            "continuity_dphi_rad": {"median": float(np.median(dphi)) if dphi else None,
                                    "max": float(np.max(dphi)) if dphi else None},
            "continuity_dfreq_rad_s": {"median": float(np.median(dfreq)) if dfreq else None,
                                       "max": float(np.max(dfreq)) if dfreq else None},
            "f0_abs_err_hz_median": float(np.median(f0err)),
            "int_doppler_abs_err_rad_s": {"intervals": len(idop_err),
                                          "median": float(np.median(idop_err)) if idop_err else None,
                                          "max": float(np.max(idop_err)) if idop_err else None}}
    print(json.dumps(line))
    tr.close()
    ctx.close()
    return 0


def run_seed(args):
    """The FFT-seeded fit (Sec. 3.1.1): pt_seed_bounds on the loaded block, then
    the DE fit (pop 64, 1250 generations) inside the seeded ranges (A and f0
    +- 10 %), on 10 synthetic blocks: four 4 s blocks at 1 kHz, three 40 s
    blocks at 10 kHz (N = 400,000) and three 2 s cuts of them. A fit reaches
    the truth's basin when its SSE is at or below the SSE at the truth (the
    block's f0 sign normalised: a real tone cannot tell f0 from -f0). Reports
    that fraction, and the seed's and the fit's times (host wall, after a
    warm-up call)."""
    import oracle
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    blocks = [synth.single4096(s) for s in range(4)] + [synth.paper400k(s) for s in range(3)] + \
        [synth.paper400k(s, n=20_000) for s in range(3)]
    ctx = pt.Context(0)
    ctx.load_block(blocks[0].samples, blocks[0].fs, blocks[0].t0, blocks[0].scale)
    ctx.seed_bounds()
    ok, inside, seed_ms, fit_ms, rows = 0, 0, [], [], []
    for blk in blocks:
        ctx.load_block(blk.samples, blk.fs, blk.t0, blk.scale)
        t = time.perf_counter()
        g = ctx.seed_bounds()
        seed_ms.append((time.perf_counter() - t) * 1e3)
        b = g["bounds"][:5]
        tr = blk.truth.copy()
        if tr[2] < 0:
            tr[1:5] = -tr[1:5]
        inside += all(b[j, 0] <= tr[j] <= b[j, 1] for j in (2, 3, 4))
        t = time.perf_counter()
        p, f = ctx.de_solve(b, 64, 1250, 0.7, 0.9, 5, pt.TIER_F64)
        fit_ms.append((time.perf_counter() - t) * 1e3)
        f_truth = oracle.sse(blk.values(), blk.fs, blk.t0, blk.truth)
        ok += f <= f_truth * (1 + 1e-6)
        rows.append({"n": blk.n, "fs": blk.fs, "f0_seed": g["f0"], "f0_fit": float(p[2]), "f0_true": float(tr[2]),
                     "sse_over_truth": f / f_truth})
    line = {"metric": "seeded fits reaching the truth's basin", "value": ok / len(blocks), "unit": "fraction",
            "n_gpus": 1, "steps": len(blocks), "warmup": 1, "ms_per_step": float(np.mean(fit_ms) + np.mean(seed_ms)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "fft_seed_then_fit_10_blocks", "pop": 64, "gens": 1250, "f0_rel": 0.1},
            "truth_inside_seeded_ranges": inside / len(blocks), "seed_ms_median": float(np.median(seed_ms)),
            "fit_ms_median": float(np.median(fit_ms)), "blocks": rows}
    print(json.dumps(line))
    ctx.close()
    return 0


def run_precision(args):
    """Precision sweep on the 400K block: samples stored as int8 / FP16 / FP32,
    phase evaluated by the FP64-anchored default tier, the double-float FP32
    tier and the naive FP32 tier. Per (storage, tier) over `--seeds` seeds:
    the objective's relative error against the oracle's SSE at the same
    parameters, and the fitted phi0/f0/f1/f2 errors against the oracle's own
    fits (tests/golden/precision_oracle_fits.json, written by the oracle alone)."""
    import oracle
    import paper_1906_10598_b300 as pt
    from paper_1906_10598_b300 import build
    build.build()
    if args.model == "full":
        return run_precision_full(args)
    ref_path = os.path.join(ROOT, "tests", "golden", "precision_oracle_fits.json")
    ref = json.load(open(ref_path)) if os.path.exists(ref_path) else {}
    ctx = pt.Context(0)
    tiers = {"f64-anchored": pt.TIER_F64, "double-float": pt.TIER_DF32, "naive-f32": pt.TIER_F32}
    rows = {}
    for st in ("i8", "f16", "f32"):
        for seed in range(args.seeds):
            b = synth.precision(seed, synth.STORAGE_NAMES[st])
            ctx.load_block(b.samples, b.fs, b.t0, b.scale)
            vals = b.values()
            r = ref.get(f"{st}/{seed}")
            for name, tier in tiers.items():
                p, f = ctx.de_solve(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, tier)
                ms = ctx.last_kernel_ms()
                want = oracle.sse(vals, b.fs, b.t0, p)
                d = rows.setdefault((st, name), {"sse_rel": [], "ms": [], "dphi0": [], "df0": [], "df1": [],
                                                 "df2": [], "truth_df0": [], "n_ref": 0, "in_basin": []})
                d["sse_rel"].append(abs(f - want) / want)
                d["ms"].append(ms)
                d["truth_df0"].append(abs(p[2] - b.truth[2]))
                if r is not None:
                    q = np.array(r["params"])
                    d["dphi0"].append(abs(float(np.angle(np.exp(1j * (p[1] - q[1]))))))
                    d["df0"].append(abs(p[2] - q[2]))
                    d["df1"].append(abs(p[3] - q[3]))
                    d["df2"].append(abs(p[4] - q[4]))
                    # the oracle's own DE reached the truth's basin (its SSE at or below the truth's)
                    d["in_basin"].append(r["sse"] <= r["sse_truth"] * (1 + 1e-6))
                    d["n_ref"] += 1
    table = []
    for (st, name), d in rows.items():
        e = {"storage": st, "tier": name, "seeds": len(d["sse_rel"]), "oracle_fits": d["n_ref"],
             "sse_rel_err_max": float(np.max(d["sse_rel"])), "sse_rel_err_median": float(np.median(d["sse_rel"])),
             "fit_ms_median": float(np.median(d["ms"])),
             "f0_err_vs_truth_hz_median": float(np.median(d["truth_df0"]))}
        for k in ("dphi0", "df0", "df1", "df2"):
            if d[k]:
                e[k + "_vs_oracle_median"] = float(np.median(d[k]))
                e[k + "_vs_oracle_max"] = float(np.max(d[k]))
        if d["dphi0"]:
            ok = [(a <= 1e-3 and c <= 1e-5) for a, c, ib in zip(d["dphi0"], d["df0"], d["in_basin"]) if ib]
            e["oracle_fits_in_basin"] = len(ok)
            e["within_1e-3rad_1e-5Hz_of_oracle_in_basin"] = float(np.mean(ok)) if ok else None
        table.append(e)
    print(json.dumps({"metric": "precision sweep", "workload": "paper400k x storage x tier", "rows": table}))
    ctx.close()
    return 0


def run_precision_full(args):
    """Precision of the full model's tiers on the perigee-shaped 400K block
    (int8 / FP16 / FP32 storage, `--seeds` seeds, 8 by default here): the
    objective's relative error against the oracle's SSE at each tier's fitted
    parameters, and the fits' phi0 / f0 / f3 errors against the truth (the
    full model has no stored oracle fits: each takes the oracle minutes)."""
    import oracle
    import paper_1906_10598_b300 as pt
    ctx = pt.Context(0)
    tiers = {"f64-anchored": pt.TIER_F64, "all-f64": pt.TIER_PLAIN, "double-float": pt.TIER_DF32,
             "naive-f32": pt.TIER_F32}
    seeds = min(args.seeds, 8)
    rows = {}
    for st in ("i8", "f16", "f32"):
        for seed in range(seeds):
            b = synth.perigee400k(seed, storage=synth.STORAGE_NAMES[st])
            ctx.load_block(b.samples, b.fs, b.t0, b.scale)
            vals = b.values()
            sse_truth = oracle.sse_full(vals, b.fs, b.t0, b.truth)
            for name, tier in tiers.items():
                p, f = ctx.de_solve_full(b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed, tier=tier)
                ms = ctx.last_kernel_ms()
                want = oracle.sse_full(vals, b.fs, b.t0, p)
                d = rows.setdefault((st, name), {"sse_rel": [], "ms": [], "dphi0": [], "df0": [], "df3": [],
                                                 "at_or_below_truth": []})
                d["sse_rel"].append(abs(f - want) / want)
                d["ms"].append(ms)
                d["dphi0"].append(abs(float(np.angle(np.exp(1j * (p[1] - b.truth[1]))))))
                d["df0"].append(abs(p[2] - b.truth[2]))
                d["df3"].append(abs(p[6] - b.truth[6]))
                d["at_or_below_truth"].append(want <= sse_truth * (1 + 1e-6))
    table = []
    for (st, name), d in rows.items():
        table.append({"storage": st, "tier": name, "seeds": len(d["sse_rel"]),
                      "sse_rel_err_max": float(np.max(d["sse_rel"])),
                      "sse_rel_err_median": float(np.median(d["sse_rel"])),
                      "fit_ms_median": float(np.median(d["ms"])),
                      "phi0_err_vs_truth_median": float(np.median(d["dphi0"])),
                      "f0_err_vs_truth_hz_median": float(np.median(d["df0"])),
                      "f3_err_vs_truth_median": float(np.median(d["df3"])),
                      "fits_at_or_below_truth_sse": float(np.mean(d["at_or_below_truth"]))})
    print(json.dumps({"metric": "precision sweep (full model)", "workload": "perigee400k x storage x tier",
                      "rows": table}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="single: skip the batch / all-FP64 / serving measurements added to the line")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="single: simulated seconds of the serving replay added to the line")
    ap.add_argument("--mode", default="single",
                    choices=["single", "batch", "serve", "precision", "track", "objective", "seed", "peaks"],
                    help="single: the 400K-block fit (default); batch: 256 uneven blocks in one launch; "
                         "serve: 4 station streams through pt_submit/pt_poll; track: one stream through pt_track")
    ap.add_argument("--track-blocks", type=int, default=60, help="track: blocks of the tracked stream")
    ap.add_argument("--ncand", type=int, default=4096, help="objective: candidates per call")
    ap.add_argument("--objective", default="chi2", choices=["chi2", "cor"],
                    help="single: the objective minimised (cor: Eq. 2-2-5 with A held at the block's amplitude)")
    ap.add_argument("--model", default="cubic", choices=["cubic", "full"],
                    help="single: the cubic model (default) or the full model (amplitude slope, order-4 phase) "
                         "on the perigee-shaped 400K block; track: a perigee-like stream tracked with the full model")
    ap.add_argument("--nblocks", type=int, default=256)
    ap.add_argument("--speedup", type=float, default=20.0, help="serve: real-time compression factor")
    ap.add_argument("--sim-seconds", type=float, default=120.0, help="serve: simulated stream duration")
    ap.add_argument("--inflight", type=int, default=4, help="serve: blocks on the device at once")
    ap.add_argument("--seeds", type=int, default=32, help="precision: seeds per storage")
    ap.add_argument("--gens", type=int, default=1250,
                    help="single: DE generations (the workload is 1250; smaller only for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "track":
        return run_track(args)
    if args.mode == "objective":
        return run_objective(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.mode == "seed":
        return run_seed(args)
    if args.mode == "peaks":
        return run_peaks(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
