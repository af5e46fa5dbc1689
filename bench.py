"""Benchmark: one GNN re-ranking (Algorithm 1) of the Market-scale workload per step.

Workload: 3,368 queries + 19,732 gallery vectors (N = 23,100), d = 2048, FP32
features drawn as 1,501 clustered identities plus 2,000 distractors
(synthetic stand-ins for Market-1501), k1 = 26, k2 = 7, 2 layers, full
ranked lists (every gallery index per query).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp8|fp32]
                  [--impl ours|reference] [--workload market|large50k|tiny|batched64|serving]

Prints one JSON line.  `value` is ms per re-rank with inputs resident in HBM
on the BF16 tensor-core path (FP32 rescoring, exact neighbour lists), timed
with CUDA events on the launching stream, L2 flushed before every step;
`e2e` is the same re-rank through the C ABI with pinned host buffers (copies
inside the timed region).  At N = 1 the line also carries, each with its own
roofline: `fp32_path` and `fp8_path` (the other precisions on the same
instance), `large_50k` (5,000 + 45,000 vectors, d = 512, in BF16, FP8 and
FP32), `batched64` (64 independent instances per rerank_run_batch call
against 64 sequential calls), `serving` (a 60 s Poisson session at 200 req/s
against the resident 40k-vector gallery, p50/p99 latency) and `cpu_baseline`
(the FP64 oracle's whole Algorithm 1 on the same instance on the host cores).
With N > 1 (torchrun) every rank runs an independent replica (the method
needs no exchange between instances), the time is the max over ranks and
`value` divides it by all ranks' re-ranks.  `--impl reference` times the
FP64 oracle's whole Algorithm 1 on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "market": dict(spec="MARKET_SCALE", k1=26, k2=7, layers=2),
    "large50k": dict(spec="LARGE_50K", k1=26, k2=7, layers=2),
    "tiny": dict(spec="TINY", k1=26, k2=7, layers=2),
    "market_hard": dict(spec="MARKET_HARD", k1=26, k2=7, layers=2),
    "batched64": dict(spec=None, k1=0, k2=0, layers=0),
    "serving": dict(spec=None, k1=26, k2=7, layers=2),
}
METRIC = "ms per N=23.1k re-rank (FP32 vs BF16+FP32 rescore); served p50/p99 ms; %roofline"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# Arm "CPU part" numbers of the cores this may run on (from Arm's published part list).
_ARM_PARTS = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1", "0xd49": "Neoverse-N2",
              "0xd83": "Neoverse-V3"}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name"):
                    return line.split(":", 1)[1].strip()
                if low.startswith("cpu part"):
                    part = line.split(":", 1)[1].strip().lower()
                    return f"Arm {_ARM_PARTS.get(part, 'core')} (CPU part {part})"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _blas_threads():
    threads = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        threads = max((i.get("num_threads", 1) for i in threadpool_info()), default=threads)
    except ImportError:
        pass
    return threads


def cpu_oracle_full(xq, xg, k1, k2, layers):
    """One run of the FP64 oracle's whole Algorithm 1 (sparse mode: Eq. 7-8 S
    rows with a full stable sort per row, A and A*, k2-edge weights, L layers
    of Eq. 14, cos(h_q, h_g) and a full stable sort per query) on the real
    instance, on the host cores.  Returns (ms, per-stage ms)."""
    from oracle import rerank_oracle
    t = {}
    t0 = time.perf_counter()
    rerank_oracle.rerank(xq, xg, k1=k1, k2=k2, layers=layers, mode="sparse", timings=t)
    ms = (time.perf_counter() - t0) * 1e3
    return ms, {k: v * 1e3 for k, v in t.items()}


def _cpu_sample_text(n, nq, ng, d):
    return (f"whole Algorithm 1 by the FP64 oracle (sparse mode) on the full instance, {nq} + {ng} = {n} "
            f"vectors, d={d}: no row sampling, no scaling; {os.cpu_count()} host cores "
            f"({_cpu_model()}); BLAS threads {_blas_threads()}, per-row sorts single-threaded")


def run_reference(args, world, rank):
    """The reference arm: the oracle's whole Algorithm 1, one run per step.  A
    run takes tens of seconds, so the arm runs as many of the requested
    warm-up steps as fit in a quarter of --ref-seconds (at least one) and as
    many timed steps as fit in the rest (at least one), and reports the counts
    it really ran."""
    from paper_2012_07620_gb300 import synthetic
    wl = WORKLOADS[args.workload]
    if rank != 0:
        return
    w = synthetic.make_workload(getattr(synthetic, wl["spec"]))
    k1, k2, L = wl["k1"], wl["k2"], wl["layers"]
    t_start = time.perf_counter()
    warm, run_ms = 0, None
    for _ in range(args.warmup):
        # warm-ups take at most a quarter of the budget (the first one always runs)
        if run_ms is not None and (time.perf_counter() - t_start) + run_ms / 1e3 > args.ref_seconds / 4:
            break
        run_ms, _ = cpu_oracle_full(w.xq, w.xg, k1, k2, L)
        warm += 1
    vals, stages = [], {}
    for _ in range(args.steps):
        if vals and (time.perf_counter() - t_start) + float(np.mean(vals)) / 1e3 > args.ref_seconds:
            break
        v, st = cpu_oracle_full(w.xq, w.xg, k1, k2, L)
        vals.append(v)
        for k, x in st.items():
            stages[k] = stages.get(k, 0.0) + x
    ms = float(np.mean(vals))
    stages = {k: x / len(vals) for k, x in stages.items()}
    n, d = len(w.xq) + len(w.xg), w.spec.dim
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": len(vals), "warmup": warm, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(args, w),
            "requested": {"steps": args.steps, "warmup": args.warmup, "budget_s": args.ref_seconds},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": _blas_threads(), "kind": "oracle",
                             "sample": _cpu_sample_text(n, len(w.xq), len(w.xg), d), "stages_ms": stages,
                             "cpu_model": _cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _config(args, w):
    spec = w.spec
    return {"workload": f"{spec.name}: {spec.n_query} queries + {spec.n_gallery} gallery, d={spec.dim}, "
                        f"{spec.n_clusters} clusters + {spec.n_distractors} distractors, "
                        f"k1={WORKLOADS[args.workload]['k1']}, k2={WORKLOADS[args.workload]['k2']}, "
                        f"L={WORKLOADS[args.workload]['layers']}, full ranked lists",
            "n_vertices": spec.n, "dim": spec.dim, "precision": args.precision,
            "l2": "flushed before every step (256 MiB write)", "parallelism": f"replicas x{args.gpus}"}


# DRAM bytes (read + write) of one similarity launch, from `ncu --set full` captures
# of the current kernel (profiles/); None where no capture of it exists.
SIM_TRAFFIC_BYTES = {("bf16", "market"): 314.9e6}  # profiles/k1_tc2_topk_bf16_market_23k_d2048.md
# DRAM bytes of the refinement's first pass, same source
# (profiles/k2_refine_cta_bf16_market_23k_d2048.md).
REFINE_DRAM_BYTES = {("bf16", "market"): 1.682e9}


def _stage_rooflines(precision, stages, nq, ng, d, k1, k2, rescore_m, h_nnz, layers, workload):
    """Bytes each memory-side stage must move at least, against the measured
    copy bandwidth.  normalize: the FP32 rows read once, the unit rows and
    their low-precision copies written once (rows padded to the tile);
    propagate: per layer, the k2 + 1 message rows of every row gathered (on
    average k2 + 1 times each input row) and the output written, CSR entries
    of 8 bytes; rank: the ranked lists written (index + distance).
    refine is a gather: its floor is every distinct FP32 unit row read once
    (N d_p 4 bytes); the rows its first rescoring batch gathers (most served
    by L1/L2) are reported as a gather rate, not as a fraction of HBM."""
    peaks, which = _peaks()
    hbm = peaks["hbm_gbs"]
    n = nq + ng
    tc = precision != "fp32"
    np_ = -(-n // (256 if tc else 128)) * (256 if tc else 128)
    dp = -(-d // (128 if precision == "fp8" else 64)) * (128 if precision == "fp8" else 64)
    per_el = {"fp32": 4, "bf16": 8, "fp8": 9}[precision]
    first = min(k1 + max(rescore_m, 0), (k1 + 7) & ~3)
    out = {}
    byts = {"normalize": n * d * 4 + np_ * dp * per_el,
            "propagate": sum(((k2 + 1) * h_nnz[l - 1] + h_nnz[l]) * 8 for l in range(1, min(layers, 8) + 1)),
            "rank": nq * ng * 8}
    for k, b in byts.items():
        ms = stages.get(k)
        if not ms or b <= 0:
            continue
        gbs = b / (ms * 1e-3) / 1e9
        out[k] = {"bytes": int(b), "ms": ms, "achieved_gbs": gbs, "frac_of_hbm": gbs / hbm}
    ms = stages.get("refine")
    if ms:
        floor = n * dp * 4
        gathered = n * first * dp * 4
        out["refine"] = {"ms": ms, "floor_bytes": int(floor),
                         "floor_frac_of_hbm": floor / (ms * 1e-3) / 1e9 / hbm,
                         "gathered_bytes": int(gathered), "gather_rate_gbs": gathered / (ms * 1e-3) / 1e9,
                         "dram_bytes_ncu": REFINE_DRAM_BYTES.get((precision, workload)),
                         "note": "gather rate of candidate rows (mostly L1/L2 hits), not an HBM fraction"}
    out["peak_gbs"] = hbm
    out["peak_source"] = f"{which} copy bandwidth"
    return out


def _roofline(precision, sim_ms, n, d, workload):
    """Roofline of the dominant kernel, the similarity GEMM with its fused top-K:
    2 n^2 d flops per launch (the full square; the kernel computes every tile)."""
    peaks, which = _peaks()
    flops = 2.0 * n * n * d
    achieved = flops / (sim_ms * 1e-3) / 1e12
    if precision == "fp32":
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"FP32 FMA pipe: 152 SMs x 128 lanes x 2 flop x {mhz} MHz (derived)"}
    else:
        peak = peaks["bf16_tflops"] * (2.0 if precision == "fp8" else 1.0)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"{which} bf16 burst" + (" x2 (fp8 nominal ratio)" if precision == "fp8" else "")}
    roof["frac"] = achieved / peak
    roof["traffic"] = SIM_TRAFFIC_BYTES.get((precision, workload))
    roof["kernel"] = "similarity_topk (k1_tc_topk / k1_sim_fp32)"
    roof["flops_per_launch"] = flops
    return roof


def _tune(rerank, local, precision, xq, xg, k1, k2, L, path):
    """Launch shapes from the autotuner, measured on this instance before any timed region."""
    T = rerank.Reranker(device=local, precision=precision, autotune_path=path)
    tuned = T.autotune(xq, xg, k1, k2, L)
    T.close()
    return tuned


def _time_instance(rerank, local, precision, xq, xg, k1, k2, L, steps, warmup, stream, flush, tune_path,
                   world=1, feature="astar"):
    """CUDA-event time of `steps` re-ranks (after `warmup`), L2 flushed before
    each; per-stage times from the library's own events.  Returns a dict."""
    import torch
    nq, ng = xq.shape[0], xg.shape[0]
    out_i = torch.empty((nq, ng), dtype=torch.int32, device=xq.device)
    out_d = torch.empty((nq, ng), dtype=torch.float32, device=xq.device)
    R = rerank.Reranker(device=local, precision=precision, stage_timing=True, autotune_path=tune_path,
                        feature=feature)
    for _ in range(warmup):
        R.run(xq, xg, k1, k2, L, 0, out_i, out_d, stream)
    launches = R.last_info()["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stage_sum = {}
    _barrier(world)
    torch.cuda.synchronize()
    for s in range(steps):
        flush.fill_(s & 255)
        ev[s][0].record(stream)
        R.run(xq, xg, k1, k2, L, 0, out_i, out_d, stream)
        ev[s][1].record(stream)
        for k, v in R.stage_times().items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v
    torch.cuda.synchronize()
    _barrier(world)
    total = _max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
    info = R.last_info()
    R.close()
    return {"ms": total / steps, "stages_ms": {k: v / steps for k, v in stage_sum.items()}, "steps": steps,
            "launches_per_step": int(launches), "fp64_rescored": info["fp64_rescored"],
            "fallback_rows": info["fallback_rows"], "exact_scan_rows": info["exact_scan_rows"],
            "h_nnz": info["h_nnz"]}


def measure_workload(rerank, synthetic, local, dev, spec_name, precisions, steps, warmup, stream, flush,
                     tune_dir, k1=26, k2=7, L=2, workload_key="market"):
    """Each precision on one workload (autotuned first), with its roofline."""
    import torch
    w = synthetic.make_workload(getattr(synthetic, spec_name))
    xq = torch.from_numpy(w.xq).to(dev)
    xg = torch.from_numpy(w.xg).to(dev)
    nq, ng, d = len(w.xq), len(w.xg), w.spec.dim
    res = {"workload": f"{w.spec.name}: {nq} queries + {ng} gallery, d={d}, {w.spec.n_clusters} clusters + "
                       f"{w.spec.n_distractors} distractors, k1={k1}, k2={k2}, L={L}, full ranked lists"}
    for prec in precisions:
        path = os.path.join(tune_dir, f"tune_{spec_name}_{prec}.json")
        with ClockSampler(local) as clocks:
            tuned = _tune(rerank, local, prec, xq, xg, k1, k2, L, path)
            st = steps if prec != "fp32" else max(1, min(steps, 5))
            r = _time_instance(rerank, local, prec, xq, xg, k1, k2, L, st, warmup, stream, flush, path)
        r["roofline"] = _roofline(prec, r["stages_ms"].get("similarity_topk", float("nan")), nq + ng, d,
                                  workload_key)
        r["autotune"] = tuned
        r["clocks"] = clocks.summary()
        res[prec] = r
    del xq, xg
    torch.cuda.empty_cache()
    return res


def batched_measure(rerank, synthetic, local, dev, precision, steps, warmup, stream, flush, world=1):
    """64 independent instances (N log-uniform 500-8000, d in {256, 512, 2048}, BF16 features)
    per step through one rerank_run_batch call; beside it the same 64 as sequential rerank_run calls."""
    import torch
    specs = synthetic.batched_specs()
    jobs, host = [], []
    for s in specs:
        w = synthetic.make_workload(s["spec"])
        xq = torch.from_numpy(w.xq).bfloat16()
        xg = torch.from_numpy(w.xg).bfloat16()
        nq, ng = xq.shape[0], xg.shape[0]
        jobs.append(dict(xq=xq.to(dev), xg=xg.to(dev), k1=s["k1"], k2=s["k2"], layers=s["layers"],
                         out_idx=torch.empty((nq, ng), dtype=torch.int32, device=dev),
                         out_dist=torch.empty((nq, ng), dtype=torch.float32, device=dev)))
        host.append(dict(xq=xq.pin_memory(), xg=xg.pin_memory(), k1=s["k1"], k2=s["k2"], layers=s["layers"],
                         out_idx=torch.empty((nq, ng), dtype=torch.int32).pin_memory(),
                         out_dist=torch.empty((nq, ng), dtype=torch.float32).pin_memory()))
    flops = sum(2.0 * (j["xq"].shape[0] + j["xg"].shape[0]) ** 2 * j["xq"].shape[1] for j in jobs)
    # Launch shapes from the autotuner: one tuning run per (d, half-octave of N) among the instances.
    tune_path = os.path.join(tempfile.mkdtemp(), "tune.json")
    t_tune = time.perf_counter()
    T = rerank.Reranker(device=local, precision=precision, autotune_path=tune_path)
    seen = set()
    for j in jobs:
        n = j["xq"].shape[0] + j["xg"].shape[0]
        key = (j["xq"].shape[1], int(np.floor(2 * np.log2(n))))
        if key not in seen:
            seen.add(key)
            T.autotune(j["xq"], j["xg"], j["k1"], j["k2"], j["layers"])
    T.close()
    t_tune = time.perf_counter() - t_tune
    R = rerank.Reranker(device=local, precision=precision, autotune_path=tune_path)

    def timed(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for _ in range(warmup):
            fn()
        _barrier(world)
        torch.cuda.synchronize()
        for s in range(steps):
            flush.fill_(s & 255)
            ev[s][0].record(stream)
            fn()
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        _barrier(world)
        return _max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world) / steps

    def sequential():
        for j in jobs:
            R.run(j["xq"], j["xg"], j["k1"], j["k2"], j["layers"], 0, j["out_idx"], j["out_dist"], stream)

    with ClockSampler(local) as clocks:
        batch_ms = timed(lambda: R.run_batch(jobs, stream))
        launches = R.last_info()["kernel_launches"]
    seq_ms = timed(sequential)
    R.run_batch(host, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(steps, 5))
    for _ in range(e2e_steps):
        R.run_batch(host, stream)
    e2e_ms = _max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps, world)
    R.close()
    peaks, which = _peaks()
    n_tot = sum(j["xq"].shape[0] + j["xg"].shape[0] for j in jobs)
    return {"batch_ms": batch_ms, "sequential_ms": seq_ms, "speedup_vs_sequential": seq_ms / batch_ms,
            "steps": steps, "launches_per_step": int(launches),
            "workload": f"64 instances, N log-uniform 500-8000 (total {n_tot}), d in {{256, 512, 2048}}, "
                        "BF16 features, k1 20-30, k2 5-7, 1-3 layers, full ranked lists",
            "gemm_tflop": flops / 1e12, "autotune": {"entries": len(seen), "seconds": t_tune},
            "instances_per_s": 64.0 * world / (batch_ms * 1e-3),
            "e2e": {"value": e2e_ms, "unit": "ms",
                    "h2d_bytes_per_step": int(sum(h["xq"].numel() * 2 + h["xg"].numel() * 2 for h in host)),
                    "d2h_bytes_per_step": int(sum(h["out_idx"].numel() * 8 for h in host))},
            "clocks": clocks.summary(),
            "roofline": {"bound": "tensor", "achieved": flops / (batch_ms * 1e-3) / 1e12,
                         "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": flops / (batch_ms * 1e-3) / 1e12 / peaks["bf16_tflops"], "traffic": None,
                         "kernel": "whole batch (GEMM flops / batch time)", "peak_source": f"{which} bf16 burst"}}


def run_batched(args, world, rank, local):
    import torch
    import __graft_entry__
    from paper_2012_07620_gb300 import rerank, synthetic

    __graft_entry__.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    b = batched_measure(rerank, synthetic, local, dev, args.precision, args.steps, args.warmup, stream, flush,
                        world)
    line = {"metric": "ms per batch of 64 independent re-ranks (rerank_run_batch) vs 64 sequential rerank_run",
            "value": b["batch_ms"] / world, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["batch_ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": b["workload"], "gemm_tflop": b["gemm_tflop"],
                       "l2": "flushed before every step (256 MiB write)", "parallelism": f"replicas x{world}"},
            "sequential_ms": b["sequential_ms"], "speedup_vs_sequential": b["speedup_vs_sequential"],
            "autotune": b["autotune"], "instances_per_s": b["instances_per_s"], "e2e": b["e2e"],
            "gpu_launches": int(b["launches_per_step"] * args.steps), "clocks": b["clocks"],
            "roofline": b["roofline"]}
    if rank == 0:
        print(json.dumps(line))


def serving_session(rerank, synthetic, dev, seconds, rate=200.0, precision="bf16", slots=0, stream=None):
    """Poisson arrivals against the resident 40,000 x 2048 BF16 gallery; each request
    brings 1-512 queries (log-uniform), k1=26, k2=7, 2 layers, top-100 lists.
    Returns a dict of latency percentiles and throughput."""
    import torch
    w = synthetic.make_workload(synthetic.SERVING_GALLERY)
    reqs = synthetic.serving_requests(w, rate_hz=rate, duration_s=seconds)
    # A pool of query rows drawn around the gallery's identities; request r takes
    # nq rows at a request-specific offset (fresh rows for every request would
    # cost the generator minutes, not the GPU).
    pool_rows = 4096
    pool = torch.from_numpy(synthetic.request_queries(w, 0, pool_rows)).bfloat16().to(dev)
    xg = torch.from_numpy(w.xg).bfloat16().to(dev)
    budget = 80 << 30
    R = rerank.Reranker(device=dev.index or 0, precision=precision, hbm_budget=budget)
    t_load = time.perf_counter()
    R.load_gallery(xg, max_query=512, k1=26, k2=7, layers=2, slots=slots)
    t_load = time.perf_counter() - t_load
    torch.cuda.synchronize()
    # warm-up requests (first launches, lazy module loading)
    for q in (1, 64, 512):
        t, _, _ = R.submit(pool[:q], 100)
        R.wait(t)
    tickets = []
    lat, qms = [], []
    done = threading.Event()

    def waiter():
        k = 0
        while True:
            while k >= len(tickets):
                if done.is_set() and k >= len(tickets):
                    return
                time.sleep(0.0005)
            info = R.wait(tickets[k])
            lat.append(info["total_ms"])
            qms.append(info["queue_ms"])
            k += 1

    th = threading.Thread(target=waiter)
    th.start()
    t0 = time.perf_counter()
    for r in reqs:
        delay = r["t_arrival"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        nq = r["n_query"]
        off = (r["request_id"] * 2654435761) % (pool_rows - nq + 1)
        t, _, _ = R.submit(pool[off:off + nq], 100)
        tickets.append(t)
    done.set()
    th.join()
    wall = time.perf_counter() - t0
    info = R.serve_info()
    R.close()
    lat = np.array(lat)
    nqs = np.array([r["n_query"] for r in reqs])
    return {"requests": len(reqs), "seconds": seconds, "rate_hz": rate, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "queue_p99_ms": float(np.percentile(qms, 99)), "requests_per_s": len(reqs) / wall,
            "queries_per_request_mean": float(nqs.mean()), "slots": info["slots"],
            "max_in_flight": info["max_in_flight"], "touched_rows_per_request": info["touched_rows"] / max(1, info["completed"]),
            "layer_reuse": bool(info["reuse_layers"]),
            "recomputed_layer_rows_per_request": info["recomputed_rows"] / max(1, info["completed"]),
            "slot_bytes": info["slot_bytes"], "resident_bytes": info["resident_bytes"], "gallery_load_s": t_load,
            "workload": "resident gallery 40,000 x 2048 BF16 (2,500 clusters x 16); Poisson arrivals; 1-512 "
                        "queries per request (log-uniform) from a 4,096-row pool around the gallery's identities; "
                        "k1=26, k2=7, L=2, top-100 lists; hbm_budget 80 GB",
            "latency": "submit -> results in device memory, host steady clock"}


def run_serving(args, world, rank, local):
    import torch
    import __graft_entry__
    from paper_2012_07620_gb300 import rerank, synthetic

    __graft_entry__.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    precision = args.precision if args.precision != "fp32" else "bf16"
    with ClockSampler(local) as clocks:
        res = serving_session(rerank, synthetic, dev, args.serve_seconds, precision=precision)
    line = {"metric": "served re-rank latency p50 (ms), Poisson 200 req/s on a 40k resident gallery",
            "value": res["p50_ms"], "unit": "ms", "n_gpus": world, "steps": res["requests"], "warmup": 3,
            "ms_per_step": res["mean_ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": precision, "data": "synthetic",
            "config": {"workload": res["workload"], "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (gallery 164 MB BF16 + slot copies)"},
            "p99_ms": res["p99_ms"], "requests_per_s": res["requests_per_s"], "serving": res,
            "clocks": clocks.summary()}
    if rank == 0:
        print(json.dumps(line))


def run_ours(args, world, rank, local):
    import torch
    import __graft_entry__
    from paper_2012_07620_gb300 import rerank, synthetic

    __graft_entry__.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]
    w = synthetic.make_workload(getattr(synthetic, wl["spec"]))
    k1, k2, L = wl["k1"], wl["k2"], wl["layers"]
    nq, ng, d = len(w.xq), len(w.xg), w.spec.dim
    xq = torch.from_numpy(w.xq).to(dev)
    xg = torch.from_numpy(w.xg).to(dev)
    out_i = torch.empty((nq, ng), dtype=torch.int32, device=dev)
    out_d = torch.empty((nq, ng), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    tune_dir = tempfile.mkdtemp()
    tune_path, tuned = None, None
    if args.tune_file and os.path.exists(args.tune_file):
        # Launch shapes from an earlier run's table (e.g. to profile the shapes a bench run chose).
        tune_path = args.tune_file
        tuned = rerank.tuning_lookup(tune_path, args.precision, nq + ng, d)
    elif not args.no_autotune:
        tune_path = args.tune_file or os.path.join(tune_dir, "tune.json")
        tuned = _tune(rerank, local, args.precision, xq, xg, k1, k2, L, tune_path)
    R = rerank.Reranker(device=local, precision=args.precision, stage_timing=True, autotune_path=tune_path)

    for _ in range(args.warmup):
        R.run(xq, xg, k1, k2, L, 0, out_i, out_d, stream)
    launches = R.last_info()["kernel_launches"]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_sum = {}
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for s in range(args.steps):
            flush.fill_(s & 255)
            ev[s][0].record(stream)
            R.run(xq, xg, k1, k2, L, 0, out_i, out_d, stream)
            ev[s][1].record(stream)
            for k, v in R.stage_times().items():
                stage_sum[k] = stage_sum.get(k, 0.0) + v
        torch.cuda.synchronize()
    _barrier(world)
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms = _max_over_ranks(total_ms, world)
    ms = total_ms / (args.steps * world)
    stages = {k: v / args.steps for k, v in stage_sum.items()}

    # End to end through the C ABI with pinned host buffers.
    hq = torch.from_numpy(w.xq).pin_memory()
    hg = torch.from_numpy(w.xg).pin_memory()
    ho_i = torch.empty((nq, ng), dtype=torch.int32).pin_memory()
    ho_d = torch.empty((nq, ng), dtype=torch.float32).pin_memory()
    R.run(hq, hg, k1, k2, L, 0, ho_i, ho_d, stream)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        R.run(hq, hg, k1, k2, L, 0, ho_i, ho_d, stream)  # returns after the results are in host memory
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = float(np.median(e2e_times))  # host-clock noise: the median step
    e2e_ms = _max_over_ranks(e2e_ms, world) / world

    n = nq + ng
    roof = _roofline(args.precision, stages.get("similarity_topk", float("nan")), n, d, args.workload)

    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms * world, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
            "data": "synthetic", "config": _config(args, w),
            "e2e": {"value": e2e_ms, "unit": "ms", "steps": e2e_steps, "statistic": "median",
                    "h2d_bytes_per_step": int(hq.numel() * 4 + hg.numel() * 4),
                    "d2h_bytes_per_step": int(ho_i.numel() * 4 + ho_d.numel() * 4)},
            "roofline": roof, "stages_ms": stages, "gpu_launches": int(launches * args.steps),
            "clocks": clocks.summary(), "autotune": tuned}
    info = R.last_info()
    m_used = (tuned or {}).get("rescore_m", -1)
    line["stage_rooflines"] = _stage_rooflines(args.precision, stages, nq, ng, d, k1, k2,
                                               m_used if m_used is not None and m_used >= 0 else 16,
                                               info["h_nnz"], L, args.workload)
    line["fp64_rescored"] = info["fp64_rescored"]
    line["fallback_rows"] = info["fallback_rows"]
    line["exact_scan_rows"] = info["exact_scan_rows"]
    R.close()
    del hq, hg, ho_i, ho_d, out_i, out_d
    extras = world == 1 and not args.no_extras
    if extras:
        # The other precisions on the same instance, each autotuned, with its own roofline.
        for prec in ("fp32", "fp8"):
            if prec == args.precision or (prec == "fp32" and args.no_fp32_path):
                continue
            path = os.path.join(tune_dir, f"tune_{prec}.json")
            with ClockSampler(local) as ck:
                ptuned = _tune(rerank, local, prec, xq, xg, k1, k2, L, path)
                r = _time_instance(rerank, local, prec, xq, xg, k1, k2, L,
                                   args.steps if prec != "fp32" else max(1, min(args.steps, 5)),
                                   args.warmup, stream, flush, path)
            r["roofline"] = _roofline(prec, r["stages_ms"].get("similarity_topk", float("nan")), n, d,
                                      args.workload)
            r["autotune"] = ptuned
            r["clocks"] = ck.summary()
            r[f"speedup_of_{args.precision}"] = r["ms"] / ms
            line[f"{prec}_path"] = r
        # Dense x_i initial features (Table 1, first column) on the same instance:
        # dense layers, final cosines over d (2 Q G d flop) and a radix ranking.
        with ClockSampler(local) as ck:
            r = _time_instance(rerank, local, args.precision, xq, xg, k1, k2, L, max(1, min(args.steps, 5)),
                               args.warmup, stream, flush, tune_path, feature="x")
        r["clocks"] = ck.summary()
        r["final_cosines_tflop"] = 2.0 * nq * ng * d / 1e12
        line["x_features"] = r
    del xq, xg
    torch.cuda.empty_cache()
    if extras and args.workload == "market":
        line["large_50k"] = measure_workload(rerank, synthetic, local, dev, "LARGE_50K", ("bf16", "fp8", "fp32"),
                                             args.steps, args.warmup, stream, flush, tune_dir,
                                             workload_key="large50k")
        torch.cuda.empty_cache()
        b = batched_measure(rerank, synthetic, local, dev, "bf16", args.steps, args.warmup, stream, flush)
        line["batched64"] = b
        torch.cuda.empty_cache()
    if extras and args.serve_seconds_default > 0 and args.workload == "market":
        try:
            line["serving"] = serving_session(rerank, synthetic, dev, args.serve_seconds_default,
                                              precision=args.precision if args.precision != "fp32" else "bf16")
        except Exception as e:  # reported, never fatal for the headline line
            line["serving"] = {"error": repr(e)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, st = cpu_oracle_full(w.xq, w.xg, k1, k2, L)
        line["cpu_baseline"] = {"value": v, "unit": "ms", "cores": _blas_threads(), "kind": "oracle",
                                "sample": _cpu_sample_text(n, nq, ng, d), "stages_ms": st,
                                "cpu_model": _cpu_model(), "nproc": os.cpu_count()}
    if rank == 0:
        print(json.dumps(line))


def run_sweep(args, world, rank, local):
    """Synthetic accuracy sweeps (no timing): mAP and Rank-1 of the re-ranked
    lists against the identity labels, for the layer count L (Table 2's trend)
    or for (k1, k2) around the Eq. 15 value, beside the initial cosine ranking."""
    import torch
    from paper_2012_07620_gb300 import metrics, rerank, synthetic
    if rank != 0:
        return
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]
    w = synthetic.make_workload(getattr(synthetic, wl["spec"]))
    nq, ng = len(w.xq), len(w.xg)
    xq = torch.from_numpy(w.xq).to(dev)
    xg = torch.from_numpy(w.xg).to(dev)
    # initial ranking: cosine of the (unit) input rows, ties to the lower index
    s0 = w.xq.astype(np.float32) @ w.xg.astype(np.float32).T
    base = metrics.retrieval_metrics(np.argsort(-s0, axis=1, kind="stable"), w.yq, w.yg)
    del s0
    k1r = metrics.k1_from_classes(nq + ng, w.spec.n_clusters)
    if args.sweep == "layers":
        grid = [(wl["k1"], wl["k2"], L) for L in range(0, 5)]
    else:
        grid = [(k1, k2, wl["layers"]) for k1 in sorted({max(2, k1r // 2), k1r, wl["k1"], 2 * k1r})
                for k2 in (3, 5, 7, 10) if k2 <= k1]
    rows = []
    with rerank.Reranker(device=local, precision=args.precision) as R:
        for k1, k2, L in grid:
            idx, _ = R.run(xq, xg, k1, k2, L)
            torch.cuda.synchronize()
            m = metrics.retrieval_metrics(idx.cpu().numpy(), w.yq, w.yg)
            rows.append({"k1": k1, "k2": k2, "layers": L, "mAP": round(m["mAP"], 4), "R1": round(m["R1"], 4)})
    print(json.dumps({"sweep": args.sweep, "workload": wl["spec"], "precision": args.precision,
                      "data": "synthetic", "k1_eq15": k1r,
                      "initial_ranking": {"mAP": round(base["mAP"], 4), "R1": round(base["R1"], 4)},
                      "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--workload", default="market", choices=list(WORKLOADS))
    ap.add_argument("--ref-seconds", type=float, default=200.0,
                    help="reference arm: wall-time budget for its warm-up and timed oracle runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline line: no other precisions, 50k, batched or serving keys")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-seconds-default", type=float, default=60.0,
                    help="length of the serving session added to the market line (0 = none)")
    ap.add_argument("--no-fp32-path", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes instead of autotuned ones")
    ap.add_argument("--tune-file", default=None,
                    help="autotuner table: used as is when the file exists, else written by this run's tuning")
    ap.add_argument("--sweep", default=None, choices=["layers", "k1k2"],
                    help="synthetic accuracy sweep (mAP / Rank-1) instead of the timed run; "
                         "use with --workload market_hard (the default set is separable)")
    args = ap.parse_args()
    world, rank, local = _dist_setup()
    if args.sweep:
        run_sweep(args, world, rank, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched64":
        run_batched(args, world, rank, local)
    elif args.workload == "serving":
        run_serving(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
