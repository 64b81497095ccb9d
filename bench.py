#!/usr/bin/env python3
"""Benchmark of the particle-particle ladder (R += sum_cd (ac|bd) t2) on GB300.

One step = one ladder_apply (all steps of the hot path: operand preparation,
Cholesky->ERI GEMM, ladder GEMM, a<=b unpack) on the synthetic workload.
Default workload: no=20, nv=400, nchol=1260 (seed 1237), the nv = 400 shape
the tensor-roofline target is stated at, emulated FP64 (BF16 digit slices)
with the ladder form the planner picks; seeded generators of ``ladder_inputs``.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision emu|fp64]
                    [--config c3] [--impl ours|reference] [--mode replicas|shard]

Prints one JSON line (rank 0).  ``value`` = algorithmic TFLOP/s
(2 X v^2 p + 2 o^2 v^2 p with p = v(v+1)/2, per instance) summed over ranks,
timed with CUDA events on the launching stream between barriers, max over
ranks; inputs resident in HBM.  ``e2e`` repeats the measurement through the
same public call with the inputs copied from pinned host memory and R read
back every step.  ``fp64`` times the native FP64 (DMMA) path on the same
workload (``speedup_vs_fp64`` = its ms/call over the emulated one) and
``accuracy`` states both results' error against the CPU oracle: sampled
(a, b) pairs against the oracle's pair mode, E_L against the stored oracle
value, and the whole R of one path against the other.  Multi-GPU runs
(torchrun): ``--mode shard`` (default) splits one contraction's block pairs
over the ranks (ladder_plan_shard) and sums E_L with one scalar all-reduce
(strong scaling); ``--mode replicas`` gives each rank its own independent
instance (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from ladder_inputs import CONFIGS, LadderShape, make_inputs  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
NOMINAL_BF16_TFLOPS = 2250.0
NOMINAL_FP64_TFLOPS = 1.25


# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant
# kernel, from a single-pass capture of this workload.  It is reported only while the sources
# holding device code hash to the value recorded with the capture and the plan has the blocking
# it had then; any change to either makes it null.
TRAFFIC_CAPTURES = {
    # (precision, workload): (device sources sha256 prefix, bytes per launch, profiles/ summary,
    #                         (n_a, n_b))
    ("emu", "c2"): ("efd514e3bd5bd3a9", 12063834880 + 10939927808, "profiles/dram_traffic_no10_nv200_nchol630.md",
                    (200, 200)),
    ("fp64", "c2"): ("efd514e3bd5bd3a9", 49657817856 + 6438093312, "profiles/dram_traffic_no10_nv200_nchol630.md",
                     (200, 200)),
    # mean of the call's two ERI launches (20100 and 60100 pair rows)
    ("emu", "c3"): ("97af10a6ecc01af8", (118275270912 + 32870906112 + 308907295488 + 93364802304) // 2,
                    "profiles/dram_traffic_no20_nv400_nchol1260_emu.md", (400, 200)),
}
KERNEL_SOURCE_DIR = os.path.join(ROOT, "paper_2603_20912_gb300", "csrc")
HOST_ONLY_SOURCES = {"api.cu"}   # the planner and the C ABI glue: no device code


def kernel_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in sorted(os.listdir(KERNEL_SOURCE_DIR)):
        if name.endswith((".cu", ".cuh", ".h")) and name not in HOST_ONLY_SOURCES:
            with open(os.path.join(KERNEL_SOURCE_DIR, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def captured_traffic(precision: str, workload: str, blocking):
    rec = TRAFFIC_CAPTURES.get((precision, workload))
    if rec is None or rec[0] != kernel_sources_sha() or tuple(rec[3]) != tuple(blocking):
        return None, None
    return rec[1], rec[2]


def eri_products(nv: int, n_a: int, n_b: int) -> int:
    """Row-column products (each over K = nchol) that the emulated ERI of one call needs, for
    the blocking n_a x n_b (blocks: b outer, a inner, kept when they hold a pair a <= b).  L^P is
    symmetric, so only the rows (x, y) of L^T with x <= y are multiplied: a block with a range
    [a0, a1) uses the rows (x, [x, nv)) for x in the range, which store to V rows (x, b >= x),
    and (x, [a0, a1)) for x < a0, which store to (y, b >= y); each row meets the nv columns (b, d)
    of every b in the block's b range at or above that first index."""
    total = 0
    for b0 in range(0, nv, n_b):
        b1 = min(nv, b0 + n_b)
        for a0 in range(0, nv, n_a):
            a1 = min(nv, a0 + n_a)
            if a0 > b1 - 1:
                continue
            for x in range(a0, a1):
                total += (nv - x) * nv * max(0, b1 - max(b0, x))
            for y in range(a0, a1):
                total += a0 * nv * max(0, b1 - max(b0, y))
    return total


def ladder_products(no: int, nv: int, form: str) -> int:
    """Row-column products of the ladder GEMM of one call over all a <= b pairs: rows (i,j) and
    K = (c,d) in the plain form; rows i <= j with K = c <= d plus rows i < j with K = c < d in the
    symmetric/antisymmetric form."""
    pairs = nv * (nv + 1) // 2
    if form == "pm":
        return pairs * ((no * (no + 1) // 2) * (nv * (nv + 1) // 2) + (no * (no - 1) // 2) * (nv * (nv - 1) // 2))
    return pairs * no * no * nv * nv


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": FALLBACK_BF16_TFLOPS,
                "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
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
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline_sample(L, t2, target_s=15.0):
    """Time the oracle (as it stands) on a bounded sample of (a, b) pairs."""
    import oracle
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    per_pair = 2.0 * nchol * nv * nv + 2.0 * no * no * nv * nv
    rng = np.random.default_rng(7)
    n = max(1, oracle.num_threads())
    a = rng.integers(0, nv, n)
    b = rng.integers(0, nv, n)
    t0 = time.perf_counter()
    oracle.ladder_pairs(L, t2, a, b)
    dt = time.perf_counter() - t0
    n2 = int(max(1, min(nv * nv, n * max(1.0, target_s / max(dt, 1e-3)))))
    a = rng.integers(0, nv, n2)
    b = rng.integers(0, nv, n2)
    t0 = time.perf_counter()
    oracle.ladder_pairs(L, t2, np.minimum(a, b), np.maximum(a, b))
    dt = time.perf_counter() - t0
    return {"value": n2 * per_pair / dt / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n2} random (a<=b) pairs of the workload, all (i,j), {dt:.1f} s wall"}, n2, dt


def run_reference(args, cfg):
    """The CPU oracle as the reference arm (rank 0 only)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    L, t2, _, _ = make_inputs(cfg.no, cfg.nv, cfg.nchol, cfg.seed)
    import oracle
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    per_pair = 2.0 * nchol * nv * nv + 2.0 * no * no * nv * nv
    rng = np.random.default_rng(11)
    # Size one step to ~ (few minutes / (steps + warmup)).
    n = max(1, oracle.num_threads())
    t0 = time.perf_counter()
    oracle.ladder_pairs(L, t2, rng.integers(0, nv, n), rng.integers(0, nv, n))
    probe = time.perf_counter() - t0
    step_s = min(20.0, 150.0 / max(1, args.steps + args.warmup))
    npairs = int(max(1, min(nv * nv, n * step_s / max(probe, 1e-3))))
    times = []
    for k in range(args.warmup + args.steps):
        a = rng.integers(0, nv, npairs)
        b = rng.integers(0, nv, npairs)
        t0 = time.perf_counter()
        oracle.ladder_pairs(L, t2, np.minimum(a, b), np.maximum(a, b))
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = args.steps * npairs * per_pair / tot / 1e12
    line = {
        "impl": "reference", "metric": "PP-ladder TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{cfg.name}: no={cfg.no} nv={cfg.nv} nchol={cfg.nchol} seed={cfg.seed}",
                   "sample_pairs_per_step": npairs},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{npairs} random (a<=b) pairs per step of {nv * (nv + 1) // 2}, all (i,j)"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_peaks():
    """Library matmul throughput on this GPU (context for the roofline denominators)."""
    import torch
    out = {}

    def timeit(fn, flops, reps):
        fn()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        return flops / best / 1e12

    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    out["fp64_matmul_tflops"] = timeit(lambda: a @ b, 2.0 * n ** 3, 3)
    del a, b
    a = torch.randn(n, n, dtype=torch.bfloat16, device="cuda")
    b = torch.randn(n, n, dtype=torch.bfloat16, device="cuda")
    out["bf16_matmul_tflops"] = timeit(lambda: a @ b, 2.0 * n ** 3, 10)
    del a, b
    try:
        a = torch.randint(-64, 64, (n, n), dtype=torch.int8, device="cuda")
        b = torch.randint(-64, 64, (n, n), dtype=torch.int8, device="cuda").t()
        out["int8_mm_tops"] = timeit(lambda: torch._int_mm(a, b), 2.0 * n ** 3, 10)
    except Exception as e:  # pragma: no cover - depends on the library build
        out["int8_mm_tops"] = f"unavailable: {e}"
    out["gpu"] = torch.cuda.get_device_name()
    out["sms"] = torch.cuda.get_device_properties(0).multi_processor_count
    print(json.dumps(out), flush=True)


def batched_record(args, lad, local, world, device_inputs, steps, warmup, fp64_sequential=False):
    """The 24-instance uneven batch (no ~ U{5..30}, nv ~ U{60..320}, nchol = 3(no+nv), seed 1239)
    in one ladder_apply_batched call per step: the measured tuner picks the schedule and the
    ladder tile width on these buffers, the call is captured once into a CUDA graph and replayed
    `steps` times after `warmup` replays, timed with CUDA events on the current stream."""
    import torch
    from ladder_inputs import batched_shapes, make_batched_inputs, make_device_inputs
    shapes = batched_shapes()
    if device_inputs:
        pairs = [make_device_inputs(s.no, s.nv, s.nchol, s.seed, device=f"cuda:{local}") for s in shapes]
        Ls = [L for L, _ in pairs]
        ts = [t for _, t in pairs]
    else:
        host = make_batched_inputs(shapes)
        Ls = [torch.from_numpy(L).cuda() for L, _ in host]
        ts = [torch.from_numpy(t).cuda() for _, t in host]
    Rs = [torch.zeros_like(t) for t in ts]
    precision = lad.LADDER_EMU_BF16 if args.precision == "emu" else lad.LADDER_FP64
    torch.cuda.empty_cache()
    plan = lad.ladder_plan_batched([s.no for s in shapes], [s.nv for s in shapes], [s.nchol for s in shapes],
                                   precision, nslices=args.nslices, device=local)
    ws = plan.workspace()
    scratch = [torch.zeros_like(t) for t in ts]
    k = lad.ladder_tune_batched(plan, Ls, ts, scratch, ws)
    del scratch
    flops = sum(lad.ladder_flops(s.no, s.nv, s.nchol) for s in shapes)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        lad.ladder_apply_batched(plan, Ls, ts, Rs, ws, stream=stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        lad.ladder_apply_batched(plan, Ls, ts, Rs, ws, stream=stream)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    barrier(world)
    sampler.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    ev0.record(cur)
    for _ in range(steps):
        g.replay()
    ev1.record(cur)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    assert plan.last_status() == lad.LADDER_OK
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world)
    value = world * flops * steps / (ms_total * 1e-3) / 1e12
    # Where a call's time goes: one more call, outside the graph and after the timed region, with
    # the library's event pairs around each kernel class (the events add a little time).
    plan.set_timing(True)
    lad.ladder_apply_batched(plan, Ls, ts, Rs, ws)
    torch.cuda.synchronize()
    kms, kcounts = kernel_times(lad, plan, 1)
    plan.set_timing(False)
    split = {k: v for k, v in kms.items() if v > 0}
    fp64 = None
    if fp64_sequential:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for sh, L, t in zip(shapes, Ls, ts):   # 24 sequential FP64 calls, each with its own plan
            single = lad.ladder_plan(sh.no, sh.nv, sh.nchol, lad.LADDER_FP64, device=local)
            lad.ladder_apply(single, L, t, torch.zeros_like(t))
            torch.cuda.synchronize()
            single.close()
        fp64_s = time.perf_counter() - t0
        fp64 = {"seconds": fp64_s, "tflops": flops / fp64_s / 1e12,
                "speedup": fp64_s / (ms_total * 1e-3 / steps)}
    peaks, peak_src = load_peaks()
    peak_key = "bf16_tflops_sustained" if ms_total >= 1000.0 else "bf16_tflops"
    peak = peaks.get(peak_key, peaks.get("bf16_tflops", FALLBACK_BF16_TFLOPS))
    roof = None
    forms = []
    if precision == lad.LADDER_EMU_BF16:
        # executed slice products of the work each instance needs (one block pair per instance:
        # every instance's V fits the budget; each instance's ladder form from the planner's model)
        S = args.nslices or 6
        forms = ["pm" if lad.ladder_form_model(s.no, s.nv, s.nchol, args.nslices) == 1 else "plain" for s in shapes]
        useful = sum(2.0 * s.nchol * eri_products(s.nv, s.nv, s.nv) + 2.0 * ladder_products(s.no, s.nv, f)
                     for s, f in zip(shapes, forms))
        achieved = useful * (S * (S + 1) // 2) * steps / (ms_total * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "frac_of_burst": achieved / peaks.get("bf16_tflops", FALLBACK_BF16_TFLOPS),
                "traffic": None, "kernel": "whole batched call (executed slice products, all kernels)",
                "peak_source": f"{peak_key} ({peak_src})", "executed_slice_products": S * (S + 1) // 2}
    tuned = plan.batched_choice()
    rec = {"workload": "c5: 24 uneven instances, no~U{5..30}, nv~U{60..320}, nchol=3(no+nv), seed 1239",
           "value": value, "unit": "TFLOP/s", "ms_per_step": ms_total / steps, "steps": steps, "warmup": warmup,
           "instances": len(shapes), "total_flops": flops,
           "schedule": (f"{-k} instance groups, one ERI launch and one ladder launch per shape per group"
                        if k < 0 else f"{k} worker streams"),
           "tuned": tuned,
           "split_form_instances": sum(1 for f in forms if f == "pm"),
           "graph": "one CUDA graph replay per step",
           "kernel_ms_one_call": split, "launches_one_call": sum(kcounts.values()),
           "inputs": "drawn on the GPU (timing)" if device_inputs else "ladder_inputs host generators",
           "roofline": roof, "clocks": clocks, "fp64_sequential": fp64}
    del ws, Ls, ts, Rs
    plan.close()
    torch.cuda.empty_cache()
    return rec, precision


def run_batched(args):
    """The uneven batch as the bench line (--config c5)."""
    import torch
    import paper_2603_20912_gb300 as lad
    from paper_2603_20912_gb300 import build
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    build.build()
    rec, precision = batched_record(args, lad, local, world, args.device_inputs, args.steps, args.warmup,
                                    fp64_sequential=args.fp64_reference)
    if rank == 0:
        line = {
            "metric": "PP-ladder TFLOP/s", "value": rec["value"], "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64-emulated(bf16 slices)" if precision == lad.LADDER_EMU_BF16 else "f64",
            "data": "synthetic",
            "config": {"workload": rec["workload"], "instances": rec["instances"], "total_flops": rec["total_flops"],
                       "schedule": rec["schedule"], "tuned": rec["tuned"], "graph": rec["graph"]},
            "roofline": rec["roofline"], "clocks": rec["clocks"], "fp64_sequential": rec["fp64_sequential"],
            "kernel_ms_one_call": rec["kernel_ms_one_call"], "gpu_launches": rec["launches_one_call"] * args.steps,
        }
        print(json.dumps(line), flush=True)


GOLDEN_FILE = os.path.join(ROOT, "tests", "golden", "energies.json")


def golden_for(cfg):
    """E_L and ||R||_F of the workload as the oracle computed them (stored by oracle/make_golden.py),
    or None when the workload is not one of the stored ones."""
    try:
        with open(GOLDEN_FILE) as f:
            g = json.load(f).get(cfg.name)
    except Exception:
        return None
    if not g or (g["no"], g["nv"], g["nchol"], g["seed"]) != (cfg.no, cfg.nv, cfg.nchol, cfg.seed):
        return None
    return g


def sampled_error(L, t2, R_host_list, npairs=48, seed=5):
    """||R - R_oracle||_F / ||R_oracle||_F over `npairs` random (a <= b) pairs, all (i,j), for
    each R in R_host_list (the oracle's pair mode computes the pairs once)."""
    import oracle
    nv = L.shape[1]
    rng = np.random.default_rng(seed)
    a = rng.integers(0, nv, npairs)
    b = rng.integers(0, nv, npairs)
    a, b = np.minimum(a, b), np.maximum(a, b)
    ref = oracle.ladder_pairs(L, t2, a, b)                    # [k, i, j]
    den = float(np.linalg.norm(ref.ravel()))
    out = []
    for R in R_host_list:
        got = R[:, :, a, b].transpose(2, 0, 1)
        out.append(float(np.linalg.norm((got - ref).ravel())) / den if den > 0 else 0.0)
    return out, f"{npairs} random (a<=b) pairs (seed {seed}), all (i,j), against the oracle's pair mode"


def measure_dgemm_tflops(n=8192, reps=2):
    """torch/cuBLAS FP64 matmul throughput now, on this GPU (the FP64 roofline denominator)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / best / 1e12


def kernel_times(lad, plan, steps):
    kms, counts = {}, {}
    for kind, name in [(lad.LADDER_KERNEL_PREP, "prep"), (lad.LADDER_KERNEL_ERI, "eri"),
                       (lad.LADDER_KERNEL_LADDER, "ladder"), (lad.LADDER_KERNEL_FINISH, "finish"),
                       (lad.LADDER_KERNEL_COMBINE, "combine"), (lad.LADDER_KERNEL_FACT_W, "fact_w"),
                       (lad.LADDER_KERNEL_FACT_R, "fact_r"), (lad.LADDER_KERNEL_FUSED, "fused")]:
        ms, n = plan.timing(kind)
        kms[name] = ms
        counts[name] = n
    return kms, counts


FP64_PATHS = {"eri": 0, "fused": 2}


def set_fp64_path(lad, plan, args):
    """Hold an FP64 plan to the path --fp64-path names (auto: the planner's choice)."""
    if args.fp64_path != "auto":
        plan.set_path(FP64_PATHS[args.fp64_path])


def fp64_roofline(lad, plan, cfg, kms, steps, dgemm):
    """DMMA roofline of the kernel that carries an FP64 call's flops: the ERI GEMM of the
    rebuild order (its 2 X v^2 p flops), or the fused kernel (all of the call's packed flops)."""
    src = "torch float64 matmul 8192^3 measured in this run (cuBLAS DGEMM)"
    if plan.path() == lad.LADDER_PATH_FUSED:
        flops, ms, kernel = lad.ladder_flops(cfg.no, cfg.nv, cfg.nchol), kms.get("fused", 0.0), \
            "ladder_fused_fp64_kernel (DMMA m8n8k4 f64, ERI chunks contracted on chip)"
    else:
        flops, ms, kernel = 2.0 * cfg.nchol * cfg.nv * cfg.nv * (cfg.nv * (cfg.nv + 1) // 2), kms.get("eri", 0.0), \
            "eri_fp64_kernel (DMMA m8n8k4 f64)"
    tf = flops * steps / (ms * 1e-3) / 1e12 if ms > 0 else None
    return {"bound": "tensor", "kernel": kernel, "achieved": tf, "peak": dgemm, "unit": "TFLOP/s",
            "frac": tf / dgemm if tf else None, "peak_source": src}


def run_fp64_compare(args, cfg, lad, Ld, td, local, stream):
    """Native FP64 (DMMA) path on the same workload: a warm-up call on a small shape (loads the
    kernels), then `--fp64-steps` timed calls with CUDA events on the launching stream.  Returns the
    record, the R of the last call (a single application) and the plan's ERI time share."""
    import torch
    dgemm = measure_dgemm_tflops()
    warm = lad.ladder_plan(5, 19, 72, lad.LADDER_FP64, device=local)
    Lw = torch.zeros((72, 19, 19), dtype=torch.float64, device="cuda")
    tw = torch.zeros((5, 5, 19, 19), dtype=torch.float64, device="cuda")
    lad.ladder_apply(warm, Lw, tw, torch.zeros_like(tw))
    torch.cuda.synchronize()
    warm.close()
    torch.cuda.empty_cache()
    plan = lad.ladder_plan(cfg.no, cfg.nv, cfg.nchol, lad.LADDER_FP64, device=local)
    set_fp64_path(lad, plan, args)
    ws = plan.workspace()
    desc = plan.describe()
    R = torch.zeros_like(td)
    plan.set_timing(True)
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.fp64_steps):
        R.zero_()   # every call into a zeroed R (a memset of R inside the timed region)
        lad.ladder_apply(plan, Ld, td, R, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.fp64_steps
    kms, counts = kernel_times(lad, plan, args.fp64_steps)
    plan.set_timing(False)
    assert plan.last_status() == lad.LADDER_OK
    E = lad.ladder_energy(plan, td, R)
    rec = {"ms_per_call": ms, "path": {0: "eri", 1: "factorised", 2: "fused"}[plan.path()], "tflops": lad.ladder_flops(cfg.no, cfg.nv, cfg.nchol) / (ms * 1e-3) / 1e12,
           "steps": args.fp64_steps, "warmup": "one call on a no=5 nv=19 nchol=72 shape (loads the kernels)",
           "kernel_ms_per_call": {k: v / args.fp64_steps for k, v in kms.items()},
           "gpu_launches": sum(counts.values()), "n_a": desc["n_a"], "n_b": desc["n_b"],
           "block_pairs": desc["n_block_pairs"], "E_L": E,
           "roofline": fp64_roofline(lad, plan, cfg, kms, args.fp64_steps, dgemm),
           "clocks": clocks}
    del ws
    plan.close()
    torch.cuda.empty_cache()
    return rec, R


def run_single(args, cfg):
    import torch
    import paper_2603_20912_gb300 as lad
    from paper_2603_20912_gb300 import build
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    build.build()
    precision = lad.LADDER_EMU_BF16 if args.precision == "emu" else lad.LADDER_FP64
    shard = args.mode == "shard" and world > 1
    # replicas: each rank its own independent instance (seed offset by rank); shard: one instance
    seed = cfg.seed + (0 if shard else 7919 * rank)
    if args.device_inputs:
        # timing-only shapes: inputs drawn on the GPU, no host copies (no e2e, no CPU baseline)
        from ladder_inputs import make_device_inputs
        Ld, td = make_device_inputs(cfg.no, cfg.nv, cfg.nchol, seed, device=f"cuda:{local}")
        args.no_e2e = args.no_cpu_baseline = True
        args.fp64 = "off"
        L = t2 = Lh = th = None
    else:
        L, t2, _, _ = make_inputs(cfg.no, cfg.nv, cfg.nchol, seed)
        Lh = torch.from_numpy(L).pin_memory()
        th = torch.from_numpy(t2).pin_memory()
        Ld = Lh.to("cuda", non_blocking=True)
        td = th.to("cuda", non_blocking=True)
    R = torch.zeros_like(td)
    torch.cuda.synchronize()
    budget = int(args.budget_gb * 1e9)
    if shard and budget == 0:
        # every rank must plan under the same budget to see the same blocking
        import torch.distributed as dist
        free_b, _ = torch.cuda.mem_get_info()
        b = torch.tensor([float(free_b) * 0.98 * 0.9], dtype=torch.float64, device="cuda")
        dist.all_reduce(b, op=dist.ReduceOp.MIN)
        budget = int(b.item())
    plan = lad.ladder_plan(cfg.no, cfg.nv, cfg.nchol, precision, nslices=args.nslices,
                           ws_budget_bytes=budget, device=local)
    if args.form != "auto":
        plan.set_form(1 if args.form == "pm" else 0)
    if precision == lad.LADDER_FP64:
        set_fp64_path(lad, plan, args)
    if shard:
        plan.shard(rank, world)
    form_used = "pm" if plan.form() == 1 else "plain"
    ws = plan.workspace()
    desc = plan.describe()
    stream = torch.cuda.current_stream()
    flops = lad.ladder_flops(cfg.no, cfg.nv, cfg.nchol)

    for _ in range(args.warmup):
        lad.ladder_apply(plan, Ld, td, R, ws)
    torch.cuda.synchronize()
    plan.set_timing(True)
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        lad.ladder_apply(plan, Ld, td, R, ws)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    # replicas: every rank did a whole contraction; shard: the ranks together did one
    value = (1 if shard else world) * flops * args.steps / (ms_total * 1e-3) / 1e12
    kms, counts = kernel_times(lad, plan, args.steps)
    plan.set_timing(False)
    launches = sum(counts.values())
    assert plan.last_status() == lad.LADDER_OK

    # Dominant kernel: the ERI GEMM.  Algorithmic flops per launch = 2 X v^2 (pairs in the block);
    # the emulated kernel executes S(S+1)/2 BF16 slice products per FP64 product.
    nv2 = cfg.nv * cfg.nv
    pairs_total = cfg.nv * (cfg.nv + 1) // 2
    eri_flops_call = 2.0 * cfg.nchol * nv2 * pairs_total
    if precision == lad.LADDER_EMU_BF16:   # only the rows (x <= y) of L^T are multiplied
        eri_flops_call = 2.0 * cfg.nchol * eri_products(cfg.nv, desc["n_a"], desc["n_b"])
    if shard:
        eri_flops_call = None   # a shard's share of the block pairs: no per-call count here
    peaks, peak_src = load_peaks()
    # Burst peak for a timed region under a second, the sustained (power-capped) one for longer.
    long_region = ms_total >= 1000.0
    peak_key = "bf16_tflops_sustained" if long_region else "bf16_tflops"
    bf16 = peaks.get(peak_key, peaks.get("bf16_tflops", FALLBACK_BF16_TFLOPS))
    traffic, traffic_src = captured_traffic(args.precision, cfg.name, (desc["n_a"], desc["n_b"]))
    burst = peaks.get("bf16_tflops", FALLBACK_BF16_TFLOPS)
    if precision == lad.LADDER_EMU_BF16:
        S = desc["nslices"]
        slice_products = S * (S + 1) // 2
        achieved = (eri_flops_call * slice_products * args.steps / (kms["eri"] * 1e-3) / 1e12
                    if kms["eri"] > 0 and eri_flops_call else None)
        peak = bf16
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "kernel": "eri_emu_kernel (tcgen05 BF16 slice GEMM)", "peak_source": f"{peak_key} ({peak_src})",
                "frac_of_burst": (achieved / burst) if achieved else None,
                "executed_slice_products": slice_products}
        dtype = "f64-emulated(bf16 slices)"
    else:
        dgemm = measure_dgemm_tflops()
        roof = fp64_roofline(lad, plan, cfg, kms, args.steps, dgemm)
        if shard:
            roof["achieved"] = roof["frac"] = None   # a shard's share: no per-call flop count here
        roof["traffic"] = traffic if plan.path() == lad.LADDER_PATH_ERI else None
        dtype = "f64"
    if traffic_src:
        roof["traffic_source"] = traffic_src
    if form_used == "pm" and kms.get("combine", 0.0) > 0 and not shard:
        # The split form's combine pass is HBM work: it reads V as int64 and writes the V' and V''
        # digit planes, (8 + 2S) bytes per V element of the a <= b pairs.
        comb_bytes = (8 + 2 * desc["nslices"]) * nv2 * pairs_total
        comb_gbs = comb_bytes * args.steps / (kms["combine"] * 1e-3) / 1e9
        hbm = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
        roof["combine"] = {"bound": "hbm", "achieved": comb_gbs, "peak": hbm, "unit": "GB/s",
                           "frac": comb_gbs / hbm, "kernel": "vpm_combine_kernel",
                           "bytes_per_call": comb_bytes}
    # The whole call against the same peak (every kernel of the step, executed flops).
    if precision == lad.LADDER_EMU_BF16 and not shard:
        useful = eri_flops_call + 2.0 * ladder_products(cfg.no, cfg.nv, form_used)
        call_exec = useful * desc["nslices"] * (desc["nslices"] + 1) // 2
        roof["call_frac"] = call_exec / (ms_step * 1e-3) / 1e12 / peak

    # End to end through the public host-buffer call (ladder_apply_host): every step copies L and t2
    # from pinned host memory to the device, forms R there and copies it back; the library runs
    # each call's host-to-device copies on its own copy stream during the previous call's
    # contraction (two staging sets).  The last step leaves one application in Rh.
    e2e = None
    Rh = None
    if not args.no_e2e:
        Rh = torch.empty(t2.shape, dtype=torch.float64).pin_memory()
        stage = plan.host_staging()

        def e2e_step():
            lad.ladder_apply_host(plan, Lh, th, Rh, stage, ws)

        for _ in range(args.warmup):   # untimed, like the device-timed region's warm-up
            e2e_step()
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)   # the device is idle here: the first copy starts after this event
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)   # after the last call's device-to-host copy of R
        torch.cuda.synchronize()
        wall_ms = (time.perf_counter() - w0) * 1e3
        ms_e2e = max_over_ranks(e0.elapsed_time(e1), world)
        del stage
        R.copy_(Rh)   # the host result of the last call, for E_L and the accuracy check below
        # the copies alone, one step's worth, on the caller's stream (context for the difference)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c2 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        Ld.copy_(Lh, non_blocking=True)
        td.copy_(th, non_blocking=True)
        c1.record(stream)
        Rh.copy_(R, non_blocking=True)
        c2.record(stream)
        torch.cuda.synchronize()
        h2d_ms, d2h_ms = c0.elapsed_time(c1), c1.elapsed_time(c2)
        e2e = {"value": (1 if shard else world) * flops * args.steps / (ms_e2e * 1e-3) / 1e12, "unit": "TFLOP/s",
               "ms_per_step": ms_e2e / args.steps, "wall_ms_per_step": wall_ms / args.steps,
               "h2d_bytes_per_step": int(L.nbytes + t2.nbytes), "d2h_bytes_per_step": int(t2.nbytes),
               "api": "ladder_apply_host (host buffers; copies of call k+1 overlap the contraction of call k)",
               "copies_alone_ms": {"h2d": h2d_ms, "d2h": d2h_ms},
               "host_buffers_pinned": bool(Lh.is_pinned() and th.is_pinned() and Rh.is_pinned())}
    elif L is not None:
        R.zero_()
        lad.ladder_apply(plan, Ld, td, R, ws)
        torch.cuda.synchronize()
    E_main = lad.ladder_energy(plan, td, R)
    if shard:
        import torch.distributed as dist
        Et = torch.tensor([E_main], dtype=torch.float64, device="cuda")
        dist.all_reduce(Et)   # the one exchange of the sharded contraction: a scalar
        E_main = float(Et.item())
    del ws
    plan.close()
    torch.cuda.empty_cache()

    # FP64 (DMMA) path on the same workload, and both results against the oracle.
    fp64 = None
    accuracy = None
    want_fp64 = args.fp64 == "on" or (args.fp64 == "auto" and precision == lad.LADDER_EMU_BF16 and world == 1)
    R64 = None
    if want_fp64 and L is not None:
        fp64, R64 = run_fp64_compare(args, cfg, lad, Ld, td, local, stream)
        fp64["speedup_vs_fp64"] = fp64["ms_per_call"] / ms_step
    if L is not None and rank == 0 and not shard and not args.no_accuracy:
        gold = golden_for(cfg)
        R_host = Rh.numpy() if Rh is not None else R.cpu().numpy()
        hosts = [R_host] + ([R64.cpu().numpy()] if R64 is not None else [])
        errs, how = sampled_error(L, t2, hosts)
        accuracy = {"tolerance": {"R_rel_fro": 1e-10 if precision == lad.LADDER_EMU_BF16 else 1e-12,
                                  "E_L_abs_Eh": 1e-8},
                    "sample": how, "R_rel_fro_sampled": errs[0], "E_L": E_main,
                    "E_L_oracle": gold["E_L"] if gold else None,
                    "E_L_abs_err": abs(E_main - gold["E_L"]) if gold else None,
                    "R_fro": float(np.linalg.norm(R_host.ravel())),
                    "R_fro_oracle": gold["R_fro"] if gold else None}
        if R64 is not None:
            accuracy["fp64_R_rel_fro_sampled"] = errs[1]
            accuracy["fp64_E_L_abs_err"] = abs(fp64["E_L"] - gold["E_L"]) if gold else None
            # the whole R of the two paths against each other (every element, on the device)
            accuracy["R_rel_fro_vs_fp64_whole"] = float(torch.linalg.norm((R - R64).ravel()) /
                                                        torch.linalg.norm(R64.ravel()))
    # The 24-instance uneven batch, tuned and graph-captured, as a sub-record (inputs drawn on
    # the GPU: timing; its parity is the batched GPU tests').
    batched = None
    want_batched = args.batched == "on" or (args.batched == "auto" and world == 1 and not args.shape
                                             and not args.device_inputs and precision == lad.LADDER_EMU_BF16)
    if want_batched:
        del R64
        R64 = None
        torch.cuda.empty_cache()
        batched, _ = batched_record(args, lad, local, world, True, steps=3, warmup=3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, _, _ = cpu_baseline_sample(L, t2)

    if rank == 0:
        line = {
            "metric": "PP-ladder TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": f"{cfg.name}: no={cfg.no} nv={cfg.nv} nchol={cfg.nchol} seed={cfg.seed}",
                       "precision": args.precision, "form": form_used, "nslices": desc["nslices"],
                       "n_a": desc["n_a"], "n_b": desc["n_b"], "block_pairs": desc["n_block_pairs"],
                       "l2": "inputs+workspace > L2 (V block written and re-read every step)",
                       "parallelism": (f"one contraction, block pairs sharded over {world} GPUs, E_L all-reduced"
                                       if shard else f"independent instance per GPU x{world}")},
            "ms_per_call": ms_step,
            "kernel_ms_per_call": {k: v / args.steps for k, v in kms.items()},
            "gpu_launches": launches,
            "roofline": roof,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fp64": fp64,
            "speedup_vs_fp64": fp64["speedup_vs_fp64"] if fp64 else None,
            "accuracy": accuracy,
            "batched": batched,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# The paper's random-array contraction sweep (Table 3): N = nocc + nvir, nvec Cholesky vectors,
# and its best C-split seconds per contraction (FP64 on Hopper, host transfers included) as context:
# (N, nocc, nvec, nvir, GH200 CuPy, GH200 PyTorch, H100 CuPy, H100 PyTorch); None: not computed.
TABLE3 = [
    (800, 200, 8000, 600, 706.8, 1573.6, 1364.7, 1485.3),
    (900, 225, 9000, 675, None, None, 2529.6, 3042.2),
    (1000, 250, 10000, 750, None, None, 7759.1, 6233.1),
    (800, 100, 4000, 700, 306.6, 355.9, 461.5, 330.5),
    (900, 100, 4500, 800, 495.0, 587.1, 809.7, 496.2),
    (1000, 100, 5000, 900, 829.1, 805.8, 1338.7, 827.1),
    (1100, 100, 5500, 1000, 1282.7, 1401.7, 1860.9, 1223.4),
    (1200, 100, 6000, 1100, None, None, 12329.8, 1864.7),
    (1300, 100, 6500, 1200, None, None, 18426.4, 2679.1),
    (800, 150, 4000, 650, 532.8, 475.3, 940.9, 651.2),
    (900, 150, 4500, 750, 911.6, 1261.1, 1654.1, 1044.4),
    (1000, 150, 5000, 850, 1489.2, 1924.4, 2945.2, 1739.7),
    (1100, 150, 5500, 950, None, None, 4241.5, 3234.4),
    (1000, 50, 10000, 950, 763.0, 574.6, 1006.4, 673.0),
    (1200, 50, 12000, 1150, 2155.2, 1756.0, 2429.5, 2031.5),
]


def run_sweep(args):
    """Table 3 shapes, emulated path, inputs drawn on the GPU, one timed call per shape after a
    warm-up call on a small shape (calls of tens of seconds: launch costs are negligible).  A
    shape is skipped, with the reason, when its inputs do not fit the device or no blocking fits
    the workspace budget left beside them, or when the blocking needs more than 400 block pairs."""
    import torch
    import paper_2603_20912_gb300 as lad
    from paper_2603_20912_gb300 import build
    from ladder_inputs import make_device_inputs
    torch.cuda.set_device(0)
    build.build()
    warm = lad.ladder_plan(20, 64, 300, lad.LADDER_EMU_BF16)
    Lw, tw = make_device_inputs(20, 64, 300, 1)
    lad.ladder_apply(warm, Lw, tw, torch.zeros_like(tw))
    torch.cuda.synchronize()
    warm.close()
    del Lw, tw
    total_mem = torch.cuda.get_device_properties(0).total_memory
    for (N, no, nchol, nv, gh_cupy, gh_torch, h_cupy, h_torch) in TABLE3:
        paper = {"GH200_CuPy_C-split_s": gh_cupy, "GH200_PyTorch_C-split_s": gh_torch,
                 "H100_CuPy_C-split_s": h_cupy, "H100_PyTorch_C-split_s": h_torch}
        rec = {"sweep": "Table 3", "N": N, "nocc": no, "nvir": nv, "nvec": nchol, "paper_seconds": paper}
        inputs = 8.0 * (nchol * nv * nv + 2 * no * no * nv * nv)
        torch.cuda.empty_cache()
        if inputs > 0.8 * total_mem:
            rec["skipped"] = f"L, t2 and R alone take {inputs / 1e9:.0f} GB of the {total_mem / 1e9:.0f} GB device"
            print(json.dumps(rec), flush=True)
            continue
        plan = ws = Ld = td = R = None
        try:
            Ld, td = make_device_inputs(no, nv, nchol, 4242 + N + no, device="cuda:0")
            R = torch.zeros_like(td)
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            plan = lad.ladder_plan(no, nv, nchol, lad.LADDER_EMU_BF16)
        except torch.cuda.OutOfMemoryError:
            rec["skipped"] = f"drawing the inputs ({inputs / 1e9:.0f} GB) ran out of device memory"
        except lad.LadderError as e:
            rec["skipped"] = f"ladder_plan: {e} (L, t2 and R take {inputs / 1e9:.0f} GB)"
        if "skipped" not in rec and plan.describe()["n_block_pairs"] > 400:
            d = plan.describe()
            rec["skipped"] = (f"the workspace left beside {inputs / 1e9:.0f} GB of inputs holds {d['max_pairs_per_block']} "
                              f"pairs per block: {d['n_block_pairs']} block pairs, not timed")
        if "skipped" in rec:
            print(json.dumps(rec), flush=True)
            del plan, Ld, td, R
            continue
        ws = plan.workspace()
        desc = plan.describe()
        plan.set_timing(True)
        sampler = ClockSampler(0)
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        lad.ladder_apply(plan, Ld, td, R, ws)
        e1.record()
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        kms, _ = kernel_times(lad, plan, 1)
        assert plan.last_status() == lad.LADDER_OK
        flops = lad.ladder_flops(no, nv, nchol)
        unpacked = 2.0 * nv ** 4 * (nchol + no * no)
        best_paper = min(x for x in (gh_cupy, gh_torch, h_cupy, h_torch) if x is not None)
        rec.update({"seconds": ms * 1e-3, "tflops_packed": flops / (ms * 1e-3) / 1e12,
                    "tflops_unpacked_count": unpacked / (ms * 1e-3) / 1e12,
                    "form": "pm" if plan.form() == 1 else "plain", "n_a": desc["n_a"], "n_b": desc["n_b"],
                    "block_pairs": desc["n_block_pairs"], "workspace_gb": plan.workspace_bytes() / 1e9,
                    "kernel_s": {k: v * 1e-3 for k, v in kms.items()}, "clocks": clocks,
                    "best_paper_over_ours": best_paper / (ms * 1e-3),
                    "data": "synthetic, drawn on the GPU (torch generator), shapes of Table 3"})
        print(json.dumps(rec), flush=True)
        del ws, Ld, td, R
        plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="c3", choices=sorted(CONFIGS) + ["c5"])
    ap.add_argument("--shape", default=None, help="no,nv,nchol overriding --config (profiling runs)")
    ap.add_argument("--precision", default="emu", choices=["emu", "fp64"])
    ap.add_argument("--nslices", type=int, default=0)
    ap.add_argument("--form", default="auto", choices=["auto", "plain", "pm"],
                    help="emulated ladder form: the planner's choice, plain, or the symmetric/antisymmetric split")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="shard", choices=["replicas", "shard"],
                    help="N>1: one contraction sharded over the GPUs (default), or an independent instance per GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the error report against the oracle")
    ap.add_argument("--fp64", default="auto", choices=["auto", "on", "off"],
                    help="also time the native FP64 path on the workload (auto: emulated runs on one GPU)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp64-path", default="auto", choices=["auto", "eri", "fused"],
                    help="FP64 evaluation order (auto: the planner's choice)")
    ap.add_argument("--batched", default="auto", choices=["auto", "on", "off"],
                    help="also time the 24-instance uneven batch (auto: emulated default runs on one GPU)")
    ap.add_argument("--device-inputs", action="store_true",
                    help="draw L and t2 on the GPU (timing-only runs at large shapes)")
    ap.add_argument("--budget-gb", type=float, default=0.0, help="workspace budget (0: 0.9*0.98*free)")
    ap.add_argument("--fp64-reference", action="store_true",
                    help="c5: also time 24 sequential native-FP64 calls (slow)")
    ap.add_argument("--sweep", default=None, choices=["table3"],
                    help="time the paper's Table 3 shapes that fit one GB300 (one JSON line each)")
    ap.add_argument("--measure-peaks", action="store_true",
                    help="print torch/cuBLAS matmul throughput for fp64, bf16 and int8 and exit")
    args = ap.parse_args()
    if args.measure_peaks:
        measure_peaks()
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.config == "c5":
        run_batched(args)
        return
    cfg = CONFIGS[args.config]
    if args.shape:
        no, nv, nchol = (int(x) for x in args.shape.split(","))
        cfg = LadderShape(no=no, nv=nv, nchol=nchol, seed=4242, name="custom")
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    run_single(args, cfg)


if __name__ == "__main__":
    main()
