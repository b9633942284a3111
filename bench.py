"""Throughput of the Householder-chain transforms on GB300.

One step = one pass of every built hot-path row over one resident batch of
synthetic vectors: for the FP32 chain at n=4096, h=16, batch 262,144 the
kernels y = W x, y = W^T x and y = S x (S = D W diag(d) W^T D), each reading
and writing every vector once.  `value` is vectors per second through the
whole step (all ranks), timed with CUDA events on the launching stream.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]
                    [--gpus N] [--no-e2e] [--no-cpu]

With torchrun (N > 1) each rank runs its own replica of the workload (the
transforms share nothing across vectors, so there is no collective on the
data path); rank 0 prints the JSON line.  `--impl reference` times the FP64
CPU oracle on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vectors/s + HBM GB/s % of peak, Householder-chain apply, BF16-WY vs FP32 plain"
WORKLOAD = dict(n=4096, h=16, batch=262_144, seed=0)
ROWS = ("W", "WT", "SYM")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return j, "of measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "of fallback"


KERNEL_SOURCES = ["paper_1811_07624_gb300/csrc/hh_staged.cuh", "paper_1811_07624_gb300/csrc/hh_fused_f32.cu",
                  "paper_1811_07624_gb300/csrc/hh_fused.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "staged_chain_n4096_h16_ncu_full.md")


def profiled_traffic(mode, batch):
    """DRAM bytes of one launch from the committed ncu summary, scaled by the
    vector count; None when the kernel sources changed since the capture."""
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    sha = h.hexdigest()[:16]
    if not os.path.exists(TRAFFIC_FILE):
        return None
    for line in open(TRAFFIC_FILE):
        if line.startswith("TRAFFIC ") and f"mode={mode} " in line:
            kv = dict(t.split("=", 1) for t in line.split()[1:])
            if kv.get("sources_sha256") == sha:
                return float(kv["bytes_per_vector"]) * batch
    return None


def algorithmic(mode, n, h, batch, esize=4):
    """Bytes and flops one launch must move / do (the paper's op counts)."""
    bytes_ = 2 * batch * n * esize + h * n * esize
    if mode == "SYM":
        bytes_ += n * esize
        flops = (8 * h + 1) * n * batch  # §III-A
    else:
        flops = 4 * n * h * batch  # §II-A
    return bytes_, flops


class ClockSampler:
    """nvidia-smi SM-clock samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                mx.append(float(row[2]))
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_rate(workload, rows, budget_s=12.0, threads=0):
    """Vectors/s of the FP64 oracle through `rows` on a bounded sample."""
    import oracle
    import synthetic_inputs as si

    n, h = workload["n"], workload["h"]
    U = si.reflectors(n, h, seed=workload["seed"])
    d = si.spectrum(n, seed=workload["seed"])
    s = si.sign(n, seed=workload["seed"])

    def run(count):
        X = si.vectors(count, n, seed=123)
        t0 = time.perf_counter()
        for mode in rows:
            oracle.apply(mode, U, X, sign=s, d=d, threads=threads)
        return time.perf_counter() - t0

    probe = 256
    t = run(probe)
    count = int(max(probe, min(1 << 20, probe * budget_s / max(t, 1e-6))))
    t = run(count)
    return count / t, count, t


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    threads = oracle.max_threads()
    _, count, t = oracle_sample_rate(WORKLOAD, ROWS, budget_s=2.0)
    per_step = count
    times = []
    for i in range(args.warmup + args.steps):
        rate, c, dt = oracle_sample_rate_fixed(WORKLOAD, ROWS, per_step)
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "vectors/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(),
        "cpu_baseline": {"value": value, "unit": "vectors/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} vectors per step through W, W^T and S (FP64 oracle)"},
        "e2e": {"value": value, "unit": "vectors/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


_REF_CACHE = {}


def oracle_sample_rate_fixed(workload, rows, count):
    import oracle
    import synthetic_inputs as si

    key = (workload["n"], workload["h"], count)
    if key not in _REF_CACHE:
        n, h = workload["n"], workload["h"]
        _REF_CACHE[key] = (si.reflectors(n, h, seed=workload["seed"]),
                           si.spectrum(n, seed=workload["seed"]),
                           si.sign(n, seed=workload["seed"]), si.vectors(count, n, seed=123))
    U, d, s, X = _REF_CACHE[key]
    t0 = time.perf_counter()
    for mode in rows:
        oracle.apply(mode, U, X, sign=s, d=d)
    dt = time.perf_counter() - t0
    return count / dt, count, dt


def config_dict():
    w = WORKLOAD
    return {"workload": f"FP32 fused reflector chain n={w['n']} h={w['h']} batch={w['batch']}: "
                        "y = W x, y = W^T x, y = W diag(d) W^T x per vector (sign D on)",
            "n": w["n"], "h": w["h"], "batch": w["batch"], "rows": list(ROWS),
            "l2": "inputs larger than L2 (4.3 GB per buffer), no flush needed",
            "parallelism": "replicas"}


def main():
    global ROWS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch", type=int, default=None,
                    help="override the batch (profiling a smaller case); not a bench line")
    ap.add_argument("--rows", default=",".join(ROWS), help="subset of W,WT,SYM to run")
    args = ap.parse_args()
    ROWS = tuple(r for r in args.rows.split(",") if r)
    if args.batch:
        WORKLOAD["batch"] = args.batch
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    import __graft_entry__

    __graft_entry__.build()
    import oracle
    import synthetic_inputs as si
    from paper_1811_07624_gb300 import Plan

    dev = torch.device("cuda", local)
    n, h, B, seed = WORKLOAD["n"], WORKLOAD["h"], WORKLOAD["batch"], WORKLOAD["seed"]
    U = si.reflectors(n, h, seed=seed)
    d = si.spectrum(n, seed=seed)
    s = si.sign(n, seed=seed)
    plan = Plan(torch.tensor(U, device=dev, dtype=torch.float32),
                d=torch.tensor(d, device=dev, dtype=torch.float32), sign=torch.tensor(s, device=dev))
    g = torch.Generator(device=dev).manual_seed(seed + 1000 * rank)
    X = torch.randn(B, n, device=dev, generator=g, dtype=torch.float32)
    Ys = {m: torch.empty_like(X) for m in ROWS}
    fns = {"W": plan.apply, "WT": plan.apply_T, "SYM": plan.apply_sym}
    stream = torch.cuda.current_stream()

    # parity on sampled rows, outside the timed region
    for m in ROWS:
        fns[m](X, out=Ys[m])
    torch.cuda.synchronize()
    idx = np.linspace(0, B - 1, 64).astype(np.int64)
    Xs = X[idx].double().cpu().numpy()
    U32 = torch.tensor(U, dtype=torch.float32).double().numpy()
    d32 = torch.tensor(d, dtype=torch.float32).double().numpy()
    parity = {}
    for m in ROWS:
        ref = oracle.apply(m, U32, Xs, sign=s, d=d32)
        got = Ys[m][idx].double().cpu().numpy()
        parity[m] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    for _ in range(args.warmup):
        for m in ROWS:
            fns[m](X, out=Ys[m])
    torch.cuda.synchronize()

    ev = {m: [] for m in ROWS}
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ
                           else int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local]))
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        for m in ROWS:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fns[m](X, out=Ys[m])
            b.record(stream)
            ev[m].append((a, b))
    t_end.record(stream)
    torch.cuda.synchronize()
    plan.sync()  # raises if any kernel in the timed region gave up a bounded wait
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    total_ms = t_start.elapsed_time(t_end)
    ms_step = total_ms / args.steps
    if pg:
        t = torch.tensor([ms_step], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms_step = float(t.item())
    kernel_ms = {m: statistics.mean(a.elapsed_time(b) for a, b in ev[m]) for m in ROWS}
    value = world * B / (ms_step / 1e3)

    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # TFLOP/s
    ridge = fp32_peak * 1e12 / (peaks["hbm_gbs"] * 1e9)
    rows = {}
    for m in ROWS:
        by, fl = algorithmic(m, n, h, B)
        t = kernel_ms[m] / 1e3
        gbs = by / t / 1e9
        tfl = fl / t / 1e12
        rows[m] = {"ms": kernel_ms[m], "vectors_per_s": B / t, "GB_s": gbs,
                   "dram_traffic_bytes": profiled_traffic(m, B),
                   "hbm_frac": gbs / peaks["hbm_gbs"], "TFLOP_s": tfl, "alu_frac": tfl / fp32_peak,
                   "intensity_flop_per_byte": fl / by, "bound": "hbm" if fl / by < ridge else "alu",
                   "rel_l2_vs_oracle": parity[m]}
    dom = max(ROWS, key=lambda m: kernel_ms[m])
    r = rows[dom]
    if r["bound"] == "hbm":
        roof = {"bound": "hbm", "achieved": r["GB_s"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": r["hbm_frac"], "traffic": profiled_traffic(dom, B),
                "kernel": f"staged_chain_kernel mode {dom}", "peak_source": f"hbm_gbs {peak_src}"}
    else:
        roof = {"bound": "alu", "achieved": r["TFLOP_s"], "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": r["alu_frac"], "traffic": profiled_traffic(dom, B),
                "kernel": f"staged_chain_kernel mode {dom}",
                "peak_source": f"FP32 FMA: {sms} SMs x 128 lanes x 2 flops x "
                               f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz (sm_max_mhz {peak_src})"}

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(torch, fns, X, B, n, dev, stream, world, pg, steps=max(3, min(args.steps, 10)))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = oracle.max_threads()
        rate, count, secs = oracle_sample_rate(WORKLOAD, ROWS, budget_s=12.0)
        cpu = {"value": rate, "unit": "vectors/s", "cores": threads, "kind": "oracle",
               "sample": f"{count} vectors (FP64, W + W^T + S each) in {secs:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "vectors/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (Gaussian vectors and reflectors, seeded)", "config": config_dict(),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps * len(ROWS), "clocks": clocks, "rows": rows,
            "fp32_peak_tflops": fp32_peak,
        }
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


def measure_e2e(torch, fns, X, B, n, dev, stream, world, pg, steps):
    """Same step through the public API from pinned host memory, results read back."""
    Xh = torch.empty((B, n), dtype=torch.float32, pin_memory=True)
    Xh.copy_(X.cpu())
    Yh = torch.empty((B, n), dtype=torch.float32, pin_memory=True)
    Xd = torch.empty_like(X)
    Yd = torch.empty_like(X)

    def step():
        Xd.copy_(Xh, non_blocking=True)
        for m in ROWS:
            fns[m](Xd, out=Yd)
            Yh.copy_(Yd, non_blocking=True)

    step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    if pg:
        t = torch.tensor([ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    nbytes = B * n * 4
    return {"value": world * B / (ms / 1e3), "unit": "vectors/s", "ms_per_step": ms,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes * len(ROWS),
            "steps": steps}


if __name__ == "__main__":
    sys.exit(main())
