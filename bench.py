"""Throughput of the Householder-chain hot path on GB300.

One step = one pass of every built hot-path row over its own resident batch of
synthetic vectors (inputs larger than L2, so no flush is needed):

  chain_W, chain_WT, chain_SYM   FP32 chain, n=4096, h=16, 262,144 vectors:
                                 y = sigma.*(W x), W^T(sigma.*x), sigma.*W(d.*W^T(sigma.*x))
  c2_n<n>_h<h>_<W|WT|SYM>        the same three applies at scale: n=1024, h in {10, 32},
                                 1,048,576 vectors; n=4096, h in {12, 64}, 262,144 vectors
  wy_h64, wy_h256, wy_h1024      BF16 compact-WY (tcgen05), n=4096, 262,144 vectors, y = W x
  mahalanobis                    FP32 fast Mahalanobis distance, n=256, h=16, 1,048,576 pairs
  mahalanobis_grad               its gradient w.r.t. U and d (metric-learning loss)
  adjoint_SYM                    FP32 forward + adjoint of S x, n=1024, h=32, 65,536 vectors
  trunc_qr                       Result 3's partial-QR reflectors (k - 1 leading zeros), n=1024,
                                 h=512, 262,144 vectors, zero prefixes skipped (timed beside
                                 the same apply without skipping)
  batched_C5                     512 independent FP32 transforms, n in {128..2048}, h in
                                 [4, 64], 1,024-16,384 vectors each, y = W x, in ONE
                                 persistent graph-replayed launch (autotuned tile shapes)

`value` is vectors per second through the whole step (the sum of the rows'
vectors over the step time, vectors of mixed n; a Mahalanobis pair counts as
the one difference vector it transforms), timed with CUDA events on the
launching stream.  The "c2" object gives the same rate over the FP32-chain-at-
scale rows alone.
Each row also reports its own time, vectors/s, algorithmic GB/s and FLOP/s
and roofline fraction; the FP32 chain on the WY rows' shapes and data is
timed beside them ("BF16-WY vs FP32 plain"), and the 512 transforms of
batched_C5 are also timed as 512 separate launches ("batched_vs_separate"), and
"shf_su_fit" times SHF-SU's start and one iteration (n = 128, h = 16) through the
kernels beside the FP64 oracle.  `--impl reference` times the
FP64 CPU oracle on a bounded sample of the same rows.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--gpus N]
                    [--rows a,b,...] [--batch-scale f] [--no-e2e] [--no-cpu] [--no-compare]
"""

from __future__ import annotations

import argparse
import csv
import hashlib
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
N_CHAIN, H_CHAIN, B_CHAIN = 4096, 16, 262_144
B_WY = 262_144
N_MAHAL, H_MAHAL, P_MAHAL, PTS_MAHAL = 256, 16, 1 << 20, 100_000
N_ADJ, H_ADJ, B_ADJ = 1024, 32, 65_536
C5_COUNT, C5_SCALE = 512, 1.0
C5_TUNE_H, C5_TUNE_ROWS = [4, 8, 16, 32, 64], 32_768
E2E_CHUNKS = 16    # chunks per large row in the pipelined end-to-end step
TUNE_TABLE = None  # --tune-table: load the batched launch's shapes from here, or tune and save
# the FP32 chain at the configurations of the "plain FP32 chain at scale" workload:
# (n, h, batch) for each of W, W^T and S
C2_SHAPES = [(1024, 10, 1_048_576), (1024, 32, 1_048_576), (4096, 12, 262_144), (4096, 64, 262_144)]
C2_ROWS = [f"c2_n{n}_h{h}_{m}" for n, h, _ in C2_SHAPES for m in ("W", "WT", "SYM")]
ALL_ROWS = (["chain_W", "chain_WT", "chain_SYM"] + C2_ROWS
            + ["wy_h64", "wy_h256", "wy_h1024", "mahalanobis", "mahalanobis_grad", "adjoint_SYM",
               "batched_C5", "trunc_qr"])

_CSRC = "paper_1811_07624_gb300/csrc/"
_CHAIN_SRC = [_CSRC + f for f in ("hh_split.cuh", "hh_staged.cuh", "hh_fused.cuh",
                                  "hh_fused_f32.cu")]
# kernel sources behind each row kind: a traffic figure is used only while they
# hash to the value recorded with it
ROW_SOURCES = {
    "chain": _CHAIN_SRC, "c2": _CHAIN_SRC,
    "wy": [_CSRC + "hh_wy.cu", _CSRC + "hh_tc.cuh"],
    "mahalanobis": [_CSRC + "hh_mahalanobis.cu", _CSRC + "hh_fused.cuh"],
    "mahalanobis_grad": [_CSRC + "hh_backward.cu", _CSRC + "hh_fused.cuh"] + _CHAIN_SRC,
    "adjoint": [_CSRC + "hh_backward.cu", _CSRC + "hh_fused.cuh"] + _CHAIN_SRC,
    "batched": [_CSRC + "hh_batched.cu", _CSRC + "hh_staged.cuh", _CSRC + "hh_fused.cuh",
                _CSRC + "hh_split.cuh"],
    "trunc": _CHAIN_SRC,
}
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "of measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "of fallback"


def sources_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def row_kind(name):
    return name if name == "mahalanobis_grad" else name.split("_")[0]


def profiled_traffic(row, units, path=None):
    """DRAM bytes (read + write) of one call of `row` over `units` vectors, from
    the ncu figures recorded in profiles/traffic.json, scaled by units; None
    when there is no figure or the row's kernel sources changed since."""
    path = path or TRAFFIC_JSON
    if not os.path.exists(path):
        return None
    with open(path) as f:
        entries = json.load(f).get("entries", [])
    for e in entries:
        if e.get("row") != row:
            continue
        if e.get("sources_sha256") != sources_sha(ROW_SOURCES[row_kind(row)]):
            return None
        return (float(e["dram_read_bytes"]) + float(e["dram_write_bytes"])) * units / e["units"]
    return None


_NCU_UNITS = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}


def ncu_dram_bytes(csv_path):
    """[(read, write)] DRAM bytes of each launch, in launch order, in an ncu --csv
    log of dram__bytes_read.sum and dram__bytes_write.sum."""
    text = open(csv_path).read()
    start = text.find('"ID"')
    if start < 0:
        raise ValueError(f"{csv_path}: no ncu CSV table")
    order, got = [], {}
    for row in csv.DictReader(io.StringIO(text[start:])):
        name = row["Metric Name"]
        if name not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        if row["ID"] not in got:
            order.append(row["ID"])
            got[row["ID"]] = {}
        val = float(row["Metric Value"].replace(",", ""))
        got[row["ID"]][name] = val * _NCU_UNITS[row["Metric Unit"]]
    return [(got[i]["dram__bytes_read.sum"], got[i]["dram__bytes_write.sum"]) for i in order]


def ingest_traffic(csv_path, rows, out_path, command, per_row=None):
    """Record the DRAM bytes of the launches captured in an ncu log: the log
    holds the first call of each of rows (at its full batch) in order, per_row[i]
    consecutive launches for rows[i] (default 1), summed."""
    entries = []
    if os.path.exists(out_path):
        with open(out_path) as f:
            entries = json.load(f).get("entries", [])
    per_row = per_row or [1] * len(rows)
    if len(per_row) != len(rows):
        raise ValueError("one launch count per row")
    launches = ncu_dram_bytes(csv_path)
    if len(launches) < sum(per_row):
        raise ValueError(f"{csv_path}: {len(launches)} launches for {sum(per_row)}")
    full = step_vectors(rows)
    summed, k = [], 0
    for c in per_row:
        part = launches[k:k + c]
        summed.append((sum(p[0] for p in part), sum(p[1] for p in part)))
        k += c
    for row, (rd, wr) in zip(rows, summed):
        entries = [e for e in entries if e.get("row") != row]
        entries.append({"row": row, "units": full[row], "dram_read_bytes": rd,
                        "dram_write_bytes": wr, "sources": ROW_SOURCES[row_kind(row)],
                        "sources_sha256": sources_sha(ROW_SOURCES[row_kind(row)]),
                        "command": command})
    entries.sort(key=lambda e: e["row"])
    with open(out_path, "w") as f:
        json.dump({"about": "DRAM bytes of one call per row, summed over its launches (ncu "
                            "dram__bytes_read.sum and dram__bytes_write.sum, one pass, "
                            "--clock-control none), at the row's full batch; bench.py uses a "
                            "figure only while the row's kernel sources hash to sources_sha256",
                   "entries": entries}, f, indent=1)
        f.write("\n")


class ClockSampler:
    """nvidia-smi SM-clock samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu, self.proc = gpu_index, None

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
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                mx.append(float(row[2]))
                pw.append(float(row[3]))
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "power_w_max": max(pw) if pw else None, "samples": len(sm)}


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


# --------------------------------------------------------------------------------------
# rows: resident inputs, one call per step.  Each row's e2e() gives the bytes it moves per
# step and its end-to-end work as chunks (copy in, compute, copy out), which
# measure_e2e() pipelines over three streams.

def pinned_copy(torch, t):
    """A pinned host copy of device tensor t."""
    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    h.copy_(t)
    return h


def row_chunks(B, parts):
    """Split [0, B) into `parts` contiguous row ranges."""
    step = -(-B // parts)
    return [(r, min(B, r + step)) for r in range(0, B, step)]



_SHARED = {}
_CHAIN_ROWS = []


class ChainRow:
    def __init__(self, torch, dev, mode, n, h, batch, seed=0, name=None):
        import synthetic_inputs as si
        from paper_1811_07624_gb300 import Plan

        self.name = name or f"chain_{mode}"
        self.mode, self.n, self.h, self.B = mode, n, h, batch
        self.U = si.reflectors(n, h, seed=seed)
        self.d = si.spectrum(n, seed=seed)
        self.s = si.sign(n, seed=seed)
        self.plan = Plan(torch.tensor(self.U, device=dev, dtype=torch.float32),
                         d=torch.tensor(self.d, device=dev, dtype=torch.float32),
                         sign=torch.tensor(self.s, device=dev))
        key = (n, batch, seed)
        if key not in _SHARED:  # the chain rows of one (n, batch) read the same vectors
            g = torch.Generator(device=dev).manual_seed(seed + 1)
            _SHARED[key] = torch.randn(batch, n, device=dev, generator=g)
            _SHARED[("Y",) + key] = torch.empty_like(_SHARED[key])
        self.X = _SHARED[key]
        # ... and write one output buffer (each row's parity is read right after
        # its own first call)
        self.Y = _SHARED[("Y",) + key]
        self.torch = torch
        # 2048 < n <= 4096 with 25 < h <= 100 at a large batch: the eight-CTA cluster
        # kernel and, on the SMs its clusters leave, the staged kernel beside it
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        self.launches = 2 if (2048 < n <= 4096 and 25 < h <= 100 and batch >= sms * 64) else 1
        self.bound = "hbm" if (self.flops() / self.bytes()) < 11.9 else "alu"
        _CHAIN_ROWS.append(self)

    def vectors(self):
        return self.B

    def bytes(self):
        return 2.0 * self.B * self.n * 4 + self.h * self.n * 4

    def flops(self):
        per = (8 * self.h + 1) * self.n if self.mode == "SYM" else 4 * self.n * self.h
        return float(per) * self.B

    def run(self):
        self.plan.apply_mode(self.mode, self.X, out=self.Y)

    def parity(self):
        import oracle

        t = self.torch
        idx = t.linspace(0, self.B - 1, 64, device=self.X.device).long()
        ref = oracle.apply(self.mode, t.tensor(self.U, dtype=t.float32).double().numpy(),
                           self.X[idx].double().cpu().numpy(), sign=self.s,
                           d=t.tensor(self.d, dtype=t.float32).double().numpy())
        return rel_l2(self.Y[idx].double().cpu().numpy(), ref)

    def e2e(self, torch):
        # The chain rows of one (n, batch) transform the same vectors (as in the
        # device-resident step): the first of them copies the vectors in once and
        # runs every row on each chunk; the others add nothing.  Each row's
        # results go through a ring of two chunk buffers on the device and on the
        # host; chunk c reuses the buffers of chunk c - 2 once their copy out has
        # finished (the pipeline's per-key ordering).
        key = ("e2e", self.n, self.B)
        if key in _SHARED:
            return 0, 0, []
        rows = [r for r in _CHAIN_ROWS if (r.n, r.B) == (self.n, self.B)]
        _SHARED[key] = True
        Xh = pinned_copy(torch, self.X)
        Xd = torch.empty_like(self.X)
        spans = row_chunks(self.B, E2E_CHUNKS)
        rows_max = max(b - a for a, b in spans)
        ring = [[(torch.empty(rows_max, self.n, device=self.X.device),
                  torch.empty(rows_max, self.n, pin_memory=True)) for _ in range(2)] for _ in rows]
        chunks = []
        for c, (r0, r1) in enumerate(spans):
            def comp(a=r0, b=r1, c=c):
                for r, slots in zip(rows, ring):
                    r.plan.apply_mode(r.mode, Xd[a:b], out=slots[c % 2][0][:b - a])

            def cout(a=r0, b=r1, c=c):
                for slots in ring:
                    Yd, Yh = slots[c % 2]
                    Yh[:b - a].copy_(Yd[:b - a], non_blocking=True)
            chunks.append((lambda a=r0, b=r1: Xd[a:b].copy_(Xh[a:b], non_blocking=True), comp, cout,
                           ("chain ring", self.n, self.B, c % 2)))
        return Xh.numel() * 4, Xh.numel() * 4 * len(rows), chunks


class WYRow:
    def __init__(self, torch, dev, n, h, batch, seed=0):
        import synthetic_inputs as si
        from paper_1811_07624_gb300 import Plan

        self.name, self.n, self.h, self.B = f"wy_h{h}", n, h, batch
        self.U = si.reflectors(n, h, seed=seed + h)
        self.Ub = torch.tensor(self.U, device=dev, dtype=torch.bfloat16)
        self.plan = Plan(self.Ub)
        h64 = -(-h // 64) * 64
        self.launches = -(-h64 // 256)  # one launch per panel of <= 256 reflectors
        g = torch.Generator(device=dev).manual_seed(seed + h + 1)
        self.X = torch.randn(batch, n, device=dev, generator=g).bfloat16()
        self.Y = torch.empty_like(self.X)
        self.torch = torch
        ridge = 1700.6e12 / 6765.7e9
        self.bound = "hbm" if self.flops() / self.bytes() < ridge else "tensor"

    def vectors(self):
        return self.B

    def bytes(self):
        return 2.0 * self.B * self.n * 2 + self.h * self.n * 2

    def flops(self):
        return 4.0 * self.n * self.h * self.B

    def run(self):
        self.plan.apply(self.X, out=self.Y)

    def parity(self):
        import oracle

        t = self.torch
        idx = t.linspace(0, self.B - 1, 32, device=self.X.device).long()
        ref = oracle.apply("W", self.Ub.double().cpu().numpy(), self.X[idx].double().cpu().numpy())
        return rel_l2(self.Y[idx].double().cpu().numpy(), ref)

    def e2e(self, torch):
        Xh = pinned_copy(torch, self.X)
        Yh = torch.empty(Xh.shape, dtype=Xh.dtype, pin_memory=True)
        Xd, Yd = torch.empty_like(self.X), torch.empty_like(self.X)
        chunks = []
        for r0, r1 in row_chunks(self.B, E2E_CHUNKS):
            chunks.append((lambda a=r0, b=r1: Xd[a:b].copy_(Xh[a:b], non_blocking=True),
                           lambda a=r0, b=r1: self.plan.apply(Xd[a:b], out=Yd[a:b]),
                           lambda a=r0, b=r1: Yh[a:b].copy_(Yd[a:b], non_blocking=True)))
        return Xh.numel() * 2, Yh.numel() * 2, chunks


class MahalanobisRow:
    def __init__(self, torch, dev, grad=False, seed=0):
        import synthetic_inputs as si
        from paper_1811_07624_gb300 import Plan

        self.name = "mahalanobis_grad" if grad else "mahalanobis"
        self.grad = grad
        self.n, self.h, self.P = N_MAHAL, H_MAHAL, P_MAHAL
        X, labels = si.gaussian_mixture(PTS_MAHAL, n=self.n, seed=seed)
        ia, ib, _ = si.labelled_pairs(labels, self.P, seed=seed)
        self.U = si.reflectors(self.n, self.h, seed=seed + 7)
        self.d = si.spectrum(self.n, seed=seed + 7)
        self.ia_np, self.ib_np = ia, ib
        self.X = torch.tensor(X, device=dev, dtype=torch.float32)
        self.ia = torch.tensor(ia, device=dev)
        self.ib = torch.tensor(ib, device=dev)
        self.plan = Plan(torch.tensor(self.U, device=dev, dtype=torch.float32),
                         d=torch.tensor(self.d, device=dev, dtype=torch.float32))
        self.out = torch.empty(self.P, device=dev)
        self.gout = torch.ones(self.P, device=dev) / self.P
        self.torch = torch
        # gradient: the walk, two batch contractions, three fixed-order sums, the combine
        self.launches = 7 if grad else 1
        self.bound = "alu" if grad else "hbm"

    def vectors(self):
        return self.P

    def bytes(self):
        return 2.0 * self.P * self.n * 4 + self.P * (16 + 4)

    def flops(self):
        per = 4 * self.n * self.h + 3 * self.n
        return float(per) * self.P * (4 if self.grad else 1)

    def run(self):
        if self.grad:
            self.plan.mahalanobis_backward(self.X, self.ia, self.ib, self.gout)
        else:
            self.plan.mahalanobis(self.X, self.ia, self.ib, out=self.out)

    def parity(self):
        import oracle

        t = self.torch
        sel = np.linspace(0, self.P - 1, 256).astype(np.int64)
        selt = t.tensor(sel, device=self.X.device)
        U32 = t.tensor(self.U, dtype=t.float32).double().numpy()
        d32 = t.tensor(self.d, dtype=t.float32).double().numpy()
        X32 = self.X.double().cpu().numpy()
        if not self.grad:
            self.plan.mahalanobis(self.X, self.ia, self.ib, out=self.out)
            ref = oracle.mahalanobis(U32, X32, self.ia_np[sel], self.ib_np[sel], d32)
            return rel_l2(self.out[selt].double().cpu().numpy(), ref)
        gU, gd = self.plan.mahalanobis_backward(self.X, self.ia[selt], self.ib[selt],
                                                t.ones(sel.shape[0], device=self.X.device))
        delta = X32[self.ia_np[sel]] - X32[self.ib_np[sel]]
        z = oracle.apply("WT", U32, delta)
        _, gU_ref, _ = oracle.backward("WT", U32, delta, 2.0 * d32[None, :] * z)
        return max(rel_l2(gU.double().cpu().numpy(), gU_ref),
                   rel_l2(gd.double().cpu().numpy(), (z * z).sum(0)))

    def e2e(self, torch):
        Xh = pinned_copy(torch, self.X)
        iah, ibh = pinned_copy(torch, self.ia), pinned_copy(torch, self.ib)
        oh = torch.empty(self.P, pin_memory=True)
        gUh = torch.empty(self.h, self.n, pin_memory=True)
        Xd, iad, ibd = torch.empty_like(self.X), torch.empty_like(self.ia), torch.empty_like(self.ib)
        res = {}

        def h2d():
            Xd.copy_(Xh, non_blocking=True)
            iad.copy_(iah, non_blocking=True)
            ibd.copy_(ibh, non_blocking=True)

        def comp():
            if self.grad:
                res["gU"], _ = self.plan.mahalanobis_backward(Xd, iad, ibd, self.gout)
            else:
                self.plan.mahalanobis(Xd, iad, ibd, out=self.out)

        def d2h():
            if self.grad:
                res["gU"].record_stream(torch.cuda.current_stream())
                gUh.copy_(res["gU"], non_blocking=True)
            else:
                oh.copy_(self.out, non_blocking=True)
        h2d_bytes = Xh.numel() * 4 + 2 * iah.numel() * 8
        d2h_bytes = gUh.numel() * 4 if self.grad else oh.numel() * 4
        return h2d_bytes, d2h_bytes, [(h2d, comp, d2h)]


class AdjointRow:
    def __init__(self, torch, dev, seed=0):
        import synthetic_inputs as si
        from paper_1811_07624_gb300 import Plan

        self.name = "adjoint_SYM"
        self.n, self.h, self.B = N_ADJ, H_ADJ, B_ADJ
        self.U = si.reflectors(self.n, self.h, seed=seed + 9)
        self.d = si.spectrum(self.n, seed=seed + 9)
        self.plan = Plan(torch.tensor(self.U, device=dev, dtype=torch.float32),
                         d=torch.tensor(self.d, device=dev, dtype=torch.float32))
        g = torch.Generator(device=dev).manual_seed(seed + 10)
        self.X = torch.randn(self.B, self.n, device=dev, generator=g)
        self.G = torch.randn(self.B, self.n, device=dev, generator=g)
        self.Y = torch.empty_like(self.X)
        self.P = torch.empty_like(self.X)
        self.torch = torch
        # forward S x keeping p; the adjoint from (p, y): the two walks, three batch
        # contractions, four fixed-order sums, the combine
        self.launches = 10
        self.bound = "alu"

    def vectors(self):
        return self.B

    def bytes(self):
        return 4.0 * self.B * self.n * 4

    def flops(self):
        # forward S x, (8h+1) n, and the adjoint: its recomputed forward plus about
        # three times the forward arithmetic
        return float((8 * self.h + 1) * self.n * 5) * self.B

    def run(self):
        self.plan.apply_sym_p(self.X, out=self.Y, p_out=self.P)
        self.res = self.plan.backward("SYM", None, self.G, Y=self.Y, P=self.P)

    def parity(self):
        import oracle

        t = self.torch
        sub = 64
        Ysub, Psub = self.plan.apply_sym_p(self.X[:sub].contiguous())
        gX, gU, gd = self.plan.backward("SYM", None, self.G[:sub].contiguous(), Y=Ysub, P=Psub)
        U32 = t.tensor(self.U, dtype=t.float32).double().numpy()
        d32 = t.tensor(self.d, dtype=t.float32).double().numpy()
        rX, rU, rd = oracle.backward("SYM", U32, self.X[:sub].double().cpu().numpy(),
                                     self.G[:sub].double().cpu().numpy(), d=d32)
        return max(rel_l2(gX.double().cpu().numpy(), rX), rel_l2(gU.double().cpu().numpy(), rU),
                   rel_l2(gd.double().cpu().numpy(), rd))

    def e2e(self, torch):
        Xh, Gh = pinned_copy(torch, self.X), pinned_copy(torch, self.G)
        gUh = torch.empty(self.h, self.n, pin_memory=True)
        Xd, Gd, Yd = torch.empty_like(self.X), torch.empty_like(self.G), torch.empty_like(self.X)
        Pd = torch.empty_like(self.X)
        res = {}

        def h2d():
            Xd.copy_(Xh, non_blocking=True)
            Gd.copy_(Gh, non_blocking=True)

        def comp():
            self.plan.apply_sym_p(Xd, out=Yd, p_out=Pd)
            _, res["gU"], _ = self.plan.backward("SYM", None, Gd, need_gX=False, Y=Yd, P=Pd)

        def d2h():
            res["gU"].record_stream(torch.cuda.current_stream())
            gUh.copy_(res["gU"], non_blocking=True)
        return (Xh.numel() + Gh.numel()) * 4, gUh.numel() * 4, [(h2d, comp, d2h)]


N_TRQ, H_TRQ, B_TRQ = 1024, 512, 262_144


class TruncRow:
    """Result 3's partial-QR reflectors (§II-D) of a random orthonormal U: j_k has
    k - 1 leading zeros, and the plan skips them (4(n - k + 1) per reflector).
    y = J_1 ... J_h D x (apply_T of the plan of the reversed reflectors, sign D)."""

    def __init__(self, torch, dev, seed=0):
        import synthetic_inputs as si
        from paper_1811_07624_gb300 import factor

        self.name, self.torch = "trunc_qr", torch
        self.n, self.h, self.B = N_TRQ, H_TRQ, B_TRQ
        Q = si.random_orthonormal(self.n, seed + 31)
        R, d, _ = factor.result3(Q, self.h)
        self.R, self.d = R, d
        self.plan, self.mode = factor.plan("result3", R, d, device=dev, dtype=torch.float32)
        self.skip_auto = self.plan.skip_prefix()
        g = torch.Generator(device=dev).manual_seed(seed + 32)
        self.X = torch.randn(self.B, self.n, device=dev, generator=g)
        self.Y = torch.empty_like(self.X)
        self.launches = 1
        self.bound = "alu"
        # first non-zero column of each reflector of the plan (reversed order)
        Rr = R.flip(0).float().numpy()
        self.starts = [int(np.flatnonzero(r)[0]) if np.any(r) else self.n for r in Rr]

    def vectors(self):
        return self.B

    def bytes(self):
        return 2.0 * self.B * self.n * 4 + sum(self.n - s for s in self.starts) * 4

    def flops(self):
        return 4.0 * sum(self.n - s for s in self.starts) * self.B

    def run(self):
        self.plan.apply_mode(self.mode, self.X, out=self.Y)

    def parity(self):
        import oracle

        t = self.torch
        idx = t.linspace(0, self.B - 1, 64, device=self.X.device).long()
        Rr = self.R.flip(0).float().double().numpy()
        ref = oracle.apply("WT", Rr, self.X[idx].double().cpu().numpy(),
                           sign=self.d.numpy().astype(np.int8))
        return rel_l2(self.Y[idx].double().cpu().numpy(), ref)

    def compare(self):
        """The same apply with the skipping turned off (every reflector over all n)."""
        t = self.torch

        def timed(reps=3):
            self.run()
            t.cuda.synchronize()
            a, b = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                self.run()
            b.record()
            t.cuda.synchronize()
            return a.elapsed_time(b) / reps
        on = timed()
        self.plan.skip_prefix(0)
        off = timed()
        self.plan.skip_prefix(-1)
        full = 4.0 * self.n * self.h * self.B
        return {"skip_ms": on, "no_skip_ms": off, "speedup": off / on,
                "work_fraction": self.flops() / full, "skip_chosen_at_create": self.skip_auto}

    def e2e(self, torch):
        Xh = pinned_copy(torch, self.X)
        Yh = torch.empty(Xh.shape, dtype=Xh.dtype, pin_memory=True)
        Xd, Yd = torch.empty_like(self.X), torch.empty_like(self.X)
        chunks = []
        for r0, r1 in row_chunks(self.B, E2E_CHUNKS):
            chunks.append((lambda a=r0, b=r1: Xd[a:b].copy_(Xh[a:b], non_blocking=True),
                           lambda a=r0, b=r1: self.plan.apply_mode(self.mode, Xd[a:b],
                                                                   out=Yd[a:b]),
                           lambda a=r0, b=r1: Yh[a:b].copy_(Yd[a:b], non_blocking=True)))
        return Xh.numel() * 4, Yh.numel() * 4, chunks


def fitting_compare(torch, dev, n=128, h=16, seed=0):
    """SHF-SU (Algorithm 1) on a random symmetric n x n target: the start of step
    2 and one outer iteration through the library's kernels, beside the FP64
    oracle doing the same, with both runs' relative errors (Eq. (32))."""
    import synthetic_inputs as si
    from oracle import shf as O
    from paper_1811_07624_gb300 import shf

    S = si.random_symmetric(n, seed)
    # warm-up: the first GPU eigendecomposition loads the solver library
    torch.linalg.eigh(torch.eye(4, device=dev, dtype=torch.float64))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = shf.SHF(torch.tensor(S, device=dev), h)
    st.iterate(spectrum_update=True, inner=20)
    err_gpu = st.objective() / (4.0 * st.norm_S2)
    torch.cuda.synchronize()
    gpu_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ref = O.shf(S, h, K=1, spectrum_update_=True, inner=20, tol=0.0)
    cpu_s = time.perf_counter() - t0
    return {"n": n, "h": h, "gpu_s": gpu_s, "oracle_s": cpu_s,
            "relative_error_gpu": err_gpu, "relative_error_oracle": ref["relative_error"][-1],
            "what": "SHF-SU start (step 2) and one outer iteration, inner <= 20 steps per reflector"}


def c5_specs():
    """The 512 transforms: (n, h, batch, seed), batches scaled by --batch-scale."""
    import synthetic_inputs as si

    return [(t["n"], t["h"], max(1, int(t["batch"] * C5_SCALE)), t["seed"])
            for t in si.ragged_transforms(C5_COUNT)]


class BatchedRow:
    """512 ragged transforms (y = W x, FP32) in one graph-replayed persistent launch."""

    def __init__(self, torch, dev):
        import synthetic_inputs as si
        import paper_1811_07624_gb300 as hh

        self.name, self.torch = "batched_C5", torch
        self.specs = c5_specs()
        ns = sorted({n for n, _, _, _ in self.specs})
        t0 = time.perf_counter()
        hh.tune_clear()
        if TUNE_TABLE and os.path.exists(TUNE_TABLE):
            hh.tune_load(TUNE_TABLE)  # shapes of an earlier tuning run on this GPU
            self.tune_source = f"loaded from {TUNE_TABLE}"
        else:
            hh.tune(ns, C5_TUNE_H, rows=C5_TUNE_ROWS)
            self.tune_source = f"tuned here: n in {ns[0]}..{ns[-1]}, h in {C5_TUNE_H}"
            if TUNE_TABLE:
                hh.tune_save(TUNE_TABLE)
        self.tune_s = time.perf_counter() - t0
        self.U = [si.reflectors(n, h, seed=sd) for n, h, _, sd in self.specs]
        self.plans = [hh.Plan(torch.tensor(U, device=dev, dtype=torch.float32)) for U in self.U]
        self.batch = hh.Batch(self.plans, [b for _, _, b, _ in self.specs])
        self.plan = self.batch  # sync() after the timed region
        total = sum(n * b for n, _, b, _ in self.specs)
        g = torch.Generator(device=dev).manual_seed(77)
        self.Xbuf = torch.randn(total, device=dev, generator=g)
        self.Ybuf = torch.empty_like(self.Xbuf)
        self.Xs, self.Ys, off = [], [], 0
        for n, _, b, _ in self.specs:
            self.Xs.append(self.Xbuf[off:off + n * b].view(b, n))
            self.Ys.append(self.Ybuf[off:off + n * b].view(b, n))
            off += n * b
        self.bound = "hbm" if self.flops() / self.bytes() < 11.9 else "alu"
        info = self.batch.info()
        shapes = hh.batch_shapes()
        # kernels in the graph: one per cluster size of the resident shape in use,
        # and one for the staged shapes
        kinds = set()
        for (n, _, b, _), k in zip(self.specs, info["shapes"]):
            if b > 0:
                cl = shapes[k]["max_cluster"]
                kinds.add(-(-n // (shapes[k]["cover"] // cl)) if cl else 0)
        self.launches = len(kinds)

        def label(k):
            s = shapes[k]
            base = f"{k}:G{s['G']}xNG{s['NG']}xRT{s['RT']}"
            return base + (f" resident, <= {s['max_cluster']} CTAs" if s["max_cluster"] else "")

        self.info = {"items": info["items"], "grid": info["grid"], "tune_s": self.tune_s,
                     "tune": self.tune_source, "launches": self.launches,
                     "shape_use": {label(k): info["shapes"].count(k)
                                   for k in sorted(set(info["shapes"]))}}

    def vectors(self):
        return sum(b for _, _, b, _ in self.specs)

    def bytes(self):
        return float(sum(8 * n * b + 4 * n * h for n, h, b, _ in self.specs))

    def flops(self):
        return float(sum(4 * n * h * b for n, h, b, _ in self.specs))

    def run(self):
        self.batch.apply(self.Xs, self.Ys, mode="W")

    def parity(self):
        """Every transform on a 64-vector subset against the oracle; the worst error."""
        import oracle

        t = self.torch
        worst = 0.0
        for U, X, Y in zip(self.U, self.Xs, self.Ys):
            idx = t.linspace(0, X.shape[0] - 1, min(64, X.shape[0]), device=X.device).long()
            U32 = t.tensor(U, dtype=t.float32).double().numpy()
            ref = oracle.apply("W", U32, X[idx].double().cpu().numpy())
            worst = max(worst, rel_l2(Y[idx].double().cpu().numpy(), ref))
        return worst

    def separate(self):
        """The same transforms as 512 hh_apply calls: issued from Python one by one,
        and the same calls captured in one CUDA graph."""
        t = self.torch
        Ys = [t.empty_like(X) for X in self.Xs]

        def all_apply():
            for p, X, Y in zip(self.plans, self.Xs, Ys):
                p.apply(X, out=Y)

        def timed(fn, reps=3):
            fn()
            t.cuda.synchronize()
            a, b = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            t.cuda.synchronize()
            return a.elapsed_time(b) / reps

        ms_loop = timed(all_apply)
        s = t.cuda.Stream()
        s.wait_stream(t.cuda.current_stream())
        with t.cuda.stream(s):
            all_apply()
        t.cuda.current_stream().wait_stream(s)
        t.cuda.synchronize()
        graph = t.cuda.CUDAGraph()
        with t.cuda.graph(graph, capture_error_mode="relaxed"):
            all_apply()
        ms_graph = timed(graph.replay)
        same = max(rel_l2(a[:8].double().cpu().numpy(), b[:8].double().cpu().numpy())
                   for a, b in zip(Ys, self.Ys))
        del graph, Ys
        return {"separate_launches_ms": ms_loop, "separate_launches_graph_ms": ms_graph,
                "max_rel_diff_vs_batched": same}

    def e2e(self, torch):
        import paper_1811_07624_gb300 as hh

        Xh = pinned_copy(torch, self.Xbuf)
        Yh = torch.empty(self.Ybuf.shape, dtype=self.Ybuf.dtype, pin_memory=True)
        Xd, Yd = torch.empty_like(self.Xbuf), torch.empty_like(self.Ybuf)
        chunks, off, groups = [], 0, E2E_CHUNKS
        per = -(-len(self.specs) // groups)
        for g0 in range(0, len(self.specs), per):
            specs = self.specs[g0:g0 + per]
            batch = hh.Batch(self.plans[g0:g0 + per], [b for _, _, b, _ in specs])
            Xs, Ys, o = [], [], off
            for n, _, b, _ in specs:
                Xs.append(Xd[o:o + n * b].view(b, n))
                Ys.append(Yd[o:o + n * b].view(b, n))
                o += n * b
            chunks.append((lambda a=off, z=o: Xd[a:z].copy_(Xh[a:z], non_blocking=True),
                           lambda bt=batch, xs=Xs, ys=Ys: bt.apply(xs, ys, mode="W"),
                           lambda a=off, z=o: Yh[a:z].copy_(Yd[a:z], non_blocking=True)))
            self._e2e_batches = getattr(self, "_e2e_batches", []) + [batch]
            off = o
        return Xh.numel() * 4, Yh.numel() * 4, chunks


def make_rows(torch, dev, names):
    rows = []
    for nm in names:
        if nm.startswith("chain_"):
            rows.append(ChainRow(torch, dev, nm.split("_")[1], N_CHAIN, H_CHAIN, B_CHAIN))
        elif nm.startswith("c2_"):
            n, h, b, mode = c2_shape(nm)
            rows.append(ChainRow(torch, dev, mode, n, h, b, name=nm))
        elif nm.startswith("wy_h"):
            rows.append(WYRow(torch, dev, N_CHAIN, int(nm[4:]), B_WY))
        elif nm == "mahalanobis":
            rows.append(MahalanobisRow(torch, dev, grad=False))
        elif nm == "mahalanobis_grad":
            rows.append(MahalanobisRow(torch, dev, grad=True))
        elif nm == "adjoint_SYM":
            rows.append(AdjointRow(torch, dev))
        elif nm == "batched_C5":
            rows.append(BatchedRow(torch, dev))
        elif nm == "trunc_qr":
            rows.append(TruncRow(torch, dev))
        else:
            raise ValueError(f"unknown row {nm}")
    return rows


def c2_shape(name):
    """(n, h, batch, mode) of a row named c2_n<n>_h<h>_<mode>."""
    _, ns, hs, mode = name.split("_")
    n, h = int(ns[1:]), int(hs[1:])
    for n2, h2, b in C2_SHAPES:
        if (n2, h2) == (n, h):
            return n, h, b, mode
    raise ValueError(f"unknown row {name}")


def scale_batches(f):
    global B_CHAIN, B_WY, P_MAHAL, B_ADJ, C5_SCALE, C2_SHAPES, B_TRQ
    B_TRQ = max(1, int(B_TRQ * f))
    C2_SHAPES = [(n, h, max(1, int(b * f))) for n, h, b in C2_SHAPES]
    B_CHAIN, B_WY = max(1, int(B_CHAIN * f)), max(1, int(B_WY * f))
    P_MAHAL, B_ADJ = max(1, int(P_MAHAL * f)), max(1, int(B_ADJ * f))
    C5_SCALE = f


def config_dict(names):
    c2 = ", ".join(f"n={n} h={h} batch={b}" for n, h, b in C2_SHAPES)
    return {"workload": "Householder-chain hot path, one step = every row once: FP32 chain "
                        f"n={N_CHAIN} h={H_CHAIN} batch={B_CHAIN} (W, W^T, S); FP32 chain at "
                        f"scale {c2} (W, W^T, S each); BF16 compact-WY "
                        f"n={N_CHAIN} h=64/256/1024 batch={B_WY} (W); fast Mahalanobis n={N_MAHAL} "
                        f"h={H_MAHAL} {P_MAHAL} pairs (+ gradient); adjoint of S n={N_ADJ} "
                        f"h={H_ADJ} batch={B_ADJ}; {C5_COUNT} ragged FP32 transforms (n 128-2048, "
                        f"h 4-64, batch 1024-16384 x {C5_SCALE:g}) in one batched launch",
            "rows": list(names), "l2": "every row's inputs are larger than L2 (no flush)",
            "value_counts": "vectors transformed per second over the whole step, mixed n: a "
                            "Mahalanobis pair counts as the one difference vector it transforms; "
                            "each row's own rate and roofline fraction is under rows",
            "parallelism": "replicas (one independent copy per rank)"}


# --------------------------------------------------------------------------------------
# FP64 oracle on the host cores (cpu_baseline, --impl reference)


def oracle_units(names):
    """Host-only workloads of the rows (same shapes and seeds), each a function of
    a unit count returning nothing; units are vectors (or pairs)."""
    import oracle
    import synthetic_inputs as si

    fns = {}
    for nm in names:
        if nm.startswith("chain_") or nm.startswith("c2_"):
            if nm.startswith("chain_"):
                n, h, mode = N_CHAIN, H_CHAIN, nm.split("_")[1]
            else:
                n, h, _, mode = c2_shape(nm)
            U, d, s = si.reflectors(n, h), si.spectrum(n), si.sign(n)
            Xs = si.vectors(1024, n, seed=123)
            fns[nm] = lambda c, m=mode, U=U, d=d, s=s, Xs=Xs, n=n: oracle.apply(
                m, U, np.resize(Xs, (c, n)), sign=s, d=d)
        elif nm.startswith("wy_h"):
            h = int(nm[4:])
            U = si.reflectors(N_CHAIN, h, seed=h)
            Xs = si.vectors(64, N_CHAIN, seed=124)
            fns[nm] = lambda c, U=U, Xs=Xs: oracle.apply("W", U, np.resize(Xs, (c, N_CHAIN)))
        elif nm.startswith("mahalanobis"):
            X, labels = si.gaussian_mixture(20_000, n=N_MAHAL, seed=0)
            ia, ib, _ = si.labelled_pairs(labels, 1 << 16, seed=0)
            U, d = si.reflectors(N_MAHAL, H_MAHAL, seed=7), si.spectrum(N_MAHAL, seed=7)
            if nm.endswith("grad"):
                def f(c, X=X, ia=ia, ib=ib, U=U, d=d):
                    sel = np.arange(c) % ia.shape[0]
                    delta = X[ia[sel]] - X[ib[sel]]
                    z = oracle.apply("WT", U, delta)
                    oracle.backward("WT", U, delta, 2.0 * d[None, :] * z)
            else:
                def f(c, X=X, ia=ia, ib=ib, U=U, d=d):
                    sel = np.arange(c) % ia.shape[0]
                    oracle.mahalanobis(U, X, ia[sel], ib[sel], d)
            fns[nm] = f
        elif nm == "batched_C5":
            specs = c5_specs()
            Us = [si.reflectors(n, h, seed=sd) for n, h, _, sd in specs]
            pools = [si.vectors(16, n, seed=sd + 1) for n, _, _, sd in specs]
            wts = np.array([b for _, _, b, _ in specs], dtype=np.float64)
            wts /= wts.sum()

            def f(c, Us=Us, pools=pools, wts=wts):
                # exactly c vectors, spread over the transforms in proportion to
                # their batches (largest remainders take the leftover vectors)
                share = c * wts
                k = np.floor(share).astype(int)
                k[np.argsort(k - share)[:c - int(k.sum())]] += 1
                for U, P, ki in zip(Us, pools, k):
                    if ki > 0:
                        oracle.apply("W", U, np.resize(P, (ki, P.shape[1])))
            fns[nm] = f
        elif nm == "trunc_qr":
            from oracle import factor as OF

            R, d, _, _ = OF.result3(si.random_orthonormal(N_TRQ, 31), H_TRQ)
            Rr = R[::-1].copy()
            Xs = si.vectors(256, N_TRQ, seed=127)
            fns[nm] = lambda c, Rr=Rr, d=d, Xs=Xs: oracle.apply(
                "WT", Rr, np.resize(Xs, (c, N_TRQ)), sign=d.astype(np.int8))
        elif nm == "adjoint_SYM":
            U, d = si.reflectors(N_ADJ, H_ADJ, seed=9), si.spectrum(N_ADJ, seed=9)
            Xs, Gs = si.vectors(256, N_ADJ, seed=125), si.vectors(256, N_ADJ, seed=126)

            def f(c, U=U, d=d, Xs=Xs, Gs=Gs):
                X, G = np.resize(Xs, (c, N_ADJ)), np.resize(Gs, (c, N_ADJ))
                oracle.apply("SYM", U, X, d=d)
                oracle.backward("SYM", U, X, G, d=d)
            fns[nm] = f
    return fns


def oracle_rates(names, budget_s):
    """Per row: (units, seconds) of the oracle on a bounded sample."""
    fns = oracle_units(names)
    out = {}
    for nm, f in fns.items():
        f(4)  # first call: thread start-up, not timed
        c = 4
        while True:  # grow the sample until it takes a measurable time
            t0 = time.perf_counter()
            f(c)
            dt = time.perf_counter() - t0
            if dt >= 0.05 * budget_s or c >= (1 << 18):
                break
            c *= 4
        count = int(max(4, min(1 << 20, c * budget_s / max(dt, 1e-6))))
        t0 = time.perf_counter()
        f(count)
        out[nm] = (count, time.perf_counter() - t0)
    return out, fns


def step_vectors(names):
    per = {"chain": B_CHAIN, "wy": B_WY, "mahalanobis": P_MAHAL, "adjoint": B_ADJ,
           "trunc": B_TRQ}
    if "batched_C5" in names:
        per["batched"] = sum(b for _, _, b, _ in c5_specs())
    return {nm: c2_shape(nm)[2] if nm.startswith("c2_") else per[nm.split("_")[0]]
            for nm in names}


def run_reference(args, names):
    """The FP64 oracle on the host cores: each step runs a bounded sample of every
    row (about half a second of work each); the full step's time is the sum of
    the rows' per-unit times times their full batches."""
    rank, _, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    threads = oracle.max_threads()
    rates, fns = oracle_rates(names, budget_s=0.3)
    units = {nm: max(1, int(c / t * 0.5)) for nm, (c, t) in rates.items()}
    full = step_vectors(names)
    per_unit = {nm: [] for nm in names}
    for i in range(args.warmup + args.steps):
        for nm, f in fns.items():
            t0 = time.perf_counter()
            f(units[nm])
            if i >= args.warmup:
                per_unit[nm].append((time.perf_counter() - t0) / units[nm])
    step_s = sum(full[nm] * statistics.mean(per_unit[nm]) for nm in names)
    value = sum(full.values()) / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "vectors/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * step_s,
            "ms_per_step_kind": "extrapolated: each row's per-unit time on its bounded sample "
                                "times the row's full batch",
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian vectors, reflectors and mixture)",
            "config": config_dict(names),
            "cpu_baseline": {"value": value, "unit": "vectors/s", "cores": threads, "kind": "oracle",
                             "sample": "per step, units of each row: "
                                       + ", ".join(f"{k} {v}" for k, v in units.items())
                                       + "; the full step's time is extrapolated per unit"},
            "e2e": {"value": value, "unit": "vectors/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------------------


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", default=",".join(ALL_ROWS))
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="scale every row's batch (profiling a smaller case; not a bench line)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--tune-table", default=None,
                    help="batched launch: load tile shapes from this file if it exists, "
                         "else tune and save them there")
    ap.add_argument("--ingest-traffic", default=None, metavar="CSV",
                    help="record in --traffic-out the DRAM bytes of an ncu log whose launch i "
                         "is the first launch of the i-th of --rows, and exit (no GPU)")
    ap.add_argument("--traffic-out", default=TRAFFIC_JSON)
    ap.add_argument("--traffic-command", default="",
                    help="the ncu command line that wrote the log")
    ap.add_argument("--traffic-launches", default="",
                    help="launches per row in the log, comma separated (default 1 each)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    names = [r for r in args.rows.split(",") if r]
    if args.ingest_traffic:
        per = [int(c) for c in args.traffic_launches.split(",") if c] or None
        ingest_traffic(args.ingest_traffic, names, args.traffic_out, args.traffic_command, per)
        return 0
    global TUNE_TABLE
    TUNE_TABLE = args.tune_table
    if args.batch_scale != 1.0:
        scale_batches(args.batch_scale)
    if args.impl == "reference":
        return run_reference(args, names)

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

    dev = torch.device("cuda", local)
    rows = make_rows(torch, dev, names)
    stream = torch.cuda.current_stream()

    parity = {}
    for r in rows:  # first call and parity on sampled outputs, outside the timed region
        r.run()
        torch.cuda.synchronize()
        parity[r.name] = r.parity()
    for _ in range(args.warmup):
        for r in rows:
            r.run()
    torch.cuda.synchronize()

    ev = {r.name: [] for r in rows}
    gpu_index = local
    if "CUDA_VISIBLE_DEVICES" in os.environ:
        try:
            gpu_index = int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
        except ValueError:
            pass
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        for r in rows:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r.run()
            b.record(stream)
            ev[r.name].append((a, b))
    t1.record(stream)
    torch.cuda.synchronize()
    for r in rows:
        r.plan.sync()  # raises if a kernel in the timed region gave up a bounded wait
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    ms_step = t0.elapsed_time(t1) / args.steps
    if pg:
        from paper_1811_07624_gb300.sharding import reduce_max

        ms_step = reduce_max(ms_step, pg, dev)  # the slowest rank's step
    vec_per_step = sum(r.vectors() for r in rows)
    value = world * vec_per_step / (ms_step / 1e3)

    peaks, psrc = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    bf16_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))
    peak_of = {"hbm": peaks["hbm_gbs"], "alu": fp32_peak, "tensor": bf16_peak}
    out_rows = {}
    for r in rows:
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev[r.name])
        s = ms / 1e3
        gbs, tfl = r.bytes() / s / 1e9, r.flops() / s / 1e12
        ach = gbs if r.bound == "hbm" else tfl
        traffic = profiled_traffic(r.name, r.vectors())
        out_rows[r.name] = {"ms": ms, "vectors_per_s": r.vectors() / s, "GB_s": gbs,
                            "TFLOP_s": tfl, "bound": r.bound, "frac": ach / peak_of[r.bound],
                            "hbm_frac": gbs / peaks["hbm_gbs"], "launches": r.launches,
                            "rel_l2_vs_oracle": parity[r.name], "dram_traffic_bytes": traffic}
    c2_rows = [r for r in rows if r.name.startswith("c2_")]
    c2 = None
    if c2_rows:
        c2_ms = sum(out_rows[r.name]["ms"] for r in c2_rows)
        c2 = {"rows": [r.name for r in c2_rows], "ms": c2_ms,
              "vectors_per_s": sum(r.vectors() for r in c2_rows) / (c2_ms / 1e3),
              "GB_s": sum(r.bytes() for r in c2_rows) / (c2_ms / 1e3) / 1e9,
              "min_frac": min(out_rows[r.name]["frac"] for r in c2_rows),
              "max_rel_l2_vs_oracle": max(out_rows[r.name]["rel_l2_vs_oracle"] for r in c2_rows)}
    dom = max(rows, key=lambda r: out_rows[r.name]["ms"])
    d = out_rows[dom.name]
    psource = {"hbm": f"hbm_gbs {psrc}",
               "alu": f"FP32 FMA: {sms} SMs x 128 lanes x 2 flops x "
                      f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz (sm_max_mhz {psrc})",
               "tensor": f"bf16_tflops_sustained {psrc} (kernel timed inside a long step)"}
    roof = {"bound": dom.bound, "achieved": d["GB_s"] if dom.bound == "hbm" else d["TFLOP_s"],
            "peak": peak_of[dom.bound], "unit": "GB/s" if dom.bound == "hbm" else "TFLOP/s",
            "frac": d["frac"], "traffic": d["dram_traffic_bytes"], "kernel": dom.name,
            "peak_source": psource[dom.bound]}

    # The end-to-end step runs right after the device-timed steps, before the
    # auxiliary comparisons below (their allocations slowed the host copies by
    # up to 30% when they ran first).
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(torch, rows, stream, world, pg, dev, vec_per_step)

    compare = None
    if not args.no_compare and any(isinstance(r, WYRow) for r in rows):
        compare = compare_fp32(torch, dev, [r for r in rows if isinstance(r, WYRow)], out_rows)
    trunc_vs = None
    for r in rows:
        if isinstance(r, TruncRow) and not args.no_compare:
            trunc_vs = r.compare()
    batched_vs = None
    for r in rows:
        if isinstance(r, BatchedRow):
            out_rows[r.name].update(r.info)
            if not args.no_compare:
                batched_vs = r.separate()
                batched_vs["batched_ms"] = out_rows[r.name]["ms"]
                batched_vs["speedup_vs_separate"] = (batched_vs["separate_launches_ms"]
                                                     / out_rows[r.name]["ms"])
                batched_vs["speedup_vs_separate_graph"] = (batched_vs["separate_launches_graph_ms"]
                                                           / out_rows[r.name]["ms"])

    fitting = None
    if rank == 0 and not args.no_compare:
        fitting = fitting_compare(torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rates, _ = oracle_rates(names, budget_s=2.0)
        full = step_vectors(names)
        step_s = sum(full[nm] * t / c for nm, (c, t) in rates.items())
        cpu = {"value": vec_per_step / step_s, "unit": "vectors/s", "cores": oracle.max_threads(),
               "kind": "oracle",
               "sample": "; ".join(f"{k}: {c} units in {t:.2f} s" for k, (c, t) in rates.items())
                         + " (the full step's time extrapolated from each row's per-unit time)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "vectors/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 (chain, distance, adjoint); bf16 storage with f32 accumulation (WY)",
                "data": "synthetic (seeded Gaussian vectors, reflectors and mixture)",
                "config": config_dict(names), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * sum(r.launches for r in rows), "clocks": clocks,
                "rows": out_rows, "c2": c2, "bf16_wy_vs_fp32_chain": compare,
                "batched_vs_separate": batched_vs, "trunc_qr_skip_vs_dense": trunc_vs,
                "shf_su_fit": fitting,
                "fp32_peak_tflops": fp32_peak}
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


def compare_fp32(torch, dev, wy_rows, out_rows):
    """The FP32 chain on the WY rows' shapes and data: time and error vs the oracle."""
    from paper_1811_07624_gb300 import Plan
    import oracle

    out = {}
    for r in wy_rows:
        pf = Plan(torch.tensor(r.U, device=dev, dtype=torch.float32))
        X32 = r.X.float()
        Y32 = torch.empty_like(X32)
        for _ in range(2):
            pf.apply(X32, out=Y32)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            pf.apply(X32, out=Y32)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 3
        idx = torch.linspace(0, r.B - 1, 32, device=dev).long()
        ref = oracle.apply("W", r.U, r.X[idx].double().cpu().numpy())
        out[r.name] = {"fp32_chain_ms": ms, "bf16_wy_ms": out_rows[r.name]["ms"],
                       "speedup": ms / out_rows[r.name]["ms"],
                       "fp32_chain_rel_l2": rel_l2(Y32[idx].double().cpu().numpy(), ref),
                       "bf16_wy_rel_l2": rel_l2(r.Y[idx].double().cpu().numpy(), ref),
                       "errors_vs": "FP64 oracle on the unrounded reflectors and the BF16 inputs"}
        del pf, X32, Y32
    return out


def measure_e2e(torch, rows, stream, world, pg, dev, vec_per_step, steps=5, warm=2):
    """The step through the public API from pinned host memory, results read back.

    Every row's work is split into chunks (copy in, compute, copy out); the
    chunks of all rows are pipelined over three streams, so the copies of one
    chunk overlap the compute of another.  Per chunk, the copy in waits for the
    previous step's compute on that chunk, and the compute for the previous
    step's copy out."""
    parts = [r.e2e(torch) for r in rows]
    h2d = sum(p[0] for p in parts)
    d2h = sum(p[1] for p in parts)
    # a chunk is (copy in, compute, copy out[, key]): its compute waits for the
    # last copy out of the same key (by default the same chunk in the previous
    # step), i.e. for the output buffers it is about to overwrite
    chunks = [c if len(c) == 4 else tuple(c) + (("chunk", i),)
              for i, c in enumerate(c for p in parts for c in p[2])]
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    last_comp = [None] * len(chunks)
    last_out = {}

    def step():
        for i, (cin, comp, cout, key) in enumerate(chunks):
            with torch.cuda.stream(s_in):
                if last_comp[i] is not None:
                    s_in.wait_event(last_comp[i])
                cin()
                e_in = torch.cuda.Event()
                e_in.record(s_in)
            with torch.cuda.stream(s_comp):
                s_comp.wait_event(e_in)
                if key in last_out:
                    s_comp.wait_event(last_out[key])
                comp()
                last_comp[i] = torch.cuda.Event()
                last_comp[i].record(s_comp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(last_comp[i])
                cout()
                last_out[key] = torch.cuda.Event()
                last_out[key].record(s_out)

    for _ in range(warm):  # first touches of the pinned buffers are not timed
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s_in.wait_event(a)
    for _ in range(steps):
        step()
    for s in (s_in, s_comp, s_out):
        e = torch.cuda.Event()
        e.record(s)
        stream.wait_event(e)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    if pg:
        from paper_1811_07624_gb300.sharding import reduce_max

        ms = reduce_max(ms, pg, dev)
    return {"value": world * vec_per_step / (ms / 1e3), "unit": "vectors/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": steps,
            "pipelining": f"{len(chunks)} chunks over copy-in, compute and copy-out streams"}

if __name__ == "__main__":
    sys.exit(main())
