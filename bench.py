#!/usr/bin/env python3
"""Benchmark: PLS + rank, plus RREF, of a 16384 x 16384 dense GF(2) matrix.

One step = gf2_pls (PLS decomposition and rank, in place) and gf2_rref (the
same matrix through the reduced-row-echelon route) on copies of a matrix that
is already resident in HBM; the copies are restored at the start of each step.
L2 (129 MB) is flushed between timed steps by writing a 256 MB buffer; the
per-step device time excludes that flush.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gf2|reference]

Prints one JSON line (rank 0). Under torchrun (N > 1) every rank eliminates its
own matrix (replicas: the elimination of one matrix has no data-parallel
exchange step); time = max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "seconds per PLS+rank of n×n dense GF(2); effective bit-op/s, % of roofline"
N_DEFAULT = 16384
SEED = 0x10061744
PAPER_CONTEXT = {"value_s": 3.388, "machine": "2.33 GHz Xeon E5345 (CPU)",
                 "what": "PLS + RREF from PLS, random dense n=16384, Table 1", "note": "context only"}


def effective_bitops(m: int, n: int, r: int) -> float:
    """AND + XOR count of classical elimination: 2 * sum_{i<r} (m-1-i)(n-1-i)."""
    return float(sum(2 * (m - 1 - i) * (n - 1 - i) for i in range(r)))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_from_profiles(name: str):
    """DRAM bytes per launch of `name` recorded from an ncu capture in profiles/."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null") else float(v)
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(n: int):
    """The oracle as it stands (single-threaded C): Gaussian PLS + Gauss-Jordan RREF of one matrix."""
    import oracle
    from paper_1006_1744_gb300 import synth
    A = synth.dense(n, n, SEED)
    t0 = time.perf_counter()
    oracle.pls(A, n, n)
    oracle.rref(A, n, n)
    return time.perf_counter() - t0


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.n
    ns = min(n, 8192)  # bounded sample per step; time scaled by (n/ns)^3 (cubic elimination)
    scale = (n / ns) ** 3
    for _ in range(args.warmup):
        cpu_oracle_sample(ns)
    times = [cpu_oracle_sample(ns) * scale for _ in range(args.steps)]
    v = sum(times) / len(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{n}x{n} dense Bernoulli(1/2) GF(2): PLS + rank, plus RREF", "m": n, "n": n,
                   "seed": SEED},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"per step one {ns}x{ns} matrix (Gaussian PLS + Gauss-Jordan RREF, single "
                                   f"thread), time x {scale:g} for the cubic cost at {n}x{n}"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gf2", choices=["gf2", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--tile-words", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1006_1744_gb300 import build, gf2, synth_gpu
    build.build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n = m = args.n
    W = (n + 63) // 64
    stride = max(16, (W + 15) // 16 * 16)
    opts = {"tile_words": args.tile_words} if args.tile_words else None

    A0 = torch.empty((m, stride), dtype=torch.int64, device=dev)
    synth_gpu.fill(A0, n, SEED + rank)
    A1 = torch.empty_like(A0)
    A2 = torch.empty_like(A0)
    wp = gf2.new_workspace(gf2.OP_PLS, m, n, device=dev)
    wr = gf2.new_workspace(gf2.OP_RREF, m, n, device=dev)
    P = torch.empty(m, dtype=torch.int64, device=dev)
    Q = torch.empty(n, dtype=torch.int64, device=dev)
    r1 = torch.empty(1, dtype=torch.int64, device=dev)
    r2 = torch.empty(1, dtype=torch.int64, device=dev)
    piv = torch.empty(n, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        A1.copy_(A0)
        A2.copy_(A0)
        gf2.pls(A1, n, P=P, Q=Q, rank=r1, work=wp, opts=opts)
        gf2.rref(A2, n, rank=r2, pivots=piv, work=wr, opts=opts)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    # separate timing of the two calls (one extra untimed step) for the breakdown
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    flush.zero_()
    A1.copy_(A0)
    A2.copy_(A0)
    ev[0].record()
    gf2.pls(A1, n, P=P, Q=Q, rank=r1, work=wp, opts=opts)
    ev[1].record()
    flush.zero_()
    ev[2].record()
    gf2.rref(A2, n, rank=r2, pivots=piv, work=wr, opts=opts)
    ev[3].record()
    torch.cuda.synchronize()
    pls_ms = ev[0].elapsed_time(ev[1])
    rref_ms = ev[2].elapsed_time(ev[3])

    # ---- timed region ----------------------------------------------------------------
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    gf2.prof_reset()
    gf2.prof_enable(3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record()
        step()
        ends[i].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    gf2.prof_enable(0)
    clocks = sampler.stop()
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    launches = gf2.prof_launches()
    sweep_ms, sweep_n = gf2.prof_collect(gf2.PROF_SWEEP)
    pivot_ms, pivot_n = gf2.prof_collect(gf2.PROF_PIVOT)
    rref_blk_ms, rref_blk_n = gf2.prof_collect(gf2.PROF_RREF)
    gf2.prof_reset()

    t = torch.tensor([step_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    step_ms_max = float(t.item())

    rank_val = int(r1.item())
    assert rank_val == int(r2.item())
    # algorithmic bytes of the table sweeps: panel b reads and writes the (m - r_b) x (W - b)
    # trailing words (the panel word included); r_b = pivots left of column 64 b
    q = Q[:rank_val].cpu().numpy()
    rb = np.searchsorted(q, 64 * np.arange(W))
    sweep_bytes_one = float(np.sum((m - rb).clip(min=0) * (W - np.arange(W)) * 16.0))
    sweep_bytes = 2 * sweep_bytes_one * args.steps  # both calls run the elimination
    hbm, peak_kind = peaks()
    shares = {"sweep": sweep_ms, "pivot": pivot_ms, "rref_block": rref_blk_ms}
    tot = sum(shares.values()) or 1.0
    dominant = max(shares, key=shares.get)
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9 if sweep_ms > 0 else 0.0
    roofline = {"kernel": "k_sweep (table sweep: MakeTable1 + AddRowsFromTable)", "bound": "hbm",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                "traffic": traffic_from_profiles("k_sweep_16384"),
                "algorithmic_bytes_per_launch": sweep_bytes / max(sweep_n, 1),
                "avg_launch_us": sweep_ms * 1e3 / max(sweep_n, 1),
                "note": "16384^2 packed is 32 MB and stays in the 129 MB L2 within a step"}

    # ---- end to end: host buffers, copies inside the timed region ---------------------
    e2e = None
    if not args.no_e2e:
        hA = torch.empty((m, stride), dtype=torch.int64, pin_memory=True)
        hA.copy_(A0.cpu())
        hOut1 = torch.empty_like(hA, pin_memory=True)
        hOut2 = torch.empty_like(hA, pin_memory=True)
        hP = torch.empty(m, dtype=torch.int64, pin_memory=True)
        hQ = torch.empty(n, dtype=torch.int64, pin_memory=True)
        hpiv = torch.empty(n, dtype=torch.int64, pin_memory=True)
        hr = torch.empty(2, dtype=torch.int64, pin_memory=True)

        def e2e_step():
            A1.copy_(hA, non_blocking=True)
            A2.copy_(A1)
            gf2.pls(A1, n, P=P, Q=Q, rank=r1, work=wp, opts=opts)
            gf2.rref(A2, n, rank=r2, pivots=piv, work=wr, opts=opts)
            hOut1.copy_(A1, non_blocking=True)
            hOut2.copy_(A2, non_blocking=True)
            hP.copy_(P, non_blocking=True)
            hQ.copy_(Q, non_blocking=True)
            hpiv.copy_(piv, non_blocking=True)
            hr[0:1].copy_(r1, non_blocking=True)
            hr[1:2].copy_(r2, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        es.record()
        for _ in range(args.steps):
            e2e_step()
        ee.record()
        torch.cuda.synchronize()
        te = torch.tensor([es.elapsed_time(ee) / args.steps], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        bi = m * stride * 8
        bo = 2 * m * stride * 8 + (m + 2 * n + 2) * 8
        e2e = {"value": float(te.item()) / 1e3 / world, "unit": "s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": float(te.item())}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        secs = cpu_oracle_sample(n)
        cpu = {"value": secs, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"one full {n}x{n} matrix: Gaussian PLS + Gauss-Jordan RREF (C oracle, single thread)"}

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    value = step_ms_max / 1e3 / world
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{n}x{n} dense Bernoulli(1/2) GF(2): MMPF-style PLS + rank with XOR-table "
                               f"trailing updates (k = 8), plus the same matrix through gf2_rref",
                   "m": m, "n": n, "seed": SEED, "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MB write, excluded from the step time)"},
        "pls_s": pls_ms / 1e3, "rref_s": rref_ms / 1e3, "rank": rank_val,
        "bitops_per_s": effective_bitops(m, n, rank_val) / (pls_ms / 1e3),
        "wall_s_timed_region": wall,
        "roofline": roofline,
        "kernel_time_shares": {k: v / tot for k, v in shares.items()}, "dominant_kernel": dominant,
        "kernel_launches": {"sweep": sweep_n, "pivot": pivot_n, "rref_block": rref_blk_n},
        "gpu_launches": launches,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks, "paper_context": PAPER_CONTEXT,
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
