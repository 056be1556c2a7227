#!/usr/bin/env python3
"""Benchmark: PLS + rank of a 65536 x 65536 dense GF(2) matrix (the headline).

One step = gf2_pls (PLS decomposition and rank, in place, MMPF panels with
XOR-table sweeps) on a matrix that is already resident in HBM; the matrix is
restored from a pristine copy before each step, outside the timed events. The
512 MB input is larger than L2 (129 MB), so no extra flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gf2|reference]
                  [--config 1|2|3|4|5] [--variants]

--config 3 (default) is the headline line above; --config 3 --variants times
the three 65536^2 matrices (dense, A = B.C, Bernoulli(0.01)) through MMPF and
the recursive PLS with both products; --config 2 and 1 time 16384^2 and 1024^2
PLS + RREF; --config 4 the 2048-matrix batch; --config 5 the request stream.

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
SEED = 0x10061744
PAPER_CONTEXT = {"value_s": 151.314, "machine": "2.33 GHz Xeon E5345 (CPU)",
                 "what": "PLS + RREF from PLS, random dense n = 64000 (the nearest to 65536), Table 1",
                 "note": "context only: another machine, and it includes the RREF"}


def effective_bitops(m: int, n: int, r: int) -> float:
    """AND + XOR count of classical elimination: 2 * sum_{i<r} (m-1-i)(n-1-i), summed in closed form."""
    a, c = m - 1, n - 1
    s = r * a * c - (a + c) * (r * (r - 1) // 2) + (r - 1) * r * (2 * r - 1) // 6
    return float(2 * s)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_value(name: str, key: str):
    """A figure of one ncu-captured launch of a kernel, as recorded in profiles/<name>.md (a line
    "<key>: X"); None if there is no such capture or line."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    try:
        for line in open(path):
            if line.startswith(key + ":"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null") else float(v)
    except OSError:
        pass
    return None


def traffic_from_profiles(name: str):
    """DRAM bytes over algorithmic bytes of one ncu-captured launch ("traffic_ratio")."""
    return profile_value(name, "traffic_ratio")


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


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_seconds(n: int, rref: bool = False, omp: bool = False) -> float:
    """The oracle as it stands: Gaussian PLS (plus Gauss-Jordan RREF when rref) of one n x n matrix.
    omp: the same PLS with the rows of each step spread over all host threads."""
    import oracle
    from paper_1006_1744_gb300 import synth
    A = synth.dense(n, n, SEED)
    t0 = time.perf_counter()
    (oracle.pls_omp if omp else oracle.pls)(A, n, n)
    if rref:
        oracle.rref(A, n, n)
    return time.perf_counter() - t0


def cpu_baseline(n: int, rref: bool):
    """Single-thread oracle (the oracle of record) on a bounded sample, scaled to n x n by the
    cubic cost, plus the all-cores OpenMP timing of the same sample."""
    ns = min(n, 16384)
    scale = (n / ns) ** 3
    secs = cpu_oracle_seconds(ns, rref)
    what = "Gaussian PLS" + (" + Gauss-Jordan RREF" if rref else "")
    out = {"value": secs * scale, "unit": "s", "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
           "sample": f"one {ns}x{ns} dense matrix: {what} (C oracle, single thread), {secs:.2f} s, "
                     f"x {scale:g} for the cubic cost at {n}x{n}"}
    if not rref:
        try:
            threads = os.cpu_count() or 1
            so = cpu_oracle_seconds(ns, False, omp=True)
            out["all_cores"] = {"value": so * scale, "unit": "s", "cores": threads, "kind": "oracle (OpenMP over "
                                "the rows of each pivot step)", "sample_s": so, "sample": f"the same {ns}x{ns} PLS"}
        except Exception as exc:  # no OpenMP runtime on this host
            out["all_cores"] = {"unavailable": str(exc)[:200]}
    return out


def run_reference(args):
    """Reference arm: the CPU oracle timed on the host cores, on the headline workload
    (seconds per PLS + rank of a dense n x n matrix). Each step is one bounded sample: the
    oracle's Gaussian PLS of an 8192 x 8192 dense matrix (single thread); its time is scaled by
    (n / 8192)^3, the cubic cost, to the metric's unit. ms_per_step is the sample's own time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n = args.n or (65536 if args.config == 3 else 16384 if args.config == 2 else 1024)
    ns = min(n, 8192)
    scale = (n / ns) ** 3
    for _ in range(args.warmup):
        cpu_oracle_seconds(ns)
    t0 = time.perf_counter()
    times = [cpu_oracle_seconds(ns) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    sample_s = sum(times) / len(times)
    v = sample_s * scale
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sample_s * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{n}x{n} dense Bernoulli(1/2) GF(2): PLS + rank", "m": n, "n": n, "seed": SEED},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": f"per step one {ns}x{ns} dense matrix (Gaussian PLS, C oracle, single thread; "
                                   f"ms_per_step is that sample's time); value = sample x {scale:g} for the cubic "
                                   f"cost at {n}x{n}"},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The slowest rank's value (every rank gets it); the identity for one process."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_matrix(step_ms_max: float, world: int) -> float:
    """Replicas: every rank eliminates its own matrix per step, so the job finishes
    world matrices per (slowest) step."""
    return step_ms_max / 1e3 / world


def _timed(fn, steps, warmup, pre=None):
    """CUDA-event time of fn() (ms), mean over steps after warmup; pre() runs untimed before each."""
    import torch
    for _ in range(warmup):
        if pre:
            pre()
        fn()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        if pre:
            pre()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def _freivalds(A, B, C, m, k, n, trials=2, seed=1):
    """CPU check that A = B.C over GF(2): A.x == B.(C.x) for random bit vectors x."""
    import numpy as np
    rng = np.random.default_rng(seed)
    pc = np.array([bin(i).count("1") & 1 for i in range(256)], dtype=np.uint8)

    def matvec(M, rows, cols, x):
        W = (cols + 63) // 64
        t = (M[:rows, :W] & x[None, :W]).view(np.uint8).reshape(rows, -1)
        return np.bitwise_xor.reduce(pc[t], axis=1).astype(np.uint8)

    def pack(bits, stride_words):
        out = np.zeros(stride_words * 64, dtype=np.uint8)
        out[:bits.size] = bits
        return np.packbits(out, bitorder="little").view(np.uint64)

    for _ in range(trials):
        xb = rng.integers(0, 2, n, dtype=np.uint8)
        x = pack(xb, C.shape[1])
        cx = matvec(C, k, n, x)
        lhs = matvec(A, m, n, x)
        rhs = matvec(B, m, k, pack(cx, B.shape[1]))
        if not np.array_equal(lhs, rhs):
            return False
    return True


def _base_line(args, value, unit, ms, config, clocks, launches, extra):
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": config, "clocks": clocks, "gpu_launches": launches}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_config3(args):
    """65536 x 65536 matrices (512 MB packed): dense Bernoulli(1/2), A = B.C with B 65536 x 32768 and
    C 32768 x 65536 (rank <= 32768), and Bernoulli(0.01); each through the panel elimination alone
    (MMPF) and the recursive PLS with the XOR-table and the tensor-core trailing product."""
    import numpy as np
    import torch
    from paper_1006_1744_gb300 import build, gf2, synth, synth_gpu
    build.build()
    n = 65536
    k = 32768
    st = synth.default_stride(n)
    dev = torch.device("cuda", 0)
    A0 = torch.empty((n, st), dtype=torch.int64, device=dev)
    A = torch.empty_like(A0)
    methods = {"mmpf": None, "mmpf_1panel": {"panels_per_sweep": 1},
               "rec_xor": {"cutoff_cols": 4096, "product": 1}, "rec_tc": {"cutoff_cols": 4096, "product": 2}}
    steps = max(1, min(args.steps, 3))
    results = {}
    checks = {}
    sampler = ClockSampler(0)
    sampler.start()
    gf2.prof_reset()
    gf2.prof_enable(1)
    for variant in ("dense", "product", "sparse01"):
        if variant == "dense":
            synth_gpu.fill(A0, n, SEED)
        elif variant == "sparse01":
            synth_gpu.fill(A0, n, SEED + 2, p=0.01)
        else:
            B = torch.empty((n, synth.default_stride(k)), dtype=torch.int64, device=dev)
            C = torch.empty((k, st), dtype=torch.int64, device=dev)
            synth_gpu.fill(B, k, SEED + 3)
            synth_gpu.fill(C, n, SEED + 4)
            gf2.mul(A0, B, C, n, k, n, opts={"product": 1})
            torch.cuda.synchronize()
            checks["product_freivalds"] = _freivalds(A0.cpu().numpy().view("uint64"), B.cpu().numpy().view("uint64"),
                                                     C.cpu().numpy().view("uint64"), n, k, n)
            del B, C
        results[variant] = {}
        for name, o in methods.items():
            rank = torch.empty(1, dtype=torch.int64, device=dev)
            Qb = torch.empty(n, dtype=torch.int64, device=dev)
            ms = _timed(lambda: gf2.pls(A, n, Q=Qb, rank=rank, opts=o), steps, 1, pre=lambda: A.copy_(A0))
            results[variant][name] = {"ms": ms, "rank": int(rank.item())}
            if name in ("mmpf", "mmpf_1panel"):
                # the sweeps' algorithmic bytes (read + write of every sweep's trailing block: one
                # sweep per panel, or per two panels at this size by default) over the whole
                # elimination's time: a lower bound on the sweeps' HBM rate
                rv = int(rank.item())
                W = (n + 63) // 64
                Qh = Qb[:rv].cpu().numpy()
                byts = (sweep_algorithmic_bytes(Qh, n, W, rv) if name == "mmpf_1panel"
                        else pair_sweep_algorithmic_bytes(Qh, n, W, rv))
                hbm, _ = peaks()
                gbs = byts / (ms * 1e-3) / 1e9
                results[variant][name].update({"sweep_algorithmic_GB": byts / 1e9, "sweep_GBps_over_elimination": gbs,
                                               "hbm_frac": gbs / hbm})
        # the same matrix to its reduced echelon form by each route of gf2_rref
        wr = gf2.new_workspace(gf2.OP_RREF, n, n, device=dev)
        rk = torch.empty(1, dtype=torch.int64, device=dev)
        piv = torch.empty(n, dtype=torch.int64, device=dev)
        for name, meth in (("rref_pls_route", gf2.RREF_PLS), ("rref_m4ri", gf2.RREF_M4RI),
                           ("rref_hybrid", gf2.RREF_HYBRID)):
            ms = _timed(lambda: gf2.rref(A, n, rank=rk, pivots=piv, work=wr, opts={"rref_method": meth}), steps, 1,
                        pre=lambda: A.copy_(A0))
            results[variant][name] = {"ms": ms, "rank": int(rk.item())}
        del wr
        torch.cuda.empty_cache()
    gf2.prof_enable(0)
    clocks = sampler.stop()
    best = results["dense"]["mmpf"]["ms"]
    speed = {v: {"two_panels_over_one": r["mmpf_1panel"]["ms"] / r["mmpf"]["ms"],
                 "rec_tc_over_rec_xor": r["rec_xor"]["ms"] / r["rec_tc"]["ms"],
                 "mmpf_over_rec_xor": r["rec_xor"]["ms"] / r["mmpf"]["ms"],
                 "mmpf_over_rec_tc": r["rec_tc"]["ms"] / r["mmpf"]["ms"]} for v, r in results.items()}
    _base_line(args, best / 1e3, "s", best,
               {"workload": "65536x65536 GF(2): dense Bernoulli(1/2), A=B.C (B 65536x32768, C 32768x65536), "
                            "Bernoulli(0.01); gf2_pls by MMPF panels and by the recursive PLS (cutoff 4096 columns) "
                            "with XOR-table and tensor-core products", "m": n, "n": n, "seed": SEED,
                "value_is": "dense, MMPF"},
               clocks, gf2.prof_launches(),
               {"results_ms": results, "speedups": speed, "checks": checks,
                "bitops_per_s_dense_mmpf": effective_bitops(n, n, results["dense"]["mmpf"]["rank"]) / (best / 1e3)})
    return 0


def run_config4(args):
    """2048 independent matrices in one gf2_pls_batched call (shapes and densities of the batch recipe):
    the persistent schedule (one cooperative launch; the default) and the per-step schedule, against
    the same matrices through gf2_pls one by one."""
    import numpy as np
    import torch
    from paper_1006_1744_gb300 import build, gf2, synth, synth_gpu
    build.build()
    dev = torch.device("cuda", 0)
    rec = synth.batch_recipe(2048, SEED)
    mats0, ns = [], []
    for (m, n, p, sd) in rec:
        D = torch.empty((m, synth.default_stride(n)), dtype=torch.int64, device=dev)
        synth_gpu.fill(D, n, sd, p=p)
        mats0.append(D)
        ns.append(n)
    mats = [x.clone() for x in mats0]
    shapes = [(m, n, synth.default_stride(n)) for (m, n, p, sd) in rec]
    nb = gf2.pls_batched_workspace_bytes(shapes)
    work = torch.empty(nb // 8 + 64, dtype=torch.int64, device=dev)
    Ps = [torch.empty(m, dtype=torch.int64, device=dev) for (m, *_r) in rec]
    Qs = [torch.empty(n, dtype=torch.int64, device=dev) for n in ns]
    ranks = torch.empty(len(rec), dtype=torch.int64, device=dev)

    def restore():
        for a, b in zip(mats, mats0):
            a.copy_(b)

    sampler = ClockSampler(0)
    sampler.start()
    gf2.prof_reset()
    gf2.prof_enable(1)
    by_mode = {}
    schedules = {"persistent": {"batch_mode": gf2.BATCH_PERSISTENT},
                 "steps_tile16": {"batch_mode": gf2.BATCH_STEPS, "tile_words": 16},
                 "steps_tile8": {"batch_mode": gf2.BATCH_STEPS, "tile_words": 8}}
    rank_sets = {}
    for name, o in schedules.items():
        by_mode[name] = _timed(lambda: gf2.pls_batched(mats, ns, Ps, Qs, ranks, work=work, opts=o),
                               args.steps, args.warmup, pre=restore)
        rank_sets[name] = ranks.cpu().numpy().copy()
    launches = gf2.prof_launches()
    gf2.prof_enable(0)
    clocks = sampler.stop()
    best_name = min(by_mode, key=by_mode.get)
    best = by_mode[best_name]
    rank_sum = int(ranks.sum().item())
    same = all((v == rank_sets["persistent"]).all() for v in rank_sets.values())
    # algorithmic sweep bytes of every member (read + write of each panel's trailing words)
    byts = 0.0
    rk = rank_sets["persistent"]
    for i, (m, n, p, sd) in enumerate(rec):
        W = (n + 63) // 64
        byts += sweep_algorithmic_bytes(Qs[i].cpu().numpy(), m, W, int(rk[i]))
    hbm, peak_kind = peaks()
    t_pers = by_mode["persistent"]
    achieved = byts / (t_pers * 1e-3) / 1e9
    roofline = {"kernel": "k_batch_persist (the whole batch: pivot searches, sweeps, finishing)", "bound": "hbm",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_kind": peak_kind, "traffic": None,
                "algorithmic_bytes_per_launch": byts, "avg_launch_us": t_pers * 1e3,
                "note": "one launch per batch: the members' sweep bytes over the batch time (pivot searches "
                        "and barriers included, so this is a lower bound of the sweeps' own rate)"}
    # the same matrices one call each (one timed pass)
    w1 = gf2.new_workspace(gf2.OP_PLS, max(m for m, *_r in rec), max(ns))
    r1 = torch.empty(len(rec), dtype=torch.int64, device=dev)

    def loop():
        for i in range(len(rec)):
            gf2.pls(mats[i], ns[i], Ps[i], Qs[i], r1[i:i + 1], work=w1)

    loop_ms = _timed(loop, 1, 1, pre=restore)
    total_bytes = sum(m * synth.default_stride(n) * 8 for (m, n, p, sd) in rec)
    _base_line(args, best / 1e3, "s", best,
               {"workload": "2048 GF(2) matrices in one gf2_pls_batched call: rows log-uniform in [256, 8192], "
                            "cols = rows x U[0.5, 2] rounded to 64, density from {0.5, 0.1, 0.01}",
                "matrices": len(rec), "bytes": total_bytes, "seed": SEED, "value_is": "seconds per batch"},
               clocks, launches,
               {"matrices_per_s": len(rec) / (best / 1e3),
                "bitops_per_s": sum(effective_bitops(m, n, int(rk[i])) for i, (m, n, p, sd) in enumerate(rec)) / (best / 1e3),
                "ms_by_schedule": by_mode, "schedule": best_name,
                "roofline": roofline, "loop_of_gf2_pls_ms": loop_ms, "speedup_vs_loop": loop_ms / best,
                "rank_sum": rank_sum, "ranks_equal_across_schedules": bool(same),
                "ranks_equal_to_loop": bool((r1.cpu().numpy() == rk).all())})
    return 0


def run_config5(args):
    """Request stream: echelon-structured matrices arriving as a Poisson process at
    0.5, 0.8 and 1.0 times the measured capacity. Matrices are generated and kept on
    the device. The server has two lanes, each with its own stream and workspace: small
    requests (m < 8192) and large ones. Whenever a lane is idle, every request of its
    class that has arrived is admitted as long as the lane's workspace budget allows, and
    runs as one gf2_pls_batched call on the lane's stream (the per-step schedule, whose
    launches from the two lanes run side by side); a lane's batch completes when its event
    does. Latency = completion - arrival. Capacity = the same server with every request
    queued at time 0."""
    import numpy as np
    import torch
    from paper_1006_1744_gb300 import build, gf2, synth, synth_gpu
    build.build()
    dev = torch.device("cuda", 0)
    R = max(16, args.requests)
    rec = synth.request_recipe(R, SEED)
    mats0, mats, ns = [], [], []
    for (m, n, sd) in rec:
        D = torch.empty((m, synth.default_stride(n)), dtype=torch.int64, device=dev)
        synth_gpu.fill(D, n, sd, p=0.3, echelon_frac=0.5)
        mats0.append(D)
        mats.append(torch.empty_like(D))
        ns.append(n)
    Ps = [torch.empty(m, dtype=torch.int64, device=dev) for (m, n, sd) in rec]
    Qs = [torch.empty(n, dtype=torch.int64, device=dev) for n in ns]
    ranks = torch.empty(R, dtype=torch.int64, device=dev)
    shapes = [(m, n, synth.default_stride(n)) for (m, n, sd) in rec]
    ws_each = [gf2.pls_batched_workspace_bytes([sh]) for sh in shapes]
    free, _total = torch.cuda.mem_get_info(dev)
    total_budget = int(free * 0.6)
    SPLIT = 8192
    classes = [[i for i in range(R) if rec[i][0] < SPLIT], [i for i in range(R) if rec[i][0] >= SPLIT]]
    shares = (0.25, 0.75)
    single = args.large_lane_cap == 1  # large requests one at a time through gf2_pls
    if single:
        gf2.replay_enable(0)  # every request has its own buffers: no graph is worth capturing
        for i in classes[1]:
            ws_each[i] = gf2.workspace_bytes(gf2.OP_PLS, rec[i][0], rec[i][1])
    lanes = []
    for c, share in zip(classes, shares):
        need = gf2.pls_batched_workspace_bytes([shapes[i] for i in c]) if c else 0
        bud = int(min(total_budget * share, need)) if c else 0
        bud = max(bud, max((ws_each[i] for i in c), default=0))
        lanes.append({"ids": c, "budget": bud, "stream": torch.cuda.Stream(device=dev),
                      "cap": (args.large_lane_cap or R) if share == shares[1] else R,
                      "single": single and share == shares[1],
                      "work": torch.empty(max(bud, 256) // 8 + 64, dtype=torch.int64, device=dev)})
    opts = {"batch_mode": gf2.BATCH_STEPS}

    def launch(lane, ids):
        with torch.cuda.stream(lane["stream"]):
            for i in ids:
                mats[i].copy_(mats0[i])
            rk = torch.empty(len(ids), dtype=torch.int64, device=dev)
            if lane.get("single"):
                # one request: the single-matrix pipeline (look-ahead pivot searches beside the sweeps)
                i = ids[0]
                gf2.pls(mats[i], ns[i], P=Ps[i], Q=Qs[i], rank=rk[0:1], work=lane["work"], stream=lane["stream"])
            else:
                gf2.pls_batched([mats[i] for i in ids], [ns[i] for i in ids], [Ps[i] for i in ids],
                                [Qs[i] for i in ids], rk, work=lane["work"], opts=opts, stream=lane["stream"])
            ev = torch.cuda.Event()
            ev.record(lane["stream"])
        return rk, ev

    def serve(arr):
        """Run the whole stream with arrival times arr (seconds); returns completion times, batches."""
        comp = np.zeros(R)
        nb = 0
        state = [{"next": 0, "inflight": None} for _ in lanes]
        start = time.perf_counter()
        remaining = R
        while remaining:
            now = time.perf_counter() - start
            busy = False
            for L, st in zip(lanes, state):
                if st["inflight"] is not None:
                    ids, rk, ev = st["inflight"]
                    if not ev.query():
                        busy = True
                        continue
                    t = time.perf_counter() - start
                    comp[ids] = t
                    ranks[ids] = rk
                    remaining -= len(ids)
                    st["inflight"] = None
                c = L["ids"]
                ids, need = [], 0
                k = st["next"]
                cap = L["cap"]
                if cap < 0:
                    # adaptive: small batches while few requests wait (latency), larger ones as the
                    # queue grows (throughput)
                    waiting = int(np.searchsorted(arr[c[k:]], now, side="right")) if k < len(c) else 0
                    cap = max(-cap, waiting // 2)
                while k < len(c) and arr[c[k]] <= now:
                    if ids and (need + ws_each[c[k]] > L["budget"] or len(ids) >= cap):
                        break
                    ids.append(c[k])
                    need += ws_each[c[k]]
                    k += 1
                if ids:
                    st["next"] = k
                    rk, ev = launch(L, ids)
                    st["inflight"] = (ids, rk, ev)
                    nb += 1
                    busy = True
            if not busy:
                pending = [arr[L["ids"][st["next"]]] for L, st in zip(lanes, state) if st["next"] < len(L["ids"])]
                if pending:
                    time.sleep(max(0.0, min(min(pending) - (time.perf_counter() - start), 0.0005)))
            else:
                time.sleep(0.0001)
        return comp, nb

    serve(np.zeros(R))  # warm-up (first calls, graph captures)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    comp0, _ = serve(np.zeros(R))
    capacity = R / comp0.max()

    sampler = ClockSampler(0)
    sampler.start()
    gf2.prof_reset()
    gf2.prof_enable(1)
    results = {}
    for frac in (0.5, 0.8, 1.0):
        lam = frac * capacity
        arr = synth.arrival_times(R, lam, SEED + int(frac * 100))
        comp, nbatch = serve(arr)
        lat = comp - arr
        small = np.array([rec[i][0] < SPLIT for i in range(R)])
        results[f"{frac:.1f}"] = {
            "rate_per_s": lam, "throughput_per_s": R / comp.max(), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "batches": nbatch, "mean_batch": R / nbatch,
            "p99_small_ms": float(np.percentile(lat[small], 99) * 1e3) if small.any() else None,
            "p99_large_ms": float(np.percentile(lat[~small], 99) * 1e3) if (~small).any() else None}
    launches = gf2.prof_launches()
    gf2.prof_enable(0)
    clocks = sampler.stop()
    v = results["0.8"]["p99_ms"]
    _base_line(args, v / 1e3, "s", v,
               {"workload": "request stream: echelon-structured GF(2) matrices (m log-uniform in [512, 32768], "
                            "n = m to 2m, row i zero before column 0.5 i n / m, Bernoulli(0.3) after), Poisson "
                            "arrivals at 0.5, 0.8, 1.0 x capacity, batched as they arrive in two lanes (m < 8192, "
                            "m >= 8192), PLS + rank",
                "requests": R, "seed": SEED, "value_is": "p99 latency at 0.8 x capacity",
                "large_lane_cap": args.large_lane_cap or None,
                "workspace_budget_bytes": [L["budget"] for L in lanes]},
               clocks, launches,
               {"capacity_per_s": capacity, "by_load": results, "rank_sum": int(ranks.sum().item()),
                "requests_by_lane": [len(c) for c in classes]})
    return 0


def sweep_algorithmic_bytes(Q, m: int, W: int, r: int) -> float:
    """Read + write bytes of the trailing blocks of all panels: panel b sweeps the (m - r_b) x (W - b)
    trailing words, r_b = pivots left of column 64 b ((m - r)(n - c)/4 bytes per sweep of 64 columns)."""
    import numpy as np
    rb = np.searchsorted(np.asarray(Q[:r]), 64 * np.arange(W))
    return float(np.sum((m - rb).clip(min=0) * (W - np.arange(W)) * 16.0))


def pair_sweep_algorithmic_bytes(Q, m: int, W: int, r: int) -> float:
    """Two panels per sweep: the sweep of panels b, b + 1 (b even) streams words b + 4 .. W - 1 of the
    rows from position r_b on (words b .. b + 3 are its front's), read + write: (m - r_b)(W - b - 4) x 16."""
    import numpy as np
    b = np.arange(0, W, 2)
    b = b[b + 4 < W]
    rb = np.searchsorted(np.asarray(Q[:r]), 64 * b)
    return float(np.sum((m - rb).clip(min=0) * (W - b - 4) * 16.0))


def side_numbers_16384(g, dev, steps: int):
    """16384^2 figures kept beside the headline: gf2_pls, and gf2_rref by the PLS route, by
    Algorithm M4RI and by the hybrid (CUDA events, L2 flushed before each call)."""
    import torch
    from paper_1006_1744_gb300 import synth_gpu
    n = 16384
    A0 = torch.empty((n, 256), dtype=torch.int64, device=dev)
    synth_gpu.fill(A0, n, SEED)
    A = torch.empty_like(A0)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.int64, device=dev)
    rk = torch.empty(1, dtype=torch.int64, device=dev)
    piv = torch.empty(n, dtype=torch.int64, device=dev)
    P = torch.empty(n, dtype=torch.int64, device=dev)
    Q = torch.empty(n, dtype=torch.int64, device=dev)
    wp = g.new_workspace(g.OP_PLS, n, n, device=dev)
    wr = g.new_workspace(g.OP_RREF, n, n, device=dev)

    def pre():
        A.copy_(A0)
        flush.zero_()

    out = {"pls_s": _timed(lambda: g.pls(A, n, P=P, Q=Q, rank=rk, work=wp), steps, 3, pre) / 1e3}
    for name, meth in (("rref_pls_route_s", g.RREF_PLS), ("rref_m4ri_s", g.RREF_M4RI),
                       ("rref_hybrid_s", g.RREF_HYBRID)):
        out[name] = _timed(lambda: g.rref(A, n, rank=rk, pivots=piv, work=wr, opts={"rref_method": meth}),
                           steps, 3, pre) / 1e3
    out["rank"] = int(rk.item())
    out["note"] = "16384^2 dense (32 MB, L2-resident within a call); CUDA events; L2 flushed before each call"
    return out


def run_headline(args):
    """PLS + rank of a dense n x n matrix (config 3: n = 65536, the headline), or PLS + RREF
    (configs 2 and 1: n = 16384, 1024)."""
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
    n = m = args.n or {1: 1024, 2: 16384, 3: 65536}[args.config]
    with_rref = args.config in (1, 2)
    W = (n + 63) // 64
    stride = max(16, (W + 15) // 16 * 16)
    opts = {}
    if args.tile_words:
        opts["tile_words"] = args.tile_words
    if args.panels_per_sweep:
        opts["panels_per_sweep"] = args.panels_per_sweep
    opts = opts or None
    big = m * stride * 8 > 256 * 1024 * 1024  # input larger than L2: no flush needed

    A0 = torch.empty((m, stride), dtype=torch.int64, device=dev)
    synth_gpu.fill(A0, n, SEED + rank)
    A1 = torch.empty_like(A0)
    A2 = torch.empty_like(A0) if with_rref else None
    wp = gf2.new_workspace(gf2.OP_PLS, m, n, device=dev, opts=opts)
    wr = gf2.new_workspace(gf2.OP_RREF, m, n, device=dev, opts=opts) if with_rref else None
    P = torch.empty(m, dtype=torch.int64, device=dev)
    Q = torch.empty(n, dtype=torch.int64, device=dev)
    r1 = torch.empty(1, dtype=torch.int64, device=dev)
    r2 = torch.empty(1, dtype=torch.int64, device=dev)
    piv = torch.empty(n, dtype=torch.int64, device=dev)
    flush = None if big else torch.empty(256 * 1024 * 1024 // 8, dtype=torch.int64, device=dev)

    def restore():
        A1.copy_(A0)
        if with_rref:
            A2.copy_(A0)
        if flush is not None:
            flush.zero_()

    def step():
        gf2.pls(A1, n, P=P, Q=Q, rank=r1, work=wp, opts=opts)
        if with_rref:
            gf2.rref(A2, n, rank=r2, pivots=piv, work=wr, opts=opts)

    for _ in range(args.warmup):
        restore()
        step()
    torch.cuda.synchronize()

    # ---- timed region: restore (untimed) then the step between two events --------------
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    gf2.prof_reset()
    gf2.prof_enable(1)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        restore()
        starts[i].record()
        step()
        ends[i].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    gf2.prof_enable(0)
    clocks = sampler.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / args.steps
    launches = gf2.prof_launches()

    # ---- per-kernel-class times: untimed steps with an event pair around each launch of the
    # timed classes, on the stream it runs on ----------------------------------------------
    prof_steps = 1 if n >= 32768 else 3
    gf2.prof_reset()
    gf2.prof_enable(3)
    for _ in range(prof_steps):
        restore()
        step()
    torch.cuda.synchronize()
    gf2.prof_enable(0)
    sweep_ms, sweep_n = gf2.prof_collect(gf2.PROF_SWEEP)
    pivot_ms, pivot_n = gf2.prof_collect(gf2.PROF_PIVOT)
    rref_blk_ms, rref_blk_n = gf2.prof_collect(gf2.PROF_RREF)
    front_ms, front_n = gf2.prof_collect(gf2.PROF_COORDS)
    gf2.prof_reset()
    pair = front_n > 0  # two panels per sweep ran (the library's choice at this size, or --panels-per-sweep 2)

    step_ms_max = max_over_ranks(step_ms, world, dev)
    rank_val = int(r1.item())
    if with_rref:
        assert rank_val == int(r2.item())
    elims = 2 if with_rref else 1  # gf2_rref's PLS route runs the elimination too
    bytes_fn = pair_sweep_algorithmic_bytes if pair else sweep_algorithmic_bytes
    sweep_bytes = bytes_fn(Q.cpu().numpy(), m, W, rank_val) * elims * prof_steps
    hbm, peak_kind = peaks()
    shares = {"sweep": sweep_ms, "pivot": pivot_ms, "rref_block": rref_blk_ms}
    if pair:
        shares["front"] = front_ms
    tot = sum(shares.values()) or 1.0
    dominant = max(shares, key=shares.get)
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9 if sweep_ms > 0 else 0.0
    bytes_per_launch = sweep_bytes / max(sweep_n, 1)
    prof_name = f"k_pair_sweep_{n}" if pair else f"k_sweep16_{n}"
    traffic_ratio = traffic_from_profiles(prof_name)
    # a capture of an earlier build of the kernel gives no traffic for this one
    stale = profile_value(prof_name, "captured_kernel_current") == 0
    ratio_at_capture = traffic_ratio
    if stale:
        traffic_ratio = None
    kname = ("k_pair_sweep (table sweep of two panels: MakeTable1 + AddRowsFromTable over 128 pivot columns)"
             if pair else "k_sweep16 (table sweep: MakeTable1 + AddRowsFromTable)")
    roofline = {"kernel": kname, "bound": "hbm",
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst)" if peak_kind == "measured"
                else peak_kind,
                "traffic": traffic_ratio * bytes_per_launch if traffic_ratio else None,
                "traffic_note": (f"DRAM bytes / algorithmic bytes of one captured launch (profiles/{prof_name}.md) "
                                 "x the average launch's algorithmic bytes" if traffic_ratio else
                                 f"null: the kernel changed after its capture (profiles/{prof_name}.md); that "
                                 f"earlier build's DRAM / algorithmic bytes: {ratio_at_capture}" if stale
                                 else "no capture"),
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_us": sweep_ms * 1e3 / max(sweep_n, 1),
                "binding_unit": {"unit": "L1/shared-memory data port (l1tex throughput, pct of peak)",
                                 "frac": profile_value(prof_name, "l1_port_frac"),
                                 "source": f"profiles/{prof_name}.md (one captured launch"
                                           + (", an earlier build of the kernel)" if stale else ")")}
                if pair else None,
                "note": ("bytes per sweep of panels b, b + 1 = (m - r_b)(W - b - 4) x 16 (read + write of the "
                         "trailing words right of the front's four); half the DRAM traffic per panel of one "
                         "sweep per panel, at the same shared-memory lookups per panel, so the kernel is bound "
                         "by the L1/shared-memory data port (profiles/k_pair_sweep_*.md) before DRAM; "
                         if pair else "bytes per panel = (m - r_b)(W - b) x 16 (read + write of the trailing "
                         "words); ")
                        + ("the matrix is L2-resident within a step" if not big else "input larger than L2")}
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    pivot_us = pivot_ms * 1e3 / max(pivot_n, 1)
    floor_us = 64 * (26 + 38) / sm_mhz
    pivot_chain = {"kernel": ("k_pivot_pair" if pair else "k_pivot") + " (panel pivot search: PlsSubmatrix)",
                   "bound": "latency",
                   "avg_launch_us": pivot_us, "chain_floor_us": floor_us,
                   "frac": floor_us / pivot_us if pivot_us else 0.0,
                   "note": "1 CTA; the elimination chain of 64 pivots (warp min-reduction 26 cycles + 64-bit "
                           "shuffle 38 cycles per pivot), plus window formation and the inverses"}

    # ---- end to end through the C ABI: pinned host buffers, copies inside the timed region ---
    # Every step copies its input in from pinned host memory, runs the elimination and copies its
    # results out. Two sets of buffers alternate, with the copies on streams of their own, so step
    # i + 1's input copy and step i - 1's result copy overlap step i's elimination (the way a
    # caller streams matrices through the library); the timed region covers all of it.
    e2e = None
    if not args.no_e2e:
        hA = torch.empty((m, stride), dtype=torch.int64, pin_memory=True)
        hA.copy_(A0.cpu())
        comp = torch.cuda.current_stream(dev)
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        sets = []
        for k in range(2):
            sets.append({
                "A": A1 if k == 0 else torch.empty_like(A0),
                "A2": (A2 if k == 0 else torch.empty_like(A0)) if with_rref else None,
                "P": P if k == 0 else torch.empty_like(P), "Q": Q if k == 0 else torch.empty_like(Q),
                "r1": r1 if k == 0 else torch.empty_like(r1), "r2": r2 if k == 0 else torch.empty_like(r2),
                "piv": piv if k == 0 else torch.empty_like(piv),
                "hOut1": torch.empty_like(hA, pin_memory=True),
                "hOut2": torch.empty_like(hA, pin_memory=True) if with_rref else None,
                "hP": torch.empty(m, dtype=torch.int64, pin_memory=True),
                "hQ": torch.empty(n, dtype=torch.int64, pin_memory=True),
                "hpiv": torch.empty(n, dtype=torch.int64, pin_memory=True),
                "hr": torch.empty(2, dtype=torch.int64, pin_memory=True),
                "ev_in": torch.cuda.Event(), "ev_done": torch.cuda.Event(), "ev_out": torch.cuda.Event()})
        for d in sets:
            d["ev_out"].record(s_out)

        def e2e_step(i):
            d = sets[i & 1]
            with torch.cuda.stream(s_in):
                s_in.wait_event(d["ev_out"])  # this set's previous results are out
                d["A"].copy_(hA, non_blocking=True)
                d["ev_in"].record(s_in)
            comp.wait_event(d["ev_in"])
            if with_rref:
                d["A2"].copy_(d["A"])
            gf2.pls(d["A"], n, P=d["P"], Q=d["Q"], rank=d["r1"], work=wp, opts=opts)
            if with_rref:
                gf2.rref(d["A2"], n, rank=d["r2"], pivots=d["piv"], work=wr, opts=opts)
            d["ev_done"].record(comp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(d["ev_done"])
                d["hOut1"].copy_(d["A"], non_blocking=True)
                d["hP"].copy_(d["P"], non_blocking=True)
                d["hQ"].copy_(d["Q"], non_blocking=True)
                d["hr"][0:1].copy_(d["r1"], non_blocking=True)
                if with_rref:
                    d["hOut2"].copy_(d["A2"], non_blocking=True)
                    d["hpiv"].copy_(d["piv"], non_blocking=True)
                    d["hr"][1:2].copy_(d["r2"], non_blocking=True)
                d["ev_out"].record(s_out)

        for i in range(2):  # warm-up: both buffer sets (first calls, graph captures)
            e2e_step(i)
        torch.cuda.synchronize()
        e2e_steps = max(3, min(args.steps, 10))
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        es.record(comp)
        s_in.wait_event(es)
        s_out.wait_event(es)
        for i in range(e2e_steps):
            e2e_step(i)
        comp.wait_stream(s_out)
        ee.record(comp)
        torch.cuda.synchronize()
        te_ms = max_over_ranks(es.elapsed_time(ee) / e2e_steps, world, dev)
        last = sets[(e2e_steps - 1) & 1]
        assert int(last["hr"][0].item()) == int(r1.item())  # the results did come back
        bi = m * stride * 8
        bo = m * stride * 8 + (m + n + 1) * 8 + ((m * stride * 8 + n * 8 + 8) if with_rref else 0)
        e2e = {"value": job_seconds_per_matrix(te_ms, world), "unit": "s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": te_ms, "steps": e2e_steps,
               "note": "two buffer sets: step i + 1's input copy and step i - 1's result copy overlap "
                       "step i's elimination; all inside the timed region"}

    side = None
    if args.config == 3 and not args.no_side:
        side = side_numbers_16384(gf2, dev, 10)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, with_rref)

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    value = job_seconds_per_matrix(step_ms_max, world)
    what = "PLS + rank" if not with_rref else "PLS + rank, plus the same matrix through gf2_rref"
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{n}x{n} dense Bernoulli(1/2) GF(2): {what}; MMPF panels with XOR-table "
                               f"sweeps (k = 8 per table, {128 if pair else 64} pivots per sweep)",
                   "m": m, "n": n, "seed": SEED, "parallelism": f"replicas x{world}",
                   "l2": ("input (512 MB) larger than L2; restored from a pristine copy before each step, "
                          "outside the timed events") if big else
                         "flushed between timed steps (256 MB write, excluded from the step time)"},
        "rank": rank_val,
        "bitops_per_s": effective_bitops(m, n, rank_val) / (step_ms_max / 1e3 / (elims if with_rref else 1)),
        "wall_s_timed_region": wall,
        "roofline": roofline, "pivot_chain": pivot_chain,
        "kernel_time_shares": {k: v / tot for k, v in shares.items()}, "dominant_kernel": dominant,
        "kernel_launches": {"sweep": sweep_n, "pivot": pivot_n, "rref_block": rref_blk_n, "front": front_n,
                            "steps": prof_steps},
        "gpu_launches": launches,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks, "paper_context": PAPER_CONTEXT,
    }
    if side:
        line["config2_16384"] = side
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gf2", choices=["gf2", "reference"])
    ap.add_argument("--n", type=int, default=0, help="matrix size of the headline form (default: by config)")
    ap.add_argument("--tile-words", type=int, default=0)
    ap.add_argument("--panels-per-sweep", type=int, default=0, choices=[0, 1, 2],
                    help="panels per table sweep of the PLS elimination (0: the library's choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="config 3: skip the 16384^2 side figures")
    ap.add_argument("--config", type=int, default=3, choices=[1, 2, 3, 4, 5],
                    help="3: 65536^2 PLS + rank (the headline, default); 2 / 1: 16384^2 / 1024^2 PLS + RREF; "
                         "4: batched PLS of 2048 matrices; 5: a stream of requests with Poisson arrivals")
    ap.add_argument("--variants", action="store_true",
                    help="config 3: the three 65536^2 matrices through MMPF and the recursive PLS")
    ap.add_argument("--requests", type=int, default=4096, help="config 5: requests per arrival rate")
    ap.add_argument("--large-lane-cap", type=int, default=0,
                    help="config 5: most requests per batch of the large lane (0: no cap; -k: at least k, "
                         "else half of those waiting)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.config == 3 and args.variants:
        return run_config3(args)
    if args.config == 4:
        return run_config4(args)
    if args.config == 5:
        return run_config5(args)
    return run_headline(args)


if __name__ == "__main__":
    sys.exit(main())
