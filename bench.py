#!/usr/bin/env python3
"""Benchmark: stable Merge Path merge of the large unbalanced key-value
workload on GB300.

Workload: A = 2^28 and B = 2^26 uint64 keys, each with a uint32 payload
(its global source index); keys uniform over the full 64-bit range, sorted
(other distributions: --dist a_gt_b | interleaved | distinct16).  One step
= one mp_merge_pairs call (partition kernel + merge-tile kernel) over the
whole workload, inputs resident in HBM.  Inputs and outputs (8.05 GB per
pass) are far larger than the 129 MB L2, so no flush is needed between
steps.

Printed (rank 0, one JSON line): Gkeys/s of merged output, the roofline of
the merge-tile kernel (algorithmic bytes 2 * n * (8 + 4) per launch over
its CUDA-event duration, against the measured HBM copy peak), the CPU
oracle timed on the host, the end-to-end rate through the host-buffer C
entry point (copies included), the SM clocks seen while timing, and the
number of kernels launched in the timed region.

--impl reference times the plain CPU oracle (the program this library is
checked against) on a bounded sample of the same workload.

Multi-GPU (torchrun): every rank merges its own copy of the workload (weak
scaling, no data-path collective); time = max over ranks.
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

import numpy as np  # noqa: E402

METRIC = "merge Gkeys/s & % of HBM peak; batched/served vs per-call on same GPU; p99"
UNIT = "Gkeys/s"
NOMINAL_HBM_GBS = 7900.0
PEAK_FALLBACK_GBS = 6800.0
KERNEL_SOURCES = ["paper_1406_2628_gb300/csrc/merge_bulk.cu", "paper_1406_2628_gb300/csrc/mp_tile.cuh",
                  "paper_1406_2628_gb300/csrc/mp_device.cuh", "paper_1406_2628_gb300/csrc/mp_bulk.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "merge_tile_kernel_large_kv_traffic.json")
SORT_BLOCK_4B = 512 * 33  # keys per block-sort tile for 4-byte keys alone (the first of the sort's HBM passes)


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--dist", default="uniform", choices=["uniform", "a_gt_b", "interleaved", "distinct16"])
    p.add_argument("--log2-a", type=int, default=28)
    p.add_argument("--log2-b", type=int, default=26)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--plan", default=None, help="NT,VT tile plan (default: automatic)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the other workloads (plain keys, sort, batched, serving)")
    p.add_argument("--extras", default="dists,plain,sort,batched,serving,setops,wide,crossover,tiles",
                   help="comma list of extra workloads to run after the headline")
    p.add_argument("--serving-requests", type=int, default=50000)
    p.add_argument("--sort-log2-n", type=int, default=28, help="keys of the sort extra (log2)")
    p.add_argument("--tiles-log2-n", type=int, default=27, help="keys per side of the tiles extra (log2)")
    p.add_argument("--batched-segments", type=int, default=16384, help="segments of the batched extra")
    p.add_argument("--setops-log2-universe", type=int, default=28,
                   help="key universe of the set-operation extra (log2; each set holds about half)")
    return p.parse_args()


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return PEAK_FALLBACK_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_key):
    """DRAM bytes per merge-kernel launch from a committed ncu summary, if it
    was taken on the current kernel source; else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    entry = d.get("workloads", {}).get(workload_key)
    return None if entry is None else float(entry["traffic_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi SM clock / throttle samples every 100 ms in the background,
    kept for the span from the first warm-up step to the end of a ~1 s soak
    of the same step after the timed region and the per-kernel timing."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "utilization.gpu")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 11:
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        rows = [r for (t, r) in self.rows if t0 <= t <= t1]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        busy = [r for r in rows if (num(r[10]) or 0) > 0] or rows
        sm = [num(r[2]) for r in busy if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in busy:
            for name, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max((num(r[3]) or 0) for r in busy),
                "reasons": sorted(reasons), "samples": len(busy),
                "power_w_max": max((num(r[4]) or 0) for r in busy)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (all ranks get it)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: int, ms: float, world: int) -> float:
    """Whole-job rate in G units/s: every rank processed units_per_rank in at
    most ms milliseconds (the max over ranks)."""
    return units_per_rank * world / (ms * 1e-3) / 1e9


def workload(args, seed_offset=0):
    import gen
    n_a, n_b = 1 << args.log2_a, 1 << args.log2_b
    return gen.large_kv(args.dist, n_a=n_a, n_b=n_b, seed=gen.BASE_SEED + seed_offset)


def config_dict(args, n_ranks):
    return {"workload": "large_kv_merge", "n_a": 1 << args.log2_a, "n_b": 1 << args.log2_b,
            "key": "uint64", "value": "uint32 (global source index)", "dist": args.dist,
            "bytes_per_pass": 2 * ((1 << args.log2_a) + (1 << args.log2_b)) * 12,
            "l2": "no flush: inputs+outputs 8.05 GB per pass >> 129 MB L2",
            "parallelism": f"replicas x{n_ranks}" if n_ranks > 1 else "single GPU",
            "plan": args.plan or "auto"}


# --------------------------------------------------------------------- oracle

def oracle_rate(a, av, b, bv, target_s=10.0, max_s=30.0):
    """Time the CPU oracle on the full workload, repeated to ~target_s."""
    import oracle
    oracle.build()
    n = a.size + b.size
    t0 = time.perf_counter()
    oracle.merge(a, b, av, bv)
    t1 = time.perf_counter() - t0
    reps = 1
    extra = max(0, min(int(math.ceil(target_s / max(t1, 1e-3))) - 1, int(max_s / max(t1, 1e-3)) - 1))
    total = t1
    if extra:
        t0 = time.perf_counter()
        for _ in range(extra):
            oracle.merge(a, b, av, bv)
        total += time.perf_counter() - t0
        reps += extra
    return n * reps / total / 1e9, reps, total


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    a, av, b, bv = workload(args)
    n = a.size + b.size
    # Bounded sample: the first m outputs of the merge (a true sub-merge:
    # A[:a(m)] with B[:m - a(m)]), m sized so the whole run stays within
    # about two minutes.
    calib = min(n, 1 << 24)
    sa, _ = oracle.split(a, b, calib)
    t0 = time.perf_counter()
    oracle.merge(a[:sa], b[:calib - sa], av[:sa], bv[:calib - sa])
    rate = calib / (time.perf_counter() - t0)
    budget_per_step = 100.0 / max(1, args.steps + args.warmup)
    m = int(min(n, max(1 << 20, rate * budget_per_step)))
    sa, _ = oracle.split(a, b, m)
    A, AV, B, BV = a[:sa], av[:sa], b[:m - sa], bv[:m - sa]
    for _ in range(args.warmup):
        oracle.merge(A, B, AV, BV)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.merge(A, B, AV, BV)
    el = time.perf_counter() - t0
    value = m * args.steps / el / 1e9
    sample = f"first {m} outputs of the workload (A[:{sa}] + B[:{m - sa}]), {args.steps} steps"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": config_dict(args, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- extras
#
# The other workloads, reported under "extras" in the same JSON line.  Inputs
# for these are generated on the device (torch / mp_generate): they measure
# speed; their exactness is covered by the parity tests.

def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def extra_plain(mp, torch, dev, reps=50):
    """2 x 2^20 int32 keys, uniform in [0, 2^24), sorted; warm (L2-resident)
    and cold (L2 flushed by a 512 MB write before each call)."""
    import gen
    a, b = gen.plain_keys()
    A, B = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    out = torch.empty(a.size + b.size, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(5):
        mp.mp_merge_keys(A, B, out)
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(reps):
        mp.mp_merge_keys(A, B, out)
    e1.record()
    torch.cuda.synchronize(dev)
    warm_us = e0.elapsed_time(e1) / reps * 1e3
    cold = []
    for _ in range(reps // 2):
        flush.fill_(1)
        e0.record()
        mp.mp_merge_keys(A, B, out)
        e1.record()
        torch.cuda.synchronize(dev)
        cold.append(e0.elapsed_time(e1) * 1e3)
    n = a.size + b.size
    cold_us = statistics.median(cold)
    # The same merge through the partitioned tile path (partition + merge
    # kernels), which automatic plans use above the streaming threshold.
    tile = (0, 0, mp.MP_STAGE_BULK)
    tcold = []
    for _ in range(reps // 2):
        flush.fill_(1)
        e0.record()
        mp.mp_merge_plan(A, B, out_keys=out, plan=tile)
        e1.record()
        torch.cuda.synchronize(dev)
        tcold.append(e0.elapsed_time(e1) * 1e3)
    return {"n": n, "call": "mp_merge_keys (automatic plan: streaming merge, one launch)",
            "warm_us": warm_us, "cold_us": cold_us, "gkeys_s_warm": n / warm_us / 1e3,
            "gkeys_s_cold": n / cold_us / 1e3, "gbs_cold": 2 * n * 4 / cold_us / 1e3,
            "partitioned_cold_us": statistics.median(tcold)}


def extra_tiles(mp, torch, dev, log2_n=27, reps=10):
    """Keys-only merges of 2 x 2^log2_n keys through the TMA tile path at
    several tile shapes (block threads, items per thread): uniform int32 and
    int64 keys, and int32 runs with every A below every B (each tile then
    comes from one side, the case where an even count per thread puts a
    warp's serial walks into two banks).  Partition + merge per call."""
    g = torch.Generator(device=dev)
    g.manual_seed(0x2628)
    n = 1 << log2_n
    e0, e1 = _events(torch)
    res = {"n_a": n, "n_b": n}
    bulk = mp.MP_STAGE_BULK
    cases = [("i32_uniform", torch.int32, False, [(256, 16), (256, 12), (256, 33), (128, 33)]),
             ("i32_a_below_b", torch.int32, True, [(256, 16), (256, 12), (256, 33), (128, 33)]),
             ("i64_uniform", torch.int64, False, [(256, 12), (128, 16), (128, 27)])]
    for name, dt, ordered, shapes in cases:
        if ordered:
            A = torch.arange(n, dtype=dt, device=dev)
            B = torch.arange(n, 2 * n, dtype=dt, device=dev)
        else:
            hi = (1 << 31) - 1 if dt == torch.int32 else 1 << 62
            A = torch.sort(torch.randint(-hi, hi, (n,), dtype=dt, device=dev, generator=g)).values
            B = torch.sort(torch.randint(-hi, hi, (n,), dtype=dt, device=dev, generator=g)).values
        out = torch.empty(2 * n, dtype=dt, device=dev)
        row = {}
        for nt, vt in shapes:
            plan = (nt, vt, bulk)
            for _ in range(3):
                mp.mp_merge_plan(A, B, out_keys=out, plan=plan)
            e0.record()
            for _ in range(reps):
                mp.mp_merge_plan(A, B, out_keys=out, plan=plan)
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            row[f"{nt}x{vt}"] = {"ms": ms, "gbs": 2 * 2 * n * A.element_size() / ms / 1e6}
        res[name] = row
        del A, B, out
    return res


def extra_crossover(mp, torch, dev, reps=15):
    """Small merges: the streaming plan (one launch) against partition + TMA
    tiles, sorted uniform keys, L2 flushed before each call (median of reps),
    at 2^16 .. 2^24 outputs, int32 keys and uint64 keys with values."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    e0, e1 = _events(torch)
    res = {}
    for name, kd, vals in [("i32", torch.int32, False), ("u64_pairs", torch.int64, True)]:
        for lg in (16, 18, 20, 21, 22, 23, 24):
            n = 1 << (lg - 1)
            g = torch.Generator(device=dev)
            g.manual_seed(lg)
            x = torch.sort(torch.randint(0, 1 << 30, (n,), device=dev, dtype=kd, generator=g)).values
            y = torch.sort(torch.randint(0, 1 << 30, (n,), device=dev, dtype=kd, generator=g)).values
            o = torch.empty(2 * n, dtype=kd, device=dev)
            xv = torch.arange(n, dtype=torch.int32, device=dev)
            ov = torch.empty(2 * n, dtype=torch.int32, device=dev)
            row = {}
            for plan_name, plan in [("stream", (0, 0, mp.MP_STAGE_STREAM)), ("tiles", (0, 0, mp.MP_STAGE_BULK))]:
                def call():
                    if vals:
                        mp.mp_merge_plan(x, y, xv, xv, o, ov, plan=plan)
                    else:
                        mp.mp_merge_plan(x, y, out_keys=o, plan=plan)
                for _ in range(3):
                    call()
                ts = []
                for _ in range(reps):
                    flush.fill_(1)
                    e0.record()
                    call()
                    e1.record()
                    torch.cuda.synchronize(dev)
                    ts.append(e0.elapsed_time(e1) * 1e3)
                row[plan_name + "_us"] = statistics.median(ts)
            res[f"{name}_2^{lg}"] = row
    return res


def extra_wide(mp, torch, dev, log2_n=25, reps=5):
    """128-bit keys (two 64-bit words, low first), unsigned: merge of two
    sorted arrays of 2^25 keys each (uniform random words), and a sort of
    2^25 random keys.  Inputs are made sorted on the device with mp_sort
    (outside the timed region)."""
    g = torch.Generator(device=dev)
    g.manual_seed(0x1406_2628)
    n = 1 << log2_n
    lo, hi = -(1 << 63), (1 << 63) - 1

    def rand_keys():
        return torch.randint(lo, hi, (n, 2), dtype=torch.int64, device=dev, generator=g)
    A, B = rand_keys(), rand_keys()
    mp.mp_sort(A, wide="u128")
    mp.mp_sort(B, wide="u128")
    out = torch.empty((2 * n, 2), dtype=torch.int64, device=dev)
    res = {"n_a": n, "n_b": n, "key": "uint128 (2 x uint64, low word first)"}
    e0, e1 = _events(torch)
    for name, plan in [("merge_auto", None), ("merge_stream", (128, 8, mp.MP_STAGE_STREAM))]:
        mp.mp_merge_plan(A, B, out_keys=out, plan=plan, wide="u128")
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(reps):
            mp.mp_merge_plan(A, B, out_keys=out, plan=plan, wide="u128")
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms": ms, "gkeys_s": 2 * n / ms / 1e6, "gbs": 2 * 2 * n * 16 / ms / 1e6}
    X = rand_keys()
    W = torch.empty(mp.mp_sort_workspace_bytes(mp.MP_U128, n, False), dtype=torch.uint8, device=dev)
    ts = []
    for _ in range(3):
        Y = X.clone()
        torch.cuda.synchronize(dev)
        e0.record()
        mp.mp_sort(Y, workspace=W, wide="u128")
        e1.record()
        torch.cuda.synchronize(dev)
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    res["sort"] = {"n": n, "ms": ms, "gkeys_s": n / ms / 1e6}
    return res


def extra_setops(mp, torch, dev, log2_universe=28, reps=5):
    """Set operations on two duplicate-free sorted sets of ~2^27 uint32 keys,
    each key of [0, 2^28) in each set with probability 1/2 (independent), so
    about half of each set is in the other; keys only, and union with values."""
    g = torch.Generator(device=dev)
    g.manual_seed(0x14062628)
    u = 1 << log2_universe
    A = torch.nonzero(torch.rand(u, device=dev, generator=g) < 0.5).flatten().to(torch.int32)
    B = torch.nonzero(torch.rand(u, device=dev, generator=g) < 0.5).flatten().to(torch.int32)
    na, nb = A.numel(), B.numel()
    out = torch.empty(na + nb, dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    res = {"na": na, "nb": nb, "key": "uint32 (as int32 < 2^28)"}
    e0, e1 = _events(torch)
    for op in ["union", "intersection", "difference", "symmetric_difference"]:
        mp.mp_set_operation(op, A, B, out_keys=out, count=cnt, trim=False)
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(reps):
            mp.mp_set_operation(op, A, B, out_keys=out, count=cnt, trim=False)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        k = int(cnt.item())
        res[op] = {"ms": ms, "out": k, "gkeys_s": (na + nb) / ms / 1e6,
                   "gbs": (na + nb + k) * 4 / ms / 1e6}
    AV = torch.arange(na, dtype=torch.int32, device=dev)
    BV = torch.arange(nb, dtype=torch.int32, device=dev)
    OV = torch.empty(na + nb, dtype=torch.int32, device=dev)
    mp.mp_set_operation("union", A, B, AV, BV, out, OV, count=cnt, trim=False)
    torch.cuda.synchronize(dev)
    e0.record()
    for _ in range(reps):
        mp.mp_set_operation("union", A, B, AV, BV, out, OV, count=cnt, trim=False)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    k = int(cnt.item())
    res["union_pairs"] = {"ms": ms, "out": k, "gkeys_s": (na + nb) / ms / 1e6,
                          "gbs": (na + nb + k) * 8 / ms / 1e6}
    return res


def _fill_large_kv(torch, dev, dist, A, B, seed):
    """Overwrite the resident key buffers A (n_a) and B (n_b) (uint64) with
    the large key-value recipe's other distributions, drawn on the device
    (payloads stay the global source indices):
    a_gt_b: A uniform in [2^63, 2^64), B uniform in [0, 2^63), each sorted;
    interleaved: output rank r dealt to B iff floor((r+1) n_b / n) >
    floor(r n_b / n), key r * floor(2^64 / n);
    distinct16: 16 random 64-bit values, each element a uniform choice."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    n_a, n_b = A.numel(), B.numel()
    a64, b64 = A.view(torch.int64), B.view(torch.int64)
    top = -(1 << 63)  # the top bit as an int64 bit pattern
    if dist == "a_gt_b":
        a64.copy_(torch.sort(torch.randint(0, (1 << 63) - 1, (n_a,), dtype=torch.int64, device=dev,
                                           generator=g)).values | top)
        b64.copy_(torch.sort(torch.randint(0, (1 << 63) - 1, (n_b,), dtype=torch.int64, device=dev,
                                           generator=g)).values)
    elif dist == "interleaved":
        n = n_a + n_b
        r = torch.arange(n, dtype=torch.int64, device=dev)
        to_b = ((r + 1) * n_b) // n > (r * n_b) // n
        keys = r * ((1 << 64) // n)  # wraps as uint64 bits
        a64.copy_(keys[~to_b])
        b64.copy_(keys[to_b])
        del r, to_b, keys
    elif dist == "distinct16":
        vals = torch.randint(-(1 << 63), (1 << 63) - 1, (16,), dtype=torch.int64, device=dev, generator=g)
        vals = torch.sort(vals ^ top).values ^ top  # ascending as uint64
        for t, m in ((a64, n_a), (b64, n_b)):
            idx = torch.sort(torch.randint(0, 16, (m,), dtype=torch.int64, device=dev, generator=g)).values
            t.copy_(vals[idx])
            del idx
    else:
        raise ValueError(dist)


def extra_dists(mp, torch, dev, A, AV, B, BV, OK, OV, peak, reps=20):
    """The large key-value merge under the other three key distributions of
    its recipe, on the same resident buffers: the whole step (partition +
    merge) and the merge kernel alone, CUDA events on the launching stream."""
    n = A.numel() + B.numel()
    alg = 2 * n * 12
    stream = torch.cuda.current_stream(dev)
    res = {}
    for i, dist in enumerate(("a_gt_b", "interleaved", "distinct16")):
        _fill_large_kv(torch, dev, dist, A, B, 0x14062628 + i)
        torch.cuda.synchronize(dev)
        for _ in range(3):
            mp.mp_merge_pairs(A, AV, B, BV, OK, OV)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        for _ in range(reps):
            mp.mp_merge_pairs(A, AV, B, BV, OK, OV)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        step_ms = e0.elapsed_time(e1) / reps
        tile = mp.mp_merge_tile_items(torch.uint64, True, n, None)
        splits = mp.mp_merge_path_partition(A, B, tile)
        torch.cuda.synchronize(dev)
        e1.record(stream)
        for _ in range(reps):
            mp.mp_merge_partitioned(A, B, splits, AV, BV, OK, OV)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        merge_ms = e1.elapsed_time(e2) / reps
        res[dist] = {"ms": step_ms, "gkeys_s": n / step_ms / 1e6, "kernel_ms": merge_ms,
                     "kernel_gbs": alg / merge_ms / 1e6, "frac": alg / merge_ms / 1e6 / peak}
        del splits
    return res


def _device_sort_input(torch, dev, dtype, order, n, seed):
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    if dtype == "i32":
        x = torch.randint(-(1 << 31), 1 << 31, (n,), dtype=torch.int64, device=dev, generator=g).to(torch.int32)
    else:
        bits = torch.randint(-(1 << 31), 1 << 31, (n,), dtype=torch.int64, device=dev, generator=g).to(torch.int32)
        x = bits.view(torch.float32)
        # NaN is excluded from the key order: redraw those bit patterns
        # (uniform over the non-NaN ones) until none is left.
        while True:
            nan = torch.nonzero(torch.isnan(x)).flatten()
            if nan.numel() == 0:
                break
            fresh = torch.randint(-(1 << 31), 1 << 31, (nan.numel(),), dtype=torch.int64, device=dev,
                                  generator=g).to(torch.int32)
            bits[nan] = fresh
    if order == "sorted":
        x = torch.sort(x).values
    elif order == "reverse":
        x = torch.sort(x, descending=True).values
    elif order == "distinct256":
        vals = x[:256].clone()
        idx = torch.randint(0, 256, (n,), device=dev, generator=g)
        x = vals[idx]
    return x.contiguous()


def extra_sort(mp, torch, dev, n=1 << 28, reps=3):
    res = {}
    work = None
    ws = None
    for dtype in ("i32", "f32"):
        for order in ("random", "sorted", "reverse", "distinct256"):
            x = _device_sort_input(torch, dev, dtype, order, n, 1234)
            if work is None:
                work = torch.empty_like(x)
                ws = torch.empty(mp.mp_sort_workspace_bytes(torch.int32, n, False), dtype=torch.uint8, device=dev)
            w = work.view(x.dtype)
            times = []
            for r in range(reps + 1):
                w.copy_(x)
                e0, e1 = _events(torch)
                e0.record()
                mp.mp_sort(w, workspace=ws)
                e1.record()
                torch.cuda.synchronize(dev)
                if r:
                    times.append(e0.elapsed_time(e1))
            ms = min(times)
            blocks = (n + SORT_BLOCK_4B - 1) // SORT_BLOCK_4B
            passes = 1 + max(0, math.ceil(math.log2(blocks)))
            res[f"{dtype}_{order}"] = {"ms": ms, "gkeys_s": n / ms / 1e6,
                                       "eff_gbs": passes * 2 * n * 4 / ms / 1e6, "hbm_passes": passes}
            del x
    res["n"] = n
    return res


def extra_batched(mp, torch, dev, n_seg=16384, log2_max=18.0, reps=5):
    """16,384 int32 merge pairs, per-side length floor(2^U), U ~ U[0, 18];
    one batched call, its CUDA-graph replay, a grouped launch, and 16,384
    per-call mp_merge_keys launches."""
    import gen
    la, lb = gen.batched_lengths(n_seg, log2_max)
    a_off = np.concatenate([[0], np.cumsum(la)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(lb)]).astype(np.int64)

    def side(lens, seed):
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        total = int(lens.sum())
        keys = torch.randint(0, 1 << 31, (total,), dtype=torch.int64, device=dev, generator=g)
        seg = torch.repeat_interleave(torch.arange(lens.size, device=dev), torch.from_numpy(lens).to(dev))
        return (torch.sort((seg << 32) | keys).values & 0xFFFFFFFF).to(torch.int32)

    A, B = side(la, 41), side(lb, 42)
    AO, BO = torch.from_numpy(a_off).to(dev), torch.from_numpy(b_off).to(dev)
    n = A.numel() + B.numel()
    out = torch.empty(n, dtype=torch.int32, device=dev)
    # Tile shape, items per thread and staging picked by the autotuner on
    # this very problem (it times every compiled shape), then used below.
    t0 = time.perf_counter()
    tuned = mp.mp_autotune_batched(A, AO, B, BO, out=out, reps=3)
    tune_s = time.perf_counter() - t0
    for _ in range(2):
        mp.mp_merge_batched(A, AO, B, BO, out=out, plan=tuned)
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(reps):
        mp.mp_merge_batched(A, AO, B, BO, out=out, plan=tuned)
    e1.record()
    torch.cuda.synchronize(dev)
    batched_ms = e0.elapsed_time(e1) / reps
    g = mp.mp_graph_batched_create(A, AO, B, BO, out, plan=tuned)
    g.replay()
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize(dev)
    graph_ms = e0.elapsed_time(e1) / reps
    g.close()
    # Per-call baseline and grouped launch over the same segments.
    ao, bo = a_off.tolist(), b_off.tolist()
    views = [(A[ao[s]:ao[s + 1]], B[bo[s]:bo[s + 1]], out[ao[s] + bo[s]:ao[s + 1] + bo[s + 1]])
             for s in range(n_seg)]
    # The descriptor table is built once in Python (its cost is reported
    # apart: walking 16,384 tuples), and the timed call is the C call.
    t0 = time.perf_counter()
    descs = mp.mp_merge_grouped_descs(views)
    grouped_host_ms = (time.perf_counter() - t0) * 1e3
    mp.mp_merge_grouped(descs)
    e0.record()
    mp.mp_merge_grouped(descs)
    e1.record()
    torch.cuda.synchronize(dev)
    grouped_ms = e0.elapsed_time(e1)
    for v in views[:64]:
        mp.mp_merge_keys(*v)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0.record()
    for v in views:
        mp.mp_merge_keys(v[0], v[1], v[2])
    e1.record()
    torch.cuda.synchronize(dev)
    per_call_ms = e0.elapsed_time(e1)
    per_call_wall_ms = (time.perf_counter() - t0) * 1e3
    byt = 2 * n * 4
    return {"segments": n_seg, "keys": n, "tuned_plan": {"block_threads": tuned[0], "items_per_thread": tuned[1],
                                                         "staging": {1: "vector", 2: "bulk"}.get(tuned[2])},
            "tune_s": tune_s, "batched_ms": batched_ms, "graph_ms": graph_ms,
            "grouped_ms": grouped_ms, "grouped_descs_host_ms": grouped_host_ms, "per_call_ms": per_call_ms, "per_call_wall_ms": per_call_wall_ms,
            "batched_gkeys_s": n / batched_ms / 1e6, "batched_gbs": byt / batched_ms / 1e6,
            "graph_gbs": byt / graph_ms / 1e6, "per_call_gbs": byt / per_call_ms / 1e6,
            "speedup_batched_vs_per_call": per_call_ms / batched_ms,
            "speedup_graph_vs_per_call": per_call_ms / graph_ms}


def _serving_trace(n_req, seed=0x5E7):
    import gen
    u = (gen.splitmix64(seed, 1, n_req) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    is_sort = u < 0.3
    def logu(stream):
        v = (gen.splitmix64(seed, stream, n_req) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
        return np.floor(np.exp2(10 + 14 * v)).astype(np.int64)
    na, nb = logu(2), logu(3)
    nb[is_sort] = 0
    return is_sort, na, nb


def _run_queue_trace(mp, is_sort, na, nb, arrivals, budget, max_active=4096):
    """Submit each request at its arrival time (seconds from t0); returns
    per-request latencies (done - arrival) and the makespan."""
    q = mp.Queue(budget_bytes=budget, max_active=max_active)
    n_req = len(na)
    tickets = [None] * n_req
    results = [None] * n_req
    t0 = mp.mp_clock_seconds() + 0.05

    def waiter():
        for i in range(n_req):
            while tickets[i] is None:
                time.sleep(0.0002)
            results[i] = q.wait(tickets[i])

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    i = 0
    while i < n_req:
        now = mp.mp_clock_seconds() - t0
        while i < n_req and arrivals[i] <= now:
            op = mp.MP_OP_SORT if is_sort[i] else mp.MP_OP_MERGE
            tickets[i] = q.submit_generated(op, mp.MP_U32, int(na[i]), int(nb[i]), seed=i, with_values=True)
            i += 1
        if i < n_req:
            wait = arrivals[i] - (mp.mp_clock_seconds() - t0)
            if wait > 0.0005:
                time.sleep(wait - 0.0003)
    th.join()
    stats = q.stats()
    q.close()
    lat = np.array([results[j].t_done - (t0 + arrivals[j]) for j in range(n_req)])
    bad = sum(1 for r in results if r.status != 0)
    makespan = max(r.t_done for r in results) - t0
    return lat, makespan, stats, bad


def _run_serial_trace(mp, torch, dev, is_sort, na, nb, arrivals):
    """The same trace served one request at a time with plain calls (inputs
    generated on the device by the same generator, then mp_merge_pairs or
    mp_sort), each finished before the next starts."""
    maxn = int(max((na + nb).max(), 2))
    ka = torch.empty(maxn, dtype=torch.int32, device=dev)
    kb = torch.empty(maxn, dtype=torch.int32, device=dev)
    va = torch.empty(maxn, dtype=torch.int32, device=dev)
    vb = torch.empty(maxn, dtype=torch.int32, device=dev)
    ko = torch.empty(maxn, dtype=torch.int32, device=dev)
    vo = torch.empty(maxn, dtype=torch.int32, device=dev)
    ws = torch.empty(mp.mp_sort_workspace_bytes(mp.MP_U32, maxn, True), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    n_req = len(na)
    lat = np.zeros(n_req)
    t0 = mp.mp_clock_seconds() + 0.05
    for i in range(n_req):
        while mp.mp_clock_seconds() - t0 < arrivals[i]:
            pass
        a, b = int(na[i]), int(nb[i])
        if is_sort[i]:
            mp.mp_generate(mp.MP_U32, ka, a, i, 3, False, vals=va, val_base=0)
            k = ka[:a].view(torch.uint32)
            mp.mp_sort(k, va[:a], workspace=ws)
        else:
            mp.mp_generate(mp.MP_U32, ka, a, i, 1, True, vals=va, val_base=0)
            mp.mp_generate(mp.MP_U32, kb, b, i, 2, True, vals=vb, val_base=a)
            mp.mp_merge_pairs(ka[:a].view(torch.uint32), va[:a], kb[:b].view(torch.uint32), vb[:b],
                              ko[:a + b].view(torch.uint32), vo[:a + b])
        stream.synchronize()
        lat[i] = mp.mp_clock_seconds() - (t0 + arrivals[i])
    makespan = mp.mp_clock_seconds() - t0
    return lat, makespan


def extra_serving(mp, torch, dev, n_req=50000, budget=8 << 30, rhos=(0.5, 0.9)):
    """Poisson arrivals of merge (70 %) and sort (30 %) requests, uint32 keys
    + uint32 values, sizes log-uniform in [2^10, 2^24], generated on the
    device at admission; the queue (continuous batching under an 8 GB
    budget) against serial per-request plain calls on the same trace."""
    is_sort, na, nb = _serving_trace(n_req)
    items = int((na + nb).sum())
    # Capacity: the whole trace submitted at once (closed loop).
    lat, makespan, st, bad = _run_queue_trace(mp, is_sort, na, nb, np.zeros(n_req), budget)
    cap_req_s = n_req / makespan
    out = {"requests": n_req, "items": items, "budget_bytes": budget,
           "capacity": {"req_s": cap_req_s, "gitems_s": items / makespan / 1e9, "makespan_s": makespan,
                        "steps": st["steps"], "launches": st["launches"], "failed": bad}}
    rng = np.random.default_rng(7)
    for rho in rhos:
        lam = rho * cap_req_s
        arrivals = np.cumsum(rng.exponential(1.0 / lam, n_req))
        arrivals -= arrivals[0]
        lat, makespan, st, bad = _run_queue_trace(mp, is_sort, na, nb, arrivals, budget)
        slat, smake = _run_serial_trace(mp, torch, dev, is_sort, na, nb, arrivals)
        out[f"rho_{rho}"] = {
            "rate_req_s": lam,
            "queue": {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                      "throughput_gitems_s": items / makespan / 1e9, "makespan_s": makespan,
                      "steps": st["steps"], "failed": bad},
            "serial": {"p50_ms": float(np.percentile(slat, 50) * 1e3), "p99_ms": float(np.percentile(slat, 99) * 1e3),
                       "throughput_gitems_s": items / smake / 1e9, "makespan_s": smake}}
    return out


# --------------------------------------------------------------------- digest

def _r(x, digits=4):
    """x rounded to a few significant digits (None stays None)."""
    if x is None or not isinstance(x, (int, float)) or x == 0 or not math.isfinite(x):
        return x
    return round(x, max(0, digits - 1 - int(math.floor(math.log10(abs(x))))))


def summarize(line):
    """The headline and every extra, a few numbers each (ms, GB/s, fractions
    of the measured peak, latencies), in well under 1.5 kB of JSON."""
    ex = line.get("extras", {})
    rf = line.get("roofline", {})
    sm = {"merge": {"gkeys_s": _r(line["value"]), "ms": _r(line["ms_per_step"]), "frac": _r(rf.get("frac")),
                    "e2e_gkeys_s": _r(line.get("e2e", {}).get("value")),
                    "e2e_ms": _r(line.get("e2e", {}).get("ms_per_step"))}}
    d = ex.get("dists", {})
    if "uniform" in d:
        sm["dists"] = {k: [_r(v["ms"]), _r(v["frac"], 3)] for k, v in d.items()
                       if isinstance(v, dict) and "frac" in v}
    p = ex.get("plain", {})
    if "cold_us" in p:
        sm["plain_us"] = {"cold": _r(p["cold_us"], 3), "warm": _r(p["warm_us"], 3)}
    so = ex.get("sort", {})
    if "i32_random" in so:
        sm["sort_ms"] = {dt: [_r(so[f"{dt}_{o}"]["ms"]) for o in ("random", "sorted", "reverse", "distinct256")
                              if f"{dt}_{o}" in so] for dt in ("i32", "f32")}
    b = ex.get("batched", {})
    if "batched_ms" in b:
        tp = b.get("tuned_plan", {})
        sm["batched"] = {"ms": _r(b["batched_ms"]), "gbs": _r(b["batched_gbs"]), "graph_ms": _r(b["graph_ms"]),
                         "per_call_ms": _r(b["per_call_ms"]), "x": _r(b["speedup_batched_vs_per_call"], 3),
                         "plan": f"{tp.get('block_threads')}x{tp.get('items_per_thread')}{tp.get('staging', '')[:1]}"}
    sv = ex.get("serving", {})
    if "capacity" in sv:
        sm["serving"] = {"cap_req_s": _r(sv["capacity"]["req_s"], 3)}
        for k, v in sv.items():
            if k.startswith("rho_"):
                q, se = v["queue"], v["serial"]
                sm["serving"][k] = {"q": [_r(q["p50_ms"], 3), _r(q["p99_ms"], 3), _r(q["throughput_gitems_s"], 3)],
                                    "serial": [_r(se["p50_ms"], 3), _r(se["p99_ms"], 3),
                                               _r(se["throughput_gitems_s"], 3)],
                                    "failed": q["failed"]}
    st = ex.get("setops", {})
    if "union" in st:
        short = {"union": "union", "intersection": "inter", "difference": "diff",
                 "symmetric_difference": "sym", "union_pairs": "union_kv"}
        sm["setops_ms"] = {v: _r(st[k]["ms"]) for k, v in short.items() if k in st}
    w = ex.get("wide", {})
    if "merge_auto" in w:
        sm["u128_ms"] = {"merge": _r(w["merge_auto"]["ms"]), "sort": _r(w["sort"]["ms"])}
    ro = ex.get("readonly_merge", {})
    if "ms" in ro:
        sm["readonly_ms"] = _r(ro["ms"])
    sm["legend"] = ("dists: [step ms, merge-kernel frac of peak]; sort_ms: random, sorted, reverse, "
                    "256 values; serving q/serial: [p50 ms, p99 ms, Gitems/s]")
    return sm


# --------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1406_2628_gb300 as mp
    from paper_1406_2628_gb300 import build as mpbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or not os.path.exists(mpbuild.LIB_PATH):
        mpbuild.build()
    if world > 1:
        dist.barrier()
    mp.lib()
    plan = tuple(int(x) for x in args.plan.split(",")) if args.plan else None

    a, av, b, bv = workload(args)
    n = a.size + b.size

    def dev_t(x, tdt=None):
        t = torch.from_numpy(x.view(np.int64) if x.dtype == np.uint64 else x.view(np.int32))
        t = t.to(dev)
        return t.view(torch.uint64) if x.dtype == np.uint64 else t

    A, AV, B, BV = dev_t(a), dev_t(av), dev_t(b), dev_t(bv)
    OK = torch.empty(n, dtype=torch.uint64, device=dev)
    OV = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        if plan is None:
            mp.mp_merge_pairs(A, AV, B, BV, OK, OV)
        else:
            mp.mp_merge_plan(A, B, AV, BV, OK, OV, plan=plan)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t_load0 = time.time()
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    if world > 1:
        ms = max_over_ranks(ms, dist, dev)

    # Per-kernel timing on the same stream: partition alone, merge alone.
    tile = mp.mp_merge_tile_items(torch.uint64, True, n, plan)
    resolved = mp.mp_merge_resolve_plan(torch.uint64, True, n, plan)
    splits = mp.mp_merge_path_partition(A, B, tile)
    torch.cuda.synchronize(dev)
    reps = max(args.steps, 10)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(reps):
        mp.mp_merge_path_partition(A, B, tile, out=splits)
    e1.record(stream)
    for _ in range(reps):
        mp.mp_merge_partitioned(A, B, splits, AV, BV, OK, OV, plan=plan)
    e2.record(stream)
    torch.cuda.synchronize(dev)
    part_ms = e0.elapsed_time(e1) / reps
    merge_ms = e1.elapsed_time(e2) / reps
    # The timed region is short next to the sampler's 100 ms period: keep the
    # same step running for about a second more so the clock record covers
    # this kernel under load.
    soak_end = time.time() + 1.2
    while time.time() < soak_end:
        for _ in range(20):
            step()
        torch.cuda.synchronize(dev)
    t_load1 = time.time()
    sampler.stop()
    clocks = sampler.summary(t_load0, t_load1)

    # End to end through the host-buffer C entry point (pinned host memory).
    e2e = None
    if not args.no_e2e:
        def pin(x, tdt):
            return torch.from_numpy(x.view(tdt)).pin_memory()
        hA, hB = pin(a, np.int64).view(torch.uint64), pin(b, np.int64).view(torch.uint64)
        hAV, hBV = pin(av, np.int32), pin(bv, np.int32)
        hOK = torch.empty(n, dtype=torch.int64).pin_memory().view(torch.uint64)
        hOV = torch.empty(n, dtype=torch.int32).pin_memory()
        mp.mp_merge_pairs_host(hA, hAV, hB, hBV, hOK, hOV)  # warm the pool
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            mp.mp_merge_pairs_host(hA, hAV, hB, hBV, hOK, hOV)
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        if world > 1:
            e2e_s = max_over_ranks(e2e_s, dist, dev)
        e2e = {"value": weak_scaling_value(n, e2e_s * 1e3, world), "unit": UNIT,
               "h2d_bytes_per_step": int(a.nbytes + av.nbytes + b.nbytes + bv.nbytes),
               "d2h_bytes_per_step": int(n * 12), "ms_per_step": e2e_s * 1e3,
               "call": "mp_merge_pairs_host (pinned host buffers, copies in and out inside the call)"}
        # The result that came back must be the merge of the inputs.
        chk = hOK.view(torch.int64).numpy().view(np.uint64)
        if not np.all(chk[1:] >= chk[:-1]):
            raise RuntimeError("end-to-end result is not sorted")

    peak, peak_kind = measured_peak()
    alg_bytes = 2 * n * 12
    achieved = alg_bytes / (merge_ms * 1e-3) / 1e9
    value = weak_scaling_value(n, ms, world)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config_dict(args, world),
        "roofline": {"bound": "hbm", "kernel": "merge_tile_bulk_kernel (TMA-staged merge tiles)",
                     "plan": {"block_threads": resolved[0], "items_per_thread": resolved[1],
                              "staging": {1: "vector", 2: "bulk", 3: "warp", 4: "stream"}.get(resolved[2]),
                              "tile": tile},
                     "achieved": achieved,
                     "peak": peak, "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy)",
                     "unit": "GB/s", "frac": achieved / peak,
                     "frac_of_nominal_7900": achieved / NOMINAL_HBM_GBS,
                     "traffic": recorded_traffic(f"{args.log2_a}_{args.log2_b}_{args.dist}"),
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "kernel_ms": merge_ms, "partition_ms": part_ms,
                     "step_bytes_per_s_GBs": alg_bytes / (ms * 1e-3) / 1e9},
        "clocks": clocks,
        "gpu_launches": 2 * args.steps,
    }
    if e2e is not None:
        line["e2e"] = e2e
    # The merge with results kept on chip (Sec. VI, Fig. 5: results written
    # to a register): the read side alone.
    readonly = None
    if not args.no_extras:
        cs = mp.mp_merge_checksum(A, B, AV, BV)
        torch.cuda.synchronize(dev)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        for _ in range(reps):
            mp.mp_merge_checksum(A, B, AV, BV, out=cs)
        r1.record(stream)
        torch.cuda.synchronize(dev)
        ro_ms = r0.elapsed_time(r1) / reps
        readonly = {"call": "mp_merge_checksum (partition + merge, outputs folded on chip)",
                    "ms": ro_ms, "read_gbs": n * 12 / ro_ms / 1e6,
                    "gkeys_s": n / ro_ms / 1e6}
    if not args.no_extras:
        extras = {}
        wanted = [x for x in args.extras.split(",") if x]
        if "dists" in wanted:
            t0 = time.perf_counter()
            try:
                extras["dists"] = extra_dists(mp, torch, dev, A, AV, B, BV, OK, OV, peak)
            except Exception as exc:  # an extra never breaks the headline line
                extras["dists"] = {"error": f"{type(exc).__name__}: {exc}"}
            extras["dists"]["wall_s"] = time.perf_counter() - t0
            extras["dists"]["uniform"] = {"ms": ms, "gkeys_s": n / ms / 1e6, "kernel_ms": merge_ms,
                                          "kernel_gbs": achieved, "frac": achieved / peak}
            wanted.remove("dists")
        runners = {"plain": lambda: extra_plain(mp, torch, dev),
                   "sort": lambda: extra_sort(mp, torch, dev, n=1 << args.sort_log2_n),
                   "batched": lambda: extra_batched(mp, torch, dev, n_seg=args.batched_segments),
                   "serving": lambda: extra_serving(mp, torch, dev, n_req=args.serving_requests),
                   "setops": lambda: extra_setops(mp, torch, dev, log2_universe=args.setops_log2_universe),
                   "wide": lambda: extra_wide(mp, torch, dev),
                   "crossover": lambda: extra_crossover(mp, torch, dev),
                   "tiles": lambda: extra_tiles(mp, torch, dev, log2_n=args.tiles_log2_n)}
        del OK, OV
        for name in wanted:
            t0 = time.perf_counter()
            try:
                extras[name] = runners[name]()
            except Exception as exc:  # an extra never breaks the headline line
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}
            extras[name]["wall_s"] = time.perf_counter() - t0
            torch.cuda.empty_cache()
        if readonly is not None:
            extras["readonly_merge"] = readonly
        line["extras"] = extras
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, reps_o, secs = oracle_rate(a, av, b, bv)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"the full workload merged {reps_o}x by the single-threaded "
                                          f"oracle ({secs:.1f} s)",
                                "host_cpus": os.cpu_count()}
    # Last key of the line: a compact digest of every workload, so that a
    # reader keeping only the tail of the output still has all of them.
    line["summary"] = summarize(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
