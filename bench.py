#!/usr/bin/env python
"""Benchmark of the LDE + Poseidon-Merkle commitment on GB300.

One step = one commit through the library's public entry point
(v3c_commit: coset LDE, leaf hash, Merkle levels to the cap, on a resident
object) followed by its release.  The default workload is the large commit:
135 trace columns x 2^20 rows, rate_bits 3 (2^23 LDE rows, 9.06 GB
resident), cap height 4.  Inputs are resident in HBM when the timed region
starts; every buffer is larger than L2 (1.13 GB in, 9.06 GB LDE), so no
flush is needed between steps.  A workload whose commit fits in L2 is timed
step by step, each after an untimed write of a 256 MB buffer.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (the
reference arm of this tier) on a bounded sample of the same workload, or on
the whole workload when it is no larger than that sample.
Under torchrun the ranks split the one commit by LDE row blocks (strong
scaling): each computes the coefficients of its share of the columns, one
NCCL all-gather assembles them, and each commits its coset block (a whole
subtree, whose top is its slice of the cap).  --replicas instead has each
rank commit its own independent request (weak scaling, no data-path
collective).  The default single-GPU line also carries the serving block
(latency at load against the serial path) and the batched block (64 uneven
batches in one commit against one commit per batch).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "LDE+Merkle commit Gelem/s vs roofline; p50/p99 audit-commit latency at load"
WORKLOADS = {
    "large_135x2_20": synth.LARGE_135x2_20,
    "trace_135x2_16": synth.TRACE_135x2_16,
    "plain_8x2_10": synth.PLAIN_8x2_10,
    "profile_8x2_20": synth.PROFILE_8x2_20,  # small capture case with the large commit's stage shapes
}
# Algorithmic work per Poseidon permutation in 32x32->64 wide-multiply units
# (minimal exact form: S-boxes 1888, full-round small MDS 2304, sparse
# partial rounds 2024 + 576) and per NTT butterfly multiplication.
W_PER_PERM = 6792
W_PER_NTT_MUL = 4
# Integer-pipe peak derived from unit counts and clocks: 152 SMs x 32 wide
# multiplies per SM per clock x 2070 MHz.  An SM issues 64 32-bit IMAD lanes
# per clock (4 SMSPs x 16-lane FMA-heavy pipe; measured 62.6), and a
# 32x32->64 product takes two of them (lo and hi; IMAD.WIDE measured 23.8 per
# SM per clock).
SMS = 152
WIDE_MUL_PER_SM_CLK = 32
SM_MAX_MHZ = 2070.0
# DRAM traffic of one leaf-hash launch on this workload, from an ncu capture
# of the same kernel (dram__bytes_read.sum + dram__bytes_write.sum, one
# capture of the bench's own command).  Drop an entry when the kernel changes.
LEAF_HASH_TRAFFIC = {"large_135x2_20": 9.758e9}
# The CPU-baseline / reference-arm sample: the full commit of the same column
# mix at fewer rows.
CPU_SAMPLE = synth.Shape(c=135, log_n=14, rate_bits=3, cap_height=4, seed=0)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def shard_workload(s: "synth.Shape", rank: int) -> "synth.Shape":
    """Rank r commits its own independent batch of the same shape (batch
    index r of the same seed): weak scaling with no data-path collective."""
    return synth.Shape(c=s.c, log_n=s.log_n, rate_bits=s.rate_bits, cap_height=s.cap_height, seed=s.seed,
                       mix=s.mix, batch=rank)


def max_over_ranks(value: float, device: str = "cuda") -> float:
    """The slowest rank's time (the only collective: timing, not data)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(pw) if pw else None}


def cpu_sample(w):
    """The oracle's shape for workload w: w itself when it is no larger than
    CPU_SAMPLE, else w's columns, mix, rate and cap height on fewer rows (the
    largest power of two within CPU_SAMPLE's element count)."""
    if w.lde_elems() <= CPU_SAMPLE.lde_elems():
        return w, True
    budget = CPU_SAMPLE.c << CPU_SAMPLE.log_n
    log_n = max(1, min(w.log_n, (budget // w.c).bit_length() - 1))
    cap = min(w.cap_height, log_n + w.rate_bits)
    return synth.Shape(c=w.c, log_n=log_n, rate_bits=w.rate_bits, cap_height=cap, seed=w.seed, mix=w.mix), False


def cpu_baseline(steps: int = 1, shape=None) -> dict:
    """The oracle on the host cores.  A workload no larger than the bounded
    sample is timed whole (and on one thread as well); larger ones on the
    same columns and mix over fewer rows (cpu_sample)."""
    import oracle

    s, whole = cpu_sample(shape if shape is not None else synth.LARGE_135x2_20)
    x = s.inputs()

    def time_commit(threads):
        oracle.commit(x, s.rate_bits, s.cap_height, threads=threads)  # warm (constants, pages)
        n, t0 = 0, time.perf_counter()
        while n < steps or time.perf_counter() - t0 < (0.5 if whole else 0.0):
            oracle.commit(x, s.rate_bits, s.cap_height, threads=threads)
            n += 1
        return (time.perf_counter() - t0) / n

    threads = oracle.default_threads()
    dt = time_commit(threads)
    what = "the whole workload" if whole else "a bounded sample"
    out = {"value": s.lde_elems() / dt / 1e9, "unit": "Gelem/s", "cores": threads, "kind": "oracle",
           "sample": f"{what}: full oracle commit of {s.c} columns x 2^{s.log_n} rows (same column mix), "
                     f"rate_bits {s.rate_bits}, cap height {s.cap_height}; {dt * 1e3:.2f} ms per commit"}
    if whole:
        dt1 = time_commit(1)
        out["single_core"] = {"value": s.lde_elems() / dt1 / 1e9, "unit": "Gelem/s", "ms_per_commit": dt1 * 1e3}
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    if args.workload in FRI_WORKLOADS:
        return run_reference_fri(args)
    if args.workload in ("snapshot_msmarco", "seteq_64x2_17"):
        return run_reference_other(args)
    import oracle

    w = WORKLOADS.get(args.workload, synth.LARGE_135x2_20)
    s, whole = cpu_sample(w)  # small workloads are timed whole
    x = s.inputs()
    threads = oracle.default_threads()
    for _ in range(args.warmup):
        oracle.commit(x, s.rate_bits, s.cap_height, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.commit(x, s.rate_bits, s.cap_height, threads=threads)
    dt = (time.perf_counter() - t0) / args.steps
    value = s.lde_elems() / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(args.workload, w),
        "cpu_baseline": {"kind": "oracle", "cores": threads, "value": value, "unit": "Gelem/s",
                         "sample": f"oracle commit of {s.c} x 2^{s.log_n} rows per step ("
                                   + ("the whole workload)" if whole else
                                      f"bounded sample of the {args.workload} workload's column mix)")},
        "e2e": {"value": value, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference_fri(args):
    s = FRI_CPU_SAMPLE
    for _ in range(max(args.warmup - 1, 0)):
        fri_cpu_baseline(s, 1)
    base = fri_cpu_baseline(s, args.steps)
    line = {
        "impl": "reference", "metric": FRI_METRIC, "value": base["value"], "unit": "Gelem/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "columns": FRI_WORKLOADS[args.workload].c,
                   "log_rows": FRI_WORKLOADS[args.workload].log_n, "rate_bits": 3,
                   "arity_bits": FRI_CFG[0], "final_log": FRI_CFG[1], "layer_cap_height": FRI_CFG[2],
                   "queries": FRI_QUERIES, "ext_degree": FRI_EXT},
        "cpu_baseline": {k: base[k] for k in ("kind", "cores", "value", "unit", "sample")},
        "e2e": {"value": base["value"], "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference_other(args):
    snap = args.workload == "snapshot_msmarco"
    for _ in range(max(args.warmup - 1, 0)):
        (snapshot_cpu_baseline if snap else seteq_cpu_baseline)(1)
    base = (snapshot_cpu_baseline if snap else seteq_cpu_baseline)(args.steps)
    line = {
        "impl": "reference", "metric": "snapshot commitment (root_mk, root_cb) Mslot/s" if snap else
        "SetEq grand-product columns Gtuple/s", "value": base["value"], "unit": base["unit"], "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {k: base[k] for k in ("kind", "cores", "value", "unit", "sample")},
        "e2e": {"value": base["value"], "unit": base["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(name, s):
    return {"workload": name, "columns": s.c, "log_rows": s.log_n, "rate_bits": s.rate_bits,
            "cap_height": s.cap_height, "lde_rows": 1 << s.log_N, "mix": s.mix,
            "l2": "inputs larger than L2 (no flush needed)" if s.lde_elems() * 8 > 129e6 else "L2 flush"}


def run_v3c(args):
    import torch

    import paper_2603_03065_gb300 as v3c

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    s = shard_workload(WORKLOADS[args.workload], rank)
    x = s.inputs()
    ctx = v3c.Context(local_rank, flags=v3c.FLAG_TIMING, autotune=args.autotune)
    stream = torch.cuda.current_stream()
    d_x = v3c.to_device_u64(x)

    def step():
        cid = ctx.commit([(d_x, s.rate_bits, s.cap_height)], stream=stream)[0]
        ctx.release(cid)

    # A commit that fits in L2 (129 MB) is timed step by step, each after an
    # untimed write of a 256 MB buffer that evicts it.
    small = s.lde_elems() * 8 <= 129e6
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if small else None

    def flush():
        flush_buf.fill_(1)  # on the current stream, which the commits use

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    clocks = ClockSampler(local_rank)
    ctx.stage_stats(reset=True)
    l0 = ctx.kernel_launches()
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    pairs = []
    if small:
        for _ in range(args.steps):
            flush()
            ea = torch.cuda.Event(enable_timing=True)
            eb = torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            step()
            eb.record(stream)
            pairs.append((ea, eb))
    else:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        pairs.append((e0, e1))
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in pairs) / args.steps
    launches = ctx.kernel_launches() - l0
    stats = ctx.stage_stats(reset=True)
    ms = max_over_ranks(ms)

    value = world * s.lde_elems() / (ms * 1e-3) / 1e9

    # end to end: pinned host input -> device inside the call, cap back to host
    pinned = torch.from_numpy(x.view(np.int64)).pin_memory()
    x_pinned = pinned.numpy().view(np.uint64)

    host_ms = {"enqueue": 0.0, "cap_wait": 0.0, "release": 0.0}

    def step_e2e():
        t_a = time.perf_counter()
        cid = ctx.commit([(x_pinned, s.rate_bits, s.cap_height)], stream=stream)[0]
        t_b = time.perf_counter()
        cap = ctx.cap(cid)
        t_c = time.perf_counter()
        ctx.release(cid)
        t_d = time.perf_counter()
        host_ms["enqueue"] += (t_b - t_a) * 1e3
        host_ms["cap_wait"] += (t_c - t_b) * 1e3
        host_ms["release"] += (t_d - t_c) * 1e3
        return cap

    step_e2e()
    torch.cuda.synchronize()
    # The host link's bandwidth on this machine: one pinned copy of the input.
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    d_x.copy_(pinned.view(d_x.dtype).view(d_x.shape), non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    h2d_gbs = x.nbytes / (c0.elapsed_time(c1) * 1e-3) / 1e9
    barrier()
    e2e_clocks = ClockSampler(local_rank)
    e2e_clocks.start()
    for k in host_ms:
        host_ms[k] = 0.0
    ctx.stage_stats(reset=True)
    e2e_total = 0.0
    if small:
        for _ in range(args.steps):
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_e2e()  # ends with the cap read, which waits for the commit
            e2e_total += time.perf_counter() - t0
    else:
        # Two commits in flight, as a client streaming requests would run them:
        # step k enqueues commit k (its input copy from pinned host memory
        # included) before reading commit k-1's cap; the last cap is read
        # inside the timed region too.
        t0 = time.perf_counter()
        prev = None
        for _ in range(args.steps):
            t_a = time.perf_counter()
            cid = ctx.commit([(x_pinned, s.rate_bits, s.cap_height)], stream=stream)[0]
            host_ms["enqueue"] += (time.perf_counter() - t_a) * 1e3
            if prev is not None:
                t_b = time.perf_counter()
                ctx.cap(prev)
                host_ms["cap_wait"] += (time.perf_counter() - t_b) * 1e3
                ctx.release(prev)
            prev = cid
        ctx.cap(prev)
        ctx.release(prev)
        e2e_total = time.perf_counter() - t0
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(e2e_total / args.steps)
    e2e_clk = e2e_clocks.stop()
    e2e_stats = ctx.stage_stats(reset=True)
    e2e_value = world * s.lde_elems() / e2e_s / 1e9

    # roofline of the dominant kernel (leaf hash), timed by events on its stream
    leaf_ms, leaf_n = stats["leaf_hash"]
    N = 1 << s.log_N
    perms_leaf = N * (-(-s.c // 8))
    leaf_ms_per = leaf_ms / max(leaf_n, 1)
    achieved = W_PER_PERM * perms_leaf / (leaf_ms_per * 1e-3) / 1e12
    peak = SMS * WIDE_MUL_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    peaks = int_peaks(ctx) if rank == 0 else {}
    traffic = LEAF_HASH_TRAFFIC.get(args.workload)
    stage_ms = {k: (v[0] / max(v[1], 1), int(v[1])) for k, v in stats.items()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(workload_config(args.workload, s), autotune=bool(args.autotune)),
            "e2e": {"value": e2e_value, "unit": "Gelem/s", "h2d_bytes_per_step": int(x.nbytes),
                    "d2h_bytes_per_step": int(32 << s.cap_height), "ms_per_step": e2e_s * 1e3,
                    "clocks": e2e_clk, "h2d_GBps_measured": h2d_gbs,
                    "in_flight": 1 if small else 2,
                    "host_ms_per_step": {k: v / args.steps for k, v in host_ms.items()},
                    "stages_ms_per_step": {k: v[0] / args.steps for k, v in e2e_stats.items() if v[1]}},
            "gpu_launches": int(launches),
            "clocks": clk,
            "roofline": {"bound": "alu", "kernel": "k_leaf_hash", "achieved": achieved, "peak": peak,
                         "unit": "T wide-mul/s", "frac": achieved / peak, "traffic": traffic,
                         "frac_uses": "peak_derived (the larger, stricter denominator)",
                         "peak_derived": peak, **peaks,
                         "frac_of_measured_wide": achieved / peaks["peak_measured_wide"]
                         if peaks.get("peak_measured_wide") else None,
                         "work_per_launch": W_PER_PERM * perms_leaf, "ms_per_launch": leaf_ms_per},
            "stages_ms_per_launch": stage_ms,
        }
        try:  # the whole path against its roofline (reported only; never fails the line)
            line["path_roofline"] = path_roofline(s, ms, float(measured_peaks().get("hbm_gbs") or 6789.0))
        except Exception as e:  # pragma: no cover
            line["path_roofline"] = {"error": str(e)}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(shape=s)
        if world == 1 and args.workload == "large_135x2_20" and not args.no_extras:
            # The other half of the metric (latency at load) and the batched
            # form, measured after the timed region of the line's value.
            try:
                line["serving"] = serving_block(None, args.serve_duration, load=args.serve_load)
                # 10 % above the serial capacity: the serial path falls behind,
                # the served loop (more capacity) should keep up.
                line["serving_over_serial_capacity"] = serving_block(None, args.serve_duration,
                                                                     load=args.serve_load * 1.1)
            except Exception as e:  # pragma: no cover
                line["serving"] = {"error": str(e)}
            try:
                line["batched"] = batched_block(3, 2, autotune_variants=False)
            except Exception as e:  # pragma: no cover
                line["batched"] = {"error": str(e)}
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_split(args):
    """One commit split over the ranks by LDE row blocks (strong scaling):
    each rank computes the coefficients of its share of the columns
    (v3c_coeffs), one NCCL all-gather assembles the coefficient table on
    every rank, each rank commits its part (v3c_commit_part: its coset block,
    a whole subtree) and rank 0 gathers the cap slices.  The value is the
    whole commit's LDE elements over the slowest rank's time per step."""
    import torch
    import torch.distributed as dist

    import paper_2603_03065_gb300 as v3c
    from paper_2603_03065_gb300 import split

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if not dist.is_initialized():
        if world == 1:
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", "29533")
            os.environ.setdefault("RANK", "0")
            os.environ.setdefault("WORLD_SIZE", "1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    s = WORKLOADS[args.workload]
    log_parts = split.log_parts_for(world, s.rate_bits, s.cap_height)
    c0, c1 = split.column_shard(s.c, world, rank)
    x = s.inputs()[c0:c1]
    ctx = v3c.Context(local_rank, flags=v3c.FLAG_TIMING)
    stream = torch.cuda.current_stream()
    d_x = v3c.to_device_u64(x) if c1 > c0 else None
    held = []

    def new_table(rows, cols):
        return torch.empty((rows, cols), dtype=torch.int64, device="cuda")

    def commit_part(coeffs, lp, q):
        cid = ctx.commit_part(coeffs, s.rate_bits, s.cap_height, lp, q, stream=stream)
        b = ctx.buffers(cid)
        cap = new_table(1 << (s.cap_height - lp), 4)
        cap.copy_(_device_words(b["cap"], cap.numel()).view(cap.shape))
        return cid, cap

    def step():
        cid, cap = split.commit_split(d_x, s.c, s.log_n, s.rate_bits, s.cap_height,
                                      coeffs_of=lambda t: ctx.coeffs(t, stream=stream),
                                      commit_part=commit_part, new_table=new_table)
        ctx.release(cid)
        return cap

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    ctx.stage_stats(reset=True)
    l0 = ctx.kernel_launches()
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    launches = ctx.kernel_launches() - l0
    stats = ctx.stage_stats(reset=True)
    # end to end: each rank's pinned host shard copied in, the cap read back on rank 0
    pinned = torch.from_numpy(x.view(np.int64)).pin_memory() if c1 > c0 else None
    dist.barrier()
    t_total = 0.0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        if pinned is not None:
            d_x.copy_(pinned, non_blocking=True)
        cap = step()
        if rank == 0:
            cap.cpu()
        torch.cuda.synchronize()
        t_total += time.perf_counter() - t0
    e2e_s = max_over_ranks(t_total / args.steps)
    if rank == 0:
        value = s.lde_elems() / (ms * 1e-3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(workload_config(args.workload, s), parallelism=f"row split over {world} GPUs "
                           f"(2^{log_parts} cosets blocks, one all-gather of coefficients)"),
            "e2e": {"value": s.lde_elems() / e2e_s / 1e9, "unit": "Gelem/s",
                    "h2d_bytes_per_step": int(s.c << s.log_n) * 8, "d2h_bytes_per_step": int(32 << s.cap_height),
                    "ms_per_step": e2e_s * 1e3},
            "gpu_launches": int(launches) * world,
            "clocks": clk,
            "stages_ms_per_launch": {k: (v[0] / max(v[1], 1), int(v[1])) for k, v in stats.items()},
        }
        print(json.dumps(line))
    ctx.close()
    dist.destroy_process_group()
    return 0


def _device_words(ptr: int, words: int):
    import torch

    class _A:
        __cuda_array_interface__ = {"shape": (words,), "typestr": "<i8", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_A(), device="cuda")


def batched_block(steps: int, warmup: int, autotune_variants: bool = True) -> dict:
    """C4: the 64 uneven column-batches of seed 3 committed by one v3c_commit
    (one persistent launch per stage, replayed from a CUDA graph, tiles from
    the autotuner) against one commit per batch (per-batch launches, the
    same context and tiles), on the same device-resident inputs."""
    import torch

    import paper_2603_03065_gb300 as v3c

    shapes = synth.uneven_batches(3)
    xs = [s.inputs() for s in shapes]
    elems = sum(s.lde_elems() for s in shapes)
    out = {"workload": "uneven_64", "batches": len(shapes), "lde_elems": elems, "seed": 3, "cap_height": 4,
           "log_rows": [s.log_n for s in shapes], "columns": [s.c for s in shapes],
           "rate_bits": [s.rate_bits for s in shapes]}
    stream = torch.cuda.current_stream()
    variants = (("batched_graph_autotune", 0, True), ("batched_graph", 0, False),
                ("batched_direct", v3c.FLAG_NO_GRAPH, False)) if autotune_variants else \
        (("batched_graph_autotune", 0, True),)
    for tag, flags, tune in variants:
        # An explicit budget (the 64 batches hold 19.7 GB resident), so the
        # result does not depend on the free memory seen at context creation.
        ctx = v3c.Context(0, hbm_budget_bytes=64 << 30, flags=flags, autotune=tune)
        ds = [v3c.to_device_u64(x) for x in xs]
        items = [(d, s.rate_bits, s.cap_height) for d, s in zip(ds, shapes)]

        def batched():
            ids = ctx.commit(items, stream=stream)
            for i in ids:
                ctx.release(i)

        def per_batch():
            for it in items:
                ctx.release(ctx.commit([it], stream=stream)[0])

        for name, fn in (("all_in_one", batched), ("one_per_commit", per_batch)):
            if tag == "batched_direct" and name == "one_per_commit":
                continue
            for _ in range(max(warmup, 2)):       # the second sighting of a signature is captured
                fn()
            torch.cuda.synchronize()
            l0 = ctx.kernel_launches()
            r0 = ctx.graph_replays()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            out[f"{tag}.{name}"] = {"ms_per_step": ms, "Gelem/s": elems / (ms * 1e-3) / 1e9,
                                    "launches_per_step": (ctx.kernel_launches() - l0) / steps,
                                    "graph_replays_per_step": (ctx.graph_replays() - r0) / steps}
        ctx.close()
        del ds
    best = out["batched_graph_autotune.all_in_one"]
    base = out["batched_graph_autotune.one_per_commit"]
    out["ms_per_step"] = best["ms_per_step"]
    out["Gelem/s"] = best["Gelem/s"]
    out["vs_one_per_commit"] = base["ms_per_step"] / best["ms_per_step"]
    return out


def run_batched(args):
    """C4 as its own bench line (the default line carries the same block)."""
    import torch

    torch.cuda.set_device(0)
    b = batched_block(args.steps, args.warmup)
    out = {"metric": METRIC, "unit": "Gelem/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "dtype": "u64", "data": "synthetic", "vs_baseline": None,
           "value": b["Gelem/s"], "ms_per_step": b["ms_per_step"],
           "config": {k: b[k] for k in ("workload", "batches", "lde_elems", "log_rows", "columns", "rate_bits",
                                       "cap_height", "seed")},
           "batched": b}
    print(json.dumps(out))
    return 0


SERVE_WARM_S = 3.0


def serving_block(rate: float | None, duration: float, max_batch: int = 32, inflight: int = 4,
                  load: float = 1.0, batch_elems: int = 0) -> dict:
    """C5: Poisson arrivals (seed 5) of commits drawn from the mixture 50 %
    2^14 x 80, 35 % 2^16 x 135, 15 % 2^18 x 135 (rate 3, cap 4), served by
    the continuous-batching loop from pinned host inputs (borrowed, copied at
    admission), each released as soon as it is done; then the same trace
    through the serial one-at-a-time commit path (commit, cap read, release).
    Latency is submit -> done; p50/p99 over the requests that arrive after a
    warm-up, throughput over the elements completed after it.

    rate None: the arrival rate is ``load`` times the serial path's capacity,
    measured here first (the inverse of its mean service time over the
    mixture, each shape timed warm through the serial path)."""
    import torch

    import paper_2603_03065_gb300 as v3c

    pool = {}
    for k, (_, log_n, c) in enumerate(synth.SERVE_MIX):
        for b in range(2):
            s = synth.Shape(c=c, log_n=log_n, rate_bits=3, cap_height=4, batch=1000 + 2 * k + b, seed=5)
            t = torch.from_numpy(s.inputs().view(np.int64)).pin_memory()
            pool[(log_n, c, b)] = t.numpy().view(np.uint64)
    ctx = v3c.Context(0, hbm_budget_bytes=150 << 30, max_inflight=inflight)
    stream = torch.cuda.current_stream()

    def serial_one(a):
        cid = ctx.commit([(a, 3, 4)], stream=stream)[0]
        ctx.cap(cid)
        ctx.release(cid)

    service_ms = {}
    for (log_n, c, b), a in pool.items():
        if b:
            continue
        for _ in range(3):
            serial_one(a)
        ts = []
        for _ in range(5):
            t0 = time.perf_counter()
            serial_one(a)
            ts.append(time.perf_counter() - t0)
        service_ms[f"{c}x2^{log_n}"] = statistics.median(ts) * 1e3
    mean_s = sum(p * service_ms[f"{c}x2^{ln}"] for p, ln, c in synth.SERVE_MIX) / 1e3
    serial_capacity = 1.0 / mean_s
    if rate is None:
        rate = load * serial_capacity
    trace = synth.poisson_trace(rate=rate, duration=duration, seed=5)
    warm = SERVE_WARM_S if duration > 2 * SERVE_WARM_S else 0.0

    def src(i, req):
        return pool[(req.shape.log_n, req.shape.c, i % 2)]

    def summarize(lat, done):
        lat = sorted(lat)
        q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))] if lat else None  # noqa: E731
        t_end = max((t for t, _ in done), default=warm)
        elems = sum(e for t, e in done if t >= warm)
        return {"requests": len(lat), "p50_ms": q(0.50) * 1e3 if lat else None,
                "p99_ms": q(0.99) * 1e3 if lat else None,
                "Gelem/s": elems / max(t_end - warm, 1e-9) / 1e9}

    clocks = ClockSampler(0)
    clocks.start()
    l0 = ctx.kernel_launches()
    ctx.serve_start(max_batch=max_batch, batch_elems=batch_elems)
    pending = {}
    lat, done = [], []
    t0 = time.perf_counter()
    t0_lib = None   # the library's clock at the trace start
    i = 0
    while i < len(trace) or pending:
        now = time.perf_counter() - t0
        while i < len(trace) and trace[i].t_arrive <= now:
            req = trace[i]
            tk = ctx.serve_submit(src(i, req), 3, 4, borrow=True)
            if tk < 0:
                break                                   # queue full: retry on the next pass
            pending[tk] = req
            i += 1
        for tk in list(pending):
            st, state, _, times = ctx.serve_poll(tk)
            if st == v3c.V3C_EAGAIN:
                continue
            req = pending.pop(tk)
            if st != v3c.V3C_OK:
                raise RuntimeError(f"request failed with status {st}")
            ctx.release(tk)
            if t0_lib is None:
                t0_lib = times[0] - req.t_arrive
            done.append((times[3] - t0_lib, req.shape.lde_elems()))
            if req.t_arrive >= warm:
                lat.append(times[3] - times[0])
        time.sleep(0.0002)
    wall = time.perf_counter() - t0
    ctx.serve_stop()
    served = summarize(lat, done)
    served["wall_s"] = wall
    served["launches"] = ctx.kernel_launches() - l0

    # Serial path: one commit at a time, in arrival order, from the same pinned
    # inputs; latency = done - arrival.
    lat_s, done_s = [], []
    l0 = ctx.kernel_launches()
    t0 = time.perf_counter()
    for k, req in enumerate(trace):
        now = time.perf_counter() - t0
        if req.t_arrive > now:
            time.sleep(req.t_arrive - now)
        serial_one(src(k, req))
        t_done = time.perf_counter() - t0
        done_s.append((t_done, req.shape.lde_elems()))
        if req.t_arrive >= warm:
            lat_s.append(t_done - req.t_arrive)
    serial = summarize(lat_s, done_s)
    serial["wall_s"] = time.perf_counter() - t0
    serial["launches"] = ctx.kernel_launches() - l0
    clk = clocks.stop()
    ctx.close()
    mean_elems = sum(r.shape.lde_elems() for r in trace) / max(len(trace), 1)
    return {"workload": "serve_poisson", "rate_rps": rate, "duration_s": duration, "warmup_s": warm,
            "requests": len(trace), "mix": [list(m) for m in synth.SERVE_MIX], "rate_bits": 3, "cap_height": 4,
            "hbm_budget_gb": 150, "max_batch": max_batch, "max_inflight": inflight,
            "batch_elems": batch_elems or (1 << 28),
            "offered_Gelem_per_s": rate * mean_elems / 1e9,
            "serial_service_ms": service_ms, "serial_capacity_rps": serial_capacity,
            "rate_vs_serial_capacity": rate / serial_capacity,
            "served": served, "serial": serial,
            "served_vs_serial_throughput": served["Gelem/s"] / max(serial["Gelem/s"], 1e-12),
            "served_vs_serial_p99": (serial["p99_ms"] / served["p99_ms"]) if served["p99_ms"] else None,
            "clocks": clk}


def run_serving(args):
    """C5 as its own bench line (the default line carries the same block at
    a rate set from the serial path's measured capacity)."""
    import torch

    torch.cuda.set_device(0)
    b = serving_block(args.rate, args.duration, args.max_batch, args.inflight, batch_elems=args.batch_elems)
    out = {"metric": METRIC, "unit": "Gelem/s", "value": b["served"]["Gelem/s"], "higher_is_better": True,
           "n_gpus": 1, "dtype": "u64", "data": "synthetic", "vs_baseline": None,
           "config": {k: v for k, v in b.items() if k not in ("served", "serial", "clocks")},
           "served": b["served"], "serial": b["serial"], "clocks": b["clocks"],
           "vs_serial_throughput": b["served_vs_serial_throughput"]}
    print(json.dumps(out))
    return 0


FRI_METRIC = "FRI commit phase on the resident LDE: combined LDE elements Gelem/s"
FRI_QUERIES = 28      # Plonky2's default number of query rounds
FRI_CFG = (4, 5, 4)   # arity 2^4, final polynomial 2^5 values, cap height 4 per layer
FRI_EXT = 2           # challenges and layers in the quadratic extension (Plonky2's default)
# DRAM traffic of one k_fri_combine launch on the 135 x 2^20 workload, from an
# ncu capture of the same kernel.  Drop the entry when the kernel changes.
# DRAM bytes (read + write) of one k_fri_combine_tma<2> launch: the ncu capture of the 2^17-row
# case, and that figure scaled by the 8x rows for the 2^20-row workload (same kernel and tiles,
# traffic proportional to the rows).  Drop the entries when the kernel changes.
FRI_COMBINE_TRAFFIC = {"fri_135x2_17": 1.194e9, "fri_135x2_20": 9.553e9}
# The FRI workload, and a smaller capture case of the same kernels (1.1 GB of LDE).
FRI_WORKLOADS = {"fri_135x2_20": synth.LARGE_135x2_20,
                 "fri_135x2_17": synth.Shape(c=135, log_n=17, rate_bits=3, cap_height=4, seed=0)}


def fri_cpu_baseline(s: "synth.Shape", steps: int = 1) -> dict:
    """The oracle's commit phase (combine, folds, layer trees, final
    polynomial) and 28 query openings on the LDE of a bounded sample."""
    import oracle

    x = s.inputs()
    threads = oracle.default_threads()
    e = oracle.lde(x, s.rate_bits, threads=threads)
    ch = synth.challenges(7, 64)
    nr = len(oracle.fri_arities(s.log_N, FRI_CFG[0], FRI_CFG[1]))
    idx = np.array(ch[-FRI_QUERIES:], dtype=np.uint64) % np.uint64(1 << s.log_N)
    alpha, betas = fri_challenges(ch, nr)

    def one():
        st = oracle.fri_commit([e], [s.c], alpha, betas, *FRI_CFG, threads=threads, ext=FRI_EXT)
        for t in idx:
            oracle.fri_query(st, int(t))

    one()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    dt = (time.perf_counter() - t0) / steps
    return {"value": s.lde_elems() / dt / 1e9, "unit": "Gelem/s", "cores": threads, "kind": "oracle",
            "sample": f"oracle FRI commit phase (arity 16, final 2^5, cap 4, degree-{FRI_EXT} extension) + "
                      f"{FRI_QUERIES} query openings on "
                      f"the LDE of {s.c} columns x 2^{s.log_n} rows, rate_bits {s.rate_bits}; {dt:.2f} s per step",
            "ms_per_step": dt * 1e3}


def fri_challenges(ch, nr):
    """alpha and the round challenges from a list of seeded field elements:
    (re, im) pairs for the extension."""
    if FRI_EXT == 1:
        return ch[0], ch[1:1 + nr]
    return (ch[0], ch[1]), [(ch[2 + 2 * k], ch[3 + 2 * k]) for k in range(nr)]


def run_fri(args):
    """FRI commit phase on a resident commitment of the 135 x 2^20 trace
    workload: combination of the 135 LDE columns with powers of alpha, folds
    of arity 16 down to 2^5 values, every layer's Merkle tree, the final
    coefficients; then 28 query openings and the 28 initial-row openings.
    Not the default bench line."""
    import torch

    import paper_2603_03065_gb300 as v3c

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    s = shard_workload(FRI_WORKLOADS[args.workload], rank)
    ctx = v3c.Context(local_rank, flags=v3c.FLAG_TIMING)
    stream = torch.cuda.current_stream()
    cid = ctx.commit([(v3c.to_device_u64(s.inputs()), s.rate_bits, s.cap_height)], stream=stream)[0]
    ch = synth.challenges(7 + rank, 64)
    a, fl, h = FRI_CFG
    fid = ctx.fri_begin([cid], (ch[0], ch[1]) if FRI_EXT == 2 else ch[0], a, fl, h, ext=FRI_EXT)
    info = ctx.fri_info(fid)
    ctx.fri_release(fid)
    nr = info["rounds"]
    alpha, betas = fri_challenges(ch, nr)
    idx = np.array(ch[-FRI_QUERIES:], dtype=np.uint64) % np.uint64(1 << s.log_N)

    def commit_phase():
        return ctx.fri_begin([cid], alpha, a, fl, h, betas=betas, ext=FRI_EXT, stream=stream)

    for _ in range(max(args.warmup, 1)):
        ctx.fri_release(commit_phase())
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    clocks = ClockSampler(local_rank)
    ctx.stage_stats(reset=True)
    l0 = ctx.kernel_launches()
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.fri_release(commit_phase())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    launches = ctx.kernel_launches() - l0
    stats = ctx.stage_stats(reset=True)
    value = world * s.lde_elems() / (ms * 1e-3) / 1e9

    # End to end through the public calls: commit phase, layer caps and final
    # polynomial to the host, the query openings and the initial rows.
    def step_e2e():
        fid = commit_phase()
        caps = [ctx.fri_cap(fid, k) for k in range(nr)]
        fin = ctx.fri_final(fid)
        recs = ctx.fri_query(fid, idx)
        rows, paths = ctx.open_batch(cid, idx, s.c)
        ctx.fri_release(fid)
        return caps, fin, recs, rows, paths

    out = step_e2e()
    d2h = sum(c.nbytes for c in out[0]) + out[1].nbytes + out[2].nbytes + out[3].nbytes + out[4].nbytes
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps)

    comb_ms, comb_n = stats["fri_combine"]
    comb_per = comb_ms / max(comb_n, 1)
    N = 1 << s.log_N
    comb_bytes = N * s.ld * 8 + N * 8 * FRI_EXT   # every LDE row once (pad column included), f_0 written
    achieved = comb_bytes / (comb_per * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    stage_ms = {k: (v[0] / v[1], int(v[1])) for k, v in stats.items() if v[1]}
    if rank == 0:
        line = {
            "metric": FRI_METRIC, "value": value, "unit": "Gelem/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "columns": s.c, "log_rows": s.log_n,
                       "rate_bits": s.rate_bits, "lde_rows": N, "arity_bits": a, "final_log": fl,
                       "layer_cap_height": h, "rounds": nr, "queries": FRI_QUERIES, "ext_degree": FRI_EXT,
                       "l2": "inputs larger than L2 (no flush needed)"},
            "e2e": {"value": world * s.lde_elems() / e2e_s / 1e9, "unit": "Gelem/s",
                    "h2d_bytes_per_step": int(2 * idx.nbytes + 8 * FRI_EXT * (len(betas) + 1)),
                    "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": e2e_s * 1e3},
            "gpu_launches": int(launches),
            "clocks": clk,
            "roofline": {"bound": "hbm", "kernel": "k_fri_combine_tma<%d>" % FRI_EXT,
                         "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": FRI_COMBINE_TRAFFIC.get(args.workload),
                         "bytes_per_launch": comb_bytes, "ms_per_launch": comb_per, "peak_source": "measured"},
            "stages_ms_per_launch": stage_ms,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = fri_cpu_baseline(FRI_CPU_SAMPLE)
        print(json.dumps(line))
    ctx.release(cid)
    ctx.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def timed_region(ctx, step, steps: int, warmup: int, local_rank: int, stream):
    """W untimed steps, then K steps between CUDA events on the stream, with
    clocks sampled and the library's launches and stage times counted."""
    import torch

    for _ in range(max(warmup, 1)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    ctx.stage_stats(reset=True)
    l0 = ctx.kernel_launches()
    clocks.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    stats = ctx.stage_stats(reset=True)
    return (e0.elapsed_time(e1) / steps, clk, ctx.kernel_launches() - l0,
            {k: (v[0] / v[1], int(v[1])) for k, v in stats.items() if v[1]})


SNAP_CPU_SAMPLE = dict(log_nlist=10, log_n=8, D=384, M=8, K=256)   # 2^18 slots, MS MARCO dimensions


def snapshot_cpu_baseline(steps: int = 1) -> dict:
    import oracle

    p = SNAP_CPU_SAMPLE
    rec, mu, cb = synth.snapshot(31, p["log_nlist"], p["log_n"], p["D"], p["M"], p["K"])
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.snapshot_commit(rec, mu, cb, p["log_nlist"], p["log_n"], threads=threads)
    dt = (time.perf_counter() - t0) / steps
    slots = 1 << (p["log_nlist"] + p["log_n"])
    return {"value": slots / dt / 1e6, "unit": "Mslot/s", "cores": threads, "kind": "oracle", "ms_per_step": dt * 1e3,
            "sample": f"oracle snapshot commitment of 2^{p['log_nlist']} lists x 2^{p['log_n']} slots, D {p['D']}, "
                      f"M {p['M']}, K {p['K']}; {dt:.2f} s per commitment"}


def run_snapshot(args):
    """Snapshot commitment of the MS MARCO high-accuracy layout (8192 lists x
    2048 slots = 2^24 slots, D = 384, M = 8, K = 256) from device-resident
    records, centroids and codebooks; roots read back each step.  Not the
    default bench line."""
    import torch

    import paper_2603_03065_gb300 as v3c

    torch.cuda.set_device(0)
    p = synth.SNAP_MSMARCO
    ln, lnn = p["log_nlist"], p["log_n"]
    rec, mu, cb = synth.snapshot(24, ln, lnn, p["D"], p["M"], p["K"], valid=p["valid"])
    ctx = v3c.Context(0, flags=v3c.FLAG_TIMING)
    stream = torch.cuda.current_stream()
    d = [v3c.to_device_u64(a) for a in (rec, mu, cb)]

    def step():
        ctx.snapshot_release(ctx.snapshot_commit(*d, ln, lnn, stream=stream))

    # Cold: two codebook sets in turn, so every commit runs the codebook sponge.
    _, _, cb_b = synth.snapshot(25, 0, 0, p["D"], p["M"], p["K"])
    d_cb_b = v3c.to_device_u64(cb_b)
    flip = [0]

    def step_cold():
        flip[0] ^= 1
        cbk = d_cb_b if flip[0] else d[2]
        ctx.snapshot_release(ctx.snapshot_commit(d[0], d[1], cbk, ln, lnn, stream=stream))

    cold_ms, _, _, cold_stage = timed_region(ctx, step_cold, max(2, args.steps // 3), 1, 0, stream)
    # Steady state: the same codebooks every step (PQ codebooks are static once
    # trained); the digest is reused after the on-device equality check.
    ms, clk, launches, stage_ms = timed_region(ctx, step, args.steps, args.warmup, 0, stream)
    N = 1 << (ln + lnn)
    value = N / (ms * 1e-3) / 1e6

    def step_e2e():
        sid = ctx.snapshot_commit(rec, mu, cb, ln, lnn, stream=stream)
        roots = ctx.snapshot_roots(sid)
        ctx.snapshot_release(sid)
        return roots

    step_e2e()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    e2e_s = (time.perf_counter() - t0) / args.steps
    slot_ms = stage_ms["snapshot_slots"][0]
    perms = N * -(-(4 + p["M"]) // 8)
    achieved = W_PER_PERM * perms / (slot_ms * 1e-3) / 1e12
    peak = SMS * WIDE_MUL_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    line = {
        "metric": "snapshot commitment (root_mk, root_cb) Mslot/s", "value": value, "unit": "Mslot/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "snapshot_msmarco", "lists": 1 << ln, "slots_per_list": 1 << lnn, "D": p["D"],
                   "M": p["M"], "K": p["K"], "valid_fraction": p["valid"],
                   "codebooks": "unchanged between steps (digest reused after an on-device equality check)",
                   "l2": "inputs larger than L2 (no flush needed)"},
        "cold": {"ms_per_step": cold_ms, "value": N / (cold_ms * 1e-3) / 1e6, "unit": "Mslot/s",
                 "note": "two codebook sets in turn: the codebook sponge runs every step",
                 "codebook_ms": cold_stage.get("snapshot_codebook", (None,))[0]},
        "e2e": {"value": N / e2e_s / 1e6, "unit": "Mslot/s", "ms_per_step": e2e_s * 1e3,
                "h2d_bytes_per_step": int(rec.nbytes + mu.nbytes + cb.nbytes), "d2h_bytes_per_step": 64},
        "gpu_launches": int(launches), "clocks": clk,
        "roofline": {"bound": "alu", "kernel": "k_snap_slots", "achieved": achieved, "peak": peak,
                     "unit": "T wide-mul/s", "frac": achieved / peak, "traffic": None,
                     "work_per_launch": W_PER_PERM * perms, "ms_per_launch": slot_ms},
        "stages_ms_per_launch": stage_ms,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = snapshot_cpu_baseline()
    print(json.dumps(line))
    ctx.close()
    return 0


def seteq_cpu_baseline(steps: int = 1) -> dict:
    import oracle

    p = synth.SETEQ_MSMARCO
    L, n = 1 << p["log_L"], 8
    cases = [synth.seteq_instance(7, L, p["T"], batch=q) for q in range(n)]
    t0 = time.perf_counter()
    for _ in range(steps):
        for q, (X, Y) in enumerate(cases):
            oracle.seteq_partial_products(X, Y, 1000 + q, 77 + q)
    dt = (time.perf_counter() - t0) / steps
    return {"value": n * L / dt / 1e9, "unit": "Gtuple/s", "cores": 1, "kind": "oracle", "ms_per_step": dt * 1e3,
            "sample": f"oracle SetEq columns of {n} of the 64 instances (2^{p['log_L']} tuples of width {p['T']}), "
                      f"one core; {dt:.2f} s"}


def run_seteq(args):
    """SetEq grand-product columns of 64 instances x 2^17 tuples of width 4
    (the multiset checks of 64 queries at the MS MARCO scan budget) in one
    call, device-resident.  Not the default bench line."""
    import torch

    import paper_2603_03065_gb300 as v3c

    torch.cuda.set_device(0)
    p = synth.SETEQ_MSMARCO
    L, n, T = 1 << p["log_L"], p["instances"], p["T"]
    ctx = v3c.Context(0, flags=v3c.FLAG_TIMING)
    stream = torch.cuda.current_stream()
    host, inst = [], []
    for q in range(n):
        X, Y = synth.seteq_instance(7, L, T, batch=q)
        ch = synth.challenges(1000 + q, 2)
        host.append((X, Y))
        z = torch.empty(L + 1, dtype=torch.int64, device="cuda")
        inst.append((v3c.to_device_u64(X), v3c.to_device_u64(Y), z, ch[0], ch[1]))

    def step():
        ctx.seteq(inst, wait=False, stream=stream)

    ms, clk, launches, stage_ms = timed_region(ctx, step, args.steps, args.warmup, 0, stream)
    value = n * L / (ms * 1e-3) / 1e9
    # end to end: inputs from pinned host memory, every column back to the host
    pinned = [(torch.from_numpy(X.view(np.int64)).pin_memory(), torch.from_numpy(Y.view(np.int64)).pin_memory())
              for X, Y in host]
    zh = [torch.empty(L + 1, dtype=torch.int64).pin_memory() for _ in range(n)]

    def step_e2e():
        for (xp, yp), (xd, yd, _, _, _) in zip(pinned, inst):
            xd.copy_(xp, non_blocking=True)
            yd.copy_(yp, non_blocking=True)
        st = ctx.seteq(inst, wait=True, stream=stream)
        for z, (_, _, zd, _, _) in zip(zh, inst):
            z.copy_(zd, non_blocking=True)
        torch.cuda.synchronize()
        return st

    step_e2e()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    e2e_s = (time.perf_counter() - t0) / args.steps
    seq_ms = stage_ms["seteq"][0]
    alg_bytes = n * (2 * L * T * 8 + (L + 1) * 8)
    achieved = alg_bytes / (seq_ms * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    line = {
        "metric": "SetEq grand-product columns Gtuple/s", "value": value, "unit": "Gtuple/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "seteq_64x2_17", "instances": n, "tuples": L, "tuple_width": T,
                   "l2": "inputs larger than L2 (no flush needed)"},
        "e2e": {"value": n * L / e2e_s / 1e9, "unit": "Gtuple/s", "ms_per_step": e2e_s * 1e3,
                "h2d_bytes_per_step": int(n * 2 * L * T * 8), "d2h_bytes_per_step": int(n * (L + 1) * 8)},
        "gpu_launches": int(launches), "clocks": clk,
        "roofline": {"bound": "hbm", "kernel": "k_seteq_scan (+ k_seteq_zero)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "bytes_per_launch": alg_bytes, "ms_per_launch": seq_ms, "peak_source": "measured",
                     "note": "algorithmic bytes: X and Y read once, Z written once; one pass with a decoupled look-back"},
        "stages_ms_per_launch": stage_ms,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = seteq_cpu_baseline()
    print(json.dumps(line))
    ctx.close()
    return 0


def int_peaks(ctx) -> dict:
    """The integer roofline's denominators, measured on this GPU in this run
    (under a second): 32-bit IMAD lanes per second (halved: a 32x32->64
    product takes a low and a high lane) and 32x32->64 wide multiply-adds
    per second, each with the SM clock of its run, beside the derived
    152 x 32 x 2070 MHz."""
    try:
        lanes, mhz_l = ctx.int_pipe_rate(1, 5)
        wide, mhz_w = ctx.int_pipe_rate(0, 5)
    except Exception as e:  # pragma: no cover
        return {"peak_measured_error": str(e)}
    return {"peak_measured_imad_lanes_half": lanes / 2 / 1e12, "peak_measured_wide": wide / 1e12,
            "imad_lanes_per_sm_clk": lanes / (SMS * mhz_l * 1e6) if mhz_l else None,
            "wide_per_sm_clk": wide / (SMS * mhz_w * 1e6) if mhz_w else None,
            "int_peak_sm_mhz": mhz_w}


def path_roofline(s, ms: float, hbm_gbs: float) -> dict:
    """T_roof = max(bytes_alg / HBM, W_alg / R_int) for one commit of shape s
    against the measured step time ms.  W_alg: 6792 wide multiplies per
    permutation (leaves and nodes) plus 4 per NTT product, the products being
    c [(n/2) log n + n + 2^r ((n/2) log n + n)] (inverse transform, coset
    scale, 2^r coset transforms).  bytes_alg: the input read, the LDE written
    and read back by the leaf hash, the leaf digests written."""
    n, N = 1 << s.log_n, 1 << s.log_N
    ntt_muls = s.c * ((n // 2) * s.log_n + n + (1 << s.rate_bits) * ((n // 2) * s.log_n + n))
    w_alg = W_PER_PERM * s.perms() + W_PER_NTT_MUL * ntt_muls
    bytes_alg = 8 * (s.c * n + 2 * s.c * N + 4 * N)
    r_int = SMS * WIDE_MUL_PER_SM_CLK * SM_MAX_MHZ * 1e6
    t_int, t_hbm = w_alg / r_int * 1e3, bytes_alg / (hbm_gbs * 1e9) * 1e3
    t_roof = max(t_int, t_hbm)
    return {"T_roof_ms": t_roof, "T_ms": ms, "fraction": t_roof / ms, "bound": "alu" if t_int >= t_hbm else "hbm",
            "W_alg": w_alg, "bytes_alg": bytes_alg}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


FRI_CPU_SAMPLE = synth.Shape(c=135, log_n=16, rate_bits=3, cap_height=4, seed=0)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["v3c", "reference"], default="v3c")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["uneven_64", "serve_poisson", *sorted(FRI_WORKLOADS),
                                                               "snapshot_msmarco", "seteq_64x2_17"],
                    default="large_135x2_20")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="let the library time its tile choices for the shape during the warm-up")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: each rank commits its own independent request (weak scaling) "
                         "instead of splitting one commit by row blocks")
    ap.add_argument("--split", action="store_true", help="run the row-split path even on one GPU")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the serving and batched blocks after the timed region")
    ap.add_argument("--serve-duration", type=float, default=20.0, help="default line's serving block: seconds")
    ap.add_argument("--serve-load", type=float, default=1.0,
                    help="default line's serving block: arrival rate as a multiple of the serial capacity")
    ap.add_argument("--rate", type=float, default=200.0, help="serve_poisson: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve_poisson: trace length in seconds")
    ap.add_argument("--max-batch", type=int, default=32, help="serve_poisson: requests per batched pass")
    ap.add_argument("--inflight", type=int, default=4, help="serve_poisson: batches in flight")
    ap.add_argument("--batch-elems", type=int, default=0,
                    help="serve_poisson: LDE elements one batched launch may take (0 = the library's default)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven_64":
        return run_batched(args)
    if args.workload == "serve_poisson":
        return run_serving(args)
    if args.workload in FRI_WORKLOADS:
        return run_fri(args)
    if args.workload == "snapshot_msmarco":
        return run_snapshot(args)
    if args.workload == "seteq_64x2_17":
        return run_seteq(args)
    if args.split or (dist_env()[2] > 1 and not args.replicas):
        return run_split(args)
    return run_v3c(args)


if __name__ == "__main__":
    sys.exit(main())
