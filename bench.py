#!/usr/bin/env python
"""Benchmark of the 3D DRT-of-planes hot path on GB300.

Workload (one "step"): one N=256 uint8 volume -- 1 % sparse voxels at 1..255
plus 8 embedded digital planes of 255 -- through the 12-dodecant forward
transform (int32 output, 2.4 GB) followed by the exact inverse round trip from
one dodecant.  ``value`` is whole-job volumes/s with the input resident in HBM;
``e2e`` is the same through the public API with host buffers (H2D of the
volume and D2H of the transform and the reconstructed volume inside the timed
region, each step's download overlapping the next step's compute).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank transforms its own volume (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "N=256 DRT-of-planes volumes/s and HBM GB/s vs peak; batched vs one-by-one"
UNIT = "volumes/s"
L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched / lines / lsq side measurements")
    ap.add_argument("--no-tune", action="store_true", help="use the default stage-fusion split")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------
# distributed helpers (host logic; covered by gloo tests on CPU)
# --------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world: int, backend: str):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity at world 1)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * world / seconds_max


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", self.gpu], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash(files) -> str:
    """sha256 over the named CUDA sources (under the package's csrc/): a stored
    ncu traffic figure is valid only for the sources it was taken on."""
    import hashlib

    h = hashlib.sha256()
    for name in sorted(files):
        with open(os.path.join(ROOT, "paper_2501_13664_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from profiles/ncu_traffic.json, or None
    when absent or taken on other kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            e = json.load(f).get("kernels", {}).get(kernel)
        if e is None or e.get("source_sha256") != kernel_source_hash(e["sources"]):
            return None
        return float(e["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": FALLBACK_HBM_GBS, "source": "fallback"}


# --------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# --------------------------------------------------------------------------
_ORACLE_VOL = None  # the volume, in each oracle worker process


def _oracle_worker_init(f):
    global _ORACLE_VOL
    import oracle

    oracle.build()
    _ORACLE_VOL = f


def _oracle_forward(k: int) -> int:
    """Algorithm 1 on dodecant k of the worker's volume (a small checksum goes back)."""
    import oracle

    R = oracle.planes_forward(_ORACLE_VOL, dodecants=[k])[0]
    return int(R[:, :, -1].sum())


def _oracle_inverse(k: int) -> float:
    """Exact inverse of dodecant k (after computing its forward); seconds of the inverse."""
    import oracle

    R = oracle.planes_forward(_ORACLE_VOL, dodecants=[k])[0]
    t0 = time.perf_counter()
    oracle.planes_inverse(R, k)
    return time.perf_counter() - t0


def _oracle_c4_volume(args) -> float:
    """All 12 dodecants of one batch volume (Algorithm 1); seconds."""
    import oracle

    f, = args
    t0 = time.perf_counter()
    oracle.planes_forward(f)
    return time.perf_counter() - t0


def cpu_baseline_extras(f_np, workers: int) -> dict:
    """The rest of the CPU baseline: the N=256 step single-threaded, one DJT
    sector at N=128 (x12, extrapolated), and the 96-volume mixed batch over
    the pool.  Run after the GPU work, on the host cores."""
    import multiprocessing as mp

    import oracle
    import synth

    oracle.build()
    out = {}
    # single process: the 12 dodecant forwards one after another, then the inverse
    t0 = time.perf_counter()
    R0 = None
    for k in range(12):
        R = oracle.planes_forward(f_np, dodecants=[k])[0]
        if k == 0:
            R0 = R
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.planes_inverse(R0, 0)
    t_inv = time.perf_counter() - t0
    del R, R0
    out["single_thread"] = {"value": 1.0 / (t_fwd + t_inv), "unit": UNIT, "threads": 1,
                            "sample": f"one full step in one process: Algorithm 1 on the 12 dodecants "
                                      f"({t_fwd:.2f} s) + the exact inverse of dodecant 0 ({t_inv:.2f} s)"}
    # lines: one sector of the config-3 volume, extrapolated to 12
    f3 = synth.c3_volume(128)
    t0 = time.perf_counter()
    oracle.lines_forward(f3, [0])
    t_sec = time.perf_counter() - t0
    out["lines_c3"] = {"sector_s": t_sec, "twelve_sectors_s": 12 * t_sec, "extrapolated": True, "threads": 1,
                       "value": 1.0 / (12 * t_sec), "unit": "volumes/s",
                       "sample": "Algorithm 3 on sector 0 of the N=128 int16 volume (32 lines), one process; "
                                 "the 12-sector time is that sector's time x 12 (extrapolated)"}
    # the mixed batch: each volume's 12 dodecants is one task of the pool
    vols = synth.c4_batch()
    order = sorted(range(len(vols)), key=lambda i: -vols[i].shape[0])
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_c4_volume, [(vols[i],) for i in order[-workers:]])  # warm the workers
        t0 = time.perf_counter()
        pool.map(_oracle_c4_volume, [(vols[i],) for i in order], chunksize=1)
        t_b = time.perf_counter() - t0
    out["batched_c4"] = {"s": t_b, "value": len(vols) / t_b, "unit": "volumes/s", "processes": workers,
                         "sample": f"the {len(vols)} uint8 volumes of the mixed batch (N 16..256), Algorithm 1 on "
                                   f"all 12 dodecants of each, one volume per task over {workers} processes, "
                                   "largest first"}
    out["host_cores"] = os.cpu_count()
    return out


def oracle_pool(f_u8):
    """A pool of oracle worker processes on the host cores (spawned: safe after
    CUDA initialisation), one per dodecant at most, with the volume loaded."""
    import multiprocessing as mp

    workers = max(1, min(12, os.cpu_count() or 1))
    pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_worker_init, initargs=(f_u8,))
    pool.map(_oracle_forward, [0] * workers)  # warm every worker
    return pool, workers


def oracle_step_seconds(pool) -> tuple:
    """One step of the oracle: the 12 dodecant forwards spread over the pool
    (wall seconds), and the exact inverse of dodecant 0 (seconds)."""
    t0 = time.perf_counter()
    pool.map(_oracle_forward, range(12))
    t_fwd = time.perf_counter() - t0
    t_inv = pool.apply(_oracle_inverse, (0,))
    return t_fwd, t_inv


# --------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# --------------------------------------------------------------------------
def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    import synth

    f = synth.c2_volume(args.N)
    pool, workers = oracle_pool(f)
    # A step is the 12 dodecant forwards (spread over the pool); the inverse of
    # dodecant 0 is timed on every 12th step and its mean added per volume.
    fwd, inv = [], []
    try:
        for i in range(args.warmup):
            pool.map(_oracle_forward, range(12))
        t_all = time.perf_counter()
        for i in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_forward, range(12))
            fwd.append(time.perf_counter() - t0)
            if i % 12 == 0:
                inv.append(pool.apply(_oracle_inverse, (0,)))
        wall = time.perf_counter() - t_all
    finally:
        pool.close()
        pool.join()
    t_vol = statistics.mean(fwd) + statistics.mean(inv)
    value = 1.0 / t_vol
    sample = (f"per step: Algorithm 1 on the 12 dodecants of one N={args.N} volume, spread over {workers} "
              f"processes of the plain C oracle; the exact inverse of dodecant 0 timed every 12th step; "
              f"volume time = mean step + mean inverse")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": {"workload": f"N={args.N} uint8 sparse volume + 8 planes: 12-dodecant forward + exact "
                               "inverse round trip", "N": args.N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, "nccl")

    import paper_2501_13664_gb300 as drt3d
    import synth

    N = args.N
    f_np = synth.c2_volume(N, seed=2 + rank)
    vol = torch.from_numpy(f_np).to(dev)
    plan = drt3d.get_plan(N, torch.uint8)
    tuned = {}
    if not args.no_tune:
        from paper_2501_13664_gb300 import autotune

        tuned = autotune.tune([N] + ([] if args.no_extras else sorted(set(synth.c4_sizes()))))
        plan.set_schedule(tuned[N])
    out = torch.empty((12, N, N, 3 * N), dtype=torch.int32, device=dev)
    ws = plan.workspace("planes_forward")
    inv_k = 0
    inv_out = torch.empty((N, N, N), dtype=torch.int32, device=dev)
    have_inverse = hasattr(drt3d, "planes_inverse")
    iplan = drt3d.get_plan(N, torch.int32) if have_inverse else None
    iws = iplan.workspace("planes_inverse") if have_inverse else None

    def step():
        drt3d.planes_forward(vol, drt3d.ALL, out=out, workspace=ws)
        if have_inverse:
            drt3d.planes_inverse(out[inv_k], inv_k, out=inv_out, workspace=iws, check=False)

    # correctness guard on this very launch configuration
    step()
    torch.cuda.synchronize()
    if have_inverse:
        assert torch.equal(inv_out, vol.to(torch.int32)), "round trip failed"
        assert iplan.device_error() == 0

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def timed_steps(profiled: bool) -> list:
        # K steps, L2 flushed before each (untimed), CUDA events around each.
        # With `profiled` the library also records events around every one of
        # its launches (on the launching stream): those events separate the
        # launches, so the step time is taken from a run without them.
        plan.set_profiling(profiled)
        if have_inverse:
            iplan.set_profiling(profiled)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(i)  # evict L2 between timed steps (untimed)
            starts[i].record()
            step()
            ends[i].record()
        torch.cuda.synchronize()
        barrier(world)
        return [s.elapsed_time(e) for s, e in zip(starts, ends)]

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    step_ms = timed_steps(False)
    prof_step_ms = timed_steps(True)
    clk = clocks.stop()
    ms_local = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms_local, world, dev)
    value = whole_job_rate(1.0, world, ms / 1000.0)

    launches = plan.profiled_launches() + (iplan.profiled_launches() if have_inverse else [])
    plan.set_profiling(False)
    if have_inverse:
        iplan.set_profiling(False)
    # per launch name: total ms, launches, total algorithmic bytes (a pass
    # split into several launches sums its parts)
    by_name: dict = {}
    for name, t, b in launches:
        e = by_name.setdefault(name, [0.0, 0, 0.0])
        e[0] += t
        e[1] += 1
        e[2] += b
    dom = max(by_name.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_tot, dom_cnt, dom_bytes_tot) = dom
    dom_ms = dom_tot / dom_cnt
    dom_bytes = dom_bytes_tot / dom_cnt
    peaks = measured_peaks()
    achieved = dom_bytes / (dom_ms / 1000.0) / 1e9
    floor_bytes = 12.0 * N * N * (3 * N - 2) * 4 + N ** 3  # input once + final output
    kernels = {nm: {"launches": c, "avg_ms": tot / c, "algo_bytes": b / c,
                    "gbs": b / (tot / 1000.0) / 1e9} for nm, (tot, c, b) in by_name.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i32", "data": "synthetic",
        "config": {
            "workload": f"N={N} uint8 volume (1% voxels 1..255 + 8 digital planes of 255): 12-dodecant "
                        "forward (int32) + exact inverse round trip from one dodecant",
            "N": N, "dodecants": 12, "input_dtype": "u8",
            "l2": "flushed between timed steps by writing a 258 MB buffer (untimed)",
            "kernel_times": "per-launch CUDA events in a second timed run of the same steps (the events "
                            "separate the launches, so the step time is timed without them)",
            "inverse_in_step": have_inverse,
            "schedule": list(plan.schedule()),
        },
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic(dom_name),
                     "peak_source": peaks["source"], "avg_ms": dom_ms, "algo_bytes_per_launch": dom_bytes},
        "hbm_floor_gbs": floor_bytes / (ms / 1000.0) / 1e9,
        "kernels": kernels,
        "ms_per_step_with_launch_events": sum(prof_step_ms) / len(prof_step_ms),
        "gpu_launches": len(launches),
        "clocks": clk,
    }

    if not args.no_e2e:
        # Every step copies its volume in from pinned host memory and its
        # transform (and inverse) back out.  Steps are pipelined over two
        # device output buffers: step i's device-to-host copy (on a copy
        # stream) overlaps step i+1's upload and compute.  Per-step time =
        # wall time of all steps (synchronised at both ends) / steps.
        pin_in = torch.from_numpy(f_np).pin_memory()
        pin_out = [torch.empty((12, N, N, 3 * N), dtype=torch.int32).pin_memory() for _ in range(2)]
        pin_inv = [torch.empty((N, N, N), dtype=torch.int32).pin_memory() for _ in range(2)]
        outs2 = [out, torch.empty_like(out)]
        invs2 = [inv_out, torch.empty_like(inv_out)]
        vol_d = torch.empty_like(vol)
        copy_stream = torch.cuda.Stream(device=dev)
        freed = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_run(steps: int) -> float:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(steps):
                b = i & 1
                if i >= 2:
                    torch.cuda.current_stream().wait_event(freed[b])
                vol_d.copy_(pin_in, non_blocking=True)
                drt3d.planes_forward(vol_d, drt3d.ALL, out=outs2[b], workspace=ws)
                if have_inverse:
                    drt3d.planes_inverse(outs2[b][inv_k], inv_k, out=invs2[b], workspace=iws, check=False)
                copy_stream.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(copy_stream):
                    pin_out[b].copy_(outs2[b], non_blocking=True)
                    if have_inverse:
                        pin_inv[b].copy_(invs2[b], non_blocking=True)
                    freed[b].record(copy_stream)
            torch.cuda.current_stream().wait_stream(copy_stream)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / steps

        e2e_run(2)  # warm-up
        e2e_s = max_over_ranks(e2e_run(max(2, args.e2e_steps)), world, dev)
        if have_inverse:
            assert torch.equal(pin_inv[0], pin_in.to(torch.int32)), "end-to-end round trip failed"
        line["e2e"] = {"value": whole_job_rate(1.0, world, e2e_s), "unit": UNIT,
                       "h2d_bytes_per_step": int(pin_in.numel()),
                       "d2h_bytes_per_step": int(pin_out[0].numel() * 4 + (pin_inv[0].numel() * 4 if have_inverse else 0)),
                       "pipelined": "two device output buffers; each step's device-to-host copy overlaps the next "
                                    "step's upload and compute"}
        del outs2, invs2, pin_out, pin_inv

    if not args.no_extras:
        del out, ws, flush
        torch.cuda.empty_cache()
        line["batched_c4"] = bench_batched(drt3d, synth, dev, tuned)
        torch.cuda.empty_cache()
        line["lines_c3"] = bench_lines(drt3d, synth, dev)
        torch.cuda.empty_cache()
        line["lsq_c5"] = bench_lsq(drt3d, synth, dev, tune=not args.no_tune)
        torch.cuda.empty_cache()
        line["drt2d_images"] = bench_drt2d(drt3d, synth, dev)
        torch.cuda.empty_cache()
        line["press_inverse"] = bench_press(drt3d, synth, dev)
        torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool, workers = oracle_pool(f_np)
        try:
            t_fwd, t_inv = oracle_step_seconds(pool)
        finally:
            pool.close()
            pool.join()
        sample = (f"one full step of the plain C oracle on N={N}: Algorithm 1 on all 12 dodecants spread over "
                  f"{workers} processes ({t_fwd:.2f} s wall) + the exact inverse of dodecant 0 ({t_inv:.2f} s)")
        line["cpu_baseline"] = {"value": 1.0 / (t_fwd + t_inv), "unit": UNIT, "cores": workers, "kind": "oracle",
                                "sample": sample}
        if not args.no_extras:
            line["cpu_baseline"].update(cpu_baseline_extras(f_np, workers))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def _event_ms(fn, reps: int) -> list:
    import torch

    out = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        out.append(a.elapsed_time(b))
    return out


def bench_batched(drt3d, synth, dev, tuned) -> dict:
    """Config 4: 96 uint8 volumes of uneven N, one persistent launch replayed
    from a CUDA graph vs 96 one-by-one forward calls on one stream."""
    import torch

    sizes = synth.c4_sizes()
    vols = [torch.from_numpy(v).to(dev) for v in synth.c4_batch(sizes=sizes)]
    sched = {N: tuple(tuned[N]) for N in set(sizes) if N in tuned}
    bsched = sched
    btiles = None
    if tuned:
        from paper_2501_13664_gb300 import autotune

        bsched = autotune.tune_batched(sizes)  # splits for the persistent kernel's footprint
        btiles = autotune.tune_batched_items(sizes, bsched)  # work-item size per pass
    bp = drt3d.BatchPlan(sizes, schedules=bsched, item_tiles=btiles)
    outs = bp.bind(vols)
    plans, wss = {}, {}
    for N in set(sizes):
        p = drt3d.get_plan(N, torch.uint8)
        if N in sched:
            p.set_schedule(sched[N])
        plans[N] = p
        wss[N] = p.workspace("planes_forward")
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bp.run()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bp.run()
    assert bp.device_error() == 0

    def one_by_one():
        for v, o, N in zip(vols, outs, sizes):
            drt3d.planes_forward(v, drt3d.ALL, out=o, workspace=wss[N])

    for _ in range(3):
        g.replay()
        one_by_one()
    tb = sorted(_event_ms(g.replay, 7))[3]
    t1 = sorted(_event_ms(one_by_one, 7))[3]
    # mode 1: the same batch as per-volume launches over internal streams,
    # with the single-volume splits, also replayed from a CUDA graph
    ms = {}
    for k in (2, 4, 8):
        bm = drt3d.BatchPlan(sizes, schedules=sched)
        bm.set_mode(1, k)
        bm.bind(vols, outs=outs)
        with torch.cuda.stream(s):
            bm.run()
        torch.cuda.current_stream().wait_stream(s)
        gm = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gm):
            bm.run()
        for _ in range(3):
            gm.replay()
        ms[k] = sorted(_event_ms(gm.replay, 7))[3]
        assert bm.device_error() == 0
        del gm, bm
    kbest = min(ms, key=ms.get)
    floor = sum(12.0 * N * N * (3 * N - 2) * 4 + N ** 3 for N in sizes)
    best = min(tb, ms[kbest])
    return {"volumes": len(sizes), "batched_ms": best, "one_by_one_ms": t1,
            "batched_mode": "persistent" if tb <= ms[kbest] else f"streams{kbest}",
            "persistent_ms": tb, "multistream_ms": {str(k): v for k, v in ms.items()},
            "batched_volumes_per_s": len(sizes) / (best / 1000), "one_by_one_volumes_per_s": len(sizes) / (t1 / 1000),
            "speedup": t1 / best, "floor_gbs_batched": floor / (best / 1000) / 1e9,
            "launches_persistent": 1, "launches_one_by_one": sum(len(plans[N].schedule()) for N in sizes),
            "schedules_persistent": {str(N): list(v) for N, v in sorted(bsched.items())},
            "item_tiles_persistent": ({str(N): list(v) for N, v in sorted(btiles.items())} if btiles
                                      else "library defaults"),
            "schedules_one_by_one": {str(N): list(v) for N, v in sorted(sched.items())},
            "note": "persistent = one memset + one persistent kernel; multistream = the volumes' per-pass launches "
                    "over k internal streams; both replayed from a CUDA graph; one-by-one = 96 calls on one "
                    "stream; medians of 7"}


def bench_lines(drt3d, synth, dev) -> dict:
    """Config 3: DJT of lines, N=128 int16, all 12 sectors (51.5 GB out)."""
    import torch

    N = 128
    vol = torch.from_numpy(synth.c3_volume(N)).to(dev)
    plan = drt3d.get_plan(N, torch.int16)
    out = torch.empty((12, N, N, 2 * N, 2 * N), dtype=torch.int32, device=dev)
    ws = plan.workspace("lines_forward")
    run = lambda: drt3d.lines_forward(vol, drt3d.ALL, out=out, workspace=ws)  # noqa: E731
    run()
    t = sorted(_event_ms(run, 5))[2]
    floor = 12.0 * N * N * (2 * N) * (2 * N) * 4 + N ** 3 * 2
    fwd_passes = profile_launches(plan, run)
    del ws
    # adjoint (backprojection) of the same 12 sectors, the transform as cotangent
    aplan = drt3d.get_plan(N, torch.int32)
    aws = aplan.workspace("lines_adjoint")
    vb = torch.empty((N, N, N), dtype=torch.int32, device=dev)
    arun = lambda: drt3d.lines_adjoint(out, drt3d.ALL, out=vb, workspace=aws)  # noqa: E731
    arun()
    ta = sorted(_event_ms(arun, 5))[2]
    afloor = 12.0 * N * N * (2 * N) * (2 * N) * 4 + N ** 3 * 4
    adj_passes = profile_launches(aplan, arun)
    del out, aws
    return {"ms": t, "sectors_per_s": 12 / (t / 1000), "floor_gbs": floor / (t / 1000) / 1e9, "passes": fwd_passes,
            "adjoint_ms": ta, "adjoint_floor_gbs": afloor / (ta / 1000) / 1e9, "adjoint_passes": adj_passes,
            "workload": "N=128 int16 uniform 0..1023 + 32 lines, 12 sectors, int32 out; adjoint of that "
                        "transform back to an int32 volume"}


def profile_launches(plan, run) -> dict:
    """Per-launch CUDA-event times of one call of `run` (the library's own
    profiler on the launching stream), summed by launch name."""
    import torch

    plan.set_profiling(True)
    run()
    torch.cuda.synchronize()
    passes = {}
    for name, ms, by in plan.profiled_launches():
        e = passes.setdefault(name, {"launches": 0, "ms": 0.0, "algo_bytes": 0.0})
        e["launches"] += 1
        e["ms"] += ms
        e["algo_bytes"] += by
    plan.set_profiling(False)
    for e in passes.values():
        e["gbs"] = e["algo_bytes"] / (e["ms"] / 1000) / 1e9 if e["ms"] > 0 else None
    return passes


def bench_drt2d(drt3d, synth, dev) -> dict:
    """The 2D DRT by-product: 512 uint8 images of 256^2, four quadrants, int32
    out (1.07 GB written per call, larger than L2)."""
    import torch

    N, B = 256, 512
    imgs = torch.from_numpy(synth.images_2d(N, B)).to(dev)
    out = torch.empty((B, 4, N, 2 * N), dtype=torch.int32, device=dev)
    plan = drt3d.get_plan(N, torch.uint8)
    run = lambda: drt3d.drt2d_forward(imgs, range(4), out=out)  # noqa: E731
    for _ in range(3):
        run()
    t = sorted(_event_ms(run, 7))[3]
    passes = profile_launches(plan, run)
    floor = B * N * N * 1.0 + B * 4.0 * N * 2 * N * 4
    del out
    return {"ms": t, "images_per_s": B / (t / 1000), "floor_gbs": floor / (t / 1000) / 1e9, "passes": passes,
            "workload": "512 uint8 images 256x256 (5 % pixels 1..255 + 4 lines of 255 each), four quadrants, "
                        "int32 out; one CTA per (image, quadrant), 16-bit intermediate rows in shared memory"}


def bench_press(drt3d, synth, dev) -> dict:
    """Section 5.2's iterative inverse on a 128^3 float32 phantom (the size
    of the paper's MRI inversions): error after 5, 10 and 20 iterations and
    the time of 10."""
    import torch

    N = 128
    f = torch.from_numpy(synth.phantom(N)).to(dev)
    R = drt3d.planes_forward(f)
    steps = drt3d.press_step_sizes(N)
    plan = drt3d.get_plan(N, torch.float32)
    ws = plan.workspace("planes_press")
    out = torch.empty_like(f)
    rng = float(f.max() - f.min())

    def nrmsd(k):
        drt3d.planes_press_inverse(R, k, 2, steps, out=out, workspace=ws)
        return float(torch.sqrt(torch.mean((out - f) ** 2)) / rng)

    errs = {k: nrmsd(k) for k in (1, 5, 10, 20)}
    run = lambda: drt3d.planes_press_inverse(R, 10, 2, steps, out=out, workspace=ws)  # noqa: E731
    t = sorted(_event_ms(run, 3))[1]
    return {"ms_10_iterations": t, "ms_per_iteration": t / 10, "nrmsd": errs, "smooth": 2, "step_factor": 1.5,
            "workload": "128^3 float32 phantom (6 solid ellipsoids), all 12 dodecants, multigrid down to N=1"}


def bench_lsq(drt3d, synth, dev, tune: bool = True) -> dict:
    """Config 5: one gradient step of the least-squares fit, 8 x 128^3 float32
    (with ``tune``, the adjoint's split autotuned first)."""
    import torch

    N, B = 128, 8
    if tune:
        from paper_2501_13664_gb300 import autotune

        autotune.tune_adjoint([N], torch.float32)  # applied to the shared float32 plan
    x = torch.from_numpy(synth.c5_batch(N=N, batch=B)).to(dev)
    b = torch.zeros((B, 12, N, N, 3 * N), dtype=torch.float32, device=dev)

    def step():
        # 0.5 ||A x - b||^2; mse_loss computes the residual and its gradient in
        # one elementwise pass each way (the same gradient, bit for bit, as
        # spelling out r = A x - b and (r * r).sum())
        xr = x.detach().requires_grad_(True)
        (0.5 * torch.nn.functional.mse_loss(drt3d.planes(xr), b, reduction="sum")).backward()
        return xr.grad

    from paper_2501_13664_gb300 import lsq

    def step_fused():
        # the library's least-squares loss: residual A x - b in the forward's
        # last pass, loss from it, adjoint of it as the gradient
        xr = x.detach().requires_grad_(True)
        lsq.least_squares_loss(xr, b).backward()
        return xr.grad

    step()
    step_fused()
    t_mse = sorted(_event_ms(step, 5))[2]
    t = sorted(_event_ms(step_fused, 5))[2]
    passes = profile_launches(drt3d.get_plan(N, torch.float32), step_fused)
    lib_ms = sum(e["ms"] for e in passes.values())
    fplan = drt3d.get_plan(N, torch.float32)
    return {"ms_per_step": t, "volumes": B, "N": N, "passes": passes, "library_ms": lib_ms,
            "schedule_forward": list(fplan.schedule()), "schedule_adjoint": list(fplan.adjoint_schedule()),
            "autograd_mse_ms_per_step": t_mse,
            "note": "one gradient step of 0.5||Ax - b||^2 for 8 volumes through torch.autograd: ms_per_step with "
                    "the library's least-squares loss (residual subtracted in the forward's last pass, "
                    "hand-written adjoint of it); autograd_mse_ms_per_step with the batched transform and "
                    "PyTorch's mse_loss (same gradient bit for bit); passes = the library's launches of one "
                    "fused step"}


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
