"""Autotuner for the planes forward's and adjoint's stage-fusion schedules.

For each size N the candidates are the ordered splits of the n = log2 N
stages into passes of 2..4 stages (each pass applies its stages on both
axes).  Each candidate is timed with CUDA events on a seeded uint8 volume
(all 12 dodecants, median of a few launches after warm-up) and the fastest
is kept.  The adjoint's split is tuned on its own (``tune_adjoint``), and the
persistent batched launch gets its own splits (``tune_batched``) and
work-item lengths (``tune_batched_items``).  Results are cached as JSON
keyed by device name, SM count, N and dtype, at $DRT3D_TUNE_CACHE or
~/.cache/drt3d/tune.json.
"""
from __future__ import annotations

import itertools
import json
import os

import torch

from . import ALL, get_plan, planes_adjoint, planes_forward


def splits(n: int, lo: int = 2, hi: int = 4) -> list:
    """Ordered compositions of n into parts in [lo, hi] (n < lo: the single part n)."""
    if n < lo:
        return [(n,)]
    out = []
    for k in range(1, n // lo + 1):
        for parts in itertools.product(range(lo, hi + 1), repeat=k):
            if sum(parts) == n:
                out.append(tuple(parts))
    return out


def _cache_path() -> str:
    return os.environ.get("DRT3D_TUNE_CACHE", os.path.expanduser("~/.cache/drt3d/tune.json"))


def _key(N: int, dtype: torch.dtype) -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|{p.multi_processor_count}|{N}|{str(dtype).replace('torch.', '')}"


def load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(d: dict) -> None:
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def time_schedule(vol: torch.Tensor, groups, reps: int = 5) -> float:
    """Median milliseconds of the 12-dodecant forward under ``groups``."""
    N = int(vol.shape[0])
    plan = get_plan(N, vol.dtype)
    old = plan.schedule()
    plan.set_schedule(groups)
    try:
        out = torch.empty((12, N, N, 3 * N), dtype=torch.int32, device=vol.device)
        ws = plan.workspace("planes_forward")
        for _ in range(2):
            planes_forward(vol, ALL, out=out, workspace=ws)
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            planes_forward(vol, ALL, out=out, workspace=ws)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        times.sort()
        return times[len(times) // 2]
    finally:
        plan.set_schedule(old)


def time_adjoint(N: int, groups, dtype: torch.dtype = torch.float32, reps: int = 7, seed: int = 13) -> float:
    """Median milliseconds of the 12-dodecant planes adjoint under ``groups``
    (the plan's adjoint schedule is restored afterwards)."""
    plan = get_plan(N, dtype)
    old = plan.adjoint_schedule() if plan.adjoint_schedule() != plan.schedule() else ()
    plan.set_adjoint_schedule(groups)
    try:
        g = torch.Generator(device="cpu").manual_seed(seed)
        if dtype == torch.float32:
            cot = torch.randn((12, N, N, 3 * N), generator=g).cuda()
        else:
            cot = torch.randint(-1000, 1000, (12, N, N, 3 * N), generator=g, dtype=torch.int32).cuda()
        out = torch.empty((N, N, N), dtype=cot.dtype, device=cot.device)
        ws = plan.workspace("planes_adjoint")
        for _ in range(2):
            planes_adjoint(cot, ALL, out=out, workspace=ws)
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            planes_adjoint(cot, ALL, out=out, workspace=ws)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        times.sort()
        return times[len(times) // 2]
    finally:
        plan.set_adjoint_schedule(old)


def tune_adjoint(Ns, dtype: torch.dtype = torch.float32, use_cache: bool = True, apply: bool = True) -> dict:
    """{N: best split of the planes adjoint} (timed on its own: the adjoint's
    transposed passes favour other splits than the forward's), applied to the
    shared plans with ``apply``."""
    cache = load_cache() if use_cache else {}
    best = {}
    for N in sorted(set(int(n) for n in Ns)):
        key = "adjoint|" + _key(N, dtype)
        if key in cache:
            best[N] = tuple(cache[key]["groups"])
        else:
            n = N.bit_length() - 1
            results = {str(s): time_adjoint(N, s, dtype) for s in splits(n)}
            pick = min(results, key=results.get)
            best[N] = tuple(int(x) for x in pick.strip("()").split(",") if x.strip())
            cache[key] = {"groups": list(best[N]), "ms": results}
            torch.cuda.empty_cache()
        if apply:
            get_plan(N, dtype).set_adjoint_schedule(best[N])
    if use_cache:
        save_cache(cache)
    return best


def tune(Ns, dtype: torch.dtype = torch.uint8, use_cache: bool = True, seed: int = 11) -> dict:
    """{N: best split} for the given sizes (and record the timings)."""
    cache = load_cache() if use_cache else {}
    best = {}
    for N in sorted(set(int(n) for n in Ns)):
        key = _key(N, dtype)
        if key in cache:
            best[N] = tuple(cache[key]["groups"])
            continue
        g = torch.Generator(device="cpu").manual_seed(seed)
        vol = torch.randint(0, 256, (N, N, N), generator=g, dtype=torch.int32).to(dtype).cuda()
        n = N.bit_length() - 1
        results = {str(s): time_schedule(vol, s) for s in splits(n)}
        pick = min(results, key=results.get)
        best[N] = tuple(int(x) for x in pick.strip("()").split(",") if x.strip())
        cache[key] = {"groups": list(best[N]), "ms": results}
    if use_cache:
        save_cache(cache)
    return best


def time_batched(N: int, groups, count: int, dtype: torch.dtype = torch.uint8, reps: int = 5,
                 seed: int = 11, item_tiles=None) -> float:
    """Median milliseconds of one batched launch of ``count`` volumes of size N
    under ``groups`` (the persistent kernel has one fixed footprint, so the
    best split can differ from the per-pass launches'), with ``item_tiles``
    unit-tiles per work item of each pass (None: the defaults)."""
    from . import BatchPlan

    g = torch.Generator(device="cpu").manual_seed(seed)
    vols = [torch.randint(0, 256, (N, N, N), generator=g, dtype=torch.int32).to(dtype).cuda()
            for _ in range(count)]
    bp = BatchPlan([N] * count, dtype=dtype, schedules={N: tuple(groups)},
                   item_tiles={N: list(item_tiles)} if item_tiles is not None else None)
    bp.bind(vols)
    for _ in range(2):
        bp.run()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        bp.run()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def tune_batched(sizes, dtype: torch.dtype = torch.uint8, use_cache: bool = True, max_count: int = 4) -> dict:
    """{N: best split for the batched launch}, timing up to ``max_count``
    volumes of each size of ``sizes`` alone."""
    cache = load_cache() if use_cache else {}
    best = {}
    counts = {}
    for n in sizes:
        counts[int(n)] = counts.get(int(n), 0) + 1
    for N in sorted(counts):
        key = "batched|" + _key(N, dtype)
        if key in cache:
            best[N] = tuple(cache[key]["groups"])
            continue
        n = N.bit_length() - 1
        c = min(counts[N], max_count)
        results = {str(sp): time_batched(N, sp, c, dtype) for sp in splits(n) if len(sp) <= 4}
        pick = min(results, key=results.get)
        best[N] = tuple(int(x) for x in pick.strip("()").split(",") if x.strip())
        cache[key] = {"groups": list(best[N]), "ms": results, "count": c}
        torch.cuda.empty_cache()
    if use_cache:
        save_cache(cache)
    return best


# Work-item sizes tried for each pass of the persistent launch (unit-tiles per
# item; 0 = the library's default).
ITEM_TILES = (0, 2, 4, 8, 16, 32, 64)


def tune_batched_items(sizes, schedules: dict, dtype: torch.dtype = torch.uint8, use_cache: bool = True,
                       max_count: int = 4) -> dict:
    """{N: unit-tiles per work item of each pass} for the persistent launch:
    one sweep over the passes, each pass's candidates timed with the other
    passes at their best so far, on up to ``max_count`` volumes of size N
    alone under ``schedules[N]``."""
    cache = load_cache() if use_cache else {}
    best = {}
    counts = {}
    for n in sizes:
        counts[int(n)] = counts.get(int(n), 0) + 1
    for N in sorted(counts):
        groups = tuple(schedules[N])
        key = "batched_items|" + _key(N, dtype) + "|" + ",".join(str(g) for g in groups)
        if key in cache:
            best[N] = list(cache[key]["item_tiles"])
            continue
        c = min(counts[N], max_count)
        tiles = [0] * len(groups)
        ms = {}
        for p in range(len(groups)):
            res = {}
            for cand in ITEM_TILES:
                t = list(tiles)
                t[p] = cand
                res[cand] = time_batched(N, groups, c, dtype, item_tiles=t)
            tiles[p] = min(res, key=res.get)
            ms[str(p)] = {str(k): v for k, v in res.items()}
        best[N] = tiles
        cache[key] = {"item_tiles": tiles, "ms": ms, "count": c}
        torch.cuda.empty_cache()
    if use_cache:
        save_cache(cache)
    return best
