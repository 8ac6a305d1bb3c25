"""Autotuner for the kernels' schedule.

The schedule of a plan (``Plan.set_schedule``) has two knobs: the level-0
rows of one work unit (the tile height: 16 .. 256, a power of two) and the
number of CTAs of the persistent grid.  Results never depend on them; speed
does, and the best pair moves with the buffer's shape and size.  ``tune``
times protect + recover of synthetic bytes of a given shape for every
candidate on the current GPU and keeps the fastest; results are cached in a
JSON file per (device name, width, levels, size class) and ``apply`` sets a
plan's schedule from that cache.  ``tune_batch`` does the same for a whole
batch (which takes its schedule from its first item's plan) by timing the
batch itself over ``batch_candidates``.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, Iterable, Optional, Tuple

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_schedules.json")
CANDIDATE_ROWS = (16, 32, 64, 128)


def size_class(nbytes: int) -> int:
    """Power-of-two bucket of a buffer size (buffers in one bucket share a schedule)."""
    return max(0, int(round(math.log2(max(1, nbytes)))))


def _key(device_name: str, width: int, levels: int, nbytes: int) -> str:
    return "%s|%d|%d|%d" % (device_name, width, levels, size_class(nbytes))


def load_cache(path: str = DEFAULT_CACHE) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict[str, dict], path: str = DEFAULT_CACHE) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def candidates(sms: int) -> Iterable[Tuple[int, int]]:
    for rows in CANDIDATE_ROWS:
        for ctas in (0, 2 * sms, sms):
            yield rows, ctas


def tune(width: int, levels: int, nbytes: int, reps: int = 3, path: Optional[str] = DEFAULT_CACHE,
         device: int = 0) -> dict:
    """Time every candidate schedule for buffers of this shape; return (and
    cache, unless path is None) {"seg_rows", "ctas", "us", "timings"}."""
    import torch
    import paper_1803_04880_b300 as fr
    from . import workloads as wl

    torch.cuda.set_device(device)
    dev = torch.device("cuda", device)
    props = torch.cuda.get_device_properties(dev)
    plan = fr.Plan(width, levels)
    key = fr.Key(wl.KEY)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    data = torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device=dev, generator=g)
    _, pb, ub = plan.sizes(nbytes)
    priv = torch.empty(pb, dtype=torch.uint8, device=dev)
    pub = torch.empty(ub, dtype=torch.uint8, device=dev)
    out = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(device=dev)
    timings = {}
    for rows, ctas in candidates(props.multi_processor_count):
        plan.set_schedule(rows, ctas)
        best = float("inf")
        with torch.cuda.stream(s):
            for r in range(reps + 1):
                flush.fill_(r)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                fr.protect(plan, key, 0, data, nbytes, priv, pub, stream=s)
                fr.recover(plan, key, 0, priv, pub, nbytes, out, stream=s)
                e1.record(s)
                e1.synchronize()
                if r:
                    best = min(best, 1e3 * e0.elapsed_time(e1))
        fr.sync_status(s)
        if not torch.equal(out, data):
            raise RuntimeError("schedule %s gave a wrong round trip" % ((rows, ctas),))
        timings["%d/%d" % (rows, ctas)] = round(best, 2)
    rows, ctas = map(int, min(timings, key=timings.get).split("/"))
    result = {"seg_rows": rows, "ctas": ctas, "us": timings["%d/%d" % (rows, ctas)],
              "timings": timings}
    if path is not None:
        cache = load_cache(path)
        cache[_key(props.name, width, levels, nbytes)] = result
        save_cache(cache, path)
    return result


# a batch's schedule: fused-unit rows (0: the library's adaptive units,
# sized to the batch's work and capped when it mixes buffers), grid cap, and
# level-fusion depth (path 0: up to three levels fused per pass, the rest in
# a second pass or the level kernel; path 1: every level in the level kernel)
BATCH_ROWS = (0, 64, 128, 256)


def batch_candidates(sms: int) -> Iterable[Tuple[int, int, int]]:
    for rows in BATCH_ROWS:
        for ctas in (0, 2 * sms):
            yield rows, ctas, 0
    for ctas in (0, 2 * sms):
        yield 0, ctas, 1


def _event_ms(fn) -> float:
    """Device time of one call of fn, by CUDA events on the current stream."""
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    fn()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1)


def tune_batch(make_run: Callable[..., Callable[[], None]], cands: Iterable[Tuple[int, ...]],
               reps: int = 2, clock: Optional[Callable[[Callable[[], None]], float]] = None) -> dict:
    """Pick a batch's schedule by timing the batch itself.  make_run(rows,
    ctas, path) sets that schedule and path on the batch's plans (a batch
    takes rows and cap from its first item's plan, each buffer's path from
    its own), builds the batch and returns a callable that runs it once; the
    results do not depend on the schedule (the caller checks them
    afterwards).  clock(fn) gives the milliseconds of one call (default:
    CUDA events on the current stream).  Returns {"seg_rows", "ctas",
    "path", "ms", "timings"} with the fastest candidate."""
    clock = clock or _event_ms
    timings = {}
    for cand in cands:
        run = make_run(*cand)
        run()  # warm-up
        timings["/".join(map(str, cand))] = round(min(clock(run) for _ in range(max(1, reps))), 3)
        del run
    best = min(timings, key=timings.get)
    rows, ctas, path = (list(map(int, best.split("/"))) + [0])[:3]
    return {"seg_rows": rows, "ctas": ctas, "path": path, "ms": timings[best], "timings": timings}


def apply(plan, nbytes: int, path: str = DEFAULT_CACHE, device_name: Optional[str] = None) -> bool:
    """Set plan's schedule from the cache for buffers of nbytes; False (and
    the library's default schedule) if the shape was never tuned."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_properties(torch.cuda.current_device()).name
    hit = load_cache(path).get(_key(device_name, plan.width, plan.levels, nbytes))
    if hit is None:
        plan.set_schedule(0, 0)
        return False
    plan.set_schedule(hit["seg_rows"], hit["ctas"])
    return True
