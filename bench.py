#!/usr/bin/env python
"""Benchmark: protect + recover throughput of the fragmentation hot path on
one B300 (replicas on N GPUs under torchrun).

Workload (default "c2"): the 3-plane 4096 x 4096 synthetic bitmap, width 4096,
3 levels, nonce = plane index, key 00..0f.  One step = protect of all three
planes (one batched, dependency-ordered launch: every level and the AES pass)
followed by recover of all three (one launch).  L2 is flushed before each
direction, outside the timed events: a 512 MiB write, then a read of the same
buffer so that L2 holds clean lines and the timed launch pays for no write-back
of the flush.  The step time is the sum of the two event-timed directions on
the launch stream.  value = input bytes of all ranks / max-over-ranks time.

--impl reference times the oracle (plain single-threaded C) on the host cores
as the reference arm, one bounded sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "protect+recover GB/s on one B300 (fraction of HBM peak); batched vs per-file; p99 ms"
UNIT = "GB/s"
HBM_FALLBACK = 6400.0


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3l2", "c3l4"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def _workload(name):
    """(description, list of (width, levels, nonce, uint8 numpy array))."""
    from paper_1803_04880_b300 import workloads as wl
    if name == "c2":
        planes = wl.c2()
        return ({"workload": "bitmap 3x4096x4096 u8, 5/3 DWT 3 levels, LL_3 AES-128-CTR",
                 "planes": 3, "width": 4096, "levels": 3},
                [(4096, 3, i, planes[i].reshape(-1)) for i in range(planes.shape[0])])
    L = 2 if name == "c3l2" else 4
    return ({"workload": "256 MiB mixed buffer (uniform|text|int32 walk), width 8192, "
                         "5/3 DWT %d levels, LL_%d AES-128-CTR" % (L, L),
             "planes": 1, "width": wl.C3_WIDTH, "levels": L},
            [(wl.C3_WIDTH, L, 0, wl.c3())])


# -- clocks -----------------------------------------------------------------------

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + CLOCK_FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# -- reference arm: the oracle on the host cores -----------------------------------

def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    import oracle
    from paper_1803_04880_b300 import workloads as wl
    desc, items = _workload(args.workload)
    W, L, nonce, data = items[0]
    # a bounded sample per step: the first 1/4 of item 0 (whole rows)
    n = min(data.size, max(W * (1 << L), (data.size // 4) // (W << L) * (W << L)))
    sample = data[:n]
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        p, u = oracle.protect(sample, W, L, wl.KEY, nonce)
        oracle.recover(p, u, n, W, L, wl.KEY, nonce)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n * len(times) / total / 1e9
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / len(times), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": desc,
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d bytes (first rows of item 0) protect+recover per step"
                                       % n},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -- our arm ---------------------------------------------------------------------------

def _kernel_hash():
    h = hashlib.sha256()
    for name in ("stream_kernels.cu", "frag_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1803_04880_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(workload, kernel):
    """DRAM bytes per launch from the committed ncu summary, if it is current."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t[workload][kernel]
        if e["kernel_hash"] == _kernel_hash():
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def _cpu_baseline(items):
    import oracle
    from paper_1803_04880_b300 import workloads as wl
    W, L, nonce, data = items[0]
    n = data.size
    reps, t0 = 0, time.perf_counter()
    while True:
        p, u = oracle.protect(data, W, L, wl.KEY, nonce)
        oracle.recover(p, u, n, W, L, wl.KEY, nonce)
        reps += 1
        el = time.perf_counter() - t0
        if el >= 10.0 or reps >= 20:
            break
    return {"value": round(n * reps / el / 1e9, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "item 0 of the workload (%d bytes), protect+recover x%d, one thread"
                      % (n, reps)}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_1803_04880_b300 as fr
    from paper_1803_04880_b300 import workloads as wl

    fr.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    desc, items = _workload(args.workload)
    key = fr.Key(wl.KEY)
    plans = {}
    ins, privs, pubs, outs, pitems, ritems = [], [], [], [], [], []
    n_total = 0
    for W, L, nonce, data in items:
        plan = plans.setdefault((W, L), fr.Plan(W, L))
        n = data.size
        _, pb, ub = plan.sizes(n)
        t = torch.from_numpy(data).to(dev)
        p = torch.empty(pb, dtype=torch.uint8, device=dev)
        u = torch.empty(ub, dtype=torch.uint8, device=dev)
        o = torch.empty(n, dtype=torch.uint8, device=dev)
        ins.append(t), privs.append(p), pubs.append(u), outs.append(o)
        pitems.append((plan, nonce, n, t, p, u))
        ritems.append((plan, nonce, n, p, u, o))
        n_total += n
    bp = fr.Batch(pitems, protect=True)
    br = fr.Batch(ritems, protect=False)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    flush_words = flush.view(torch.int32)
    s = torch.cuda.Stream(device=dev)

    def flush_l2(i):
        flush.fill_(i & 255)
        torch.sum(flush_words, dtype=torch.int32)  # reads it back in place, no cast

    # correctness of what is timed: one round trip checked before timing
    with torch.cuda.stream(s):
        bp.run(key, s)
        br.run(key, s)
    torch.cuda.synchronize()
    fr.sync_status(s)
    for t, o in zip(ins, outs):
        assert torch.equal(t, o), "round trip failed"

    dist = None
    if world > 1:
        import torch.distributed as dist
    K, Wm = args.steps, args.warmup
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    sampler = ClockSampler(local_rank)
    with torch.cuda.stream(s):
        for i in range(Wm):
            flush_l2(i)
            bp.run(key, s)
            flush_l2(i)
            br.run(key, s)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with torch.cuda.stream(s):
        for i in range(K):
            e = ev[i]
            flush_l2(i)
            e[0].record(s)
            bp.run(key, s)
            e[1].record(s)
            flush_l2(i)
            e[2].record(s)
            br.run(key, s)
            e[3].record(s)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    fr.sync_status(s)
    tp = [e[0].elapsed_time(e[1]) for e in ev]
    tr = [e[2].elapsed_time(e[3]) for e in ev]
    steps_ms = [a + b for a, b in zip(tp, tr)]
    total_ms = sum(steps_ms)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / K
    value = world * n_total * K / (total_ms / 1e3) / 1e9

    # per-file: the same step as 2 x planes single-buffer calls
    pf_ms = []
    with torch.cuda.stream(s):
        for i in range(max(10, K // 10)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush_l2(i)
            e0.record(s)
            for (plan, nonce, n, t, p, u) in pitems:
                fr.protect(plan, key, nonce, t, n, p, u, stream=s)
            for (plan, nonce, n, p, u, o) in ritems:
                fr.recover(plan, key, nonce, p, u, n, o, stream=s)
            e1.record(s)
            pf_ms.append((e0, e1))
    torch.cuda.synchronize()
    pf = statistics.mean(a.elapsed_time(b) for a, b in pf_ms)

    peak, peak_kind = _peaks()
    t_prot = statistics.mean(tp)
    t_rec = statistics.mean(tr)
    dominant = "protect" if t_prot >= t_rec else "recover"
    t_dom = max(t_prot, t_rec)
    alg_bytes = 3 * n_total  # protect: read 1 + write 2; recover: read 2 + write 1 per byte
    achieved = alg_bytes / (t_dom / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": _traffic(args.workload, dominant),
                "kernel": "dag_kernel<%s> (%s: every level and the AES pass, one launch)"
                          % ("true" if dominant == "protect" else "false", dominant),
                "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes}

    # e2e through the host-buffer C-ABI calls, pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        hin = [torch.from_numpy(d).pin_memory() for (_, _, _, d) in items]
        hp = [torch.empty(p.numel(), dtype=torch.uint8).pin_memory() for p in privs]
        hu = [torch.empty(u.numel(), dtype=torch.uint8).pin_memory() for u in pubs]
        ho = [torch.empty(d.size, dtype=torch.uint8).pin_memory() for (_, _, _, d) in items]
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for (plan, nonce, n, _, _, _), a, p, u in zip(pitems, hin, hp, hu):
                fr.protect_host(plan, key, nonce, a, p, u, stream=s)
            for (plan, nonce, n, _, _, _), p, u, o in zip(pitems, hp, hu, ho):
                fr.recover_host(plan, key, nonce, p, u, n, o, stream=s)
            dt = time.perf_counter() - t0
            if i > 0:
                times.append(dt)
        for a, o in zip(hin, ho):
            assert torch.equal(a, o), "host round trip failed"
        frag_bytes = sum(p.numel() + u.numel() for p, u in zip(hp, hu))
        e2e = {"value": round(n_total / statistics.mean(times) / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": n_total + frag_bytes,
               "d2h_bytes_per_step": frag_bytes + n_total,
               "api": "frag_protect_host + frag_recover_host per item (pinned host buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(items)

    if rank == 0:
        q = sorted(steps_ms)
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": Wm, "ms_per_step": round(ms_per_step, 5),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic",
                "config": dict(desc, l2="flushed before each direction (512 MiB write, then read back)",
                               parallelism="replicas" if world > 1 else "single GPU",
                               path="frag_batch_run (one dependency-ordered launch per direction)"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": 2 * K * bp.launches,
                "protect_gbps": round(n_total / (t_prot / 1e3) / 1e9, 2),
                "recover_gbps": round(n_total / (t_rec / 1e3) / 1e9, 2),
                "hbm_frac_protect_recover": round(2 * alg_bytes / (ms_per_step / 1e3) / 1e9 / peak, 4),
                "per_file": {"ms_per_step": round(pf, 5),
                             "value": round(n_total / (pf / 1e3) / 1e9, 2),
                             "batched_over_per_file": round(pf / ms_per_step, 3)},
                "p50_ms": round(q[len(q) // 2], 5), "p99_ms": round(q[min(len(q) - 1, int(0.99 * len(q)))], 5),
                "wall_s_timed_region": round(wall, 3)}
        print(json.dumps(line), flush=True)


def main():
    args = _args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
