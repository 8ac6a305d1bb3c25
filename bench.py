#!/usr/bin/env python
"""Benchmark: protect + recover throughput of the fragmentation hot path on
one B300 (replicas on N GPUs under torchrun).

Workload (default "c3l2"): the 256 MiB format-agnostic buffer (uniform bytes |
Markov text | int32 random walk) as one buffer of width 8192, 2 levels, LL_2
(an eighth of the bytes, as int16) enciphered with AES-128-CTR, nonce 0, key
00..0f.  One step = protect of the buffer followed by its recover, each one
batch-object run on the launch stream.  L2 is flushed before each direction,
outside the timed events: a 512 MiB write, then a read of the same buffer so
that L2 holds clean lines and the timed launch pays for no write-back of the
flush.  The step time is the sum of the two event-timed directions on the
launch stream.  value = input bytes of all ranks / max-over-ranks time.  The
line carries the same measurement of the buffer at 4 levels ("c3l4") and of
the 3-plane 4096 x 4096 bitmap at 3 levels ("c2") under "sub".

--impl reference times the oracle (plain single-threaded C) on the host cores
as the reference arm, one bounded sample per step.

Workload "aesfull" is the thesis's full-encryption comparator: AES-128-CTR
over the whole 256 MiB mixed buffer (encrypt, then decrypt), the same unit
as protect+recover, so it reads beside c3l2 / c3l4.
"""
from __future__ import annotations

import argparse
import contextlib
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
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
    ap.add_argument("--workload", default="c3l2",
                    choices=["c1", "c2", "c2blocks", "c2packed", "c2keyed", "c3l2", "c3l4", "c4", "c5", "aesfull",
                             "noalloc"])
    ap.add_argument("--items", type=int, default=10000, help="c4: number of buffers")
    ap.add_argument("--requests", type=int, default=240, help="c5: requests per load level")
    ap.add_argument("--levels", default="1,2,3,4,5", help="noalloc: level counts, comma-separated")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="default workload: skip the sub-records")
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
    if name == "c1":
        return ({"workload": "256 x 256 random bytes (seed 0), 5/3 DWT 1 level, LL_1 AES-128-CTR",
                 "planes": 1, "width": 256, "levels": 1},
                [(256, 1, 0, wl.c1().reshape(-1))])
    if name == "c2":
        planes = wl.c2()
        return ({"workload": "bitmap 3x4096x4096 u8, 5/3 DWT 3 levels, LL_3 AES-128-CTR",
                 "planes": 3, "width": 4096, "levels": 3},
                [(4096, 3, i, planes[i].reshape(-1)) for i in range(planes.shape[0])])
    if name == "c2blocks":
        # the thesis's own arrangement (Sec. 5.2.1): every 8 x 8 block on its
        # own, two levels, LL_2 (4 of 64 coefficients) private
        planes = wl.c2()
        return ({"workload": "bitmap 3x4096x4096 u8 in 8x8 blocks, 5/3 DWT 2 levels per block, "
                             "LL_2 AES-128-CTR", "planes": 3, "width": 4096, "levels": 2,
                 "block": 8},
                [(4096, 2, i, planes[i].reshape(-1)) for i in range(planes.shape[0])])
    if name == "c2packed":
        # the thesis's storage of its three fragments (Sec. 5.2.3): 40 / 124 /
        # 480 bits a block for the private, first and second public fragment
        planes = wl.c2()
        return ({"workload": "bitmap 3x4096x4096 u8 in 8x8 blocks, 5/3 DWT 2 levels per block, "
                             "packed three fragments (40 / 124 / 480 bits a block), private "
                             "AES-128-CTR", "planes": 3, "width": 4096, "levels": 2, "block": 8,
                 "packed": True},
                [(4096, 2, i, planes[i].reshape(-1)) for i in range(planes.shape[0])])
    if name == "c2keyed":
        # the packed fragments with the public ones protected by the keyed
        # hashes (Sec. 5.2.1: SHA-256 of the private fragment, SHA-512 of the
        # first protected fragment, each with the key, once per block)
        planes = wl.c2()
        return ({"workload": "bitmap 3x4096x4096 u8 in 8x8 blocks, 5/3 DWT 2 levels per block, "
                             "packed three fragments, private AES-128-CTR, public protected by "
                             "keyed SHA-256 / SHA-512 per block", "planes": 3, "width": 4096,
                 "levels": 2, "block": 8, "packed": True, "keyed": True},
                [(4096, 2, i, planes[i].reshape(-1)) for i in range(planes.shape[0])])
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
        # the raw samples (the JSON line carries their summary); FRAG_CLOCKS_CSV
        # names another file to keep them
        self.path = os.environ.get("FRAG_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                      "frag_clocks_bench.csv")

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


def job_rate(dist, total_ms, bytes_per_rank_step, K, world, device):
    """(ms per step, whole-job GB/s) of K timed steps: the slowest rank's
    time (max over ranks when dist is a process group module) and the bytes
    every rank processed (each rank the same bytes a step: weak scaling)."""
    import torch
    if dist is not None:
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms / K, world * bytes_per_rank_step * K / (total_ms / 1e3) / 1e9


def _sig(v, digits=4):
    """v to `digits` significant digits (the oracle's rates are far below 1 GB/s)."""
    return float("%.*g" % (digits, v))


# -- reference arm: the oracle on the host cores -----------------------------------

def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    import oracle
    from paper_1803_04880_b300 import workloads as wl
    if args.workload == "aesfull":
        return _reference_aes(args)
    desc, items = _workload(args.workload)
    W, L, nonce, data = items[0]
    # a bounded sample per step: the first rows of item 0, at most 1/4 of it
    # and at most 16 MiB (whole rows of 2^L); the keyed hashes run in plain
    # Python, so 64 rows of it there
    n = min(data.size, max(W * (1 << L), min(data.size // 4, SAMPLE_BYTES) // (W << L) * (W << L)))
    if desc.get("keyed"):
        n = min(n, 64 * W)
    sample = data[:n]
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        if desc.get("keyed"):
            p, u = oracle.protect_keyed(sample, W, wl.KEY, nonce)
            oracle.recover_keyed(p, u, n, W, wl.KEY, nonce)
        elif desc.get("packed"):
            p, u = oracle.protect_packed(sample, W, wl.KEY, nonce)
            oracle.recover_packed(p, u, n, W, wl.KEY, nonce)
        else:
            p, u = oracle.protect(sample, W, L, wl.KEY, nonce, block=desc.get("block", 0))
            oracle.recover(p, u, n, W, L, wl.KEY, nonce, block=desc.get("block", 0))
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n * len(times) / total / 1e9
    line = {"metric": METRIC, "value": _sig(value), "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / len(times), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": desc,
            "cpu_baseline": {"value": _sig(value), "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host_info(),
                             "sample": "%d bytes (first rows of item 0) protect+recover per step"
                                       % n},
            "e2e": {"value": _sig(value), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -- our arm ---------------------------------------------------------------------------

# the keyed hashes of one 8 x 8 block as the fewest 32-bit integer
# instructions (3-input add and logic, funnel-shift rotates; a 64-bit add or
# logic op as two): SHA-256 64 x 14 per round + 48 x 10 per schedule word + 8,
# SHA-512 80 x 28 + 64 x 20 + 16
SHA_INST_PER_BLOCK = (64 * 14 + 48 * 10 + 8) + (80 * 28 + 64 * 20 + 16)
# 32-bit integer add, logic and shift instructions an SM issues a clock
ALU_LANES_PER_SM_CLOCK = 64

# the files that define the dominant kernel (the fused-level kernel; the
# keyed packed block kernel on c2keyed)
KERNEL_SOURCES = ("fused_kernels.cu", "swar.cuh", "frag_internal.cuh")
BLOCK_SOURCES = ("block_kernels.cu", "sha2.cuh", "sha2_constants.cuh", "pack_bits.cuh", "swar.cuh",
                 "frag_internal.cuh")
CTR_SOURCES = ("cipher_kernels.cu", "aes_tt.cuh", "frag_internal.cuh")
# the sources a dominant kernel of each kind is built from
KIND_SOURCES = {"fused": KERNEL_SOURCES, "fused_low": KERNEL_SOURCES, "blocks": BLOCK_SOURCES,
                "cipher": CTR_SOURCES, "levels": ("stream_kernels.cu", "swar.cuh", "frag_internal.cuh")}


def _kernel_hash(sources=KERNEL_SOURCES):
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_1803_04880_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(workload, direction, kind):
    """DRAM bytes per launch of the dominant kernel (its kind: fused, blocks,
    cipher) from the committed ncu summary, if the entry is of that kernel and
    its sources are unchanged since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t[workload][direction]
        if e.get("kind") == kind and e["kernel_hash"] == _kernel_hash(KIND_SOURCES[kind]):
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def _oracle_round_trip(W, L, nonce, data, block, packed, keyed):
    """One protect + recover of data through the oracle (the form the
    workload uses)."""
    import oracle
    from paper_1803_04880_b300 import workloads as wl
    n = data.size
    if keyed:
        p, u = oracle.protect_keyed(data, W, wl.KEY, nonce)
        oracle.recover_keyed(p, u, n, W, wl.KEY, nonce)
    elif packed:
        p, u = oracle.protect_packed(data, W, wl.KEY, nonce)
        oracle.recover_packed(p, u, n, W, wl.KEY, nonce)
    else:
        p, u = oracle.protect(data, W, L, wl.KEY, nonce, block=block)
        oracle.recover(p, u, n, W, L, wl.KEY, nonce, block=block)


def _oracle_worker(job):
    """A pool worker: wait for the common start time, run its round trips,
    return (bytes, start, end)."""
    W, L, nonce, data, block, packed, keyed, start_at, reps = job
    while time.time() < start_at:
        time.sleep(0.001)
    t0 = time.time()
    for _ in range(reps):
        _oracle_round_trip(W, L, nonce, data, block, packed, keyed)
    return data.size * reps, t0, time.time()


def _host_info():
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        nproc = len(os.sched_getaffinity(0))
    except AttributeError:
        nproc = os.cpu_count()
    return {"cpu_model": model, "nproc": nproc}


# the oracle's bounded samples: at most this many bytes an item
SAMPLE_BYTES = 16 << 20


def _slices(items):
    """The workload's items cut into samples of at most SAMPLE_BYTES (whole
    rows of 2^L), every slice its own item with the item's nonce; a buffer
    larger than that gives several disjoint slices."""
    out = []
    for W, L, nonce, data in items:
        step = max(W << L, SAMPLE_BYTES // (W << L) * (W << L))
        for o in range(0, data.size, step):
            out.append((W, L, nonce, data[o:o + step]))
    return out


def _cpu_baseline(items, block=0, packed=False, keyed=False):
    """The oracle on the host cores: one thread on the first sample (about
    10 s), then one process per core, each on a sample (round robin), all
    started together: their bytes over the span from the first start to the
    last end.  The pool is spawned (the GPU is in use by this process)."""
    import multiprocessing as mp
    items = _slices(items)
    W, L, nonce, data = items[0]
    if keyed:  # the keyed hashes run in plain Python: the first 64 rows
        data = data[:64 * W]
    n = data.size
    reps, t0 = 0, time.perf_counter()
    while True:
        _oracle_round_trip(W, L, nonce, data, block, packed, keyed)
        reps += 1
        el = time.perf_counter() - t0
        if el >= 10.0 or reps >= 20:
            break
    host = _host_info()
    procs = max(1, host["nproc"] or 1)
    jobs = []
    start_at = time.time() + 5.0  # after every worker has started and imported
    for i in range(procs):
        Wi, Li, ni, di = items[i % len(items)]
        if keyed:
            di = di[:64 * Wi]
        jobs.append((Wi, Li, ni, di, block, packed, keyed, start_at, 1))
    agg = None
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_worker, jobs, chunksize=1)
        span = max(r[2] for r in res) - min(r[1] for r in res)
        agg = {"value": _sig(sum(r[0] for r in res) / span / 1e9), "unit": UNIT, "processes": procs,
               "sample": "one protect+recover per process, process i on sample i mod %d%s"
                         % (len(items), " (its first 64 rows)" if keyed else "")}
    except Exception as e:  # the single-thread figure stands alone
        agg = {"error": str(e)[:200]}
    return {"value": _sig(n * reps / el / 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%s of the first sample of the workload (%d bytes; samples are the items cut "
                      "into pieces of at most %d bytes of whole rows), protect+recover x%d, one thread"
                      % ("the first 64 rows" if keyed else "all", n, SAMPLE_BYTES, reps),
            "host": host, "all_cores": agg}


def _prewarm(step, stream, seconds=1.0):
    """Untimed steps for at least `seconds` of wall clock, before the warm-up
    steps proper: the GPU leaves its idle clocks (a few steps are only
    milliseconds of work) while the clock sampler starts.  Returns the steps
    and seconds it took."""
    import torch
    t0 = time.perf_counter()
    n = 0
    while True:
        with torch.cuda.stream(stream):
            for _ in range(8):
                step(n)
                n += 1
        torch.cuda.synchronize()
        if n == 8:  # the clock starts after the first chunk (first-use costs)
            t0 = time.perf_counter()
            continue
        el = time.perf_counter() - t0
        if el >= seconds or n >= 100_000:
            return {"steps": n, "seconds": round(el, 3)}


def _measure(args, name, dev, s, world, dist, local_rank, K, Wm, e2e_steps, pf_reps):
    """One workload of single-buffer or few-buffer protect + recover: K timed
    steps after Wm warm-up steps, the per-launch kernel times, the per-file
    leg and (e2e_steps > 0) the host-buffer form.  Returns the record (every
    rank computes it; the timing is max over ranks)."""
    import torch
    import paper_1803_04880_b300 as fr
    from paper_1803_04880_b300 import workloads as wl

    desc, items = _workload(name)
    key = fr.Key(wl.KEY)
    plans = {}
    ins, privs, pubs, outs, pitems, ritems = [], [], [], [], [], []
    n_total = 0
    for W, L, nonce, data in items:
        if (W, L) not in plans:
            plans[(W, L)] = fr.Plan(W, L)
            plans[(W, L)].set_block(desc.get("block", 0))
            if desc.get("packed"):
                plans[(W, L)].set_packed(True)
            if desc.get("keyed"):
                plans[(W, L)].set_protect_public(True)
        plan = plans[(W, L)]
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
    frag_total = sum(p.numel() + u.numel() for p, u in zip(privs, pubs))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    flush_words = flush.view(torch.int32)

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

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    sampler = ClockSampler(local_rank)
    sampler.start()

    def step(i):
        flush_l2(i)
        bp.run(key, s)
        flush_l2(i)
        br.run(key, s)

    prewarm = _prewarm(step, s)
    with torch.cuda.stream(s):
        for i in range(Wm):
            step(i)
    torch.cuda.synchronize()
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
    fr.sync_status(s)
    # per-kernel durations: the same steps again with an event pair around
    # each launch inside the library's calls (kept out of the step timing:
    # an event between two launches keeps the second from starting early)
    bp.set_timing(True)
    br.set_timing(True)
    with torch.cuda.stream(s):
        for i in range(max(K, 50)):
            flush_l2(i)
            bp.run(key, s)
            flush_l2(i)
            br.run(key, s)
    kt = {"protect": bp.launch_times(), "recover": br.launch_times()}
    bp.set_timing(False)
    br.set_timing(False)
    clocks = sampler.stop()
    tp = [e[0].elapsed_time(e[1]) for e in ev]
    tr = [e[2].elapsed_time(e[3]) for e in ev]
    steps_ms = [a + b for a, b in zip(tp, tr)]
    ms_per_step, value = job_rate(dist, sum(steps_ms), n_total, K, world, dev)

    # per-file: the same step as one plain call per buffer and direction,
    # timed like the batched step (L2 flushed before each direction), with
    # the batched leg's warm-up and at least pf_reps timed repetitions
    def per_file_step(i, timed):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if timed else None
        flush_l2(i)
        if timed:
            e[0].record(s)
        for (plan, nonce, n, t, p, u) in pitems:
            fr.protect(plan, key, nonce, t, n, p, u, stream=s)
        if timed:
            e[1].record(s)
        flush_l2(i)
        if timed:
            e[2].record(s)
        for (plan, nonce, n, p, u, o) in ritems:
            fr.recover(plan, key, nonce, p, u, n, o, stream=s)
        if timed:
            e[3].record(s)
        return e

    with torch.cuda.stream(s):
        for i in range(max(3, Wm)):
            per_file_step(i, False)
        pf_ev = [per_file_step(i, True) for i in range(pf_reps)]
    torch.cuda.synchronize()
    pf = statistics.mean(e[0].elapsed_time(e[1]) + e[2].elapsed_time(e[3]) for e in pf_ev)
    for t, o in zip(ins, outs):
        assert torch.equal(t, o), "per-file round trip failed"

    peak, peak_kind = _peaks()
    t_prot = statistics.mean(tp)
    t_rec = statistics.mean(tr)
    # the dominant kernel: whichever kind's launch took longest over the two
    # directions (the fused pass over every byte, on every workload so far);
    # the second fused pass touches 1/64 of the bytes and is never the one
    per_launch = {}
    for d, times in kt.items():
        for kind, (ms, n) in times.items():
            if n:
                per_launch[(d, kind)] = ms / n
    dom_dir, dom_kind = max(((d, k) for (d, k) in per_launch if k != "fused_low"),
                            key=per_launch.get)
    t_dom = per_launch[(dom_dir, dom_kind)]
    # the fused kernel reads 1 byte and writes 2 (int16 bands and LL) per
    # input byte, or the reverse; the level kernel the same over all levels
    # (with a second fused pass, the first writes LL_3 to scratch instead of
    # the private fragment: the same 2 bytes a sample); the block kernel of
    # the packed storage moves the input and the three packed fragments
    alg_bytes = n_total + frag_total if desc.get("packed") else 3 * n_total
    achieved = alg_bytes / (t_dom / 1e3) / 1e9
    names = {"fused": "fuse_kernel<%s, packed=false> (%s: levels 1..3 of every buffer, one launch)",
             "levels": "dag_kernel<%s> (%s: dependency-ordered levels, one launch)",
             "blocks": "block_kernel<%s> (%s: every 8 x 8 block on its own, one launch)",
             "cipher": "ctr_kernel (%s%s: AES-128-CTR over the private fragments)"}
    if desc.get("packed"):
        names["blocks"] = "block_kernel<%s, packed=true> (%s: every 8 x 8 block, its bit records, one launch)"
    if desc.get("keyed"):
        names["blocks"] = ("block_kernel<%s, packed=true, keyed=true> (%s: every 8 x 8 block, its bit "
                           "records, SHA-256 + SHA-512 of each, one launch)")
    if dom_kind == "cipher":
        label = names["cipher"] % (dom_dir, "")
    else:
        label = names[dom_kind] % ("true" if dom_dir == "protect" else "false", dom_dir)
    traffic = _traffic(name, dom_dir, dom_kind)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "traffic_source": TRAFFIC_SOURCE if traffic is not None else
                "null: no ncu capture of this kernel's current source",
                "kernel": label, "peak_kind": peak_kind,
                "kernel_ms_per_launch": round(t_dom, 5),
                "launch_ms": {"%s/%s" % k: round(v, 5) for k, v in per_launch.items()},
                "algorithmic_bytes_per_launch": alg_bytes}
    if desc.get("keyed") and dom_kind == "blocks":
        # bound by the integer pipe: the two compressions of every block
        blocks = n_total // 64
        sm_mhz = (clocks or {}).get("sm_mhz") or 2032.0
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        inst_peak = sms * ALU_LANES_PER_SM_CLOCK * sm_mhz * 1e6
        inst = SHA_INST_PER_BLOCK * blocks / (t_dom / 1e3)
        roofline = {"bound": "alu", "achieved": round(inst / 1e9, 1), "peak": round(inst_peak / 1e9, 1),
                    "unit": "G instructions/s", "frac": round(inst / inst_peak, 4),
                    "traffic": traffic,
                    "traffic_source": TRAFFIC_SOURCE if traffic is not None else
                    "null: no ncu capture of this kernel's current source",
                    "kernel": label,
                    "peak_kind": "integer pipe: %d SMs x %d lanes a clock x %.0f MHz (median SM clock "
                                 "of the timed region)" % (sms, ALU_LANES_PER_SM_CLOCK, sm_mhz),
                    "algorithmic_instructions_per_launch": SHA_INST_PER_BLOCK * blocks,
                    "instructions_per_block": SHA_INST_PER_BLOCK,
                    "kernel_ms_per_launch": round(t_dom, 5),
                    "launch_ms": {"%s/%s" % k: round(v, 5) for k, v in per_launch.items()},
                    "hbm": {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                            "algorithmic_bytes_per_launch": alg_bytes}}

    # e2e through the host-buffer C-ABI calls, pinned host memory
    e2e = None
    if e2e_steps > 0:
        hin = [torch.from_numpy(d).pin_memory() for (_, _, _, d) in items]
        hp = [torch.empty(p.numel(), dtype=torch.uint8).pin_memory() for p in privs]
        hu = [torch.empty(u.numel(), dtype=torch.uint8).pin_memory() for u in pubs]
        ho = [torch.empty(d.size, dtype=torch.uint8).pin_memory() for (_, _, _, d) in items]
        times = []
        for i in range(e2e_steps + 1):
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
        # the pinned copy rates of this machine, for the e2e's own bound: one
        # copy of the input size each way
        dbuf = torch.empty(n_total, dtype=torch.uint8, device=dev)
        hbuf = torch.empty(n_total, dtype=torch.uint8).pin_memory()
        rates = {}
        for kind in ("h2d", "d2h"):
            ts = []
            for _ in range(4):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                (dbuf.copy_(hbuf, non_blocking=True) if kind == "h2d" else
                 hbuf.copy_(dbuf, non_blocking=True))
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            rates[kind + "_gbps"] = round(n_total / min(ts[1:]) / 1e9, 2)
        del dbuf, hbuf
        moved = n_total + frag_bytes
        h2d, d2h = rates["h2d_gbps"] * 1e9, rates["d2h_gbps"] * 1e9
        # the copies' own bounds: every copy after the other, or each
        # direction's copies in overlap with the other's (protect moves the
        # input in and the fragments out, recover the reverse)
        serial = moved / h2d + moved / d2h
        overlapped = max(n_total / h2d, frag_bytes / d2h) + max(frag_bytes / h2d, n_total / d2h)
        e2e = {"value": round(n_total / statistics.mean(times) / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": moved,
               "d2h_bytes_per_step": moved,
               "api": "frag_protect_host + frag_recover_host per item (pinned host buffers; buffers of "
                      "16 MiB and more move in row bands that overlap copies and kernels)",
               "pinned_copy": rates,
               "copy_bound_serial_gbps": round(n_total / serial / 1e9, 3),
               "copy_bound_overlapped_gbps": round(n_total / overlapped / 1e9, 3)}

    q = sorted(steps_ms)
    rec = {"value": round(value, 2), "unit": UNIT, "steps": K, "warmup": Wm,
           "ms_per_step": round(ms_per_step, 5),
           "config": dict(desc, l2="flushed before each direction (512 MiB write, then read back)",
                          parallelism="replicas" if world > 1 else "single GPU",
                          path=("frag_batch_run (the packed block kernel + AES-CTR, one launch "
                                "each per direction)" if desc.get("packed") else
                                "frag_batch_run (batch objects of the workload's buffers)")),
           "roofline": roofline, "e2e": e2e, "clocks": clocks, "prewarm": prewarm,
           "gpu_launches": 2 * K * bp.launches,
           "protect_gbps": round(n_total / (t_prot / 1e3) / 1e9, 2),
           "recover_gbps": round(n_total / (t_rec / 1e3) / 1e9, 2),
           "hbm_frac_protect_recover": round(2 * (n_total + frag_total) / (ms_per_step / 1e3) / 1e9 / peak, 4),
           "per_file": {"ms_per_step": round(pf, 5), "reps": pf_reps, "warmup": max(3, Wm),
                        "value": round(n_total / (pf / 1e3) / 1e9, 2),
                        "batched_over_per_file": round(pf / ms_per_step, 3)},
           "p50_ms": round(q[len(q) // 2], 5), "p99_ms": round(q[min(len(q) - 1, int(0.99 * len(q)))], 5),
           "wall_s_timed_region": round(wall, 3)}
    del bp, br, ins, privs, pubs, outs, pitems, ritems, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec, items, desc


# the sub-records of the default line: the same buffer at 4 levels, and the
# 3-plane bitmap
SUB_WORKLOADS = {"c3l2": ("c3l4", "c2")}
TRAFFIC_SOURCE = ("profiles/traffic.json: ncu dram__bytes_read.sum + dram__bytes_write.sum of "
                  "this kernel's current source on this workload (builder run, not this run)")


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1803_04880_b300 as fr

    fr.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    s = torch.cuda.Stream(device=dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    K, Wm = args.steps, args.warmup
    rec, items, desc = _measure(args, args.workload, dev, s, world, dist, local_rank, K, Wm,
                                args.e2e_steps, max(50, K))
    subs = {}
    if not args.no_sub:
        for sub in SUB_WORKLOADS.get(args.workload, ()):
            r, _, _ = _measure(args, sub, dev, s, world, dist, local_rank, K, Wm, 0, max(50, K))
            subs[sub] = r

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(items, desc.get("block", 0), bool(desc.get("packed")), bool(desc.get("keyed")))

    if rank == 0:
        line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": Wm, "ms_per_step": rec["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic", "config": rec["config"],
                "roofline": rec["roofline"], "cpu_baseline": cpu, "e2e": rec["e2e"],
                "clocks": rec["clocks"], "gpu_launches": rec["gpu_launches"]}
        for k in ("prewarm", "protect_gbps", "recover_gbps", "hbm_frac_protect_recover", "per_file", "p50_ms",
                  "p99_ms", "wall_s_timed_region"):
            line[k] = rec[k]
        if subs:
            line["sub"] = subs
        if args.workload in SUB_WORKLOADS:
            line["batched_workloads"] = (
                "the 10,000-buffer batch (--workload c4: batched vs one call per buffer) and the "
                "served stream (--workload c5: p50/p99 latency) run as their own invocations")
        print(json.dumps(line), flush=True)


# -- C4: thousands of uneven buffers, one launch per direction vs one per file ----

def _digest(t):
    import torch
    x = t.to(torch.int64)
    w = torch.arange(1, x.numel() + 1, device=t.device, dtype=torch.int64) % 65521
    return int(x.sum()), int((x * w).sum())


def run_c4(args, rank, world, local_rank):
    """10,000 buffers, log-uniform 4 KiB .. 64 MiB, width 2^round(log2(n)/2),
    levels 1..4, nonce = index (about 69 GB of input).  Timed: protect of all
    of them as one batch object replayed in a CUDA graph, then recover into
    the input buffers (the fragments alone hold the data meanwhile), against
    the same work as one frag_protect / frag_recover call per buffer.  Every
    buffer is checked after each recover by a digest of its regenerated
    contents; a seeded sample of small buffers is regenerated and compared."""
    import numpy as np
    import torch
    import paper_1803_04880_b300 as fr
    from paper_1803_04880_b300 import workloads as wl

    fr.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    items = wl.c4_items(count=args.items)
    key = fr.Key(wl.KEY)
    plans = {}
    data, privs, pubs, digests = [], [], [], []
    for i, (n, W, L, nonce) in enumerate(items):
        plan = plans.setdefault((W, L), fr.Plan(W, L))
        _, pb, ub = plan.sizes(n)
        t = wl.c4_content(i, n, device=dev)
        data.append(t)
        privs.append(torch.empty(pb, dtype=torch.uint8, device=dev))
        pubs.append(torch.empty(ub, dtype=torch.uint8, device=dev))
    torch.cuda.synchronize()
    n_total = sum(n for (n, _, _, _) in items)
    pentries = [(plans[(W, L)], nonce, n, d, p, u)
                for (n, W, L, nonce), d, p, u in zip(items, data, privs, pubs)]
    rentries = [(plans[(W, L)], nonce, n, p, u, d)
                for (n, W, L, nonce), d, p, u in zip(items, data, privs, pubs)]
    s = torch.cuda.Stream(device=dev)
    # the batch's schedule (fused-unit rows, grid cap), autotuned on the
    # batch itself: every candidate protects and recovers all the buffers
    # (in place: the round trip restores them)
    from paper_1803_04880_b300 import tune

    def set_schedule(rows, ctas, path=0):
        for p in plans.values():
            p.set_schedule(rows, ctas)
            p.set_path(path)

    def make_run(rows, ctas, path):
        set_schedule(rows, ctas, path)
        b1, b2 = fr.Batch(pentries, protect=True), fr.Batch(rentries, protect=False)

        def run():
            b1.run(key, s)
            b2.run(key, s)
        return run

    with torch.cuda.stream(s):
        tuned = tune.tune_batch(make_run, tune.batch_candidates(torch.cuda.get_device_properties(dev)
                                                                 .multi_processor_count))
    torch.cuda.synchronize()
    set_schedule(tuned["seg_rows"], tuned["ctas"], tuned["path"])
    bp = fr.Batch(pentries, protect=True)
    br = fr.Batch(rentries, protect=False)
    # graph: protect then recover in place
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bp.run(key, s)
        br.run(key, s)
    # a seeded sample of buffers regenerated and compared after one run (the
    # oracle parity of these classes is tests/test_gpu_parity.py's)
    rng = np.random.default_rng(11)
    small = [i for i, (n, _, _, _) in enumerate(items) if n <= (1 << 18)]
    sample = sorted(rng.choice(small, size=min(200, len(small)), replace=False).tolist())
    g.replay()
    torch.cuda.synchronize()
    fr.sync_status(s)
    bad = 0
    for i in sample:
        n, W, L, nonce = items[i]
        ref = wl.c4_content(i, n, device=dev)
        bad += int(not torch.equal(data[i], ref))
    assert bad == 0, "c4 sample round trip differs"
    K, Wm = max(1, min(args.steps, 5)), max(1, min(args.warmup, 3))
    for _ in range(Wm):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    with torch.cuda.stream(s):
        for _ in range(K):
            g.replay()
    e1.record(s)
    torch.cuda.synchronize()
    fr.sync_status(s)
    batched_ms = e0.elapsed_time(e1) / K
    # every buffer after the replays: regenerate and compare
    mism = 0
    for i, (n, _, _, _) in enumerate(items):
        mism += int(not torch.equal(data[i], wl.c4_content(i, n, device=dev)))
    assert mism == 0, "c4 round trip differs on %d buffers" % mism
    # per-file: one protect and one recover call per buffer, plain calls
    # (each plan with the library's default schedule)
    set_schedule(0, 0)
    torch.cuda.synchronize()
    e0.record(s)
    for (plan, nonce, n, d, p, u) in pentries:
        fr.protect(plan, key, nonce, d, n, p, u, stream=s)
    for (plan, nonce, n, p, u, d) in rentries:
        fr.recover(plan, key, nonce, p, u, n, d, stream=s)
    e1.record(s)
    torch.cuda.synchronize()
    fr.sync_status(s)
    per_file_ms = e0.elapsed_time(e1)
    noalloc = _noalloc_leg(fr, pentries, privs, pubs, key, wl.KEY, s)
    launches, held = bp.info()
    if rank == 0:
        value = world * n_total / (batched_ms / 1e3) / 1e9
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": Wm, "ms_per_step": round(batched_ms, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic",
                "config": {"workload": "batched: %d buffers log-uniform 4 KiB..64 MiB, width "
                                       "2^round(log2(n)/2), levels 1..4" % len(items),
                           "bytes": n_total, "l2": "inputs larger than L2",
                           "schedule": {"seg_rows": tuned["seg_rows"], "ctas": tuned["ctas"],
                                        "path": tuned["path"], "autotuned_ms": tuned["timings"],
                                        "note": "rows/ctas/path; rows 0, ctas 0: the library's "
                                                "adaptive units and full grid; path 0 fused "
                                                "levels, 1 level kernel only"},
                           "path": "Batch objects (one launch per wave and direction) in one CUDA graph"},
                "per_file": {"ms_per_step": round(per_file_ms, 3),
                             "value": round(n_total / (per_file_ms / 1e3) / 1e9, 2),
                             "batched_over_per_file": round(per_file_ms / batched_ms, 3)},
                "noalloc": noalloc,
                "gpu_launches": K * (launches + br.info()[0]),
                "checked_sample_items": len(sample), "batch_device_bytes": held}
        print(json.dumps(line), flush=True)


def _noalloc_leg(fr, pentries, privs, pubs, key, raw_key, s, reps=5):
    """Protect of the batch's first FRAG_NOALLOC_MAX_ITEMS buffers through
    the allocation-free call (the fused and CTR launches for buffers of 1..3
    levels, the shared-memory tile kernel for 4 levels) against a batch
    object's protect of the same buffers, both event-timed on the launch
    stream; the call's fragments must equal the batch's, which privs / pubs
    hold after the batched round trips."""
    import torch

    sub = pentries[:1024]
    nbytes = sum(e[2] for e in sub)
    p2 = [torch.empty_like(privs[i]) for i in range(len(sub))]
    u2 = [torch.empty_like(pubs[i]) for i in range(len(sub))]
    arr = (fr.frag_item * len(sub))()
    for i, (plan, nonce, n, d, _, _) in enumerate(sub):
        arr[i] = fr.frag_item(plan.handle, nonce, n, d.data_ptr(), p2[i].data_ptr(), u2[i].data_ptr())

    def call():
        st = fr.lib().frag_protect_batch_noalloc(arr, len(sub), bytes(raw_key), s.cuda_stream)
        assert st == fr.FRAG_OK, fr.last_error()

    call()
    torch.cuda.synchronize()
    assert fr.lib().frag_noalloc_sync_status(s.cuda_stream) == fr.FRAG_OK, fr.last_error()
    same = all(torch.equal(p2[i], privs[i]) and torch.equal(u2[i], pubs[i]) for i in range(len(sub)))
    assert same, "allocation-free fragments differ from the batch's"
    bsub = fr.Batch(sub, protect=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = {}
    for name, fn in (("noalloc", call), ("batch", lambda: bsub.run(key, s))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / reps
    assert fr.lib().frag_noalloc_sync_status(s.cuda_stream) == fr.FRAG_OK, fr.last_error()
    fr.sync_status(s)
    del p2, u2
    return {"what": "protect only, the first %d buffers (%.2f GB), allocation-free call "
                    "(fused + CTR launches at 1..3 levels, tile kernel at 4) vs a batch "
                    "object; fragments equal" % (len(sub), nbytes / 1e9),
            "ms": round(times["noalloc"], 3), "value": round(nbytes / (times["noalloc"] / 1e3) / 1e9, 2),
            "batch_ms": round(times["batch"], 3),
            "batch_value": round(nbytes / (times["batch"] / 1e3) / 1e9, 2)}


# -- C5: served stream of requests -------------------------------------------------

def run_c5(args, rank, world, local_rank):
    """Poisson stream of protect/recover requests (50/50), sizes log-uniform
    1 KiB .. 256 MiB, width 4096, 3 levels, through the continuous-batching
    server.  After a warm-up of at least a second, the saturated rate (all
    requests queued at once; the median of three passes), the peak under
    Poisson arrivals offered at that rate, then offered loads of 10 / 50 / 90
    % of the peak; per level p50 / p99 latency (submit to completion) and
    achieved GB/s of request bytes."""
    import numpy as np
    import torch
    import paper_1803_04880_b300 as fr
    from paper_1803_04880_b300 import workloads as wl
    from paper_1803_04880_b300.serve import Server

    fr.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    R = args.requests
    pool = torch.randint(0, 256, (1 << 29,), dtype=torch.uint8, device=dev)  # 512 MiB of bytes
    reqs = wl.c5_requests(R, 1.0, hi=1 << 28)
    sizes = [n for (_, _, n) in reqs]
    mean_size = float(np.mean(sizes))
    rng = np.random.default_rng(5)
    # request buffers start on 256-byte boundaries, as device allocations do
    offs = [int(rng.integers(0, pool.numel() - n + 1)) // 256 * 256 for n in sizes]
    srv = Server(wl.KEY, width=4096, levels=3, device=local_rank)
    # fragments for the recover requests, made beforehand
    frags = []
    for i, (n, o) in enumerate(zip(sizes, offs)):
        if reqs[i][1] == "recover":
            r = srv.submit_protect(pool[o:o + n], nonce=i)
            frags.append(r)
    for r in frags:
        r.wait()
    srv.check()
    fr_by_index = {r.nonce: r for r in frags}

    def run_level(rate):
        arr = wl.c5_requests(R, rate, hi=1 << 28) if rate else [(0.0, k, n) for (_, k, n) in reqs]
        out = []
        # rate 0: every request submitted while the scheduler holds, then
        # admitted at once (the same groups every run)
        hold = srv.held() if not rate else contextlib.nullcontext()
        hold.__enter__()
        t0 = time.perf_counter()
        for i, (a, kind, n) in enumerate(arr):
            while time.perf_counter() - t0 < a:
                time.sleep(0)
            o = offs[i]
            if kind == "protect":
                out.append(srv.submit_protect(pool[o:o + sizes[i]], nonce=10_000 + i))
            else:
                f = fr_by_index.get(i)
                if f is None:
                    out.append(srv.submit_protect(pool[o:o + sizes[i]], nonce=10_000 + i))
                else:
                    out.append(srv.submit_recover(f.private, f.public, f.nbytes, f.nonce))
        hold.__exit__(None, None, None)
        for r in out:
            r.wait()
        # the server's own clock: first submit to last completion
        t_first = min(r.t_submit for r in out)
        t1 = max(r.t_done for r in out)
        lat = sorted(1e3 * r.latency_s for r in out)
        nbytes = sum(r.nbytes for r in out)
        for r in out:  # outputs back to the pool (the fragments recovers read stay)
            r.release()
        return {"offered_req_per_s": round(rate, 1) if rate else None,
                "achieved_gbps": round(nbytes / (t1 - t_first) / 1e9, 2),
                "p50_ms": round(lat[len(lat) // 2], 3),
                "p99_ms": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3),
                "requests": len(out)}

    sampler = ClockSampler(local_rank)
    sampler.start()
    # warm-up: fills the allocator's cache with output blocks and brings the
    # GPU out of idle (one pass is only ~10 ms of work, so at least a second)
    tw = time.perf_counter()
    n_warm = 0
    while n_warm < 100:
        run_level(0)
        n_warm += 1
        if n_warm >= 2 and time.perf_counter() - tw >= 1.0:
            break
    # everything queued at once and admitted together: the drain rate (the
    # median of three passes)
    sat = sorted((run_level(0) for _ in range(3)), key=lambda r: r["achieved_gbps"])[1]
    # the peak under Poisson arrivals: offered at the drain rate, the server
    # carries what its batching of arriving requests allows
    peak = run_level(sat["achieved_gbps"] * 1e9 / mean_size)
    peak_gbps = peak["achieved_gbps"]
    levels = []
    for load in (0.1, 0.5, 0.9):
        rate = load * peak_gbps * 1e9 / mean_size
        lv = run_level(rate)
        lv["load"] = load
        lv["offered_gbps"] = round(load * peak_gbps, 2)
        levels.append(lv)
    clocks = sampler.stop()
    srv.check()
    srv.close()
    if rank == 0:
        top = levels[-1]
        line = {"metric": METRIC, "value": top["achieved_gbps"], "unit": UNIT, "n_gpus": world,
                "steps": len(levels), "warmup": n_warm, "ms_per_step": None,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic",
                "config": {"workload": "served: Poisson protect/recover 50/50, log-uniform "
                                       "1 KiB..256 MiB, width 4096, 3 levels",
                           "requests_per_level": R, "mean_request_bytes": int(mean_size),
                           "path": "serve.Server over the library's C++ scheduler (frag_server_*: "
                                   "continuous batching, 2 groups in flight, completions by stream "
                                   "host functions)"},
                "saturated": sat, "poisson_peak": peak,
                "load_reference": "poisson_peak (achieved GB/s with arrivals offered at the drain rate)",
                "levels": levels, "p50_ms": top["p50_ms"],
                "p99_ms": top["p99_ms"], "clocks": clocks, "gpu_launches": srv.launches}
        print(json.dumps(line), flush=True)


# -- the full-encryption comparator ------------------------------------------------

AES_DESC = {"workload": "full-buffer AES-128-CTR of the 256 MiB mixed buffer (encrypt + decrypt), "
                        "the thesis's full-encryption comparator", "planes": 1, "width": None,
            "levels": 0}
# the table AES's own ceiling: 148 four-byte table lookups per 16-byte block
# (16 in each of rounds 2..10, 4 in round 1, whose other terms depend only on
# the nonce and are computed once per chunk), at most 32 of them per SM per
# clock from shared memory -> SMs x clock x 32 / 148 blocks per second
AES_LOOKUPS_PER_BLOCK = 148
AES_LOOKUPS_PER_SM_CLOCK = 32


def _reference_aes(args):
    import oracle
    from paper_1803_04880_b300 import workloads as wl
    data = wl.c3()
    n = 8 << 20  # a bounded sample per step: the first 8 MiB
    sample = data[:n].tobytes()
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        c = oracle.aes128_ctr_xor(wl.KEY, 0, 0, sample)
        oracle.aes128_ctr_xor(wl.KEY, 0, 0, c)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n * len(times) / total / 1e9
    line = {"metric": METRIC, "value": _sig(value), "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / len(times), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": AES_DESC,
            "cpu_baseline": {"value": _sig(value), "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host_info(),
                             "sample": "first %d bytes, encrypt+decrypt per step" % n},
            "e2e": {"value": _sig(value), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_c1(args, rank, world, local_rank):
    """The 256 x 256 matrix of random bytes, one level: it fits in L2, so it
    is a latency figure: one frag_protect + one frag_recover call per step
    (device buffers; an event pair around each call), p50 / p99 per call,
    and the same through the host-buffer calls (wall clock, pinned)."""
    import numpy as np
    import torch
    import paper_1803_04880_b300 as fr
    from paper_1803_04880_b300 import workloads as wl

    fr.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    data = wl.c1().reshape(-1)
    n, W, L = data.size, 256, 1
    plan = fr.Plan(W, L)
    key = fr.Key(wl.KEY)
    _, pb, ub = plan.sizes(n)
    d = torch.from_numpy(data).to(dev)
    p = torch.empty(pb, dtype=torch.uint8, device=dev)
    u = torch.empty(ub, dtype=torch.uint8, device=dev)
    o = torch.empty(n, dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(device=dev)
    K, Wm = args.steps, max(3, args.warmup)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    with torch.cuda.stream(s):
        for _ in range(Wm):
            fr.protect(plan, key, 0, d, n, p, u, stream=s)
            fr.recover(plan, key, 0, p, u, n, o, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(o, d), "c1 round trip differs"
    sampler = ClockSampler(local_rank)
    sampler.start()

    def step(i):
        fr.protect(plan, key, 0, d, n, p, u, stream=s)
        fr.recover(plan, key, 0, p, u, n, o, stream=s)

    prewarm = _prewarm(step, s)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for e in ev:
            e[0].record(s)
            fr.protect(plan, key, 0, d, n, p, u, stream=s)
            e[1].record(s)
            fr.recover(plan, key, 0, p, u, n, o, stream=s)
            e[2].record(s)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    fr.sync_status(s)
    tp = sorted(1e3 * e[0].elapsed_time(e[1]) for e in ev)
    tr = sorted(1e3 * e[1].elapsed_time(e[2]) for e in ev)
    steps_us = [1e3 * e[0].elapsed_time(e[2]) for e in ev]
    ms_per_step = statistics.mean(steps_us) / 1e3
    value = n / (ms_per_step / 1e3) / 1e9

    def pct(v, q):
        return round(v[min(len(v) - 1, int(q * len(v)))], 2)

    # host buffers: wall clock of protect_host + recover_host
    hin = torch.from_numpy(data).pin_memory()
    hp = torch.empty(pb, dtype=torch.uint8).pin_memory()
    hu = torch.empty(ub, dtype=torch.uint8).pin_memory()
    ho = torch.empty(n, dtype=torch.uint8).pin_memory()
    wall = []
    for i in range(min(K, 2000) + Wm):
        t0 = time.perf_counter()
        fr.protect_host(plan, key, 0, hin, hp, hu, stream=s)
        fr.recover_host(plan, key, 0, hp, hu, n, ho, stream=s)
        if i >= Wm:
            wall.append(1e6 * (time.perf_counter() - t0))
    assert torch.equal(ho, hin), "c1 host round trip differs"
    wall.sort()
    # kernels a call launches: those of a one-item batch of the same buffer
    launches = (fr.Batch([(plan, 0, n, d, p, u)], protect=True).launches +
                fr.Batch([(plan, 0, n, p, u, o)], protect=False).launches)
    peak, peak_kind = _peaks()
    alg = 3 * n  # per direction
    t_dir = statistics.mean(tp + tr) / 1e6
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": Wm, "ms_per_step": round(ms_per_step, 5),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic",
                "config": {"workload": "256 x 256 random bytes (seed 0), 5/3 DWT 1 level, LL_1 "
                                       "AES-128-CTR (key 00..0f, nonce 0): latency class",
                           "planes": 1, "width": W, "levels": L,
                           "l2": "fits in L2 (64 KiB): not flushed; a latency figure",
                           "path": "frag_protect + frag_recover, one call each per step"},
                "latency_us": {"protect_p50": pct(tp, 0.5), "protect_p99": pct(tp, 0.99),
                               "recover_p50": pct(tr, 0.5), "recover_p99": pct(tr, 0.99),
                               "host_round_trip_p50": pct(wall, 0.5),
                               "host_round_trip_p99": pct(wall, 0.99)},
                "p50_ms": round(statistics.median(steps_us) / 1e3, 5),
                "p99_ms": round(sorted(steps_us)[min(K - 1, int(0.99 * K))] / 1e3, 5),
                "roofline": {"bound": "hbm", "achieved": round(alg / t_dir / 1e9, 2), "peak": peak,
                             "unit": "GB/s", "frac": round(alg / t_dir / 1e9 / peak, 5),
                             "traffic": None, "peak_kind": peak_kind,
                             "kernel": "one frag_protect / frag_recover call (its kernels and "
                                       "launch gaps): launch-latency bound at 64 KiB"},
                "cpu_baseline": (None if world > 1 or args.no_cpu_baseline
                                 else _cpu_baseline([(W, L, 0, data)])),
                "e2e": {"value": round(n / (statistics.mean(wall) / 1e6) / 1e9, 4), "unit": UNIT,
                        "h2d_bytes_per_step": n + pb + ub, "d2h_bytes_per_step": pb + ub + n,
                        "api": "frag_protect_host + frag_recover_host (pinned host buffers)"},
                "clocks": clocks, "prewarm": prewarm, "gpu_launches": K * launches}
        print(json.dumps(line), flush=True)


def run_aesfull(args, rank, world, local_rank):
    import torch
    import paper_1803_04880_b300 as fr
    from paper_1803_04880_b300 import workloads as wl

    fr.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    data = wl.c3()
    n = data.size
    key = fr.Key(wl.KEY)
    src = torch.from_numpy(data).to(dev)
    ct = torch.empty(n, dtype=torch.uint8, device=dev)
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    flush_words = flush.view(torch.int32)
    s = torch.cuda.Stream(device=dev)

    def flush_l2(i):
        flush.fill_(i & 255)
        torch.sum(flush_words, dtype=torch.int32)

    with torch.cuda.stream(s):
        fr.aes_ctr(key, 0, src, ct, stream=s)
        fr.aes_ctr(key, 0, ct, out, stream=s)
    torch.cuda.synchronize()
    fr.sync_status(s)
    assert torch.equal(src, out), "round trip failed"

    dist = None
    if world > 1:
        import torch.distributed as dist
    K, Wm = args.steps, args.warmup
    with torch.cuda.stream(s):
        for i in range(Wm):
            flush_l2(i)
            fr.aes_ctr(key, 0, src, ct, stream=s)
            flush_l2(i)
            fr.aes_ctr(key, 0, ct, out, stream=s)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    sampler = ClockSampler(local_rank)
    sampler.start()

    def step(i):
        flush_l2(i)
        fr.aes_ctr(key, 0, src, ct, stream=s)
        flush_l2(i)
        fr.aes_ctr(key, 0, ct, out, stream=s)

    prewarm = _prewarm(step, s)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with torch.cuda.stream(s):
        for i in range(K):
            e = ev[i]
            flush_l2(i)
            e[0].record(s)
            fr.aes_ctr(key, 0, src, ct, stream=s)
            e[1].record(s)
            flush_l2(i)
            e[2].record(s)
            fr.aes_ctr(key, 0, ct, out, stream=s)
            e[3].record(s)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    fr.sync_status(s)
    te = [e[0].elapsed_time(e[1]) for e in ev]
    td = [e[2].elapsed_time(e[3]) for e in ev]
    steps_ms = [a + b for a, b in zip(te, td)]
    ms_per_step, value = job_rate(dist, sum(steps_ms), n, K, world, dev)
    # one launch per direction: the event pair around it is the kernel's time
    t_launch = statistics.mean(te + td)
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2032.0
    blocks = (n + 15) // 16
    lookups_peak = props.multi_processor_count * sm_mhz * 1e6 * AES_LOOKUPS_PER_SM_CLOCK
    achieved = blocks * AES_LOOKUPS_PER_BLOCK / (t_launch / 1e3)
    peak_hbm, peak_kind = _peaks()
    roofline = {"bound": "alu", "achieved": round(achieved / 1e12, 3),
                "peak": round(lookups_peak / 1e12, 3), "unit": "T table lookups/s",
                "frac": round(achieved / lookups_peak, 4), "traffic": None,
                "kernel": "ctr_kernel (T-table AES-128-CTR over the whole buffer, one launch)",
                "peak_kind": "shared-memory lookup rate: %d SMs x %.0f MHz x %d lookups per SM "
                             "per clock" % (props.multi_processor_count, sm_mhz,
                                            AES_LOOKUPS_PER_SM_CLOCK),
                "kernel_ms_per_launch": round(t_launch, 5),
                "hbm_frac": round(2 * n / (t_launch / 1e3) / 1e9 / peak_hbm, 4),
                "hbm_peak": peak_hbm, "hbm_peak_kind": peak_kind}

    # the table form against the bitsliced form (frag_aes128_ctr_bitsliced),
    # at the comparator's size and at the private fragments of the same
    # buffer at one level (LL_1 as int16: 128 MiB) and two (LL_2: 32 MiB);
    # each launch timed alone, L2 flushed before it, the median of 20
    forms = None
    if not args.no_sub:
        forms = {}
        with torch.cuda.stream(s):
            fr.aes_ctr_bitsliced(key, 0, src, out, stream=s)
        torch.cuda.synchronize()
        assert torch.equal(ct, out), "the two AES forms differ"
        for label, m in (("comparator_256MiB", n), ("fragment_L1_128MiB", n // 2),
                         ("fragment_L2_32MiB", n // 8)):
            row = {}
            for fname, f in (("table", fr.aes_ctr), ("bitsliced", fr.aes_ctr_bitsliced)):
                evs = []
                with torch.cuda.stream(s):
                    for i in range(max(3, Wm) + 20):
                        flush_l2(i)
                        e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                        e[0].record(s)
                        f(key, 0, src[:m], out[:m], stream=s)
                        e[1].record(s)
                        if i >= max(3, Wm):
                            evs.append(e)
                torch.cuda.synchronize()
                t = sorted(a.elapsed_time(b) for a, b in evs)[len(evs) // 2]
                row[fname] = {"us_per_launch": round(t * 1e3, 1), "us_per_MiB": round(t * 1e3 / (m / 2**20), 4),
                              "GBps": round(m / (t / 1e3) / 1e9, 1)}
            row["bitsliced_over_table"] = round(row["bitsliced"]["us_per_launch"] /
                                                row["table"]["us_per_launch"], 3)
            forms[label] = row
        fr.sync_status(s)

    # e2e: pinned host buffers, copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        hin = torch.from_numpy(data).pin_memory()
        hct = torch.empty(n, dtype=torch.uint8).pin_memory()
        hout = torch.empty(n, dtype=torch.uint8).pin_memory()
        dbuf = torch.empty(n, dtype=torch.uint8, device=dev)
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(s):
                dbuf.copy_(hin, non_blocking=True)
                fr.aes_ctr(key, 0, dbuf, dbuf, stream=s)
                hct.copy_(dbuf, non_blocking=True)
                dbuf.copy_(hct, non_blocking=True)
                fr.aes_ctr(key, 0, dbuf, dbuf, stream=s)
                hout.copy_(dbuf, non_blocking=True)
            s.synchronize()
            dt = time.perf_counter() - t0
            if i > 0:
                times.append(dt)
        assert torch.equal(hin, hout), "host round trip failed"
        e2e = {"value": round(n / statistics.mean(times) / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": 2 * n, "d2h_bytes_per_step": 2 * n,
               "api": "frag_aes128_ctr on device copies of pinned host buffers, both directions"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        m = 16 << 20
        sample = data[:m].tobytes()
        reps, t0 = 0, time.perf_counter()
        while True:
            c = oracle.aes128_ctr_xor(wl.KEY, 0, 0, sample)
            oracle.aes128_ctr_xor(wl.KEY, 0, 0, c)
            reps += 1
            el = time.perf_counter() - t0
            if el >= 10.0 or reps >= 20:
                break
        cpu = {"value": round(m * reps / el / 1e9, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first %d bytes, encrypt+decrypt x%d, one thread" % (m, reps)}

    if rank == 0:
        q = sorted(steps_ms)
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": Wm, "ms_per_step": round(ms_per_step, 5),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u8", "data": "synthetic",
                "config": dict(AES_DESC, l2="flushed before each direction (512 MiB write, then read back)",
                               parallelism="replicas" if world > 1 else "single GPU",
                               path="frag_aes128_ctr, one launch per direction"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "prewarm": prewarm,
                "gpu_launches": 2 * K,
                "encrypt_gbps": round(n / (statistics.mean(te) / 1e3) / 1e9, 2),
                "decrypt_gbps": round(n / (statistics.mean(td) / 1e3) / 1e9, 2),
                "aes_forms": forms,
                "p50_ms": round(q[len(q) // 2], 5), "p99_ms": round(q[min(len(q) - 1, int(0.99 * len(q)))], 5),
                "wall_s_timed_region": round(wall, 3)}
        print(json.dumps(line), flush=True)


# -- the allocation-free protect, per level count ------------------------------------

def run_noalloc(args, rank, world, local_rank):
    """The allocation-free batched protect (frag_protect_batch_noalloc) of the
    256 MiB mixed buffer at width 8192, once per level count of --levels:
    K event-timed calls after W untimed ones on the launch stream, against a
    batch object's protect of the same buffer timed the same way; the
    fragments must be equal.  Buffers of 1..3 levels go through the fused and
    CTR launches, of 4 and 5 levels through the shared-memory tile kernel.
    The buffer and its fragments exceed L2.  value = input bytes of every
    level count's calls / their summed time (protect only)."""
    import torch
    import paper_1803_04880_b300 as fr
    from paper_1803_04880_b300 import workloads as wl

    fr.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    d = torch.from_numpy(wl.c3()).to(dev)
    n = d.numel()
    key = fr.Key(wl.KEY)
    s = torch.cuda.Stream(device=dev)
    K, Wm = max(1, min(args.steps, 50)), max(1, min(args.warmup, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(Wm):
            fn()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(K):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    levels, total_ms = {}, 0.0
    sampler = ClockSampler(local_rank)
    sampler.start()
    for L in [int(x) for x in args.levels.split(",") if x]:
        plan = fr.Plan(8192, L)
        _, pb, ub = plan.sizes(n)
        p = torch.empty(pb, dtype=torch.uint8, device=dev)
        u = torch.empty(ub, dtype=torch.uint8, device=dev)
        arr = (fr.frag_item * 1)()
        arr[0] = fr.frag_item(plan.handle, 0, n, d.data_ptr(), p.data_ptr(), u.data_ptr())

        def call():
            st = fr.lib().frag_protect_batch_noalloc(arr, 1, bytes(wl.KEY), s.cuda_stream)
            assert st == fr.FRAG_OK, fr.last_error()
        ms = timed(call)
        assert fr.lib().frag_noalloc_sync_status(s.cuda_stream) == fr.FRAG_OK, fr.last_error()
        p2, u2 = torch.empty_like(p), torch.empty_like(u)
        b = fr.Batch([(plan, 0, n, d, p2, u2)], protect=True)
        bms = timed(lambda: b.run(key, s))
        fr.sync_status(s)
        assert torch.equal(p, p2) and torch.equal(u, u2), "allocation-free fragments differ at %d levels" % L
        levels[str(L)] = {"ms": round(ms, 4), "value": round(n / ms / 1e6, 2),
                          "batch_ms": round(bms, 4), "batch_value": round(n / bms / 1e6, 2),
                          "kernels": "tile" if L > 3 else "fused + CTR"}
        total_ms += ms
        del p, u, p2, u2, b
    clocks = sampler.stop()
    if rank == 0:
        value = world * n * len(levels) / (total_ms / 1e3) / 1e9
        line = {"metric": "allocation-free protect GB/s on one B300", "value": round(value, 2),
                "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
                "ms_per_step": round(total_ms, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": "256 MiB mixed buffer (uniform|text|int32 walk), width 8192, "
                                       "protect through frag_protect_batch_noalloc, levels " + args.levels,
                           "l2": "inputs larger than L2",
                           "path": "one call per step and level count; the batch object's protect of "
                                   "the same buffer beside it"},
                "levels": levels, "clocks": clocks}
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
        if args.workload == "c1":
            run_c1(args, rank, world, local_rank)
        elif args.workload == "c4":
            run_c4(args, rank, world, local_rank)
        elif args.workload == "c5":
            run_c5(args, rank, world, local_rank)
        elif args.workload == "aesfull":
            run_aesfull(args, rank, world, local_rank)
        elif args.workload == "noalloc":
            run_noalloc(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
