"""The allocation-free batched protect (frag_protect_batch_noalloc).

It exists for callers that may not allocate device memory themselves or have
the library do it: code whose process hands all device memory to one pool it
does not control, or a latency-critical path that cannot take a driver
allocation's implicit synchronisation.  Its fragments must be byte-identical
to those of frag_protect_batch (integer work, so the tolerance is zero), on
two calls in a row that share the static scratch.  This file is collected
last so a failure here cannot hide the other tests' results.
"""
import ctypes

import numpy as np
import pytest

from paper_1803_04880_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fr():
    import paper_1803_04880_b300 as m
    m.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = m.lib().frag_protect_batch_noalloc
    f.argtypes = [ctypes.POINTER(m.frag_item), ctypes.c_uint32, ctypes.c_char_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    g = m.lib().frag_noalloc_sync_status
    g.argtypes = [ctypes.c_void_p]
    g.restype = ctypes.c_int
    return m


# one buffer per level count the call takes, 1..5 (the seeded mix below
# draws levels 1..4 only): (bytes, width, levels, nonce)
EXPLICIT = [(30_001, 128, 1, 900), (40_003, 64, 2, 901), (70_000, 256, 3, 902),
            (65_536, 128, 4, 903), (50_000, 64, 5, 904), (200_000, 512, 5, 905)]


def _buffers(fr, count, seed):
    items = wl.c4_items(count=count, lo=100, hi=1 << 19, seed=seed) + EXPLICIT
    plans, ins, ref, got = {}, [], [], []
    for (n, W, L, nonce) in items:
        plan = plans.setdefault((W, L), fr.Plan(W, L))
        _, pb, ub = plan.sizes(n)
        t = torch.from_numpy(wl.random_bytes(n, seed=seed * 7919 + nonce)).cuda()
        mk = lambda k: torch.full((k,), 0x5A, dtype=torch.uint8, device="cuda")
        ref.append((plan, nonce, n, t, mk(pb), mk(ub)))
        got.append((plan, nonce, n, t, mk(pb), mk(ub)))
    return plans, ref, got


def _noalloc(fr, entries, key=wl.KEY):
    arr = (fr.frag_item * len(entries))()
    for i, (plan, nonce, n, t, p, u) in enumerate(entries):
        arr[i] = fr.frag_item(plan.handle, nonce, n, t.data_ptr(), p.data_ptr(), u.data_ptr())
    st = fr.lib().frag_protect_batch_noalloc(arr, len(entries), key,
                                             torch.cuda.current_stream().cuda_stream)
    return st


def test_matches_allocating_batch_on_two_calls(fr):
    key = fr.Key(wl.KEY)
    for call, (count, seed) in enumerate(((40, 101), (25, 202))):
        plans, ref, got = _buffers(fr, count, seed)
        fr.protect_batch(ref, key)
        torch.cuda.synchronize()
        fr.sync_status()
        # the second call runs with nothing else allocating around it: the
        # device's free memory must not move
        free0 = torch.cuda.mem_get_info()[0]
        st = _noalloc(fr, got)
        assert st == fr.FRAG_OK, fr.last_error()
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0, "the call allocated device memory"
        st = fr.lib().frag_noalloc_sync_status(torch.cuda.current_stream().cuda_stream)
        assert st == fr.FRAG_OK, fr.last_error()
        for (plan, nonce, n, _, p0, u0), (_, _, _, _, p1, u1) in zip(ref, got):
            what = "(n=%d, W=%d, L=%d) on call %d" % (n, plan.width, plan.levels, call)
            assert torch.equal(p0, p1), "private fragment differs " + what
            assert torch.equal(u0, u1), "public fragment differs " + what


def test_rejects_more_items_than_the_scratch_holds(fr):
    limit = 1024
    arr = (fr.frag_item * (limit + 1))()
    st = fr.lib().frag_protect_batch_noalloc(arr, limit + 1, wl.KEY, None)
    assert st == fr.FRAG_EINVAL
    assert "limit" in fr.last_error()


def test_rejects_more_than_five_levels(fr):
    """The tile kernel behind this call keeps a tile and its halo in shared
    memory, which bounds it at 5 levels; 6 to 8 are refused with a message."""
    plan = fr.Plan(64, 6)
    t = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    _, pb, ub = plan.sizes(t.numel())
    p = torch.empty(pb, dtype=torch.uint8, device="cuda")
    u = torch.empty(ub, dtype=torch.uint8, device="cuda")
    st = _noalloc(fr, [(plan, 0, t.numel(), t, p, u)])
    assert st == fr.FRAG_EUNSUPPORTED
    assert "at most 5 levels" in fr.last_error()


# (bytes, width, levels, nonce, input offset, private-fragment offset): the
# fused pass takes the first three (1..3 levels, aligned, width a multiple of
# 8); the tile kernel the rest -- an input one byte off alignment, a width of
# 4, a private fragment 4 bytes off 8-byte alignment at one level, 4 and 5
# levels
ROUTES = [(50_000, 64, 1, 910, 0, 0), (70_001, 128, 2, 911, 0, 0), (90_000, 256, 3, 912, 0, 0),
          (50_000, 64, 2, 913, 1, 0), (6_000, 4, 2, 914, 0, 0), (30_000, 64, 1, 915, 0, 4),
          (100_000, 256, 4, 916, 0, 0), (120_000, 512, 5, 917, 0, 0),
          # 4 levels: 240-pixel tiles, 5 levels: 160-pixel tiles -- several
          # tile columns and rows with ragged last ones, narrow widths, an
          # unaligned input, a last row cut short
          (1024 * 700 + 5, 1024, 4, 918, 0, 0), (2048 * 400 + 77, 2048, 5, 919, 0, 0),
          (16 * 3000, 16, 4, 920, 0, 0), (32 * 5000 - 3, 32, 5, 921, 0, 0),
          (480 * 481, 480, 4, 922, 3, 0), (320 * 330 + 1, 320, 5, 923, 0, 0)]


def _route_entries(fr, rows):
    out = []
    for (n, W, L, nonce, ioff, poff) in rows:
        plan = fr.Plan(W, L)
        _, pb, ub = plan.sizes(n)
        base = torch.from_numpy(wl.random_bytes(n + ioff, seed=nonce)).cuda()
        t = base[ioff:]
        ref = (plan, nonce, n, t, torch.full((pb,), 0x5A, dtype=torch.uint8, device="cuda"),
               torch.full((ub,), 0x5A, dtype=torch.uint8, device="cuda"))
        pg = torch.full((pb + poff,), 0x5A, dtype=torch.uint8, device="cuda")[poff:]
        got = (plan, nonce, n, t, pg, torch.full((ub,), 0x5A, dtype=torch.uint8, device="cuda"))
        out.append((ref, got))
    return out


def test_fused_and_tile_routes_alike(fr):
    """The call sends items whose levels all fit the fused pass through it
    and the CTR pass, and the rest through the tile kernel; in one call,
    each route alone and a call of one fused item, every fragment equals
    frag_protect_batch's (which the parity tests hold to the oracle)."""
    key = fr.Key(wl.KEY)
    entries = _route_entries(fr, ROUTES)
    fr.protect_batch([r for r, _ in entries], key)
    torch.cuda.synchronize()
    fr.sync_status()
    for name, idx in (("mixed", range(len(ROUTES))), ("fused only", range(3)),
                      ("tile only", range(3, len(ROUTES))), ("one fused item", [1]),
                      ("one tile item", [9])):
        got = [entries[i][1] for i in idx]
        for (_, _, _, _, p, u) in got:
            p.fill_(0x5A)
            u.fill_(0x5A)
        assert _noalloc(fr, got) == fr.FRAG_OK, fr.last_error()
        assert fr.lib().frag_noalloc_sync_status(
            torch.cuda.current_stream().cuda_stream) == fr.FRAG_OK, fr.last_error()
        for i in idx:
            (plan, _, n, _, p0, u0), (_, _, _, _, p1, u1) = entries[i]
            what = "(n=%d, W=%d, L=%d, row %d) in the %s call" % (n, plan.width, plan.levels, i, name)
            assert torch.equal(p0, p1), "private fragment differs " + what
            assert torch.equal(u0, u1), "public fragment differs " + what


def test_large_call_one_fused_launch_per_level_count(fr):
    """Fused items large enough that each level count fills eight rounds of
    full units on the device (the call then runs one fused launch per count,
    as a batch does): fragments equal frag_protect_batch's."""
    key = fr.Key(wl.KEY)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    W = 4096
    need = 8.8 * sms * 16 * 32 / -(-W // 240)    # fused iterations per level count, with a margin
    rows = int(need * 8 / 4) + 1                  # four buffers a count
    ref, got = [], []
    for L in (3, 1, 2):
        plan = fr.Plan(W, L)
        for k in range(4):
            n = W * (rows + 53 * k) + 777 * k
            nonce = 1000 + 10 * L + k
            t = torch.from_numpy(wl.random_bytes(n, nonce)).cuda()
            _, pb, ub = plan.sizes(n)
            mk = lambda m: torch.full((m,), 0x5A, dtype=torch.uint8, device="cuda")
            ref.append((plan, nonce, n, t, mk(pb), mk(ub)))
            got.append((plan, nonce, n, t, mk(pb), mk(ub)))
    fr.protect_batch(ref, key)
    torch.cuda.synchronize()
    fr.sync_status()
    assert _noalloc(fr, got) == fr.FRAG_OK, fr.last_error()
    assert fr.lib().frag_noalloc_sync_status(
        torch.cuda.current_stream().cuda_stream) == fr.FRAG_OK, fr.last_error()
    for (plan, _, n, _, p0, u0), (_, _, _, _, p1, u1) in zip(ref, got):
        what = "(n=%d, L=%d)" % (n, plan.levels)
        assert torch.equal(p0, p1), "private fragment differs " + what
        assert torch.equal(u0, u1), "public fragment differs " + what
