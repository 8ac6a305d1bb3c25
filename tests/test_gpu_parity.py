"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit-exact
on every private, public and recovered byte.

Integer work, so the bar is exact equality.  Sizes run from single tiles with
ragged tails up to the full workloads (the 256 x 256 matrix, the 3-plane
4096 x 4096 bitmap and the 256 MiB buffer at 2 and 4 levels).
"""
import numpy as np
import pytest

import oracle
from paper_1803_04880_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEY = wl.KEY


@pytest.fixture(scope="module")
def fr():
    import paper_1803_04880_b300 as m
    m.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


@pytest.fixture(scope="module")
def key(fr):
    return fr.Key(KEY)


def gpu_round_trip(fr, key, data, W, L, nonce, offset=0, path=0):
    plan = fr.Plan(W, L)
    plan.set_path(path)
    n = data.size
    _, pb, ub = plan.sizes(n)
    # offset > 0 places every buffer at an odd address
    dev_in = torch.zeros(n + offset, dtype=torch.uint8, device="cuda")
    dev_in[offset:] = torch.from_numpy(np.ascontiguousarray(data).reshape(-1)).cuda()
    priv = torch.full((pb + offset,), 0xAA, dtype=torch.uint8, device="cuda")
    pub = torch.full((ub + offset,), 0xAA, dtype=torch.uint8, device="cuda")
    out = torch.full((n + offset + 64,), 0x55, dtype=torch.uint8, device="cuda")
    fr.protect(plan, key, nonce, dev_in[offset:], n, priv[offset:], pub[offset:])
    fr.recover(plan, key, nonce, priv[offset:], pub[offset:], n, out[offset:offset + n])
    fr.sync_status()
    o = out.cpu().numpy()
    assert (o[offset + n:] == 0x55).all(), "recover wrote past n"
    return priv[offset:].cpu().numpy(), pub[offset:].cpu().numpy(), o[offset:offset + n]


def check_against_oracle(fr, key, data, W, L, nonce=0, offset=0, path=0):
    data = np.ascontiguousarray(data).reshape(-1)
    p_ref, u_ref = oracle.protect(data, W, L, KEY, nonce)
    p, u, r = gpu_round_trip(fr, key, data, W, L, nonce, offset, path)
    assert np.array_equal(p, p_ref), "private fragment differs"
    if not np.array_equal(u, u_ref):
        bad = np.flatnonzero(u != u_ref)
        raise AssertionError("public fragment differs at %d bytes, first %s" % (bad.size, bad[:8]))
    assert np.array_equal(r, data), "recovered bytes differ"


def test_c1_full(fr, key):
    check_against_oracle(fr, key, wl.c1(), 256, 1, 0)


SWEEP = [
    # (n, W, L)
    (1, 2, 1), (2, 2, 1), (5, 4, 2), (64, 8, 2), (1000, 64, 3),
    (4096, 64, 1), (4097, 64, 1), (5000, 16, 4), (12345, 128, 2), (65536 + 17, 256, 3),
    (77777, 256, 5), (100000, 1024, 4), (200000, 96, 2), (300000, 160, 5), (131072, 512, 3),
    (250000, 1000, 3), (262144, 256, 4), (99999, 32, 5), (1 << 20, 2048, 2),
    # around the 224-pixel tile of the register-streaming path
    (224 * 230, 224, 3), (448 * 449 + 3, 448, 2), (240 * 500, 240, 3), (672 * 225 + 100, 672, 1),
    (16 * 1000, 16, 3), (8 * 7, 8, 3), (232 * 232, 232, 3), (456 * 456 - 1, 456, 3),
    (904 * 220, 904, 2),
    # six to eight levels (W a multiple of 2^L, ragged heights and tails)
    (64 * 130 + 5, 64, 6), (128 * 200 - 1, 128, 7), (256 * 300 + 13, 256, 8),
    (1024 * 1024 + 777, 1024, 6), (512 * 600, 512, 7), (2048 * 300 + 1, 2048, 8),
    (768 * 256, 768, 8), (320 * 999, 320, 6),
]


# path 0: fused levels where alignment allows, the private fragment through
# the AES-CTR launch (the default); 1: every level in the dependency-ordered
# kernel; 2: the fused levels with the private fragment enciphered inside the
# fused pass that reaches level L
@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("n,W,L", SWEEP)
def test_sweep_random(fr, key, n, W, L, path):
    data = wl.random_bytes(n, seed=n + W + L)
    check_against_oracle(fr, key, data, W, L, nonce=n % 7, path=path)


# the fused kernel's segment height: from one 8-row iteration per unit (the
# most warm-up per unit) up to long units, at one to three fused levels and
# with levels above them in the level kernel
@pytest.mark.parametrize("seg_rows", [16, 32, 64, 256])
@pytest.mark.parametrize("n,W,L", [(4096 * 200 + 5, 4096, 3), (1000 * 333, 1000, 2),
                                   (2048 * 97, 2048, 1), (512 * 512, 512, 5)])
def test_fused_segments(fr, key, n, W, L, seg_rows):
    data = wl.random_bytes(n, seed=seg_rows + L)
    p_ref, u_ref = oracle.protect(data, W, L, KEY, 11)
    plan = fr.Plan(W, L)
    plan.set_schedule(seg_rows, 0)
    _, pb, ub = plan.sizes(n)
    d = torch.from_numpy(data).cuda()
    priv = torch.empty(pb, dtype=torch.uint8, device="cuda")
    pub = torch.empty(ub, dtype=torch.uint8, device="cuda")
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    fr.protect(plan, key, 11, d, n, priv, pub)
    fr.recover(plan, key, 11, priv, pub, n, out)
    fr.sync_status()
    assert np.array_equal(priv.cpu().numpy(), p_ref)
    assert np.array_equal(pub.cpu().numpy(), u_ref)
    assert torch.equal(out, d)


# the second fused pass (levels 4 to 6 over the level-3 LL): level-3 widths
# from one lane's 8 columns to two strips, LL_3 heights from 2 rows up,
# ragged tails; with 7 and 8 levels the level kernel takes the levels above
# the sixth from the pass's LL_6
PASS2 = [(64 * 16, 64, 4), (64 * 16 * 3 - 7, 64, 4), (128 * 64 + 1, 128, 5), (192 * 128 - 3, 192, 5),
         (512 * 300 + 11, 512, 4), (2048 * 256, 2048, 5), (4096 * 256 + 99, 4096, 4),
         (1024 * 512, 1024, 5), (1984 * 256 - 5, 1984, 5), (8192 * 64, 8192, 5), (64 * 64 - 1, 64, 5),
         (128 * 128, 128, 6), (512 * 512 - 9, 512, 6), (4096 * 200 + 3, 4096, 6), (1984 * 1280, 1984, 6),
         (1024 * 1024, 1024, 7), (2048 * 512 + 5, 2048, 7), (4096 * 256, 4096, 8), (256 * 1024 - 1, 256, 8)]


@pytest.mark.parametrize("seg_rows", [0, 16])
@pytest.mark.parametrize("n,W,L", PASS2)
def test_second_fused_pass(fr, key, n, W, L, seg_rows):
    data = wl.random_bytes(n, seed=n + L)
    p_ref, u_ref = oracle.protect(data, W, L, KEY, 4)
    plan = fr.Plan(W, L)
    plan.set_schedule(seg_rows, 0)
    _, pb, ub = plan.sizes(n)
    d = torch.from_numpy(data).cuda()
    priv = torch.empty(pb, dtype=torch.uint8, device="cuda")
    pub = torch.empty(ub, dtype=torch.uint8, device="cuda")
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    b = fr.Batch([(plan, 4, n, d, priv, pub)], True)
    b.set_timing(True)
    b.run(key)
    assert b.launch_times()["fused_low"][1] == 1  # the case runs the second pass
    fr.recover(plan, key, 4, priv, pub, n, out)
    fr.sync_status()
    assert np.array_equal(priv.cpu().numpy(), p_ref)
    assert np.array_equal(pub.cpu().numpy(), u_ref)
    assert torch.equal(out, d)


def test_path_selects_kernels(fr, key):
    """Three fused levels take the fused launch and the CTR launch; with the
    cipher in the fused pass, one fused launch, except for a private fragment
    the fused recover cannot read with 4-byte words (an odd address), which
    goes through the CTR launch; the level path takes one dependency-ordered
    launch with in-launch cipher units."""
    n, W, L = 4096 * 64, 4096, 3
    plan = fr.Plan(W, L)
    _, pb, ub = plan.sizes(n)
    d = torch.zeros(n, dtype=torch.uint8, device="cuda")
    priv = torch.empty(pb + 1, dtype=torch.uint8, device="cuda")
    pub = torch.empty(ub, dtype=torch.uint8, device="cuda")
    assert plan.path() == fr.Plan.PATH_AUTO
    assert fr.Batch([(plan, 0, n, d, priv[:pb], pub)], True).launches == 2
    plan.set_path(fr.Plan.PATH_FUSED_CIPHER)
    assert plan.path() == fr.Plan.PATH_FUSED_CIPHER
    assert fr.Batch([(plan, 0, n, d, priv[:pb], pub)], True).launches == 1
    assert fr.Batch([(plan, 0, n, priv[:pb], pub, d)], False).launches == 1
    assert fr.Batch([(plan, 0, n, priv[1:], pub, d)], False).launches == 2
    plan.set_path(fr.Plan.PATH_LEVELS)
    assert plan.path() == fr.Plan.PATH_LEVELS
    assert fr.Batch([(plan, 0, n, d, priv[:pb], pub)], True).launches == 1


@pytest.mark.parametrize("L", [3, 4])
def test_batch_launch_times(fr, key, L):
    """The per-kernel event pairs count every launch of the timed runs; with
    four levels the second fused pass (levels 4.. over the level-3 LL) is
    counted as its own kind."""
    n, W = 4096 * 64, 4096
    plan = fr.Plan(W, L)
    _, pb, ub = plan.sizes(n)
    d = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda")
    priv = torch.empty(pb, dtype=torch.uint8, device="cuda")
    pub = torch.empty(ub, dtype=torch.uint8, device="cuda")
    b = fr.Batch([(plan, 0, n, d, priv, pub)], True)
    b.run(key)
    assert b.launch_times() == {"fused": (0.0, 0), "levels": (0.0, 0), "cipher": (0.0, 0),
                                "blocks": (0.0, 0), "fused_low": (0.0, 0)}
    b.set_timing(True)
    for _ in range(3):
        b.run(key)
    t = b.launch_times()
    low = 3 if L > 3 else 0
    assert t["fused"][1] == 3 and t["cipher"][1] == 3 and t["levels"][1] == 0 and t["blocks"][1] == 0
    assert t["fused_low"][1] == low and (t["fused_low"][0] > 0) == (low > 0)
    assert t["fused"][0] > 0 and t["cipher"][0] > 0
    assert b.launch_times()["fused"] == (0.0, 0)  # read once
    fr.sync_status()


@pytest.mark.parametrize("n,W,L", [(12345, 128, 2), (4096, 64, 3), (77777, 256, 5)])
def test_unaligned_buffers(fr, key, n, W, L):
    check_against_oracle(fr, key, wl.random_bytes(n, 5), W, L, nonce=3, offset=1)


@pytest.mark.parametrize("poff", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("n,W,L", [(4096 * 40 + 3, 4096, 1), (2048 * 64 - 7, 2048, 2),
                                   (1024 * 96, 1024, 3), (512 * 512 + 1, 512, 5)])
def test_private_fragment_offsets(fr, key, n, W, L, poff):
    """Only the private fragment moves (to an offset of 1, 2, 4 or 8 bytes):
    with the cipher in the fused pass, that pass enciphers / deciphers it on
    chip when its words are aligned for the pass, the CTR launch takes it
    otherwise; either way every byte equals the oracle's, and a protect by
    one path recovers by the other."""
    data = wl.random_bytes(n, seed=n + poff)
    p_ref, u_ref = oracle.protect(data, W, L, KEY, 6)
    d = torch.from_numpy(data).cuda()
    for pp, rp in ((0, 0), (0, 2), (2, 0)):
        plan_p, plan_r = fr.Plan(W, L), fr.Plan(W, L)
        plan_p.set_path(pp)
        plan_r.set_path(rp)
        _, pb, ub = plan_p.sizes(n)
        pbuf = torch.full((pb + 16,), 0xAA, dtype=torch.uint8, device="cuda")
        priv = pbuf[poff:poff + pb]
        pub = torch.empty(ub, dtype=torch.uint8, device="cuda")
        out = torch.full((n,), 0x55, dtype=torch.uint8, device="cuda")
        fr.protect(plan_p, key, 6, d, n, priv, pub)
        fr.recover(plan_r, key, 6, priv, pub, n, out)
        fr.sync_status()
        assert np.array_equal(priv.cpu().numpy(), p_ref), (pp, rp)
        assert np.array_equal(pub.cpu().numpy(), u_ref), (pp, rp)
        assert torch.equal(out, d), (pp, rp)
        assert (pbuf[:poff] == 0xAA).all() and (pbuf[poff + pb:] == 0xAA).all(), "wrote outside the fragment"


@pytest.mark.parametrize("kind", ["zeros", "ones", "checker", "ramp", "c3mix"])
def test_structured_inputs(fr, key, kind):
    W, L, H = 512, 4, 300
    if kind == "zeros":
        d = np.zeros(W * H, np.uint8)
    elif kind == "ones":
        d = np.full(W * H, 255, np.uint8)
    elif kind == "checker":
        d = (np.add.outer(np.arange(H), np.arange(W)) % 2 * 255).astype(np.uint8).ravel()
    elif kind == "ramp":
        d = (np.add.outer(np.arange(H), np.arange(W)) % 256).astype(np.uint8).ravel()
    else:
        d = wl.c3(total=W * H)
    check_against_oracle(fr, key, d, W, L, nonce=9)


def test_c2_full(fr, key):
    planes = wl.c2()
    for i in range(planes.shape[0]):
        check_against_oracle(fr, key, planes[i], 4096, 3, nonce=i)


@pytest.mark.parametrize("L", [2, 4])
def test_c3_full(fr, key, L):
    data = wl.c3()
    check_against_oracle(fr, key, data, wl.C3_WIDTH, L, nonce=0)


def test_c2_full_level_path(fr, key):
    planes = wl.c2()
    check_against_oracle(fr, key, planes[0], 4096, 3, nonce=0, path=1)


def test_zero_bytes_is_noop(fr, key):
    plan = fr.Plan(64, 2)
    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    fr.protect(plan, key, 0, t, 0, t, t)
    fr.recover(plan, key, 0, t, t, 0, t)
    fr.sync_status()
    assert not t.any()


def test_wrong_key_gives_other_bytes_without_error(fr, key):
    data = wl.random_bytes(50000, 1)
    plan = fr.Plan(256, 2)
    d = torch.from_numpy(data).cuda()
    priv, pub = fr.protect(plan, key, 4, d)
    other = fr.Key(bytes([1]) + KEY[1:])
    out = fr.recover(plan, other, 4, priv, pub, data.size)
    out2 = fr.recover(plan, key, 5, priv, pub, data.size)
    fr.sync_status()
    assert not np.array_equal(out.cpu().numpy(), data)
    assert not np.array_equal(out2.cpu().numpy(), data)


def test_host_buffer_forms(fr, key):
    data = wl.random_bytes(300000, 2)
    plan = fr.Plan(512, 3)
    p, u = fr.protect_host(plan, key, 11, data)
    p_ref, u_ref = oracle.protect(data, 512, 3, KEY, 11)
    assert np.array_equal(p.numpy(), p_ref) and np.array_equal(u.numpy(), u_ref)
    r = fr.recover_host(plan, key, 11, p, u, data.size)
    assert np.array_equal(r.numpy(), data)


# buffers of 16 MiB and more take the banded host form: copies in, kernels
# and copies out of row bands overlap on three streams (bands of about 32
# MiB, at least 8: the 300 MiB case runs 10); at 4..6 levels the bands run
# the first fused pass and the second pass runs whole
@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n,W,L", [((16 << 20) + 12345, 4096, 3), ((20 << 20) - 7, 8192, 2),
                                   ((17 << 20) + 1, 2048, 1), (24 << 20, 1024, 3),
                                   ((18 << 20) + 999, 4000, 2), ((300 << 20) + 77, 8192, 2),
                                   ((20 << 20) + 3, 4096, 4), ((40 << 20) - 5, 8192, 5),
                                   ((24 << 20) + 11, 2048, 6)])
def test_host_forms_in_bands(fr, key, n, W, L, pinned):
    """The banded host forms give the device calls' fragments byte for byte
    and recover every byte (and, on one case, the oracle's fragments)."""
    data = wl.random_bytes(n, seed=n % 1000 + L)
    plan = fr.Plan(W, L)
    _, pb, ub = plan.sizes(n)
    h = torch.from_numpy(data)
    hp = torch.full((pb,), 0xAA, dtype=torch.uint8)
    hu = torch.full((ub,), 0xAA, dtype=torch.uint8)
    ho = torch.full((n,), 0x55, dtype=torch.uint8)
    if pinned:
        h, hp, hu, ho = h.pin_memory(), hp.pin_memory(), hu.pin_memory(), ho.pin_memory()
    fr.protect_host(plan, key, 5, h, hp, hu)
    d = h.cuda()
    dp = torch.empty(pb, dtype=torch.uint8, device="cuda")
    du = torch.empty(ub, dtype=torch.uint8, device="cuda")
    fr.protect(plan, key, 5, d, n, dp, du)
    fr.sync_status()
    assert torch.equal(hp, dp.cpu()), "private fragment differs from the device call"
    assert torch.equal(hu, du.cpu()), "public fragment differs from the device call"
    fr.recover_host(plan, key, 5, hp, hu, n, ho)
    assert torch.equal(ho, h), "recovered bytes differ"
    if n == (16 << 20) + 12345 and pinned:
        p_ref, u_ref = oracle.protect(data, W, L, KEY, 5)
        assert np.array_equal(hp.numpy(), p_ref) and np.array_equal(hu.numpy(), u_ref)


def _mixed_items(count, seed, hi=1 << 18):
    items = wl.c4_items(count=count, lo=64, hi=hi, seed=seed)
    datas = [wl.random_bytes(n, seed=i) for i, (n, _, _, _) in enumerate(items)]
    return items, datas


def test_batch_matches_single_calls_and_oracle(fr, key):
    items, datas = _mixed_items(60, seed=31)
    plans = {}
    ins, privs, pubs, outs, entries, rentries = [], [], [], [], [], []
    for (n, W, L, nonce), d in zip(items, datas):
        plan = plans.setdefault((W, L), fr.Plan(W, L))
        _, pb, ub = plan.sizes(n)
        t = torch.from_numpy(d).cuda()
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(n, dtype=torch.uint8, device="cuda")
        ins.append(t), privs.append(p), pubs.append(u), outs.append(o)
        entries.append((plan, nonce, n, t, p, u))
        rentries.append((plan, nonce, n, p, u, o))
    fr.protect_batch(entries, key)
    fr.recover_batch(rentries, key)
    fr.sync_status()
    for (n, W, L, nonce), d, p, u, o in zip(items, datas, privs, pubs, outs):
        p_ref, u_ref = oracle.protect(d, W, L, KEY, nonce)
        assert np.array_equal(p.cpu().numpy(), p_ref)
        assert np.array_equal(u.cpu().numpy(), u_ref)
        assert np.array_equal(o.cpu().numpy(), d)


def test_batch_of_six_to_eight_levels(fr, key):
    """A batch of buffers at 6, 7 and 8 levels (with buffers of 1..5 levels
    beside them), on both kernel paths, against the oracle."""
    items = [(64 * 130 + 5, 64, 6, 1), (128 * 200 - 1, 128, 7, 2), (256 * 300 + 13, 256, 8, 3),
             (4096 * 64, 4096, 6, 4), (1024 * 512 + 1, 1024, 7, 5), (2048 * 512, 2048, 8, 6),
             (5000, 16, 4, 7), (77777, 256, 5, 8), (12345, 128, 2, 9), (40000, 512, 1, 10)]
    for path in (0, 1):
        plans = {}
        entries, rentries, refs = [], [], []
        for (n, W, L, nonce) in items:
            if (W, L) not in plans:
                plans[(W, L)] = fr.Plan(W, L)
                plans[(W, L)].set_path(path)
            plan = plans[(W, L)]
            d = wl.random_bytes(n, seed=n + 3 * L + path)
            _, pb, ub = plan.sizes(n)
            t = torch.from_numpy(d).cuda()
            p = torch.empty(pb, dtype=torch.uint8, device="cuda")
            u = torch.empty(ub, dtype=torch.uint8, device="cuda")
            o = torch.empty(n, dtype=torch.uint8, device="cuda")
            entries.append((plan, nonce, n, t, p, u))
            rentries.append((plan, nonce, n, p, u, o))
            refs.append((d, W, L, nonce, p, u, o))
        fr.protect_batch(entries, key)
        fr.recover_batch(rentries, key)
        fr.sync_status()
        for d, W, L, nonce, p, u, o in refs:
            p_ref, u_ref = oracle.protect(d, W, L, KEY, nonce)
            assert np.array_equal(p.cpu().numpy(), p_ref), (W, L, path)
            assert np.array_equal(u.cpu().numpy(), u_ref), (W, L, path)
            assert np.array_equal(o.cpu().numpy(), d), (W, L, path)


def test_batch_object_in_cuda_graph(fr, key):
    items, datas = _mixed_items(40, seed=32)
    plans = {}
    entries, rentries, outs, refs = [], [], [], []
    for (n, W, L, nonce), d in zip(items, datas):
        plan = plans.setdefault((W, L), fr.Plan(W, L))
        _, pb, ub = plan.sizes(n)
        t = torch.from_numpy(d).cuda()
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.zeros(n, dtype=torch.uint8, device="cuda")
        entries.append((plan, nonce, n, t, p, u))
        rentries.append((plan, nonce, n, p, u, o))
        outs.append(o)
        refs.append(d)
    bp = fr.Batch(entries, protect=True)
    br = fr.Batch(rentries, protect=False)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bp.run(key)
        br.run(key)
    for _ in range(3):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for o, d in zip(outs, refs):
            assert np.array_equal(o.cpu().numpy(), d)
    fr.sync_status()


def test_lone_buffer_batch_with_box_loads_in_cuda_graph(fr, key):
    """A one-buffer batch whose recover loads its level-1 bands as TMA boxes
    (width 1024, 2 levels; the maps travel in the captured launch's
    parameters), captured once and replayed: every replay recovers the
    bytes, and the fragments are the oracle's."""
    n, W, L, nonce = 1024 * 300 + 77, 1024, 2, 6
    d = wl.random_bytes(n, 41)
    plan = fr.Plan(W, L)
    _, pb, ub = plan.sizes(n)
    t = torch.from_numpy(d).cuda()
    p = torch.empty(pb, dtype=torch.uint8, device="cuda")
    u = torch.empty(ub, dtype=torch.uint8, device="cuda")
    o = torch.zeros(n, dtype=torch.uint8, device="cuda")
    bp = fr.Batch([(plan, nonce, n, t, p, u)], protect=True)
    br = fr.Batch([(plan, nonce, n, p, u, o)], protect=False)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bp.run(key)
        br.run(key)
    p_ref, u_ref = oracle.protect(d, W, L, KEY, nonce)
    for _ in range(3):
        o.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(o.cpu().numpy(), d)
    assert np.array_equal(p.cpu().numpy(), p_ref)
    assert np.array_equal(u.cpu().numpy(), u_ref)
    fr.sync_status()


def test_batch_of_large_private_fragments(fr, key):
    """A batch whose private fragments total about 16 M AES blocks (the CTR
    pass then takes chunks of several times 256 blocks): every fragment
    equals that of a single call on the same buffer (the single call's CTR
    pass is pinned against the oracle at full size), ragged chunk ends
    included, and the batch recovers every byte."""
    specs = [(8192, 1, (64 << 20) + 12345), (8192, 1, 64 << 20), (4096, 2, (48 << 20) - 7),
             (8192, 1, (64 << 20) - 4096 * 3), (256, 1, 1000)]
    entries, rentries, singles, outs, ins = [], [], [], [], []
    for i, (W, L, n) in enumerate(specs):
        plan = fr.Plan(W, L)
        g = torch.Generator(device="cuda").manual_seed(40 + i)
        t = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g)
        _, pb, ub = plan.sizes(n)
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(n, dtype=torch.uint8, device="cuda")
        entries.append((plan, 500 + i, n, t, p, u))
        rentries.append((plan, 500 + i, n, p, u, o))
        singles.append((plan, 500 + i, t))
        outs.append(o)
        ins.append(t)
    fr.protect_batch(entries, key)
    fr.recover_batch(rentries, key)
    fr.sync_status()
    for (plan, nonce, t), (_, _, _, _, p, u), o in zip(singles, entries, outs):
        p1, u1 = fr.protect(plan, key, nonce, t)
        fr.sync_status()
        assert torch.equal(p, p1), "private fragment differs from the single call"
        assert torch.equal(u, u1), "public fragment differs from the single call"
        assert torch.equal(o, t), "recovered bytes differ"
    # the small buffer against the oracle as well
    plan, nonce, t = singles[-1]
    p_ref, u_ref = oracle.protect(t.cpu().numpy(), 256, 1, KEY, nonce)
    assert np.array_equal(entries[-1][4].cpu().numpy(), p_ref)


# The recover of a lone buffer of 1-2 levels whose width is a multiple of 16
# and at least 272 loads its level-1 bands as TMA boxes (4 rows x 136 int16,
# starting 4 columns left of a strip's first lane): the narrowest such width
# (two boxes' worth), a last strip much shorter than the others, two or three
# level-1 row pairs, rows cut short by the end of the data, and two shapes
# whose band bases miss the 16-byte boundary (272 x 12 and 2064 x 20 rows at
# two levels), which fall back to per-lane copies.
BOX_CASES = [(272 * 8, 272, 1), (288 * 40 + 17, 288, 1), (1040 * 40, 1040, 2), (1040 * 37, 1040, 2),
             (4112 * 64 - 3, 4112, 2), (496 * 24, 496, 2), (2048 * 8, 2048, 1), (272 * 9 + 5, 272, 2),
             (2064 * 16 + 1, 2064, 2)]


@pytest.mark.parametrize("path", [0, 2])
@pytest.mark.parametrize("n,W,L", BOX_CASES)
def test_level1_box_loads(fr, key, n, W, L, path):
    data = wl.random_bytes(n, seed=3 * n + W)
    check_against_oracle(fr, key, data, W, L, nonce=n % 5, path=path)
