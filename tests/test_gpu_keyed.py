"""GPU parity of the keyed protection of the packed public fragments
(Sec. 5.2.1: SHA-256 of a block's private fragment and the key masks its
first public and protected fragment, SHA-512 of that protected fragment and
the key its second) against the oracle: every byte of A and B' || C' and
every recovered byte, bit-exact; odd block rows, a partial warp strip,
ragged tails, unaligned buffers; a batch that mixes keyed, plain packed and
whole-matrix buffers; and, at the 4096 x 4096 bitmap plane the benchmark
times, sampled blocks checked one by one."""
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


def _keyed_plan(fr, W):
    plan = fr.Plan(W, 2)
    plan.set_block(8)
    plan.set_packed(True)
    plan.set_protect_public(True)
    return plan


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("W,n", [(64, 64 * 16), (72, 72 * 24 - 5), (264, 264 * 40 - 3),
                                 (8, 8 * 8 * 5), (4096, 4096 * 16 + 11), (512, 512 * 40)])
def test_matches_oracle(fr, key, W, n, offset):
    data = wl.random_bytes(n, seed=W + n + 1)
    nonce = 0x1122334455667700 + W
    a_ref, pub_ref = oracle.protect_keyed(data, W, KEY, nonce)
    plan = _keyed_plan(fr, W)
    _, pb, ub = plan.sizes(n)
    assert (pb, ub) == (a_ref.size, pub_ref.size)
    src = torch.zeros(n + offset, dtype=torch.uint8, device="cuda")
    src[offset:] = torch.from_numpy(data).cuda()
    priv = torch.full((pb + offset,), 0xAA, dtype=torch.uint8, device="cuda")
    pub = torch.full((ub + offset,), 0xAA, dtype=torch.uint8, device="cuda")
    out = torch.full((n + offset + 16,), 0x55, dtype=torch.uint8, device="cuda")
    fr.protect(plan, key, nonce, src[offset:], n, priv[offset:], pub[offset:])
    fr.recover(plan, key, nonce, priv[offset:], pub[offset:], n, out[offset:offset + n])
    fr.sync_status()
    assert np.array_equal(priv[offset:].cpu().numpy(), a_ref), "private fragment A differs"
    got = pub[offset:].cpu().numpy()
    if not np.array_equal(got, pub_ref):
        bad = np.flatnonzero(got != pub_ref)
        raise AssertionError("public fragment differs at %d bytes, first %s" % (bad.size, bad[:8]))
    o = out.cpu().numpy()
    assert np.array_equal(o[offset:offset + n], data), "recovered bytes differ"
    assert (o[offset + n:] == 0x55).all(), "recover wrote past n"


def test_oracle_fragments_recover_on_the_gpu(fr, key):
    """Recover alone, from the oracle's fragments."""
    W, n = 136, 136 * 32 - 9
    data = wl.random_bytes(n, seed=21)
    a_ref, pub_ref = oracle.protect_keyed(data, W, KEY, 9)
    plan = _keyed_plan(fr, W)
    out = fr.recover(plan, key, 9, torch.from_numpy(a_ref).cuda(), torch.from_numpy(pub_ref).cuda(), n)
    fr.sync_status()
    assert np.array_equal(out.cpu().numpy(), data)


def test_wrong_key_does_not_recover(fr, key):
    W, n = 64, 64 * 16
    data = wl.random_bytes(n, seed=22)
    plan = _keyed_plan(fr, W)
    d = torch.from_numpy(data).cuda()
    priv, pub = fr.protect(plan, key, 3, d)
    other = fr.Key(bytes([KEY[0] ^ 0x80]) + KEY[1:])
    out = fr.recover(plan, other, 3, priv, pub, n)
    torch.cuda.synchronize()
    assert not torch.equal(out, d)


def test_batch_mixes_keyed_packed_and_whole_matrix(fr, key):
    specs = [("keyed", 64, 64 * 40 - 7), ("packed", 4096, 4096 * 8), ("keyed", 4096, 4096 * 16 + 5),
             ("whole", 256, 256 * 50 + 1), ("keyed", 72, 72 * 8)]
    ents, rents, refs = [], [], []
    for i, (kind, W, n) in enumerate(specs):
        data = wl.random_bytes(n, seed=200 + i)
        plan = fr.Plan(W, 2)
        nonce = 1000 + i
        if kind != "whole":
            plan.set_block(8)
            plan.set_packed(True)
        if kind == "keyed":
            plan.set_protect_public(True)
            ref = oracle.protect_keyed(data, W, KEY, nonce)
        elif kind == "packed":
            ref = oracle.protect_packed(data, W, KEY, nonce)
        else:
            ref = oracle.protect(data, W, 2, KEY, nonce)
        _, pb, ub = plan.sizes(n)
        d = torch.from_numpy(data).cuda()
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(n, dtype=torch.uint8, device="cuda")
        ents.append((plan, nonce, n, d, p, u))
        rents.append((plan, nonce, n, p, u, o))
        refs.append((data, ref, p, u, o))
    fr.protect_batch(ents, key)
    fr.recover_batch(rents, key)
    fr.sync_status()
    for data, (p_ref, u_ref), p, u, o in refs:
        assert np.array_equal(p.cpu().numpy(), p_ref)
        assert np.array_equal(u.cpu().numpy(), u_ref)
        assert np.array_equal(o.cpu().numpy(), data)


def test_full_plane_sampled_blocks(fr, key):
    """The 4096 x 4096 bitmap plane of the benchmark, through the batch call
    it times: 256 sampled blocks (the corners, the edges, random ones) each
    checked against the oracle from its 64 bytes, and the whole round trip."""
    plane = wl.c2(planes=1)[0]
    W = plane.shape[1]
    data = plane.reshape(-1)
    nonce = 0xABCDEF
    plan = _keyed_plan(fr, W)
    d = torch.from_numpy(data).cuda()
    _, pb, ub = plan.sizes(data.size)
    p = torch.empty(pb, dtype=torch.uint8, device="cuda")
    u = torch.empty(ub, dtype=torch.uint8, device="cuda")
    o = torch.empty(data.size, dtype=torch.uint8, device="cuda")
    fr.protect_batch([(plan, nonce, data.size, d, p, u)], key)
    fr.recover_batch([(plan, nonce, data.size, p, u, o)], key)
    fr.sync_status()
    assert torch.equal(o, d)
    a = p.cpu().numpy()
    pub = u.cpu().numpy()
    _, sa, sb, sc = oracle.packed_sizes(data.size, W)
    nbx, nby = W // 8, plane.shape[0] // 8
    brow = (124 * nbx + 7) // 8
    rng = np.random.default_rng(0)
    picks = {0, nbx - 1, nbx * (nby - 1), nbx * nby - 1, 31, 32, 33, nbx + 31}
    picks |= set(rng.integers(0, nbx * nby, 256 - len(picks)).tolist())
    for idx in sorted(picks):
        bi, bj = divmod(idx, nbx)
        want = oracle.keyed_block_records(plane[8 * bi:8 * bi + 8, 8 * bj:8 * bj + 8], KEY, nonce, idx)
        # A: decipher the 16-byte CTR blocks that cover its 5 bytes
        c0 = (5 * idx) // 16
        c1 = (5 * idx + 4) // 16
        plain = oracle.aes128_ctr_xor(KEY, nonce, c0, a[16 * c0:16 * (c1 + 1)].tobytes())
        got_a = plain[5 * idx - 16 * c0:5 * idx - 16 * c0 + 5]
        row = int.from_bytes(pub[bi * brow:(bi + 1) * brow].tobytes(), "little")
        got_b = (row >> (124 * bj)) & ((1 << 124) - 1)
        got_c = int.from_bytes(pub[sb + 60 * idx:sb + 60 * idx + 60].tobytes(), "little")
        assert (got_a, got_b, got_c) == want, "block %d" % idx


def test_host_buffer_forms(fr, key):
    """frag_protect_host / frag_recover_host on a keyed plan: host buffers in
    and out, the same fragments as the oracle."""
    W, n = 200, 200 * 48 + 17
    data = wl.random_bytes(n, seed=23)
    plan = _keyed_plan(fr, W)
    p, u = fr.protect_host(plan, key, 77, data)
    a_ref, pub_ref = oracle.protect_keyed(data, W, KEY, 77)
    assert np.array_equal(p.numpy(), a_ref)
    assert np.array_equal(u.numpy(), pub_ref)
    out = fr.recover_host(plan, key, 77, p, u, n)
    assert np.array_equal(out.numpy(), data)


def test_resident_batch_object(fr, key):
    """A keyed plan in a resident batch (frag_batch_create_*), run twice."""
    W = 64
    datas = [wl.random_bytes(64 * 24 + i * 64, seed=30 + i) for i in range(3)]
    plan = _keyed_plan(fr, W)
    ents, rents, refs = [], [], []
    for i, d in enumerate(datas):
        _, pb, ub = plan.sizes(d.size)
        t = torch.from_numpy(d).cuda()
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(d.size, dtype=torch.uint8, device="cuda")
        ents.append((plan, 40 + i, d.size, t, p, u))
        rents.append((plan, 40 + i, d.size, p, u, o))
        refs.append((d, oracle.protect_keyed(d, W, KEY, 40 + i), p, u, o))
    bp = fr.Batch(ents, protect=True)
    br = fr.Batch(rents, protect=False)
    for _ in range(2):
        for _, _, _, _, o in refs:
            o.zero_()
        bp.run(key)
        br.run(key)
        fr.sync_status()
        for d, (a_ref, pub_ref), p, u, o in refs:
            assert np.array_equal(p.cpu().numpy(), a_ref)
            assert np.array_equal(u.cpu().numpy(), pub_ref)
            assert np.array_equal(o.cpu().numpy(), d)
