"""GPU parity of the packed three fragments (Sec. 5.2.1 / Sec. 5.2.3: 8 x 8
blocks at two levels, 40 / 124 / 480 bits a block) against the oracle,
bit-exact on every byte of the private fragment A and of the public
fragment B || C, and on every recovered byte; block rows of an odd number
of blocks (B rows padded to a byte), a warp strip of fewer than 32 blocks,
ragged tails and unaligned buffers."""
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


def _packed_plan(fr, W):
    plan = fr.Plan(W, 2)
    plan.set_block(8)
    plan.set_packed(True)
    return plan


@pytest.mark.parametrize("offset", [0, 1, 4])
@pytest.mark.parametrize("W,n", [(64, 64 * 16), (72, 72 * 24 - 5), (264, 264 * 40 - 3),
                                 (8, 8 * 8 * 5), (4096, 4096 * 64 + 11), (512, 512 * 100)])
def test_matches_oracle(fr, key, W, n, offset):
    data = wl.random_bytes(n, seed=W + n)
    nonce = W + 3
    a_ref, pub_ref = oracle.protect_packed(data, W, KEY, nonce)
    plan = _packed_plan(fr, W)
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


def test_extremes_round_trip(fr, key):
    # blocks that drive coefficients to the thesis's bounds, and flat / checker
    Wt = np.zeros((8, 8, 8, 8))
    for i in range(8):
        for j in range(8):
            X = np.zeros((8, 8), dtype=np.int64)
            X[i, j] = 4096
            Wt[:, :, i, j] = oracle.dwt53_fwd_2d(X, 2) / 4096.0
    blocks = [np.where(s * Wt[r, c] >= 0, 255, 0).astype(np.uint8)
              for r in range(8) for c in range(8) for s in (1, -1)]
    blocks += [np.zeros((8, 8), np.uint8), np.full((8, 8), 255, np.uint8),
               (np.add.outer(np.arange(8), np.arange(8)) % 2 * 255).astype(np.uint8)]
    blocks += [blocks[0]] * (136 - len(blocks))
    img = np.concatenate(blocks, axis=1)
    data = img.reshape(-1)
    W = img.shape[1]
    plan = _packed_plan(fr, W)
    a_ref, pub_ref = oracle.protect_packed(data, W, KEY, 5)
    d = torch.from_numpy(data).cuda()
    priv, pub = fr.protect(plan, key, 5, d)
    out = fr.recover(plan, key, 5, priv, pub, data.size)
    fr.sync_status()  # no coefficient outside its width
    assert np.array_equal(priv.cpu().numpy(), a_ref)
    assert np.array_equal(pub.cpu().numpy(), pub_ref)
    assert torch.equal(out, d)


def test_batch_mixes_packed_block_and_whole_matrix(fr, key):
    """One batch per direction over packed, unpacked block-mode and
    whole-matrix buffers: every fragment as the oracle's."""
    specs = [("packed", 64, 64 * 40 - 7), ("packed", 4096, 4096 * 24), ("block", 64, 64 * 16 + 3),
             ("whole", 256, 256 * 50 + 1), ("packed", 72, 72 * 8)]
    ents, rents, refs, outs = [], [], [], []
    for i, (kind, W, n) in enumerate(specs):
        data = wl.random_bytes(n, seed=100 + i)
        plan = fr.Plan(W, 2)
        if kind != "whole":
            plan.set_block(8)
        if kind == "packed":
            plan.set_packed(True)
            ref = oracle.protect_packed(data, W, KEY, i)
        else:
            ref = oracle.protect(data, W, 2, KEY, i, block=8 if kind == "block" else 0)
        _, pb, ub = plan.sizes(n)
        d = torch.from_numpy(data).cuda()
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(n, dtype=torch.uint8, device="cuda")
        ents.append((plan, i, n, d, p, u))
        rents.append((plan, i, n, p, u, o))
        refs.append((data, ref, p, u, o))
    fr.protect_batch(ents, key)
    fr.recover_batch(rents, key)
    fr.sync_status()
    for data, (p_ref, u_ref), p, u, o in refs:
        assert np.array_equal(p.cpu().numpy(), p_ref)
        assert np.array_equal(u.cpu().numpy(), u_ref)
        assert np.array_equal(o.cpu().numpy(), data)


def test_batch_with_more_units_than_warps(fr, key):
    """Packed buffers whose units (32 blocks each) outnumber the launch's
    warps, so warps take several units across buffer boundaries (the loops'
    per-warp buffer cursor advances and is reused): every fragment and every
    recovered byte as the oracle's."""
    specs = [(4096, 4096 * 1024), (2048, 2048 * 2048 - 5), (1024, 1024 * 512 + 3), (4096, 4096 * 512)]
    ents, rents, refs = [], [], []
    for i, (W, n) in enumerate(specs):
        data = wl.random_bytes(n, seed=300 + i)
        plan = fr.Plan(W, 2)
        plan.set_block(8)
        plan.set_packed(True)
        ref = oracle.protect_packed(data, W, KEY, 40 + i)
        _, pb, ub = plan.sizes(n)
        d = torch.from_numpy(data).cuda()
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(n, dtype=torch.uint8, device="cuda")
        ents.append((plan, 40 + i, n, d, p, u))
        rents.append((plan, 40 + i, n, p, u, o))
        refs.append((data, ref, p, u, o))
    units = sum((W // 8 + 31) // 32 * ((n + W - 1) // W + 7) // 8 for W, n in specs)
    assert units > 148 * 6 * 4  # more than the warps of any packed launch
    fr.protect_batch(ents, key)
    fr.recover_batch(rents, key)
    fr.sync_status()
    for data, (p_ref, u_ref), p, u, o in refs:
        assert np.array_equal(p.cpu().numpy(), p_ref)
        assert np.array_equal(u.cpu().numpy(), u_ref)
        assert np.array_equal(o.cpu().numpy(), data)
