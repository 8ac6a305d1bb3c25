"""GPU parity of the block mode (every 8 x 8 block transformed on its own,
Sec. 5.2.1) against the oracle's block mode, bit-exact on every private,
public and recovered byte: widths that fill a warp's 32 blocks and ones that
leave most lanes idle, 1 to 3 levels, ragged lengths, odd addresses (the
byte-wise path), and batches that mix block and whole-matrix plans."""
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


def _plan(fr, W, L):
    p = fr.Plan(W, L)
    p.set_block(8)
    return p


@pytest.mark.parametrize("n,W,L", [
    (64, 8, 1), (64, 8, 3), (8 * 8 * 5 + 3, 8, 2), (256 * 8, 256, 2), (256 * 40 - 1, 256, 3),
    (264 * 31 + 5, 264, 1), (4096 * 4096, 4096, 2), (2048 * 333 + 17, 2048, 3), (40 * 1000, 40, 2)])
def test_block_mode_matches_oracle(fr, key, n, W, L):
    data = wl.random_bytes(n, seed=n + W)
    p_ref, u_ref = oracle.protect(data, W, L, KEY, 7, block=8)
    plan = _plan(fr, W, L)
    _, pb, ub = plan.sizes(n)
    assert (pb, ub) == (p_ref.size, u_ref.size)
    d = torch.from_numpy(data).cuda()
    priv = torch.empty(pb, dtype=torch.uint8, device="cuda")
    pub = torch.empty(ub, dtype=torch.uint8, device="cuda")
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    fr.protect(plan, key, 7, d, n, priv, pub)
    fr.recover(plan, key, 7, priv, pub, n, out)
    fr.sync_status()
    assert np.array_equal(priv.cpu().numpy(), p_ref)
    assert np.array_equal(pub.cpu().numpy(), u_ref)
    assert torch.equal(out, d)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_block_mode_odd_addresses(fr, key, L):
    n, W = 512 * 37 + 9, 512
    data = wl.random_bytes(n, seed=L)
    p_ref, u_ref = oracle.protect(data, W, L, KEY, 3, block=8)
    plan = _plan(fr, W, L)
    _, pb, ub = plan.sizes(n)
    din = torch.zeros(n + 1, dtype=torch.uint8, device="cuda")
    din[1:] = torch.from_numpy(data).cuda()
    priv = torch.zeros(pb + 1, dtype=torch.uint8, device="cuda")
    pub = torch.zeros(ub + 1, dtype=torch.uint8, device="cuda")
    out = torch.full((n + 1 + 16,), 0x55, dtype=torch.uint8, device="cuda")
    fr.protect(plan, key, 3, din[1:], n, priv[1:], pub[1:])
    fr.recover(plan, key, 3, priv[1:], pub[1:], n, out[1:1 + n])
    fr.sync_status()
    assert np.array_equal(priv[1:].cpu().numpy(), p_ref)
    assert np.array_equal(pub[1:].cpu().numpy(), u_ref)
    assert np.array_equal(out[1:1 + n].cpu().numpy(), data)
    assert (out[1 + n:].cpu().numpy() == 0x55).all()


def test_batch_mixes_block_and_whole_plans(fr, key):
    rng = np.random.default_rng(5)
    items, ritems, refs = [], [], []
    for i in range(8):
        W = int(rng.choice([64, 256, 1024]))
        L = int(rng.integers(1, 4))
        block = i % 2 == 0
        n = int(rng.integers(1, 40)) * W + int(rng.integers(0, W))
        plan = fr.Plan(W, L)
        if block:
            plan.set_block(8)
        data = wl.random_bytes(n, seed=100 + i)
        refs.append((data, oracle.protect(data, W, L, KEY, i, block=8 if block else 0)))
        _, pb, ub = plan.sizes(n)
        d = torch.from_numpy(data).cuda()
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(n, dtype=torch.uint8, device="cuda")
        items.append((plan, i, n, d, p, u))
        ritems.append((plan, i, n, p, u, o))
    fr.protect_batch(items, key)
    fr.recover_batch(ritems, key)
    fr.sync_status()
    for (data, (pr, ur)), it, rit in zip(refs, items, ritems):
        assert np.array_equal(it[4].cpu().numpy(), pr)
        assert np.array_equal(it[5].cpu().numpy(), ur)
        assert np.array_equal(rit[5].cpu().numpy(), data)
    b = fr.Batch(items, True)
    assert b.launches == 3  # fused, block, CTR


def test_block_batch_with_more_units_than_warps(fr, key):
    """Block-mode buffers at 1..3 levels whose units (32 blocks each)
    outnumber the launch's warps, so warps take several units across buffer
    boundaries (the per-warp buffer cursor advances and is reused), one of
    them at an odd address (the byte-wise path): every fragment and every
    recovered byte as the oracle's."""
    specs = [(4096, 1024, 2, 0), (2048, 2048, 3, 0), (1024, 512, 1, 1), (4096, 512, 2, 0)]
    items, ritems, refs = [], [], []
    for i, (W, rows, L, off) in enumerate(specs):
        n = W * rows - 7 * i
        plan = fr.Plan(W, L)
        plan.set_block(8)
        data = wl.random_bytes(n, seed=400 + i)
        refs.append((data, oracle.protect(data, W, L, KEY, 50 + i, block=8)))
        _, pb, ub = plan.sizes(n)
        d = torch.zeros(n + off, dtype=torch.uint8, device="cuda")
        d[off:] = torch.from_numpy(data).cuda()
        p = torch.empty(pb, dtype=torch.uint8, device="cuda")
        u = torch.empty(ub, dtype=torch.uint8, device="cuda")
        o = torch.empty(n, dtype=torch.uint8, device="cuda")
        items.append((plan, 50 + i, n, d[off:], p, u))
        ritems.append((plan, 50 + i, n, p, u, o))
    assert sum(W // 8 // 32 * rows // 8 for W, rows, _, _ in specs) > 148 * 8 * 4
    fr.protect_batch(items, key)
    fr.recover_batch(ritems, key)
    fr.sync_status()
    for (data, (pr, ur)), it, rit in zip(refs, items, ritems):
        assert np.array_equal(it[4].cpu().numpy(), pr)
        assert np.array_equal(it[5].cpu().numpy(), ur)
        assert np.array_equal(rit[5].cpu().numpy(), data)
