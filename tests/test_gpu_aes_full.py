"""GPU parity of the full-buffer AES-128-CTR call (the thesis's full-encryption
comparator, Sec. 5.4) against the oracle's AES-CTR, which FIPS-197 and
SP 800-38A vectors pin: bit-exact on every byte, at sizes with ragged last
blocks, unaligned buffers, in place, and as its own inverse."""
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


@pytest.mark.parametrize("offset", [0, 1, 7])
@pytest.mark.parametrize("n", [1, 15, 16, 17, 4095, 65536 + 7, 3 << 20])
def test_matches_oracle(fr, key, n, offset):
    data = wl.random_bytes(n, seed=n + offset)
    nonce = (n * 2654435761) & 0xFFFFFFFFFFFF
    want = np.frombuffer(oracle.aes128_ctr_xor(KEY, nonce, 0, data.tobytes()), dtype=np.uint8)
    src = torch.zeros(n + offset, dtype=torch.uint8, device="cuda")
    src[offset:] = torch.from_numpy(data).cuda()
    dst = torch.full((n + offset + 32,), 0x5A, dtype=torch.uint8, device="cuda")
    fr.aes_ctr(key, nonce, src[offset:], dst[offset:offset + n])
    fr.sync_status()
    got = dst.cpu().numpy()
    assert np.array_equal(got[offset:offset + n], want)
    assert (got[:offset] == 0x5A).all() and (got[offset + n:] == 0x5A).all(), "wrote outside the buffer"


def test_argument_checks(fr, key):
    L = fr.lib()
    assert L.frag_aes128_ctr(key.handle, 0, None, None, 16, None) == fr.FRAG_EINVAL
    assert L.frag_aes128_ctr(key.handle, 0, None, None, 0, None) == fr.FRAG_OK


def test_in_place_and_self_inverse(fr, key):
    n = (1 << 20) + 5
    data = wl.random_bytes(n, seed=3)
    t = torch.from_numpy(data).cuda()
    fr.aes_ctr(key, 9, t, t)
    want = np.frombuffer(oracle.aes128_ctr_xor(KEY, 9, 0, data.tobytes()), dtype=np.uint8)
    assert np.array_equal(t.cpu().numpy(), want)
    fr.aes_ctr(key, 9, t, t)
    fr.sync_status()
    assert np.array_equal(t.cpu().numpy(), data)


def test_private_fragment_is_this_cipher(fr, key):
    """The private fragment of a protect is LL_L (int16) under the same
    keystream: deciphering it with the full-buffer call gives the oracle's
    plaintext LL_L."""
    n, W, L, nonce = 4096 * 64, 4096, 3, 21
    data = wl.random_bytes(n, seed=5)
    plan = fr.Plan(W, L)
    _, pb, ub = plan.sizes(n)
    priv = torch.empty(pb, dtype=torch.uint8, device="cuda")
    pub = torch.empty(ub, dtype=torch.uint8, device="cuda")
    fr.protect(plan, key, nonce, torch.from_numpy(data).cuda(), n, priv, pub)
    plain = fr.aes_ctr(key, nonce, priv)
    fr.sync_status()
    p_ref, _ = oracle.protect(data, W, L, KEY, nonce)
    want = oracle.aes128_ctr_xor(KEY, nonce, 0, p_ref.tobytes())
    assert plain.cpu().numpy().tobytes() == want


# -- the bitsliced form (the measured alternative): the same bytes ----------

@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("n", [1, 16, 17, 4095, 16 * 1024 * 3 + 5, 3 << 20])
def test_bitsliced_matches_oracle(fr, key, n, offset):
    """Every byte against the oracle's CTR: ragged last blocks, a partial last
    warp chunk (1,024 blocks), unaligned buffers (the byte path), nothing
    written outside."""
    data = wl.random_bytes(n, seed=7 * n + offset)
    nonce = 0xF1E2D3C4B5A69788 ^ n  # every nonce byte nonzero and varied
    want = np.frombuffer(oracle.aes128_ctr_xor(KEY, nonce, 0, data.tobytes()), dtype=np.uint8)
    src = torch.zeros(n + offset, dtype=torch.uint8, device="cuda")
    src[offset:] = torch.from_numpy(data).cuda()
    dst = torch.full((n + offset + 32,), 0x5A, dtype=torch.uint8, device="cuda")
    fr.aes_ctr_bitsliced(key, nonce, src[offset:], dst[offset:offset + n])
    fr.sync_status()
    got = dst.cpu().numpy()
    assert np.array_equal(got[offset:offset + n], want)
    assert (got[:offset] == 0x5A).all() and (got[offset + n:] == 0x5A).all(), "wrote outside the buffer"


def test_bitsliced_equals_table_form_far_counters(fr, key):
    """Block indices past 2^10 and 2^20 (the chunk's own counter bits) on a
    buffer of 48 MiB: both forms give the same bytes, and sampled blocks equal
    the oracle's."""
    n = 48 << 20
    t = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda")
    a = fr.aes_ctr(key, 77, t)
    b = fr.aes_ctr_bitsliced(key, 77, t)
    fr.sync_status()
    assert torch.equal(a, b)
    host = t.cpu().numpy()
    for blk in (0, 1023, 1024, (1 << 20) - 1, 1 << 20, (n >> 4) - 1):
        o = 16 * blk
        want = oracle.aes128_ctr_xor(KEY, 77, blk, host[o:o + 16].tobytes())
        assert b[o:o + 16].cpu().numpy().tobytes() == want


def test_bitsliced_argument_checks(fr, key):
    L = fr.lib()
    assert L.frag_aes128_ctr_bitsliced(key.handle, 0, None, None, 16, None) == fr.FRAG_EINVAL
    assert L.frag_aes128_ctr_bitsliced(key.handle, 0, None, None, 0, None) == fr.FRAG_OK
    assert L.frag_aes128_ctr_bitsliced(None, 0, None, None, 16, None) == fr.FRAG_EINVAL
