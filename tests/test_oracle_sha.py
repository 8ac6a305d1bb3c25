"""Pins of the oracle's keyed protection of the public fragments (Sec. 5.2.1:
SHA-256 of the private fragment and the key protects the first public and
protected fragment, SHA-512 of that protected fragment and the key the
second; Sec. 5.3.5: a counter among the hash inputs makes identical blocks
protect differently; Sec. 5.3.7: an error stays inside its block).

SHA-2 is pinned against FIPS 180-4's published "abc" example and against
Python's hashlib over every padding case.  The framing of the hash inputs
(key, nonce, block index, record) is a reading; the tests restate it with
hashlib on sampled blocks, so a wrong operand (B instead of B', the wrong
block's A) or a wrong bit order fails, and check the properties the thesis
gives the scheme: the exact inverse, key sensitivity, identical blocks
protected differently, and errors that stay in their block."""
import hashlib

import numpy as np
import pytest

import oracle
from conftest import read_golden
from oracle import sha2

KEY = bytes(range(16))
NONCE = 0x0123456789ABCDEF


def test_sha2_published_example():
    for alg, msg, digest in read_golden("sha2_vectors.txt"):
        f = sha2.sha256 if alg == "sha256" else sha2.sha512
        assert f(bytes.fromhex(msg)).hex() == digest


@pytest.mark.parametrize("n", list(range(0, 140)) + [183, 239, 240, 255, 256, 1000])
def test_sha2_matches_hashlib_every_padding_case(n):
    msg = np.random.default_rng(n).integers(0, 256, n, dtype=np.uint8).tobytes()
    assert sha2.sha256(msg) == hashlib.sha256(msg).digest()
    assert sha2.sha512(msg) == hashlib.sha512(msg).digest()


def test_sha2_constants_are_the_root_fractions():
    # 2 ** (1/2) = 1.6a09e667f3bcc908b2f..., 2 ** (1/3) = 1.428a2f98d728ae22...
    assert sha2.H512[0] == 0x6A09E667F3BCC908 and sha2.H256[0] == sha2.H512[0] >> 32
    assert sha2.K512[0] == 0x428A2F98D728AE22 and sha2.K256[0] == sha2.K512[0] >> 32
    assert all(k >> 32 == k32 for k, k32 in zip(sha2.K512, sha2.K256))
    assert len(set(sha2.K512)) == 80


def _records(width, n, a_plain, pub):
    """(A bytes, B int, C int) per block, read with a bit reader of our own."""
    H, sa, sb, sc = oracle.packed_sizes(n, width)
    nbx, nby = width // 8, H // 8
    brow = (124 * nbx + 7) // 8
    out = {}
    for bi in range(nby):
        row = int.from_bytes(bytes(pub[bi * brow:(bi + 1) * brow]), "little")
        for bj in range(nbx):
            idx = bi * nbx + bj
            b = (row >> (124 * bj)) & ((1 << 124) - 1)
            c = int.from_bytes(bytes(pub[sb + 60 * idx:sb + 60 * idx + 60]), "little")
            out[idx] = (bytes(a_plain[5 * idx:5 * idx + 5]), b, c)
    return out


def _case(width=72, rows=40, seed=3):
    x = np.random.default_rng(seed).integers(0, 256, width * rows - 5, dtype=np.uint8)
    return x, width


def test_keyed_framing_restated_with_hashlib():
    """Sec. 5.2.1 fixes which fragment feeds which hash: the first public
    fragment is protected with SHA-256 of the private fragment and the key,
    the second with SHA-512 of the first *protected* public fragment and the
    key.  Those choices are pinned here (and the two slips that would keep
    every round trip working -- hashing B instead of B', or reading the
    digest's bits in the other order -- are shown to fail); the byte layout
    of the hash inputs (key, nonce, block index, record) is this
    implementation's reading and stays unpinned by the thesis."""
    x, W = _case()
    a, pub = oracle.protect_keyed(x, W, KEY, NONCE)
    a0, pub0 = oracle.protect_packed(x, W, KEY, NONCE)
    assert np.array_equal(a, a0)  # the private fragment is untouched
    plain_a = oracle.aes128_ctr_xor(KEY, NONCE, 0, a)
    keyed = _records(W, x.size, plain_a, pub)
    plain = _records(W, x.size, plain_a, pub0)
    for idx in (0, 1, 8, 9, 17, len(plain) - 1):
        prefix = KEY + NONCE.to_bytes(8, "big") + idx.to_bytes(8, "big")
        a_rec, b, c = plain[idx]
        h1 = int.from_bytes(hashlib.sha256(prefix + a_rec).digest(), "little") & ((1 << 124) - 1)
        b_prot = b ^ h1
        assert keyed[idx][1] == b_prot
        h2 = int.from_bytes(hashlib.sha512(prefix + b_prot.to_bytes(16, "little")).digest(),
                            "little") & ((1 << 480) - 1)
        assert keyed[idx][2] == c ^ h2
        # SHA-512 over the plain B (not B') would give other bits
        h2_plain = int.from_bytes(hashlib.sha512(prefix + b.to_bytes(16, "little")).digest(),
                                  "little") & ((1 << 480) - 1)
        assert keyed[idx][2] != c ^ h2_plain
        # the digest read big-endian (its bits in the other order) would too
        h1_rev = int.from_bytes(hashlib.sha256(prefix + a_rec).digest(), "big") & ((1 << 124) - 1)
        assert keyed[idx][1] != b ^ h1_rev


@pytest.mark.parametrize("width,n", [(8, 64), (16, 8 * 16 * 3 - 1), (72, 72 * 24), (256, 256 * 16 + 77)])
def test_keyed_round_trip(width, n):
    x = np.random.default_rng(n).integers(0, 256, n, dtype=np.uint8)
    a, pub = oracle.protect_keyed(x, width, KEY, NONCE)
    assert np.array_equal(oracle.recover_keyed(a, pub, n, width, KEY, NONCE), x)


def test_keyed_empty():
    a, pub = oracle.protect_keyed(np.zeros(0, np.uint8), 64, KEY, NONCE)
    assert a.size == 0 and pub.size == 0
    assert oracle.recover_keyed(a, pub, 0, 64, KEY, NONCE).size == 0


def test_key_sensitivity():
    x, W = _case()
    _, pub = oracle.protect_keyed(x, W, KEY, NONCE)
    key2 = bytes([KEY[0] ^ 1]) + KEY[1:]
    _, pub2 = oracle.protect_keyed(x, W, key2, NONCE)
    frac = np.unpackbits(pub ^ pub2).mean()
    assert 0.45 < frac < 0.55
    # the wrong key recovers other bytes, or none (values out of the byte range)
    a, pub = oracle.protect_keyed(x, W, KEY, NONCE)
    try:
        assert not np.array_equal(oracle.recover_keyed(a, pub, x.size, W, key2, NONCE), x)
    except RuntimeError:
        pass


def test_identical_blocks_are_protected_differently():
    W = 64
    x = np.full(W * 16, 200, dtype=np.uint8)  # 16 identical blocks
    a0, pub0 = oracle.protect_packed(x, W, KEY, NONCE)
    a, pub = oracle.protect_keyed(x, W, KEY, NONCE)
    plain_a = oracle.aes128_ctr_xor(KEY, NONCE, 0, a)
    plain = _records(W, x.size, plain_a, pub0)
    keyed = _records(W, x.size, plain_a, pub)
    assert len({v[1:] for v in plain.values()}) == 1
    assert len({v[1] for v in keyed.values()}) == len(keyed)
    assert len({v[2] for v in keyed.values()}) == len(keyed)


@pytest.mark.parametrize("which", ["B", "C"])
def test_an_error_stays_in_its_block(which):
    x, W = _case(width=64, rows=32, seed=9)
    a, pub = oracle.protect_keyed(x, W, KEY, NONCE)
    _, pub0 = oracle.protect_packed(x, W, KEY, NONCE)
    H, sa, sb, sc = oracle.packed_sizes(x.size, W)
    nbx = W // 8
    bi, bj = 2, 5
    bad = pub.copy()
    if which == "B":
        bit = 8 * bi * ((124 * nbx + 7) // 8) + 124 * bj + 7
    else:
        bit = 8 * (sb + 60 * (bi * nbx + bj)) + 100
    bad[bit // 8] ^= np.uint8(1 << (bit % 8))
    # unprotect the damaged fragment and compare it with the unprotected one
    oracle._xor_public(bad, oracle.aes128_ctr_xor(KEY, NONCE, 0, a), H, W, KEY, NONCE, False)
    plain_a = oracle.aes128_ctr_xor(KEY, NONCE, 0, a)
    got = _records(W, x.size, plain_a, bad)
    want = _records(W, x.size, plain_a, pub0)
    damaged = [i for i in want if got[i] != want[i]]
    assert damaged == [bi * nbx + bj]
    b_err = got[damaged[0]][1] ^ want[damaged[0]][1]
    c_err = got[damaged[0]][2] ^ want[damaged[0]][2]
    if which == "C":  # one bit in, one bit out
        assert b_err == 0 and c_err == 1 << 100
    else:  # the B bit itself, and the block's C through H2
        assert b_err == 1 << 7 and bin(c_err).count("1") > 100


def test_block_records_match_the_whole_buffer():
    """The per-block form (used to sample large buffers) gives every block's
    records as the whole-buffer protection does."""
    W = 64
    x = np.random.default_rng(5).integers(0, 256, W * 24, dtype=np.uint8)
    a, pub = oracle.protect_keyed(x, W, KEY, 77)
    plain_a = oracle.aes128_ctr_xor(KEY, 77, 0, a)
    recs = _records(W, x.size, plain_a, pub)
    img = x.reshape(-1, W)
    for idx, want in recs.items():
        bi, bj = divmod(idx, W // 8)
        got = oracle.keyed_block_records(img[8 * bi:8 * bi + 8, 8 * bj:8 * bj + 8], KEY, 77, idx)
        assert got == want


def test_sha512_takes_the_protected_first_fragment():
    """Sec. 5.2.1: SHA-256 keys the first public fragment from the private
    one, and SHA-512 keys the second from the first *protected* public
    fragment.  A block and the same block plus a constant have the same
    detail bands (the 5/3 high-pass of a constant is exactly zero, floors
    included) and LL_2 differing by the constant: the same unprotected B and
    C, a different A.  So their B' differ, and their C' must differ too;
    hashing the unprotected B into SHA-512 would give both the same C'."""
    rng = np.random.default_rng(17)
    x = rng.integers(0, 200, size=(8, 8), dtype=np.uint8)
    y = (x.astype(np.int32) + 40).astype(np.uint8)
    _, pub_x = oracle.protect_packed(x.reshape(-1), 8, KEY, NONCE)
    _, pub_y = oracle.protect_packed(y.reshape(-1), 8, KEY, NONCE)
    assert np.array_equal(pub_x, pub_y)  # same B and C before the keyed protection
    a0, b0, c0 = oracle.keyed_block_records(x, KEY, NONCE, 0)
    a1, b1, c1 = oracle.keyed_block_records(y, KEY, NONCE, 0)
    assert a0 != a1
    assert b0 != b1
    assert c0 != c1


def test_sha256_takes_only_the_private_fragment():
    """Sec. 5.2.1: the first public fragment is keyed by SHA-256 of the
    private fragment (with the key).  Two blocks with the same A and B whose
    C differs in one coefficient (the second made by the exact inverse from
    the first's fragments with that coefficient changed by one) get the same
    B' -- its mask depends on A alone -- and different C'."""
    rng = np.random.default_rng(23)
    x = rng.integers(40, 200, size=64, dtype=np.uint8)
    a, pub = oracle.protect_packed(x, 8, KEY, NONCE)
    pub2 = pub.copy()
    pub2[16] ^= np.uint8(1)  # the lowest bit of C's first 10-bit field
    y = oracle.recover_packed(a, pub2, 64, 8, KEY, NONCE)
    a_y, pub_y = oracle.protect_packed(y, 8, KEY, NONCE)
    assert np.array_equal(a_y, a) and np.array_equal(pub_y, pub2)  # same A and B, C one field apart
    a0, b0, c0 = oracle.keyed_block_records(x.reshape(8, 8), KEY, NONCE, 0)
    a1, b1, c1 = oracle.keyed_block_records(y.reshape(8, 8), KEY, NONCE, 0)
    assert a0 == a1
    assert b0 == b1
    assert c0 != c1
