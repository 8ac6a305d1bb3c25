"""Pins of the oracle's AES-128 / CTR and of the fragment layout (no GPU).

AES is pinned by the FIPS-197 and SP 800-38A vectors and cross-checked with the
installed OpenSSL-backed ``cryptography`` package (a second, independent AES).
The fragment layout is pinned by the size arithmetic of Sec. 5.1.1 / 5.2.1
(1/16 private at two levels), by decrypting the private fragment with that
independent AES, and by exact round trips through protect/recover.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden


def _vectors():
    return {r[0]: r[1:] for r in read_golden("aes_vectors.txt")}


def test_fips197_known_answers():
    v = _vectors()
    key, pt, ct = (bytes.fromhex(x) for x in v["fips197_c1"])
    assert oracle.aes128_encrypt_block(key, pt) == ct
    key, pt, ct = (bytes.fromhex(x) for x in v["fips197_b"])
    assert oracle.aes128_encrypt_block(key, pt) == ct
    key, rk10 = (bytes.fromhex(x) for x in v["fips197_a1_rk10"])
    assert oracle.aes128_expand_key(key)[160:176].tobytes() == rk10


def test_sp800_38a_ctr_vector():
    v = _vectors()
    key = bytes.fromhex(v["sp80038a_f51_key"][0])
    ctr = bytes.fromhex(v["sp80038a_f51_ctr"][0])
    pt = bytes.fromhex(v["sp80038a_f51_pt"][0])
    ct = bytes.fromhex(v["sp80038a_f51_ct"][0])
    nonce = int.from_bytes(ctr[:8], "big")
    first = int.from_bytes(ctr[8:], "big")
    assert oracle.aes128_ctr_xor(key, nonce, first, pt) == ct
    assert oracle.aes128_ctr_xor(key, nonce, first, ct) == pt


def _openssl_ctr(key, nonce, data):
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms, modes
    iv = nonce.to_bytes(8, "big") + bytes(8)
    enc = Cipher(algorithms.AES(key), modes.CTR(iv)).encryptor()
    return enc.update(bytes(data)) + enc.finalize()


@pytest.mark.parametrize("length", [0, 1, 15, 16, 17, 255, 4096 + 7])
def test_ctr_matches_openssl(length):
    rng = np.random.default_rng(length)
    key = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
    data = rng.integers(0, 256, length, dtype=np.uint8).tobytes()
    for nonce in (0, 1, 0x0123456789ABCDEF):
        assert oracle.aes128_ctr_xor(key, nonce, 0, data) == _openssl_ctr(key, nonce, data)


def test_sizes():
    # two levels on an 8x8 block: private = 4 of 64 coefficients (Sec. 5.2.1)
    H, pb, ub = oracle.sizes(64, 8, 2)
    assert (H, pb, ub) == (8, 2 * 4, 2 * 60)
    assert pb * 16 == pb + ub
    # ragged: 1000 bytes at width 64, 3 levels -> 16 rows (15.6 rounded up to 8s)
    H, pb, ub = oracle.sizes(1000, 64, 3)
    assert H == 16 and pb == 2 * 2 * 8 and ub == 2 * 16 * 64 - pb
    assert oracle.sizes(0, 64, 3) == (0, 0, 0)
    for bad in ((100, 0, 1), (100, 12, 3), (100, 8, 0)):
        with pytest.raises(ValueError):
            oracle.sizes(*bad)


KEY = bytes(range(16))


def _bands(coef, H, W, L):
    out = []
    for l in range(L, 0, -1):
        h, w = H >> l, W >> l
        out += [coef[:h, w:2 * w], coef[h:2 * h, :w], coef[h:2 * h, w:2 * w]]
    return out


@pytest.mark.parametrize("n,W,L", [(256 * 256, 256, 1), (1000, 64, 3), (5000, 16, 4),
                                   (64, 8, 2), (1, 2, 1), (3 * 1024 + 5, 128, 2)])
def test_protect_layout_against_independent_aes(n, W, L):
    rng = np.random.default_rng(n + W + L)
    data = rng.integers(0, 256, n, dtype=np.uint8)
    nonce = 7
    priv, pub = oracle.protect(data, W, L, KEY, nonce)
    H, pb, ub = oracle.sizes(n, W, L)
    img = np.zeros(H * W, dtype=np.int64)
    img[:n] = data
    coef = oracle.dwt53_fwd_2d((img - 128).reshape(H, W), L)
    ll = np.frombuffer(_openssl_ctr(KEY, nonce, priv.tobytes()), dtype="<i2")
    assert np.array_equal(ll.reshape(H >> L, W >> L), coef[:H >> L, :W >> L])
    want_pub = np.concatenate([b.astype("<i2").ravel() for b in _bands(coef, H, W, L)])
    assert np.array_equal(np.frombuffer(pub.tobytes(), dtype="<i2"), want_pub)


@pytest.mark.parametrize("n,W,L", [(256 * 256, 256, 1), (1000, 64, 3), (5000, 16, 4),
                                   (64, 8, 2), (1, 2, 1), (77777, 256, 5), (4096, 4096, 3)])
def test_protect_recover_round_trip(n, W, L):
    rng = np.random.default_rng(n * 3 + L)
    for data in (rng.integers(0, 256, n, dtype=np.uint8), np.full(n, 255, dtype=np.uint8),
                 np.zeros(n, dtype=np.uint8)):
        priv, pub = oracle.protect(data, W, L, KEY, 3)
        assert np.array_equal(oracle.recover(priv, pub, n, W, L, KEY, 3), data)


def test_wrong_key_or_nonce_changes_recovery():
    rng = np.random.default_rng(5)
    data = rng.integers(0, 256, 4096, dtype=np.uint8)
    priv, pub = oracle.protect(data, 64, 2, KEY, 1)
    bad_key = bytes([1]) + KEY[1:]
    for k, nn in ((bad_key, 1), (KEY, 2)):
        try:
            out = oracle.recover(priv, pub, 4096, 64, 2, k, nn)
        except RuntimeError:
            continue  # a wrong LL can leave the byte range: reported, not crashed
        assert not np.array_equal(out, data)


def test_constant_input_has_zero_public_fragment():
    priv, pub = oracle.protect(np.full(64 * 64, 77, dtype=np.uint8), 64, 3, KEY, 0)
    assert not pub.any()
    ll = np.frombuffer(_openssl_ctr(KEY, 0, priv.tobytes()), dtype="<i2")
    assert (ll == 77 - 128).all()
