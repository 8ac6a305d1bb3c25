"""Pins of the oracle's packed three fragments (Sec. 5.2.1: private, 1st and
2nd public and protected fragments; Sec. 5.2.3: their storage at 10 / 11
bits per coefficient for 8 x 8 blocks and two levels).

The field order is a reading; these tests decode every field with a plain
Python bit reader of their own and compare it with the block mode's int16
coefficients (already pinned by the thesis's matrix A and F(4,4)), check the
sizes against the thesis's bit counts, and run round trips on inputs built
to reach each coefficient's bound."""
import numpy as np
import pytest

import oracle
from conftest import read_golden

KEY = bytes(range(16))


def _bits_per_block():
    return {r[0]: int(r[1]) for r in read_golden("packed_storage_bits.txt")}


def test_sizes_are_the_thesis_bits_per_block():
    bits = _bits_per_block()
    assert bits["private"] + bits["public1"] + bits["public2"] == bits["total"]
    for W, rows in ((16, 8), (4096, 4096), (64, 24)):
        n = W * rows
        H, sa, sb, sc = oracle.packed_sizes(n, W)
        nblocks = (W // 8) * (H // 8)
        assert 8 * sa == bits["private"] * nblocks
        assert 8 * sb == bits["public1"] * nblocks  # W / 8 even: no row padding
        assert 8 * sc == bits["public2"] * nblocks
    # the printed shares of the input: 7.8 %, 24.2 %, 93.8 %
    H, sa, sb, sc = oracle.packed_sizes(4096 * 4096, 4096)
    n = 4096 * 4096
    assert (round(100 * sa / n, 1), round(100 * sb / n, 1), round(100 * sc / n, 1)) == (7.8, 24.2, 93.8)
    # an odd number of blocks a row pads each row of B to a whole byte
    H, sa, sb, sc = oracle.packed_sizes(72 * 8, 72)
    assert sb == (124 * 9 + 7) // 8


def _field(buf, pos, width):
    """Two's complement value of `width` bits at bit `pos`, LSB first."""
    u = 0
    for i in range(width):
        byte = buf[(pos + i) // 8]
        u |= ((int(byte) >> ((pos + i) % 8)) & 1) << i
    return u - (1 << width) if u >> (width - 1) else u


def _unpacked_tiles(data, W, nonce):
    """Every block's 8 x 8 Mallat layout from the block mode's int16 output."""
    H, pb, ub = oracle.sizes(data.size, W, 2, 8)
    priv, pub = oracle.protect(data, W, 2, KEY, nonce, block=8)
    ll = np.frombuffer(oracle.aes128_ctr_xor(KEY, nonce, 0, priv.tobytes()), dtype="<i2")
    ll = ll.reshape(H // 4, W // 4)
    p = pub.view("<i2")
    bands, off = {}, 0
    for l in (2, 1):
        h, w = H >> l, W >> l
        for k in ("HL", "LH", "HH"):
            bands[(k, l)] = p[off:off + h * w].reshape(h, w)
            off += h * w
    tiles = {}
    for bi in range(H // 8):
        for bj in range(W // 8):
            t = np.zeros((8, 8), dtype=np.int64)
            t[:2, :2] = ll[2 * bi:2 * bi + 2, 2 * bj:2 * bj + 2]
            t[:2, 2:4] = bands[("HL", 2)][2 * bi:2 * bi + 2, 2 * bj:2 * bj + 2]
            t[2:4, :2] = bands[("LH", 2)][2 * bi:2 * bi + 2, 2 * bj:2 * bj + 2]
            t[2:4, 2:4] = bands[("HH", 2)][2 * bi:2 * bi + 2, 2 * bj:2 * bj + 2]
            t[:4, 4:] = bands[("HL", 1)][4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4]
            t[4:, :4] = bands[("LH", 1)][4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4]
            t[4:, 4:] = bands[("HH", 1)][4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4]
            tiles[(bi, bj)] = t
    return H, tiles


@pytest.mark.parametrize("W,rows", [(64, 16), (72, 24)])
def test_fields_are_the_block_mode_coefficients(W, rows):
    rng = np.random.default_rng(W + rows)
    data = rng.integers(0, 256, W * rows - 5, dtype=np.uint8)
    H, tiles = _unpacked_tiles(data, W, 7)
    a, pub = oracle.protect_packed(data, W, KEY, 7)
    _, sa, sb, sc = oracle.packed_sizes(data.size, W)
    a = np.frombuffer(oracle.aes128_ctr_xor(KEY, 7, 0, a.tobytes()), dtype=np.uint8)
    b, c = pub[:sb], pub[sb:]
    nbx = W // 8
    brow = (124 * nbx + 7) // 8
    for (bi, bj), t in tiles.items():
        k = bi * nbx + bj
        pos = 40 * k
        for r in range(2):
            for cc in range(2):
                assert _field(a, pos, 10) == t[r, cc]
                pos += 10
        pos = 8 * brow * bi + 124 * bj
        for r0, c0, width in ((0, 2, 10), (2, 0, 10), (2, 2, 11)):
            for r in range(2):
                for cc in range(2):
                    assert _field(b, pos, width) == t[r0 + r, c0 + cc], (bi, bj, r0, c0)
                    pos += width
        pos = 480 * k
        for r0, c0 in ((0, 4), (4, 0), (4, 4)):
            for r in range(4):
                for cc in range(4):
                    assert _field(c, pos, 10) == t[r0 + r, c0 + cc]
                    pos += 10


def test_round_trip_reaches_the_bounds():
    # weights of each level-2 / level-1 output coefficient of one block
    Wt = np.zeros((8, 8, 8, 8))
    for i in range(8):
        for j in range(8):
            X = np.zeros((8, 8), dtype=np.int64)
            X[i, j] = 4096
            Wt[:, :, i, j] = oracle.dwt53_fwd_2d(X, 2) / 4096.0
    blocks = []
    for r in range(8):
        for c in range(8):
            w = Wt[r, c]
            for sgn in (1, -1):
                blocks.append(np.where(sgn * w >= 0, 255, 0).astype(np.uint8))
    W = 8 * len(blocks)
    img = np.concatenate(blocks, axis=1)  # 8 x W: one block each
    data = img.reshape(-1)
    a, pub = oracle.protect_packed(data, W, KEY, 1)
    assert np.array_equal(oracle.recover_packed(a, pub, data.size, W, KEY, 1), data)
    # and the coefficients do reach near the thesis's bounds (338 / 468 / 648)
    _, tiles = _unpacked_tiles(data, W, 1)
    m = np.max([np.abs(t) for t in tiles.values()], axis=0)
    assert m[0, 0] >= 330 and m[2, 2] >= 640 and m[0, 2] >= 460


@pytest.mark.parametrize("kind", ["random", "zeros", "ones", "checker", "ramp"])
def test_round_trip(kind):
    W, rows = 128, 40
    rng = np.random.default_rng(5)
    if kind == "random":
        data = rng.integers(0, 256, W * rows - 3, dtype=np.uint8)
    elif kind == "zeros":
        data = np.zeros(W * rows, dtype=np.uint8)
    elif kind == "ones":
        data = np.full(W * rows, 255, dtype=np.uint8)
    elif kind == "checker":
        data = (np.add.outer(np.arange(rows), np.arange(W)) % 2 * 255).astype(np.uint8).reshape(-1)
    else:
        data = (np.add.outer(np.arange(rows), np.arange(W)) % 256).astype(np.uint8).reshape(-1)
    a, pub = oracle.protect_packed(data, W, KEY, 2)
    assert np.array_equal(oracle.recover_packed(a, pub, data.size, W, KEY, 2), data)


def test_constant_block_fields():
    # a constant block v: every detail is 0 and LL_2 = v - 128 (the 5/3
    # low-pass keeps a constant), so the private record is four copies of it
    v = 133
    data = np.full(64, v, dtype=np.uint8)
    a, pub = oracle.protect_packed(data, 8, KEY, 0)
    plain = oracle.aes128_ctr_xor(KEY, 0, 0, a.tobytes())
    want = sum((v - 128) << (10 * k) for k in range(4)).to_bytes(5, "little")
    assert plain == want
    assert not pub.any()
