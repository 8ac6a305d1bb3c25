"""Pins of the oracle's block mode (Sec. 5.2.1: every chunk is processed
block by block, 8 x 8 in the thesis, each block transformed on its own).

The thesis's matrix A and its F(4,4) weights describe exactly one 8 x 8 block,
so they pin the block mode directly: every block of a larger matrix must give
A^T X A (one level) and the F(4,4) combination (two levels) of its own
samples, with the extension at its own borders, whatever its neighbours hold.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden

KEY = bytes(range(16))


def _matrix_A():
    return np.array([[float(v) for v in r] for r in read_golden("matrix_A_level1_8x8.txt")])


def _bands(data, W, L, B, nonce=5):
    """Protect in block mode and return the plaintext band images:
    {('LL', L): ..., (k, l): ...} with k in HL / LH / HH, int64."""
    n = data.size
    H, pb, ub = oracle.sizes(n, W, L, B)
    priv, pub = oracle.protect(data, W, L, KEY, nonce, block=B)
    plain = np.frombuffer(oracle.aes128_ctr_xor(KEY, nonce, 0, priv.tobytes()), dtype="<i2")
    out = {("LL", L): plain.reshape(H >> L, W >> L).astype(np.int64)}
    pubi = pub.view("<i2")
    off = 0
    for l in range(L, 0, -1):
        h, w = H >> l, W >> l
        for k in ("HL", "LH", "HH"):
            out[(k, l)] = pubi[off:off + h * w].reshape(h, w).astype(np.int64)
            off += h * w
    assert off == pubi.size
    return H, out


def _block_tile(bands, l, k, bi, bj, b):
    return bands[(k, l)][bi * b:(bi + 1) * b, bj * b:(bj + 1) * b]


def test_level1_blocks_equal_At_X_A():
    A = _matrix_A()
    rng = np.random.default_rng(21)
    H, W = 24, 40  # 3 x 5 blocks
    img = rng.choice([0, 64, 128, 192], size=(H, W)).astype(np.uint8)
    _, bands = _bands(img.reshape(-1), W, 1, 8)
    for bi in range(H // 8):
        for bj in range(W // 8):
            X = img[8 * bi:8 * bi + 8, 8 * bj:8 * bj + 8].astype(np.int64) - 128
            want = (A.T @ X @ A).astype(np.int64)
            got = np.zeros((8, 8), dtype=np.int64)
            got[:4, :4] = _block_tile(bands, 1, "LL", bi, bj, 4)
            got[:4, 4:] = _block_tile(bands, 1, "HL", bi, bj, 4)
            got[4:, :4] = _block_tile(bands, 1, "LH", bi, bj, 4)
            got[4:, 4:] = _block_tile(bands, 1, "HH", bi, bj, 4)
            assert np.array_equal(got, want), (bi, bj)


def test_level2_blocks_follow_F44_within_floor_slack():
    want = np.zeros((8, 8))
    for i, j, w in read_golden("f44_weights_level2_8x8.txt"):
        want[int(i), int(j)] = float(w)
    rng = np.random.default_rng(22)
    H, W = 32, 32
    worst = 0.0
    for _ in range(40):
        img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
        _, bands = _bands(img.reshape(-1), W, 2, 8)
        for bi in range(H // 8):
            for bj in range(W // 8):
                X = img[8 * bi:8 * bi + 8, 8 * bj:8 * bj + 8].astype(np.int64) - 128
                # output (3, 3) of the block's 2-level layout: HH_2 tile (1, 1)
                got = _block_tile(bands, 2, "HH", bi, bj, 2)[1, 1]
                worst = max(worst, abs(got - float((want * X).sum())))
    assert worst <= 9.375  # the floor slack of the whole-matrix F(4,4) test


def test_single_block_equals_whole_matrix_mode():
    rng = np.random.default_rng(23)
    for B, L in ((8, 1), (8, 2), (8, 3), (16, 2), (32, 4)):
        d = rng.integers(0, 256, B * B, dtype=np.uint8)
        pw, uw = oracle.protect(d, B, L, KEY, 9)
        pb, ub = oracle.protect(d, B, L, KEY, 9, block=B)
        assert np.array_equal(pw, pb) and np.array_equal(uw, ub), (B, L)


def test_blocks_are_independent():
    rng = np.random.default_rng(24)
    H, W, B, L = 32, 48, 16, 2
    img = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    _, ref = _bands(img.reshape(-1), W, L, B)
    img2 = img.copy()
    img2[16:32, 16:32] = rng.integers(0, 256, size=(16, 16), dtype=np.uint8)  # block (1, 1)
    _, got = _bands(img2.reshape(-1), W, L, B)
    for (k, l), band in ref.items():
        b = B >> l
        diff = np.argwhere(band != got[(k, l)])
        assert diff.size, (k, l)
        assert (diff // b == [1, 1]).all(), (k, l)


def test_block_sizes_pad_to_whole_blocks():
    for n, W, L, B in ((1, 8, 2, 8), (65, 8, 2, 8), (1000, 32, 1, 16), (4096 * 9 + 1, 4096, 3, 8)):
        H, pb, ub = oracle.sizes(n, W, L, B)
        assert H % B == 0 and H * W >= n and (H - B) * W < n
        assert pb == 2 * (H >> L) * (W >> L) and pb + ub == 2 * H * W
    with pytest.raises(ValueError):
        oracle.sizes(64, 8, 2, 12)  # width not a multiple of the block
    with pytest.raises(ValueError):
        oracle.sizes(64, 16, 3, 4)  # block smaller than 2^L


@pytest.mark.parametrize("B,L", [(8, 1), (8, 2), (8, 3), (16, 2), (16, 4), (32, 3)])
def test_block_round_trip(B, L):
    rng = np.random.default_rng(B * 10 + L)
    for W in (B, 4 * B):
        for n in (1, B * W - 3, 3 * B * W + 7):
            d = rng.integers(0, 256, n, dtype=np.uint8)
            p, u = oracle.protect(d, W, L, KEY, 1, block=B)
            assert np.array_equal(oracle.recover(p, u, n, W, L, KEY, 1, block=B), d)


def test_extremes_round_trip():
    W, B = 64, 8
    for v in (0, 255):
        d = np.full(W * 24, v, dtype=np.uint8)
        p, u = oracle.protect(d, W, 2, KEY, 2, block=B)
        assert np.array_equal(oracle.recover(p, u, d.size, W, 2, KEY, 2, block=B), d)
    chk = (np.add.outer(np.arange(24), np.arange(W)) % 2 * 255).astype(np.uint8).reshape(-1)
    p, u = oracle.protect(chk, W, 3, KEY, 2, block=B)
    assert np.array_equal(oracle.recover(p, u, chk.size, W, 3, KEY, 2, block=B), chk)
