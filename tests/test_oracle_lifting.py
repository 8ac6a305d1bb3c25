"""Pins of the oracle's 5/3 lifting and 2-D transform against what the thesis
prints and what the mathematics fixes (no GPU needed).

Each check is chosen so that a plausible slip in the oracle fails it: a wrong
update sign, a wrong boundary extension, columns before rows, truncating
instead of flooring division, a transposed operand or a dropped level.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden


def _matrix_A():
    return np.array([[float(v) for v in r] for r in read_golden("matrix_A_level1_8x8.txt")])


# -- length-2 closed form over every byte pair --------------------------------

def test_length2_closed_form_all_pairs():
    # Eq. 5.1/5.2 with x[2] = x[0], d[-1] = d[0] reduce to
    # d = x1 - x0, s = x0 + floor((d + 1) / 2) (worked in tests/golden/order_2x2.txt)
    for x0 in range(-128, 128):
        for x1 in range(-128, 128):
            d = x1 - x0
            s = x0 + (d + 1) // 2
            out = oracle.lift53_fwd_1d([x0, x1])
            assert out[0] == s and out[1] == d
            assert list(oracle.lift53_inv_1d(out)) == [x0, x1]


def test_negative_floor_worked_example():
    (inp, out) = read_golden("lift1d_negative.txt")
    x = [int(v) for v in inp[1:]]
    want = [int(v) for v in out[1:]]
    assert list(oracle.lift53_fwd_1d(x)) == want
    assert list(oracle.lift53_inv_1d(want)) == x


def test_row_before_column_worked_example():
    (inp, out) = read_golden("order_2x2.txt")
    x = np.array([int(v) for v in inp[1:]]).reshape(2, 2)
    want = np.array([int(v) for v in out[1:]]).reshape(2, 2)
    assert np.array_equal(oracle.dwt53_fwd_2d(x, 1), want)
    assert np.array_equal(oracle.dwt53_inv_2d(want, 1), x)


# -- the thesis's matrix A (Sec. 5.2.2) ---------------------------------------

def test_level1_1d_equals_matrix_A_exactly():
    # Inputs that are multiples of 64 make every floor exact (the sums being
    # floored are multiples of 4 / 8), so the integer lifting equals the linear
    # map row . A.  This pins the update sign and the extension.
    A = _matrix_A()
    rng = np.random.default_rng(11)
    for _ in range(200):
        x = rng.choice([-128, -64, 0, 64], size=8)
        got = oracle.lift53_fwd_1d(x)
        assert np.array_equal(got, (x @ A).astype(np.int64))


def test_level1_2d_equals_At_X_A_exactly():
    A = _matrix_A()
    rng = np.random.default_rng(12)
    for _ in range(200):
        X = rng.choice([0, 64, 128, 192], size=(8, 8)) - 128
        got = oracle.dwt53_fwd_2d(X, 1)
        want = A.T @ X @ A
        assert np.array_equal(got, want.astype(np.int64))


def test_matrix_A_from_impulses():
    # the oracle's impulse responses at a scale where the floors are exact
    A = _matrix_A()
    for i in range(8):
        e = np.zeros(8, dtype=np.int64)
        e[i] = 4096
        assert np.array_equal(oracle.lift53_fwd_1d(e), (4096 * A[i]).astype(np.int64))


# -- F(4,4) of the 2-level 8x8 transform (Sec. 5.2.2) --------------------------

def _level2_weights():
    # W[p, q, i, j] = weight of input (i, j) in output (p, q), 2 levels on 8x8.
    # Inputs that are multiples of 4096 keep every floor of both levels exact.
    W = np.zeros((8, 8, 8, 8))
    for i in range(8):
        for j in range(8):
            X = np.zeros((8, 8), dtype=np.int64)
            X[i, j] = 4096
            W[:, :, i, j] = oracle.dwt53_fwd_2d(X, 2) / 4096.0
    return W


def test_F44_weights_match_thesis():
    W = _level2_weights()
    want = np.zeros((8, 8))
    for i, j, w in read_golden("f44_weights_level2_8x8.txt"):
        want[int(i), int(j)] = float(w)
    assert np.array_equal(W[3, 3], want)


def test_F44_integer_output_within_floor_slack():
    want = np.zeros((8, 8))
    for i, j, w in read_golden("f44_weights_level2_8x8.txt"):
        want[int(i), int(j)] = float(w)
    rng = np.random.default_rng(13)
    worst = 0.0
    for _ in range(2000):
        X = rng.integers(-128, 128, size=(8, 8))
        got = oracle.dwt53_fwd_2d(X, 2)[3, 3]
        worst = max(worst, abs(got - float((want * X).sum())))
    # Each predict floor moves its result by (-1, 0] and each update floor
    # (with its +2) by (-1/2, 1/2] from the floor-free Eq. 5.3/5.4 form; summed
    # with the absolute gains from those 16 + 16 rounding points to F(4,4)
    # (5.125 for the predicts, 8.5 for the updates) this bounds
    # |integer - linear| by 5.125 + 8.5 / 2 = 9.375.
    assert worst <= 9.375


def test_level2_bounds_match_thesis():
    W = _level2_weights()
    bound = 128 * np.abs(W[:4, :4]).sum(axis=(2, 3))
    want = np.array([[int(v) for v in r] for r in read_golden("bounds_level2_8x8.txt")])
    assert np.array_equal(bound, want)


def test_level1_bounds_match_thesis():
    # Sec. 5.2.3: after one level, |LL_1| <= 2.25 x 128, |HL_1|,|LH_1| <= 384,
    # |HH_1| <= 511 (512 with the [-128, +128] convention).
    W = np.zeros((8, 8, 8, 8))
    for i in range(8):
        for j in range(8):
            X = np.zeros((8, 8), dtype=np.int64)
            X[i, j] = 4096
            W[:, :, i, j] = oracle.dwt53_fwd_2d(X, 1) / 4096.0
    b = 128 * np.abs(W).sum(axis=(2, 3))
    assert b[:4, :4].max() == 288
    assert b[:4, 4:].max() == 384 and b[4:, :4].max() == 384
    assert b[4:, 4:].max() == 512


def test_integer_outputs_respect_bounds_on_extremes():
    want = np.array([[int(v) for v in r] for r in read_golden("bounds_level2_8x8.txt")])
    rng = np.random.default_rng(14)
    cases = [rng.choice([-128, 127], size=(8, 8)) for _ in range(3000)]
    cases += [rng.integers(-128, 128, size=(8, 8)) for _ in range(1000)]
    for X in cases:
        c = oracle.dwt53_fwd_2d(X, 2)[:4, :4]
        assert (np.abs(c) <= want + 2).all()


# -- invariants on whole matrices ----------------------------------------------

@pytest.mark.parametrize("levels", [1, 2, 3])
def test_constant_gives_zero_details(levels):
    X = np.full((64, 64), 77 - 128)
    c = oracle.dwt53_fwd_2d(X, levels)
    h = 64 >> levels
    assert (c[:h, :h] == 77 - 128).all()
    c[:h, :h] = 0
    assert not c.any()


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_ramp_gives_zero_interior_details(levels):
    # x[i, j] = i + j: the 5/3 predict is exact on a line, so every detail is
    # zero except where the mirror at the right / bottom border bends the line
    # (last column of HL_l, last row of LH_l); HH_l is zero everywhere.
    N = 128
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    c = oracle.dwt53_fwd_2d(i + j - 128, levels)
    for l in range(1, levels + 1):
        h = N >> l
        HL = c[:h, h:2 * h]
        LH = c[h:2 * h, :h]
        HH = c[h:2 * h, h:2 * h]
        assert not HH.any()
        assert not HL[:, :-1].any() and HL[:, -1].any()
        assert not LH[:-1, :].any() and LH[-1, :].any()


@pytest.mark.parametrize("levels", [1, 2, 3, 4])
def test_level_shift_moves_only_LL(levels):
    rng = np.random.default_rng(20 + levels)
    B = rng.integers(0, 256, size=(64, 96))
    a = oracle.dwt53_fwd_2d(B, levels)
    b = oracle.dwt53_fwd_2d(B - 128, levels)
    hl, wl = 64 >> levels, 96 >> levels
    diff = a - b
    assert (diff[:hl, :wl] == 128).all()
    diff[:hl, :wl] = 0
    assert not diff.any()


@pytest.mark.parametrize("shape,levels", [((8, 8), 2), ((64, 128), 4), ((30, 40), 1),
                                          ((48, 16), 3), ((2, 2), 1), ((256, 32), 5)])
def test_round_trip_exact(shape, levels):
    rng = np.random.default_rng(hash(shape) % 1000 + levels)
    for X in (rng.integers(-128, 128, size=shape),
              np.where((np.add.outer(np.arange(shape[0]), np.arange(shape[1])) % 2) == 0, -128, 127),
              rng.integers(-3000, 3000, size=shape)):
        c = oracle.dwt53_fwd_2d(X, levels)
        assert np.array_equal(oracle.dwt53_inv_2d(c, levels), X)


def test_round_trip_random_small_blocks():
    rng = np.random.default_rng(30)
    for _ in range(3000):
        X = rng.integers(-128, 128, size=(4, 4))
        assert np.array_equal(oracle.dwt53_inv_2d(oracle.dwt53_fwd_2d(X, 2), 2), X)
        Y = rng.integers(-128, 128, size=(2, 2))
        assert np.array_equal(oracle.dwt53_inv_2d(oracle.dwt53_fwd_2d(Y, 1), 1), Y)
