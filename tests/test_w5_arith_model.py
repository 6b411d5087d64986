"""CPU model of the exact arithmetic the tensor-core stage-2 Gram relies on:
balanced base-256 digits of a chunk column, the digit-weight cells split by
plane parity, the FP32-to-integer conversion by one addition of 1.5 2^23, and
the combined integer S.  Python integers and numpy float32 only; nothing here
runs on a GPU.

Pinned: the digits reconstruct the sliced integer; every parity cell of a
64-row chunk stays within 2^22 (the exact range of the conversion) even for the
most extreme digits, while a full weight sum can exceed it; the conversion is
exact on [-2^22, 2^22]; S 2^(E_x + E_y - 50) is within the bound of the dropped
digit weights, the slicing and the tail rounding (about 2 units of
2^(E_x + E_y - 50) per row) of the exact dot product, which the most extreme
digits nearly reach."""
from fractions import Fraction
import math

import numpy as np

BIAS = 0x0080808080808080


def digits(x, E):
    """Balanced digits d_0..d_6 of x against the chunk exponent E (|x| < 2^(E+1)):
    F = trunc(|x| 2^(53 - E)), the signed integer written as bytes of F + BIAS."""
    F = math.floor(abs(Fraction(x)) * Fraction(2) ** (53 - E))
    Fs = -F if x < 0 else F
    G = Fs + BIAS
    assert 0 <= G < 1 << 56
    return [((G >> (8 * (6 - p))) & 0xFF) - 128 for p in range(7)], Fs


def cells(dx, dy):
    """cell[d][t]: the part of digit weight t whose x plane p has parity d,
    summed over the rows (p + q = t, p, q <= 6)."""
    out = [[0] * 7 for _ in range(2)]
    for a, b in zip(dx, dy):
        for t in range(7):
            for p in range(t + 1):
                out[p & 1][t] += a[p] * b[t - p]
    return out


def magic(x):
    """Bits of float32(x) + 1.5 2^23 minus 0x4B400000, as the kernel computes it."""
    y = np.float32(x) + np.float32(12582912.0)
    return int(np.array(y, dtype=np.float32).view(np.int32)) - 0x4B400000


def test_digits_reconstruct_the_sliced_integer():
    rng = np.random.default_rng(7)
    for x in list(rng.standard_normal(200)) + [1.0, -1.0, 1.9999999999999998, -0x808080808080 * 2.0 ** -53]:
        E = math.frexp(abs(x))[1] - 1 if x != 0 else 0
        d, Fs = digits(x, E)
        assert abs(d[0]) <= 64 and all(-128 <= v <= 127 for v in d)
        assert sum(v * 256 ** (6 - p) for p, v in enumerate(d)) == Fs


def test_parity_cells_stay_in_the_exact_conversion_range():
    # the most extreme digits: d_0 = -64 (|F| < 2^54 forces |d_0| <= 64), all others -128
    worst = [-64] + [-128] * 6
    c = cells([worst] * 64, [worst] * 64)
    assert max(abs(v) for row in c for v in row) <= 1 << 22
    # the rows of the GPU test: digits 1..6 all -128 under a chunk maximum of 1
    d1, _ = digits(-0x808080808080 * 2.0 ** -53, 0)
    assert d1 == [0] + [-128] * 6
    top, _ = digits(1.0, 0)
    col = [top] + [d1] * 63
    c = cells(col, col)
    assert max(abs(v) for row in c for v in row) <= 1 << 22
    # ... while the full weight-6 sum passes 2^22: it must be added as integers
    assert c[0][6] + c[1][6] == 63 * 5 * 2 ** 14 > 1 << 22


def test_magic_conversion_is_exact_on_its_range():
    pts = [0, 1, -1, 2 ** 22, -(2 ** 22), 2 ** 22 - 1, -(2 ** 22) + 1, 123456, -654321]
    pts += list(np.random.default_rng(3).integers(-(2 ** 22), 2 ** 22 + 1, 2000))
    for x in pts:
        assert magic(int(x)) == int(x)
    # one past the range it is not exact: the cells are converted one at a time
    assert magic(2 ** 22 + 1) != 2 ** 22 + 1


def test_combined_sum_matches_the_exact_product():
    rng = np.random.default_rng(11)
    for trial in range(20):
        x = rng.standard_normal(64) * 2.0 ** int(rng.integers(-20, 20))
        y = rng.standard_normal(64) * 2.0 ** int(rng.integers(-20, 20))
        if trial == 0:
            x = np.full(64, -0x808080808080 * 2.0 ** -53)
            x[0] = 1.0
            y = x.copy()
        Ex = max(math.frexp(abs(v))[1] - 1 for v in x)
        Ey = max(math.frexp(abs(v))[1] - 1 for v in y)
        dx = [digits(v, Ex)[0] for v in x]
        dy = [digits(v, Ey)[0] for v in y]
        c = cells(dx, dy)
        I = [magic(c[0][t]) + magic(c[1][t]) for t in range(7)]
        S = (I[0] * 256 + I[1]) * 2 ** 32 + I[2] * 2 ** 24 + I[3] * 2 ** 16 + I[4] * 256 + I[5] + ((I[6] + 128) >> 8)
        got = Fraction(S) * Fraction(2) ** (Ex + Ey - 50)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, y))
        # in units u = 2^(Ex + Ey - 50), per row: the dropped weights p + q > 6 (p, q >= 1,
        # |d_p d_q| <= 2^14) at most 6 2^14 2^-16 + 5 2^14 2^-24 + ... < 1.51 u, the
        # slicing (each value within 2^(E - 53) of its digits) < 0.5 u; the tail
        # rounding 0.5 u per chunk
        bound = Fraction(64 * 2 + 1) * Fraction(2) ** (Ex + Ey - 50)
        assert abs(got - exact) <= bound, (trial, float(abs(got - exact)), float(bound))
        if trial == 0:
            assert abs(got - exact) > bound / 2      # the extreme digits use most of it
