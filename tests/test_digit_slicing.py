"""The balanced base-2^7 digit split behind the sliced tensor-core products, on the host.

The product kernels cut each scaled entry X = rint(|x| 2^(56 - e)) <= 2^55 into eight
digits d_7..d_0 with X = sum_k d_k 2^(7k), |d_k| <= 64 for the seven low digits, so that
each digit is exact in BF16 and every slice product is exact in FP32.  They form the
digits with one addition: adding 64 to each of the seven low 7-bit fields lets the binary
carries do the balancing (field k of Y = X + 64 sum_k 2^(7k), minus 64, is d_k; Y >> 49
is the top digit).  These tests check that construction against the definition: the
digits reproduce X, stay in range, and equal the ones a sequential carry loop gives.
"""
import random

import pytest

NS = 8
BAL = sum(64 << (7 * k) for k in range(NS - 1))


def digits_by_carry(X):
    """Low digits first: v = field + carry; carry = v >= 64; d = v - 128 carry."""
    d, carry = [], 0
    for k in range(NS - 1):
        v = ((X >> (7 * k)) & 127) + carry
        carry = 1 if v >= 64 else 0
        d.append(v - (carry << 7))
    d.append((X >> (7 * (NS - 1))) + carry)
    return d


def digits_by_addition(X):
    Y = X + BAL
    return [((Y >> (7 * k)) & 127) - 64 for k in range(NS - 1)] + [Y >> (7 * (NS - 1))]


def _cases():
    rng = random.Random(20260)
    xs = [0, 1, 63, 64, 65, 127, 128, (1 << 55), (1 << 55) - 1, (1 << 49) - 1, 1 << 49]
    # runs of 63 and 64 fields: the carry travels through every field
    xs += [sum(63 << (7 * k) for k in range(NS - 1)) + (1 << 49) * t for t in range(3)]
    xs += [sum(64 << (7 * k) for k in range(NS - 1)), sum(127 << (7 * k) for k in range(NS - 1))]
    xs += [rng.randrange(0, (1 << 55) + 1) for _ in range(20000)]
    xs += [rng.randrange(0, 1 << rng.randrange(1, 56)) for _ in range(20000)]
    return xs


def test_balancing_constant():
    assert BAL == 0x0001020408102040


def test_addition_matches_carry_loop_and_definition():
    for X in _cases():
        a, b = digits_by_carry(X), digits_by_addition(X)
        assert a == b, X
        assert sum(dk << (7 * k) for k, dk in enumerate(b)) == X
        assert all(-64 <= dk <= 63 for dk in b[:-1]), X
        assert 0 <= b[-1] <= 65


@pytest.mark.parametrize("X", [(1 << 55), (1 << 55) - 1])
def test_top_digit_bound(X):
    # |x| < 2^(e-1) keeps X <= 2^55, so the top digit fits BF16 exactly (<= 2^8)
    assert digits_by_addition(X)[-1] <= 1 << 8
