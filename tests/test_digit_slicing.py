"""The balanced base-2^7 digit split behind the sliced tensor-core products, on the host.

The product kernels cut each scaled entry X = rint(|x| 2^(7 NS - e)) <= 2^(7 NS - 1) into
NS digits d_(NS-1)..d_0 (NS = 8 by default, 6 or 7 as a build parameter, 5 for the
refinement's correction products; 4 still exact) with X = sum_k d_k 2^(7k),
|d_k| <= 64 for the low digits, so that each digit is exact in BF16 and every slice
product is exact in FP32.  They form the digits with one addition: adding 64 to each of
the NS - 1 low 7-bit fields lets the binary carries do the balancing (field k of
Y = X + 64 sum_k 2^(7k), minus 64, is d_k; Y >> 7 (NS - 1) is the top digit).  These
tests check that construction against the definition: the digits reproduce X, stay in
range, and equal the ones a sequential carry loop gives.
"""
import random

import pytest

NS = 8
BAL = sum(64 << (7 * k) for k in range(NS - 1))


def _set_ns(ns):
    global NS, BAL
    NS = ns
    BAL = sum(64 << (7 * k) for k in range(NS - 1))


@pytest.fixture(params=[4, 5, 6, 7, 8], autouse=True)
def digit_count(request):
    _set_ns(request.param)
    yield request.param
    _set_ns(8)


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
    top = 7 * NS - 1                      # X <= 2^top
    low = 7 * (NS - 1)                    # the top digit's weight
    xs = [0, 1, 63, 64, 65, 127, 128, (1 << top), (1 << top) - 1, (1 << low) - 1, 1 << low]
    # runs of 63 and 64 fields: the carry travels through every field
    xs += [sum(63 << (7 * k) for k in range(NS - 1)) + (1 << low) * t for t in range(3)]
    xs += [sum(64 << (7 * k) for k in range(NS - 1)), sum(127 << (7 * k) for k in range(NS - 1))]
    xs += [rng.randrange(0, (1 << top) + 1) for _ in range(20000)]
    xs += [rng.randrange(0, 1 << rng.randrange(1, top + 1)) for _ in range(20000)]
    return xs


def test_balancing_constant():
    # the constants the kernels add: 64 in each of the NS - 1 low 7-bit fields
    assert BAL == {4: 0x0000000000102040, 5: 0x0000000008102040, 6: 0x0000000408102040, 7: 0x0000020408102040,
                   8: 0x0001020408102040}[NS]


def test_addition_matches_carry_loop_and_definition():
    for X in _cases():
        a, b = digits_by_carry(X), digits_by_addition(X)
        assert a == b, X
        assert sum(dk << (7 * k) for k, dk in enumerate(b)) == X
        assert all(-64 <= dk <= 63 for dk in b[:-1]), X
        assert 0 <= b[-1] <= 65


@pytest.mark.parametrize("off", [0, 1])
def test_top_digit_bound(off):
    # |x| < 2^(e-1) keeps X <= 2^(7 NS - 1), so the top digit is at most 64: exact in BF16
    X = (1 << (7 * NS - 1)) - off
    assert digits_by_addition(X)[-1] <= 64
