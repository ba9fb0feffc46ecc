"""Pins of the oracle's software rounding against the formats' definitions:
every BF16 value and midpoint, numpy's correctly rounded FP16/FP32
conversions, and the OCP E4M3 code table enumerated from its definition."""
import numpy as np
import pytest

import oracle
from inputs import doubles_spanning


def bf16_table():
    """All finite non-negative BF16 values, from the bit patterns."""
    bits = np.arange(0, 0x7F80, dtype=np.uint32) << 16
    return bits.view(np.float32).astype(np.float64)


def e4m3_table():
    """All finite non-negative OCP E4M3 values (bias 7, no infinity, S.1111.111 = NaN)."""
    vals = []
    for code in range(0x7F):
        e, m = code >> 3, code & 7
        vals.append(m / 8 * 2.0**-6 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7))
    return np.array(vals)


def check_table(values, fmt, even_of):
    v = values
    lo, hi = v[:-1], v[1:]
    mid = (lo + hi) / 2
    # representable values are fixed points
    assert np.array_equal(oracle.round_to(v, fmt), v)
    assert np.array_equal(oracle.round_to(-v, fmt), -v)
    # just below / above a midpoint round down / up
    assert np.array_equal(oracle.round_to(np.nextafter(mid, 0), fmt), lo)
    assert np.array_equal(oracle.round_to(np.nextafter(mid, np.inf), fmt), hi)
    # exact midpoints go to the neighbour with an even significand
    want = np.where(even_of(np.arange(len(lo))), lo, hi)
    assert np.array_equal(oracle.round_to(mid, fmt), want)
    assert np.array_equal(oracle.round_to(-mid, fmt), -want)


def test_bf16_all_values_and_midpoints():
    v = bf16_table()
    check_table(v, oracle.BF16, lambda k: k % 2 == 0)
    big = v[-1]
    half_ulp = 2.0 ** (127 - 8)
    assert oracle.round_to([big + half_ulp * 0.999], oracle.BF16)[0] == big
    assert np.isinf(oracle.round_to([big + half_ulp], oracle.BF16)[0])  # tie to even = overflow
    assert np.isnan(oracle.round_to([np.nan], oracle.BF16)[0])


def test_bf16_is_not_double_rounding():
    # x sits just above a BF16 midpoint by less than half an fp32 ulp: going
    # through fp32 first would land on the midpoint and round to even (down).
    lo = 1.0
    x = lo + 2.0**-8 + 2.0**-30
    assert oracle.round_to([x], oracle.BF16)[0] == 1.0 + 2.0**-7
    assert float(np.float32(x)) == 1.0 + 2.0**-8


def test_fp16_against_numpy():
    x = np.concatenate([doubles_spanning(200000, 1, -26, 17),
                        np.float16(np.arange(1, 0x7C00, dtype=np.uint16).view(np.float16)).astype(np.float64)])
    half = np.arange(1, 0x7BFF, dtype=np.uint16).view(np.float16).astype(np.float64)
    x = np.concatenate([x, (half[:-1] + half[1:]) / 2])
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    got = oracle.round_to(x, oracle.FP16)
    assert np.array_equal(got, want)


def test_fp32_against_numpy():
    x = doubles_spanning(200000, 2, -140, 120)
    assert np.array_equal(oracle.round_to(x, oracle.FP32), x.astype(np.float32).astype(np.float64))


def test_e4m3_table_midpoints_saturation():
    v = e4m3_table()
    assert v[-1] == 448.0 and len(v) == 127
    check_table(v, oracle.E4M3, lambda k: k % 2 == 0)
    for x, want in [(449.0, 448.0), (464.0, 448.0), (480.0, 448.0), (1e30, 448.0), (np.inf, 448.0),
                    (2.0**-10, 0.0), (1.5 * 2.0**-10, 2.0**-9), (2.0**-9, 2.0**-9)]:
        assert oracle.round_to([x], oracle.E4M3)[0] == want
        assert oracle.round_to([-x], oracle.E4M3)[0] == -want


def test_zero_sign_kept():
    assert np.signbit(oracle.round_to([-0.0], oracle.BF16)[0])
    assert np.signbit(oracle.round_to([-1e-300], oracle.BF16)[0])


@pytest.mark.parametrize("fmt", [oracle.BF16, oracle.FP16, oracle.E4M3])
def test_monotone(fmt):
    x = np.sort(doubles_spanning(50000, 9, -12, 8))
    y = oracle.round_to(x, fmt)
    assert np.all(np.diff(y) >= 0)
