"""Pins of the oracle's generator (section "Matrix Generation") against closed
forms, the LCG's published properties and exact integer arithmetic."""
from fractions import Fraction

import numpy as np
import pytest

import oracle

M64 = (1 << 64) - 1
KNUTH_A = 6364136223846793005  # Knuth's MMIX multiplier
KNUTH_C = 1442695040888963407  # Knuth's MMIX increment


def step_py(s: int) -> int:
    """One step of the recurrence s' = a s + c mod 2^64, written from its definition."""
    return (KNUTH_A * s + KNUTH_C) & M64


def test_first_state_closed_form():
    # from seed 0 the first state is the increment itself
    assert oracle.lcg_state(0, 1) == KNUTH_C
    assert oracle.lcg_state(12345, 0) == 12345


def test_jump_equals_stepping():
    seq = oracle.lcg_sequence(987654321, 3000)
    s = 987654321
    for t in range(3000):
        s = step_py(s)
        assert int(seq[t]) == s
    for k in [1, 2, 3, 7, 64, 1000, 2999]:
        assert oracle.lcg_state(987654321, k) == int(seq[k - 1])


def test_jump_composition_and_full_period():
    g = np.random.default_rng(5)
    for _ in range(20):
        a, b = (int(x) for x in g.integers(0, 2**63, size=2, dtype=np.uint64))
        a1, c1 = oracle.lcg_jump(a)
        a2, c2 = oracle.lcg_jump(b)
        a3, c3 = oracle.lcg_jump((a + b) & M64)
        # apply jump(b) after jump(a): s -> a2 (a1 s + c1) + c2
        assert (a2 * a1) & M64 == a3
        assert (a2 * c1 + c2) & M64 == c3
    # Hull-Dobell: c odd and a-1 divisible by 4 give the full period 2^64, so
    # jump(2^63) is not the identity but applied twice it is.
    ah, ch = oracle.lcg_jump(1 << 63)
    assert (ah, ch) != (1, 0)
    assert (ah * ah) & M64 == 1 and (ah * ch + ch) & M64 == 0


def test_value_mapping():
    n = 64
    A, b = oracle.generate(n, 7, mode=oracle.NONE, nrhs=2)
    vals = np.concatenate([A.ravel(), b.ravel()])
    q = vals * 2.0**53
    assert np.all(np.abs(vals) < 0.5) and np.all(vals != 0)
    assert np.all(q == np.round(q)) and np.all(np.mod(q, 2) == 1)
    # entry (i, j) is draw i + j n; b(i, r) is draw n^2 + i + r n
    for (i, j) in [(0, 0), (5, 3), (63, 63), (17, 40)]:
        assert A[i, j] == oracle.draw_value(7, i + j * n)
    for (i, r) in [(0, 0), (63, 1), (30, 1)]:
        assert b[i, r] == oracle.draw_value(7, n * n + i + r * n)
    # value from the state, written from the mapping's definition
    s = oracle.lcg_state(7, 1)
    u = s >> 12
    assert A[0, 0] == (2 * u + 1 - 2**52) * 2.0**-53


def test_statistics():
    A, _ = oracle.generate(400, 3, mode=oracle.NONE, nrhs=0)
    v = A.ravel()
    sd = np.sqrt(1 / 12)
    assert abs(v.mean()) < 5 * sd / np.sqrt(v.size)
    assert abs(v.var() - 1 / 12) < 0.01 * (1 / 12)


@pytest.mark.parametrize("n,margin", [(1, 1.0), (2, 1.0), (33, 1.0), (200, 0.25), (257, 655.36)])
def test_diagonal_dominance_exact(n, margin):
    A, _ = oracle.generate(n, 11, margin=margin)
    for i in range(n):
        off = [A[i, j] for j in range(n) if j != i]
        S = sum(int(Fraction(x).numerator * (2**53 // Fraction(x).denominator)) if x != 0 else 0
                for x in np.abs(off))
        # the row's absolute sum as an exact integer count of 2^-53 units
        exact = Fraction(S, 2**53) + Fraction(margin)
        a = A[i, i]
        assert abs(Fraction(a) - exact) <= Fraction(np.spacing(a))
        # two roundings: int -> fp64, then the add of the margin
        assert a == float(S) * 2.0**-53 + margin
        assert Fraction(a) - Fraction(S, 2**53) >= Fraction(margin) - Fraction(np.spacing(a))


def test_norm_inf_closed_form():
    n = 300
    A, _ = oracle.generate(n, 2, margin=1.0)
    off = np.abs(A) - np.diag(np.abs(np.diag(A)))
    expected = np.max(2 * off.sum(axis=1) + 1.0)
    assert np.linalg.norm(A, np.inf) == pytest.approx(expected, rel=1e-13)


def test_sqrtn_and_none_modes():
    n = 100
    A0, b0 = oracle.generate(n, 4, mode=oracle.NONE)
    A1, b1 = oracle.generate(n, 4, mode=oracle.SQRTN)
    off = ~np.eye(n, dtype=bool)
    assert np.array_equal(A0[off], A1[off]) and np.array_equal(b0, b1)
    d0, d1 = np.diag(A0), np.diag(A1)
    assert np.all(d1 == d0 + np.sign(d0) * np.sqrt(n))


def test_rows_by_skip_ahead_match_full_generation():
    n = 150
    A, _ = oracle.generate(n, 99, margin=2.0)
    rows = [0, 1, 77, 149]
    R = oracle.generate_rows(n, 99, rows, margin=2.0)
    for k, i in enumerate(rows):
        assert np.array_equal(R[k], A[i])


def test_bad_arguments():
    with pytest.raises(ValueError):
        oracle.generate(0, 1)


@pytest.mark.parametrize("n,rho", [(2, 1.0), (64, 0.9), (257, 0.5), (300, 1.25)])
def test_departure_from_dominance_exact(n, rho):
    """DEPARTURE: a_ii = fl(fl(S_i) 2^-53 rho), S_i the exact off-diagonal sum
    of |q_ij| (section "Matrix Generation", departure from diagonal dominance)."""
    A, _ = oracle.generate(n, 12, margin=rho, mode=oracle.DEPARTURE)
    D, _ = oracle.generate(n, 12, margin=1.0)
    for i in range(n):
        S = sum(abs(int(round(A[i, j] * 2.0**53))) for j in range(n) if j != i)
        assert A[i, i] == (float(S) * 2.0**-53) * rho
        exact = Fraction(S, 2**53) * Fraction(rho)      # rho times the exact off-diagonal sum
        assert abs(Fraction(A[i, i]) - exact) <= 2 * Fraction(np.spacing(A[i, i]))
    # the off-diagonal entries are those of every other mode
    mask = ~np.eye(n, dtype=bool)
    assert np.array_equal(A[mask], D[mask])


@pytest.mark.parametrize("c", [1.0, 0.625])
def test_sqrtn_coefficient(c):
    n = 333
    A, _ = oracle.generate(n, 5, margin=c, mode=oracle.SQRTN)
    N, _ = oracle.generate(n, 5, mode=oracle.NONE)
    r = c * np.sqrt(float(n))
    for i in range(n):
        q = N[i, i]
        assert A[i, i] == q + (r if q > 0 else -r)


def test_departure_rejects_nonpositive_ratio():
    with pytest.raises(ValueError):
        oracle.generate(10, 1, margin=0.0, mode=oracle.DEPARTURE)
