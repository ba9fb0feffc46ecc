"""Pins of the oracle's low-precision blocked LU (section "Algorithmic
Framework", Fig. 1): the exact-arithmetic special case against the textbook
factorization, an independent re-derivation of every rounding point on small
matrices, diagonal-dominance invariants and error bounds."""
from fractions import Fraction

import numpy as np
import pytest

import oracle

U_LOW = {oracle.BF16: 2.0**-8, oracle.FP16: 2.0**-11}


def doolittle(A):
    """Textbook unblocked Doolittle LU without pivoting, fp64."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    for p in range(n):
        A[p + 1:, p] /= A[p, p]
        A[p + 1:, p + 1:] -= np.outer(A[p + 1:, p], A[p, p + 1:])
    return A


@pytest.mark.parametrize("n,nb", [(1, 128), (2, 128), (3, 128), (17, 128), (129, 128), (300, 128),
                                  (300, 256), (600, 256), (700, 512), (1100, 512)])
def test_exact_special_case_is_the_textbook_lu(n, nb):
    A, _ = oracle.generate(n, 5)
    LU, rc = oracle.factor(A, oracle.FP64, nb)
    assert rc == 0
    L, U = oracle.split_lu(LU)
    assert np.linalg.norm(L @ U - A) <= 4e-16 * np.linalg.norm(A) * np.sqrt(n) + 1e-300
    assert np.allclose(LU, doolittle(A), rtol=1e-12, atol=1e-14 * np.abs(A).max())


def test_exact_case_keeps_row_dominance_excess():
    # Schur complements of a row diagonally dominant matrix stay dominant with
    # at least the original excess, so every row of U keeps the margin.
    margin = 3.0
    A, _ = oracle.generate(400, 8, margin=margin)
    LU, _ = oracle.factor(A, oracle.FP64, 256)
    U = np.triu(LU)
    excess = np.abs(np.diag(U)) - (np.abs(U).sum(axis=1) - np.abs(np.diag(U)))
    assert excess.min() >= margin * (1 - 1e-9)
    assert np.abs(U).max() <= 2 * np.abs(A).max()


@pytest.mark.parametrize("fmt", [oracle.BF16, oracle.FP16])
@pytest.mark.parametrize("n,nb", [(100, 128), (517, 128), (700, 256), (900, 512)])
def test_low_precision_error_bounds(fmt, n, nb):
    A, _ = oracle.generate(n, 6)
    LU, rc = oracle.factor(A, fmt, nb)
    assert rc == 0
    assert np.array_equal(oracle.round_to(LU, fmt), LU)  # every stored value is in the format
    L, U = oracle.split_lu(LU)
    rel = np.linalg.norm(L @ U - A) / np.linalg.norm(A)
    assert rel <= 4 * n * U_LOW[fmt]   # the stated (loose) bound
    assert rel <= U_LOW[fmt]           # sharp: one rounding per stored value dominates
    assert rel >= U_LOW[fmt] / 16      # and the rounding is really applied
    assert np.abs(U).max() <= 2 * np.abs(A).max() * (1 + 4 * U_LOW[fmt])


def test_depth_above_n_reduces_to_128():
    A, _ = oracle.generate(400, 12)
    a, _ = oracle.factor(A, oracle.BF16, 128)
    b, _ = oracle.factor(A, oracle.BF16, 512)
    assert np.array_equal(a, b)
    c, _ = oracle.factor(A, oracle.BF16, 256)
    assert not np.array_equal(a, c)   # different update depth, different rounding points


def test_fp8_update_variant():
    A, _ = oracle.generate(600, 13)
    LU8, rc = oracle.factor(A, oracle.BF16, 256, fmt_update=oracle.E4M3)
    LU16, _ = oracle.factor(A, oracle.BF16, 256)
    assert rc == 0 and not np.array_equal(LU8, LU16)
    assert np.array_equal(oracle.round_to(LU8, oracle.BF16), LU8)
    L, U = oracle.split_lu(LU8)
    assert np.linalg.norm(L @ U - A) / np.linalg.norm(A) <= 2.0**-7
    # the first panel and diagonal block do not depend on the update format
    assert np.array_equal(LU8[:, :256], LU16[:, :256]) and np.array_equal(LU8[:256, :], LU16[:256, :])


# ---------------------------------------------------------------------------
# Independent re-derivation of the rounding points, written from the method's
# description with exact fp32 fused multiply-add emulation in Python.
# ---------------------------------------------------------------------------
def _round_fraction_to_f32(fr: Fraction) -> np.float32:
    c = np.float32(float(fr))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        d = abs(Fraction(float(cand)) - fr)
        key = (d, int(np.array(cand).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return best[1]


def fmaf(a, b, c):
    a, b, c = float(a), float(b), float(c)
    p = a * b            # exact: two 24-bit significands
    s = p + c
    bp = s - c
    err = (p - bp) + (c - (s - bp))
    if err == 0.0 and np.isfinite(s):
        return np.float32(s)
    return _round_fraction_to_f32(Fraction(a) * Fraction(b) + Fraction(c))


def bf16(x):
    return float(oracle.round_to([float(x)], oracle.BF16)[0])


def reference_small_lu(A):
    """Single-level method for n <= 256 with nb = 128 (base block + one panel)."""
    n = A.shape[0]
    M = np.vectorize(bf16)(A)
    b = min(128, n)
    a = M[:b, :b].astype(np.float32)
    for p in range(b):
        for i in range(p + 1, b):
            a[i, p] = np.float32(a[i, p] / a[p, p])
        for j in range(p + 1, b):
            for i in range(p + 1, b):
                a[i, j] = fmaf(-a[i, p], a[p, j], a[i, j])
    M[:b, :b] = np.vectorize(bf16)(a)
    if n == b:
        return M
    # inverses of the stored factors
    Li = np.zeros((b, b), dtype=np.float32)
    for c in range(b):
        x = np.zeros(b, dtype=np.float32); x[c] = 1
        for r in range(c + 1, b):
            acc = np.float32(0)
            for t in range(c, r):
                acc = fmaf(-np.float32(M[r, t]), x[t], acc)
            x[r] = acc
        Li[:, c] = x
    Ui = np.zeros((b, b), dtype=np.float32)
    for c in range(b):
        y = np.zeros(b, dtype=np.float32); y[c] = np.float32(1) / np.float32(M[c, c])
        for r in range(c - 1, -1, -1):
            acc = np.float32(0)
            for t in range(c, r, -1):
                acc = fmaf(np.float32(M[r, t]), y[t], acc)
            y[r] = np.float32(-acc / np.float32(M[r, r]))
        Ui[:, c] = y
    Li = np.vectorize(bf16)(Li); Ui = np.vectorize(bf16)(Ui)
    U12 = np.zeros((b, n - b)); L21 = np.zeros((n - b, b))
    for j in range(n - b):
        for p in range(b):
            acc = np.float32(0)
            for t in range(b):
                acc = fmaf(Li[p, t], M[t, b + j], acc)
            U12[p, j] = bf16(acc)
    for i in range(n - b):
        for p in range(b):
            acc = np.float32(0)
            for t in range(b):
                acc = fmaf(M[b + i, t], Ui[t, p], acc)
            L21[i, p] = bf16(acc)
    M[:b, b:] = U12; M[b:, :b] = L21
    for j in range(b, n):
        for i in range(b, n):
            acc = np.float32(0)
            for p in range(b):
                acc = fmaf(M[i, p], M[p, j], acc)
            M[i, j] = bf16(np.float32(np.float32(M[i, j]) - acc))
    # the trailing block (<= 128) is a base block again
    t = n - b
    if t:
        a = M[b:, b:].astype(np.float32)
        for p in range(t):
            for i in range(p + 1, t):
                a[i, p] = np.float32(a[i, p] / a[p, p])
            for j in range(p + 1, t):
                for i in range(p + 1, t):
                    a[i, j] = fmaf(-a[i, p], a[p, j], a[i, j])
        M[b:, b:] = np.vectorize(bf16)(a)
    return M


@pytest.mark.slow
@pytest.mark.parametrize("n", [2, 37, 136])
def test_rounding_points_rederived(n):
    A, _ = oracle.generate(n, 21)
    LU, _ = oracle.factor(A, oracle.BF16, 128)
    assert np.array_equal(LU, reference_small_lu(A))


def test_two_by_two_closed_form():
    A, _ = oracle.generate(2, 3)
    LU, _ = oracle.factor(A, oracle.BF16, 128)
    a = np.vectorize(bf16)(A).astype(np.float32)
    l = np.float32(a[1, 0] / a[0, 0])
    assert LU[1, 0] == bf16(l)
    assert LU[1, 1] == bf16(fmaf(-l, a[0, 1], a[1, 1]))
    assert LU[0, 0] == bf16(a[0, 0]) and LU[0, 1] == bf16(a[0, 1])


def test_bad_arguments():
    A, _ = oracle.generate(8, 1)
    with pytest.raises(ValueError):
        oracle.factor(A, oracle.BF16, 100)
