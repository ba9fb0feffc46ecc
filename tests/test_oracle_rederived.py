"""Pins of the oracle's fp32 pieces and of its blocked-LU scheme against an
independent, vectorised re-derivation written from the method's description
(tests/rederive.py), bit for bit; and the distance of the method's
inverse-based panels from the plain reading of Fig. 1 (fp32 substitution).

Each re-derivation fixes a rounding point the oracle must honour, so a
plausible slip in the oracle (rounding instead of truncating A to fp32, an fp64
product where fp32 is meant, a wrong tile index or slice order in the FP8
update, a transposed W / Z operand) changes at least one bit here."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import rederive as R
from inputs import vectors

U_BF16 = 2.0**-8


# ---------------------------------------------------------------------------
# the emulated fp32 FMA itself, against exact rationals
# ---------------------------------------------------------------------------
def _correctly_rounded(a, b, c) -> np.float32:
    v = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    r = np.float32(float(v))
    best = None
    for cand in (np.nextafter(r, np.float32(-np.inf)), r, np.nextafter(r, np.float32(np.inf))):
        d = abs(Fraction(float(cand)) - v)
        key = (d, int(np.array(cand).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return best[1]


def test_fmaf_emulation_against_rationals():
    g = np.random.default_rng(7)
    a = g.standard_normal(600).astype(np.float32)
    b = g.standard_normal(600).astype(np.float32)
    c = (g.standard_normal(600) * np.exp2(g.integers(-40, 40, 600))).astype(np.float32)
    # near-ties: c = -(a*b) rounded, so that the exact sum is tiny and the fp64
    # sum can land on an fp32 midpoint; and products whose sum is a midpoint
    c[:100] = -(a[:100].astype(np.float64) * b[:100]).astype(np.float32)
    a[100:150] = np.float32(1 + 2.0**-12)
    b[100:150] = np.float32(1 + 2.0**-12)
    c[100:150] = np.float32(2.0**-24) * np.arange(50, dtype=np.float32)
    got = R.fmaf(a, b, c)
    for i in range(a.size):
        assert got[i] == _correctly_rounded(a[i], b[i], c[i]), i


# ---------------------------------------------------------------------------
# fp32 Arnoldi product
# ---------------------------------------------------------------------------
def test_matvec_f32_truncates_toward_zero():
    # 1 + 2^-23 + 2^-25 rounds up to 1 + 2^-22 but truncates to 1 + 2^-23
    a = 1 + 2.0**-23 + 2.0**-25 + 2.0**-26
    A = np.array([[a, -a], [0.0, 1.0]])
    w = oracle.matvec_f32(A, np.array([1.0, 0.0]))
    assert w[0] == 1 + 2.0**-23 and w[1] == 0.0
    w = oracle.matvec_f32(A, np.array([0.0, 1.0]))
    assert w[0] == -(1 + 2.0**-23) and w[1] == 1.0


@pytest.mark.parametrize("n,seed", [(150, 4), (257, 9)])
def test_matvec_f32_rederived(n, seed):
    A, _ = oracle.generate(n, seed)
    v = vectors(n, 1, seed + 1)[:, 0]
    want = R.matvec_f32(A, v)
    got = oracle.matvec_f32(A, v)
    assert np.array_equal(got, want)
    # and it is not the fp64 product, nor the product of the rounded-to-nearest A
    assert not np.array_equal(got, A @ v)
    Ar = A.astype(np.float32).astype(np.float64)
    assert not np.array_equal(got, R.matvec_f32(Ar, v)) or np.array_equal(Ar, R.trunc_to_f32(A))


# ---------------------------------------------------------------------------
# preconditioner by substitution
# ---------------------------------------------------------------------------
def test_precond_f32_rederived():
    n = 150
    A, _ = oracle.generate(n, 5)
    LU, _ = oracle.factor(A, oracle.BF16, 128)
    v = vectors(n, 1, 6)[:, 0]
    got = oracle.precond(LU, v, prec=1)
    assert np.array_equal(got, R.precond_f32(LU, v))
    assert not np.array_equal(got, oracle.precond(LU, v, prec=0))


def test_precond_f64_rederived():
    n = 48
    A, _ = oracle.generate(n, 5)
    LU, _ = oracle.factor(A, oracle.BF16, 128)
    v = vectors(n, 1, 7)[:, 0]
    assert np.array_equal(oracle.precond(LU, v, prec=0), R.precond_f64(LU, v))


# ---------------------------------------------------------------------------
# the method's blocked LU, every rounding point
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,nb,fp8", [
    (300, 256, False),   # two 128 sub-blocks in the diagonal block: the W / Z operands
    (456, 256, True),    # E4M3 update: two 128-row tiles (128 + 72) and two 128-deep slices
    (640, 512, True),    # four sub-blocks and four slices
    (520, 128, False),   # several depth-128 steps and a ragged last block
])
def test_blocked_lu_rederived(n, nb, fp8):
    A, _ = oracle.generate(n, 21)
    LU, rc = oracle.factor(A, oracle.BF16, nb, fmt_update=oracle.E4M3 if fp8 else None)
    assert rc == 0
    want = R.method_lu(A, nb, fp8)
    bad = np.argwhere(LU != want)
    assert bad.size == 0, (bad[:5], LU[tuple(bad[0])], want[tuple(bad[0])])


@pytest.mark.parametrize("n,nb,fp8", [(456, 256, True), (300, 256, False)])
def test_blocked_lu_rederived_fp32_storage(n, nb, fp8):
    """The same scheme with every stored value kept in fp32 instead of BF16:
    a BF16 store can absorb a one-ulp fp32 difference (e.g. the FP8 slices
    folded with a multiply and an add instead of one FMA), an fp32 store
    shows every fp32 rounding point."""
    A, _ = oracle.generate(n, 21)
    LU, rc = oracle.factor(A, oracle.FP32, nb, fmt_update=oracle.E4M3 if fp8 else None)
    assert rc == 0
    assert np.array_equal(LU, R.method_lu(A, nb, fp8, store=R.f32))


# ---------------------------------------------------------------------------
# 32-bit trailing matrix (Fig. 1 with fp32 storage of the matrix being updated)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,nb", [(300, 128), (456, 256), (520, 128)])
def test_trail32_rederived(n, nb):
    A, _ = oracle.generate(n, 22)
    LU, rc = oracle.factor(A, oracle.BF16, nb, trail32=True)
    assert rc == 0
    assert np.array_equal(LU, R.method_lu(A, nb, trail32=True))


def test_trail32_without_schur_steps_is_the_method_on_the_fp32_input():
    # nb >= n: no top-level Schur update, so the only difference from the
    # method is the input's rounding to fp32 first
    A, _ = oracle.generate(300, 23)
    LU, _ = oracle.factor(A, oracle.BF16, 512, trail32=True)
    want, _ = oracle.factor(oracle.round_to(A, oracle.FP32), oracle.BF16, 512)
    assert np.array_equal(LU, want)


@pytest.mark.parametrize("fmt", [oracle.BF16, oracle.FP16])
def test_trail32_error_bounds_and_refinement(fmt):
    n = 900
    A, b = oracle.generate(n, 24)
    LU, rc = oracle.factor(A, fmt, 256, trail32=True)
    assert rc == 0 and np.array_equal(oracle.round_to(LU, fmt), LU)
    L, U = oracle.split_lu(LU)
    u = 2.0**-8 if fmt == oracle.BF16 else 2.0**-11
    assert np.linalg.norm(L @ U - A) / np.linalg.norm(A) <= u
    X, info, rc = oracle.solve_ir(A, LU, b)
    assert rc == 0 and oracle.scaled_residual(A, X, b)[0] < 16
    # it differs from rounding the trailing matrix at every step
    LU16, _ = oracle.factor(A, fmt, 256)
    assert not np.array_equal(LU, LU16)


# ---------------------------------------------------------------------------
# the method's scheme against the plain reading of Fig. 1
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [700, 1100])
@pytest.mark.parametrize("nb", [128, 256, 512])
def test_method_within_bound_of_plain_substitution_reading(n, nb):
    """Inverse-based panels (the method) vs fp32 substitution (plain Fig. 1):
    both store every entry in BF16, so they may differ by rounding only.
    Measured: 1.7e-5 (nb 128) to 4.9e-5 (nb 512) relative at n = 700; the
    bound asserted is 2^-12 (u_bf16 / 16).  Both reconstruct A equally well
    and need the same GMRES-IR iterations (within one)."""
    A, b = oracle.generate(n, 3)
    LU, _ = oracle.factor(A, oracle.BF16, nb)
    LP, rc = oracle.factor_plain(A, oracle.BF16, nb)
    assert rc == 0
    assert np.array_equal(oracle.round_to(LP, oracle.BF16), LP)
    rel = np.linalg.norm(LU - LP) / np.linalg.norm(LP)
    assert 0 < rel <= 2.0**-12
    rec = [np.linalg.norm(L @ U - A) / np.linalg.norm(A) for L, U in (oracle.split_lu(LU), oracle.split_lu(LP))]
    assert rec[0] <= U_BF16 and abs(rec[0] - rec[1]) <= 0.01 * rec[1]
    _, i_m, rc_m = oracle.solve_ir(A, LU, b)
    _, i_p, rc_p = oracle.solve_ir(A, LP, b)
    assert rc_m == 0 and rc_p == 0 and abs(i_m[0]["iters"] - i_p[0]["iters"]) <= 1


@pytest.mark.parametrize("n,nb", [(3, 128), (300, 128), (700, 256), (1100, 512), (300, 64), (130, 64)])
def test_plain_reading_exact_arithmetic_is_doolittle(n, nb):
    from test_oracle_lu import doolittle
    A, _ = oracle.generate(n, 5)
    LP, rc = oracle.factor_plain(A, oracle.FP64, nb)
    assert rc == 0
    assert np.allclose(LP, doolittle(A), rtol=1e-12, atol=1e-14 * np.abs(A).max())


def test_plain_reading_exact_case_is_textbook():
    # with nb >= n the plain reading is one unblocked fp32 factorization: its
    # 2 x 2 case is the closed form
    A, _ = oracle.generate(2, 3)
    LP, _ = oracle.factor_plain(A, oracle.BF16, 128)
    a = R.bf16(A).astype(np.float32)
    l = np.float32(a[1, 0] / a[0, 0])
    assert LP[1, 0] == R.bf16(l) and LP[1, 1] == R.bf16(R.fmaf(-l, a[0, 1], a[1, 1]))
