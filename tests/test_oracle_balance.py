"""Pins of the oracle's balancing and scaling (section "Algorithmic Framework":
Theta(n^2) balancing from the HPL harness plus a scaling into the range of the
low-precision format, timed and undone at the end).

Reading: power-of-two row then column equilibration, then the format's scale
(2^12 for FP16, 1 otherwise).  Powers of two make the pins exact: the factors
of diag(rs) A diag(cs) are exact rescalings of the factors of A whenever
nothing leaves the format's normal range, and the refined x is the same bit
for bit; where the unbalanced values do leave FP16's range, balancing is what
makes the solve succeed."""
import numpy as np
import pytest

import oracle

ACCEPT = 16.0


def _is_pow2(v):
    m, _ = np.frexp(v)
    return np.all(m == 0.5)


def test_closed_form_3x3():
    A = np.array([[4.0, -1.0, 0.5],
                  [0.25, 3.0, -0.125],
                  [0.0, 0.0, 0.0]])
    rs, cs = oracle.balance(A, oracle.BF16)
    # row maxima 4, 3, 0 -> 2^-2, 2^-1, 1 (a zero row is left alone)
    assert list(rs) == [0.25, 0.5, 1.0]
    # column maxima of diag(rs) A: 1, 1.5, 0.125 -> 1, 1, 8
    assert list(cs) == [1.0, 1.0, 8.0]
    rs16, cs16 = oracle.balance(A, oracle.FP16)
    assert list(rs16) == [0.25 * 4096, 0.5 * 4096, 4096.0] and list(cs16) == list(cs)


@pytest.mark.parametrize("n,margin,mode", [(300, 1.0, oracle.DOMINANT), (513, 50.0, oracle.DOMINANT),
                                           (200, 1.0, oracle.NONE)])
def test_equilibrated_ranges(n, margin, mode):
    A, _ = oracle.generate(n, 3, margin=margin, mode=mode)
    A[:, 7] *= 2.0**-20          # a column of tiny entries, a row of large ones
    A[11, :] *= 2.0**30
    rs, cs = oracle.balance(A, oracle.BF16)
    assert _is_pow2(rs) and _is_pow2(cs)
    B = rs[:, None] * A * cs[None, :]
    rmax, cmax = np.abs(B).max(axis=1), np.abs(B).max(axis=0)
    assert np.all(cmax >= 1) and np.all(cmax < 2)      # columns last: exactly in [1, 2)
    assert np.all(rmax < 2) and np.all(rmax >= 1)   # column scales are >= 1, so rows keep their [1, 2) maximum


@pytest.mark.parametrize("nb", [128, 256, 512])
@pytest.mark.parametrize("fp8", [False, True])
def test_bf16_factors_are_exact_rescalings(nb, fp8):
    n = 700
    A, b = oracle.generate(n, 3, margin=3.0)
    A[:, 5] *= 2.0**-9
    A[17, :] *= 2.0**12
    rs, cs = oracle.balance(A, oracle.BF16)
    upd = oracle.E4M3 if fp8 else None
    LU, _ = oracle.factor(A, oracle.BF16, nb, fmt_update=upd)
    LUs, rc = oracle.factor(A, oracle.BF16, nb, fmt_update=upd, rs=rs, cs=cs)
    assert rc == 0
    L, U = oracle.split_lu(LU)
    Ls, Us = oracle.split_lu(LUs)
    if not fp8:
        # L' = R L R^-1 and U' = R U C, bit for bit
        assert np.array_equal(Ls, rs[:, None] * L / rs[None, :])
        assert np.array_equal(Us, rs[:, None] * U * cs[None, :])
    else:
        # the per-tile fp8 quantization is not scale-equivariant row by row: only close
        assert np.linalg.norm(Ls @ Us - rs[:, None] * A * cs[None, :]) <= \
            2.0**-7 * np.linalg.norm(rs[:, None] * A * cs[None, :])


@pytest.mark.parametrize("pp,mp", [(0, 0), (1, 0), (1, 1)])
def test_balanced_solve_is_the_unbalanced_solve_bit_for_bit(pp, mp):
    n = 600
    A, b = oracle.generate(n, 4, nrhs=2)
    rs, cs = oracle.balance(A, oracle.BF16)
    LU, _ = oracle.factor(A, oracle.BF16, 256)
    LUs, _ = oracle.factor(A, oracle.BF16, 256, rs=rs, cs=cs)
    kw = dict(precond_prec=pp, matvec_prec=mp, inner_tol=1e-5 if pp else 1e-12)
    X, i1, rc1 = oracle.solve_ir(A, LU, b, **kw)
    Xs, i2, rc2 = oracle.solve_ir(A, LUs, b, rs=rs, cs=cs, **kw)
    assert rc1 == rc2 == 0 and i1 == i2
    assert np.array_equal(X, Xs)
    v = b[:, 0]
    assert np.array_equal(oracle.precond(LU, v, pp), oracle.precond(LUs, v, pp, rs=rs, cs=cs))


def test_fp16_overflow_needs_scaling():
    # a diagonal near 1e5 does not fit FP16 (largest finite 65504): the cast
    # overflows and the factorization breaks down; balanced, the system solves
    A, b = oracle.generate(400, 5, margin=1e5)
    _, rc = oracle.factor(A, oracle.FP16, 128)
    assert rc == 1
    rs, cs = oracle.balance(A, oracle.FP16)
    LU, rc = oracle.factor(A, oracle.FP16, 128, rs=rs, cs=cs)
    assert rc == 0
    X, info, st = oracle.solve_ir(A, LU, b, rs=rs, cs=cs)
    assert st == 0 and oracle.scaled_residual(A, X, b)[0] < ACCEPT


def test_fp16_underflow_needs_scaling():
    # the same system times 2^-30: every entry is below FP16's smallest
    # subnormal (2^-24) and casts to zero; balanced, the system solves
    A, b = oracle.generate(300, 6)
    A *= 2.0**-30
    _, rc = oracle.factor(A, oracle.FP16, 128)
    assert rc == 1
    rs, cs = oracle.balance(A, oracle.FP16)
    LU, rc = oracle.factor(A, oracle.FP16, 128, rs=rs, cs=cs)
    assert rc == 0
    X, info, st = oracle.solve_ir(A, LU, b, rs=rs, cs=cs)
    assert st == 0 and oracle.scaled_residual(A, X, b)[0] < ACCEPT


def test_scales_given_together():
    A, _ = oracle.generate(8, 1)
    rs, cs = oracle.balance(A)
    with pytest.raises(ValueError):
        oracle.factor(A, oracle.BF16, 128, rs=rs)
