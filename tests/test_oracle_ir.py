"""Pins of the oracle's GMRES-IR and backward-error check (section
"Algorithmic Framework") against closed forms, exact rational solves and the
paper's qualitative claims (section "Experimental Results")."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from inputs import vectors

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
EPS = GOLDEN["eps"]["value"]
ACCEPT = GOLDEN["accept_threshold"]["value"]
MAXIT = GOLDEN["max_iters"]["value"]


def exact_solve(A, b):
    """Gaussian elimination with partial pivoting in exact rational arithmetic."""
    n = A.shape[0]
    M = [[Fraction(float(A[i, j])) for j in range(n)] + [Fraction(float(b[i]))] for i in range(n)]
    for p in range(n):
        piv = max(range(p, n), key=lambda i: abs(M[i][p]))
        M[p], M[piv] = M[piv], M[p]
        for i in range(p + 1, n):
            f = M[i][p] / M[p][p]
            if f:
                for j in range(p, n + 1):
                    M[i][j] -= f * M[p][j]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))
        x[i] = s / M[i][i]
    return x


def test_constants_from_the_paper():
    assert EPS == 2.0**-53 and ACCEPT == 16.0 and MAXIT == 50


def test_n1_closed_form():
    A, b = oracle.generate(1, 4, margin=3.0)
    assert A[0, 0] == 3.0  # no off-diagonal: the diagonal is the margin
    LU, _ = oracle.factor(A, oracle.BF16, 128)
    X, info, rc = oracle.solve_ir(A, LU, b)
    assert rc == 0 and abs(X[0, 0] - b[0, 0] / 3.0) <= 2 * EPS * abs(X[0, 0])


def test_n2_cramer():
    A, b = oracle.generate(2, 9)
    LU, _ = oracle.factor(A, oracle.BF16, 128)
    X, info, rc = oracle.solve_ir(A, LU, b)
    F = [[Fraction(float(v)) for v in row] for row in A]
    fb = [Fraction(float(v)) for v in b[:, 0]]
    det = F[0][0] * F[1][1] - F[0][1] * F[1][0]
    x0 = (fb[0] * F[1][1] - F[0][1] * fb[1]) / det
    x1 = (F[0][0] * fb[1] - fb[0] * F[1][0]) / det
    assert rc == 0
    for got, want in [(X[0, 0], x0), (X[1, 0], x1)]:
        assert abs(Fraction(float(got)) - want) <= 8 * EPS * max(abs(x0), abs(x1))


@pytest.mark.parametrize("n", [3, 8, 16, 33, 64])
def test_small_against_exact_rational_solution(n):
    A, b = oracle.generate(n, 100 + n)
    LU, _ = oracle.factor(A, oracle.BF16, 128)
    X, info, rc = oracle.solve_ir(A, LU, b)
    assert rc == 0 and info[0]["status"] == 0
    xe = exact_solve(A, b[:, 0])
    kappa = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
    err = max(abs(Fraction(float(X[i, 0])) - xe[i]) for i in range(n))
    assert float(err) / float(max(abs(v) for v in xe)) <= 64 * kappa * EPS


@pytest.mark.parametrize("fmt,nb,n,upd", [(oracle.BF16, 128, 1024, None), (oracle.BF16, 256, 777, None),
                                          (oracle.BF16, 512, 1100, None), (oracle.FP16, 128, 513, None),
                                          (oracle.BF16, 256, 900, oracle.E4M3)])
def test_converges_below_threshold(fmt, nb, n, upd):
    A, b = oracle.generate(n, 1, nrhs=3)
    LU, _ = oracle.factor(A, fmt, nb, fmt_update=upd)
    X, info, rc = oracle.solve_ir(A, LU, b)
    assert rc == 0
    sr = oracle.scaled_residual(A, X, b)
    for c in range(3):
        assert info[c]["status"] == 0 and info[c]["iters"] <= MAXIT
        assert sr[c] < ACCEPT and info[c]["scaled_resid"] == pytest.approx(sr[c])
        assert 1 <= info[c]["iters"] <= 8


def test_exact_factors_need_no_refinement():
    A, b = oracle.generate(300, 2)
    LU, _ = oracle.factor(A, oracle.FP64, 128)
    X, info, rc = oracle.solve_ir(A, LU, b)
    assert rc == 0 and info[0]["outer"] == 0 and info[0]["iters"] == 0


@pytest.mark.parametrize("pp,mp", [(1, 1), (1, 0), (0, 1)])
def test_fp32_inner_operator_options_converge(pp, mp):
    A, b = oracle.generate(700, 3)
    LU, _ = oracle.factor(A, oracle.BF16, 256)
    X, info, rc = oracle.solve_ir(A, LU, b, precond_prec=pp, matvec_prec=mp)
    assert rc == 0 and oracle.scaled_residual(A, X, b)[0] < ACCEPT


def test_scaled_residual_matches_definition():
    n = 50
    A, b = oracle.generate(n, 4)
    x = vectors(n, 1, 4)[:, 0]
    r = np.array([Fraction(float(b[i, 0])) - sum(Fraction(float(A[i, j])) * Fraction(float(x[j]))
                                                  for j in range(n)) for i in range(n)])
    rn = float(max(abs(v) for v in r))
    want = rn / ((np.linalg.norm(A, np.inf) * np.abs(x).max() + np.abs(b).max()) * n * EPS)
    got = oracle.scaled_residual(A, x, b[:, 0])[0]
    assert got == pytest.approx(want, rel=1e-6)
    rv = oracle.residual_vec(A, x, b[:, 0])
    assert np.max(np.abs(rv - r.astype(float))) <= n * EPS * np.abs(A).sum(axis=1).max() * np.abs(x).max()


def test_iteration_cap_reports_failure():
    # unscaled uniform entries without pivoting: the refinement cannot recover
    # (catastrophic growth, section "Experimental Results", Fig. 4)
    A, b = oracle.generate(400, 1, mode=oracle.NONE)
    LU, _ = oracle.factor(A, oracle.BF16, 128)
    X, info, rc = oracle.solve_ir(A, LU, b, max_iters=MAXIT)
    assert rc == 4 and info[0]["status"] == 4 and info[0]["iters"] == MAXIT


def test_no_pivoting_loses_orders_of_magnitude_on_unscaled_matrices():
    # Figs. 3-4: fp64 LU without pivoting on uniform matrices without diagonal
    # scaling gives residual norms orders of magnitude above pivoted LU.
    n = 512
    ratios = []
    for seed in range(3):
        A, b = oracle.generate(n, 50 + seed, mode=oracle.NONE)
        LU, _ = oracle.factor(A, oracle.FP64, 128)
        x_np = oracle.precond(LU, b[:, 0])
        x_pp = np.linalg.solve(A, b[:, 0])
        ratios.append(np.abs(A @ x_np - b[:, 0]).max() / np.abs(A @ x_pp - b[:, 0]).max())
    assert np.median(ratios) >= 10.0
    # with the sqrt(n) diagonal scaling the gap closes
    A, b = oracle.generate(n, 50, mode=oracle.SQRTN)
    LU, _ = oracle.factor(A, oracle.FP64, 128)
    x_np = oracle.precond(LU, b[:, 0])
    x_pp = np.linalg.solve(A, b[:, 0])
    assert np.abs(A @ x_np - b[:, 0]).max() <= 10 * np.abs(A @ x_pp - b[:, 0]).max()


def test_precond_exact_on_triangular_product():
    n = 40
    LU, _ = oracle.factor(oracle.generate(n, 6)[0], oracle.BF16, 128)
    L, U = oracle.split_lu(LU)
    v = vectors(n, 1, 8)[:, 0]
    z = oracle.precond(LU, v)
    assert np.allclose(L @ (U @ z), v, rtol=0, atol=1e-13 * np.abs(v).max())
