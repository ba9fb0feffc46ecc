"""Independent re-derivations of the solver's arithmetic, for pinning the oracle.

Written from the method's description (section "Algorithmic Framework",
Fig. 1, and the readings stated in the oracle's comments), not from the
oracle's code: numpy, vectorised over the entries that do not depend on each
other, with an exact emulation of the fp32 fused multiply-add.  Rounding to
BF16 / E4M3 goes through ``oracle.round_to``, which is pinned on its own
(tests/test_oracle_rounding.py).  Test infrastructure only.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import oracle

F32, F64 = np.float32, np.float64


# ---------------------------------------------------------------------------
# exact fp32 fused multiply-add, elementwise
# ---------------------------------------------------------------------------
def fmaf(a, b, c) -> np.ndarray:
    """fl32(a*b + c) with one rounding, for fp32 a, b, c (arrays broadcast).

    a*b of two fp32 values is exact in fp64; s = fl64(p + c) and its error e
    (Knuth's TwoSum) give the exact sum s + e.  fl32(s) is the correctly
    rounded result unless s is exactly the midpoint of two fp32 neighbours and
    e != 0, in which case the sign of e decides."""
    a = np.asarray(a, dtype=F32).astype(F64)
    b = np.asarray(b, dtype=F32).astype(F64)
    c = np.asarray(c, dtype=F32).astype(F64)
    p = a * b
    s = p + c
    bp = s - c
    e = (p - bp) + (c - (s - bp))
    r = s.astype(F32)
    r64 = r.astype(F64)
    toward = np.where(s > r64, np.inf, -np.inf).astype(F32)
    nb = np.nextafter(r, toward)
    mid = (r64 + nb.astype(F64)) / 2
    tie = (e != 0) & (s == mid) & (s != r64)
    if np.any(tie):
        up = np.where(nb > r, nb, r)
        down = np.where(nb > r, r, nb)
        r = np.where(tie, np.where(e > 0, up, down), r)
    return r


def fma64(a: float, b: float, c: float) -> float:
    """fl64(a*b + c) with one rounding (exact rationals)."""
    v = Fraction(a) * Fraction(b) + Fraction(c)
    f = float(v)                                  # Fraction -> float rounds to nearest even
    return f


def bf16(x) -> np.ndarray:
    x = np.asarray(x, dtype=F64)
    return oracle.round_to(x, oracle.BF16).reshape(x.shape)


def f32(x) -> np.ndarray:
    return np.asarray(x, dtype=F64).astype(F32).astype(F64)


def e4m3(x) -> np.ndarray:
    x = np.asarray(x, dtype=F64)
    return oracle.round_to(x, oracle.E4M3).reshape(x.shape)


# ---------------------------------------------------------------------------
# fp32 Arnoldi product: A truncated toward zero to fp32, fp32 FMAs, j ascending
# ---------------------------------------------------------------------------
def trunc_to_f32(A) -> np.ndarray:
    """fp64 -> fp32 toward zero from the bit pattern: keep the sign, the
    exponent and the top 23 fraction bits (values in the fp32 normal range)."""
    A = np.asarray(A, dtype=F64)
    bits = A.view(np.uint64)
    sign = (bits >> np.uint64(63)).astype(np.uint32)
    exp = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023 + 127
    frac = ((bits >> np.uint64(29)) & np.uint64(0x7FFFFF)).astype(np.uint32)
    assert np.all((exp > 0) & (exp < 255) | (A == 0)), "outside the fp32 normal range"
    out = (sign << np.uint32(31)) | (np.clip(exp, 0, 255).astype(np.uint32) << np.uint32(23)) | frac
    out = np.where(A == 0, sign << np.uint32(31), out)
    return out.astype(np.uint32).view(F32)


def matvec_f32(A, v) -> np.ndarray:
    At = trunc_to_f32(A)
    vf = np.asarray(v, dtype=F64).astype(F32)
    acc = np.zeros(At.shape[0], dtype=F32)
    for j in range(At.shape[1]):
        acc = fmaf(At[:, j], vf[j], acc)
    return acc.astype(F64)


# ---------------------------------------------------------------------------
# preconditioner z = U^{-1} L^{-1} v by substitution, fp32 or fp64
# ---------------------------------------------------------------------------
def precond_f32(LU, v) -> np.ndarray:
    LU = np.asarray(LU, dtype=F64)
    n = LU.shape[0]
    y = np.zeros(n, dtype=F32)
    for i in range(n):                   # unit lower, terms j ascending
        acc = F32(v[i])
        for j in range(i):
            acc = fmaf(-F32(LU[i, j]), y[j], acc)
        y[i] = acc
    for i in range(n - 1, -1, -1):       # upper, terms j ascending, then one division
        acc = y[i]
        for j in range(i + 1, n):
            acc = fmaf(-F32(LU[i, j]), y[j], acc)
        y[i] = F32(acc) / F32(LU[i, i])
    return y.astype(F64)


def precond_f64(LU, v) -> np.ndarray:
    LU = np.asarray(LU, dtype=F64)
    n = LU.shape[0]
    y = [0.0] * n
    for i in range(n):
        acc = float(v[i])
        for j in range(i):
            acc = fma64(-float(LU[i, j]), y[j], acc)
        y[i] = acc
    for i in range(n - 1, -1, -1):
        acc = y[i]
        for j in range(i + 1, n):
            acc = fma64(-float(LU[i, j]), y[j], acc)
        y[i] = acc / float(LU[i, i])
    return np.array(y)


# ---------------------------------------------------------------------------
# the method's blocked LU (BF16 storage, fp32 arithmetic; optional E4M3 update)
# ---------------------------------------------------------------------------
BASE = 128


class MethodLU:
    """Right-looking LU without pivoting with Schur-update depth nb: diagonal
    blocks wider than 128 factored by the same scheme at depth 128; 128-wide
    blocks unblocked in fp32, followed by the fp32 inverses of their stored
    factors; panels by block substitution, each output one fp32 accumulation
    over [W_s | Linv_ss] (rows) or [Z_s ; Uinv_ss] (columns); Schur update one
    fp32 accumulation over the panel width, rounded once into storage."""

    def __init__(self, A, nb: int, fp8_update: bool = False, store=bf16, trail32: bool = False):
        self.st = store                 # rounding to the storage format (bf16; f32 to expose fp32 rounding points)
        self.trail32 = trail32          # 32-bit trailing matrix: top-level Schur results kept in fp32
        self.M = f32(np.asarray(A, dtype=F64)) if trail32 else store(np.asarray(A, dtype=F64))
        self.n = self.M.shape[0]
        self.nb = nb
        self.fp8 = fp8_update
        self.Linv: dict[int, np.ndarray] = {}
        self.Uinv: dict[int, np.ndarray] = {}

    def run(self) -> np.ndarray:
        self.lu_range(0, self.n, self.nb, True)
        return self.M

    # 128-wide (or narrower) diagonal block and its inverses
    def getrf_base(self, k: int, b: int):
        M = self.M
        a = M[k:k + b, k:k + b].astype(F32)
        for p in range(b):
            a[p + 1:, p] = a[p + 1:, p] / a[p, p]
            if p + 1 < b:
                a[p + 1:, p + 1:] = fmaf(-a[p + 1:, p][:, None], a[p, p + 1:][None, :], a[p + 1:, p + 1:])
        M[k:k + b, k:k + b] = self.st(a.astype(F64))
        S = M[k:k + b, k:k + b].astype(F32)          # stored factors, fp32
        # X = L^{-1}: column c, rows r > c: X[r,c] = -sum_{t=c}^{r-1} L[r,t] X[t,c], t ascending
        X = np.zeros((b, b), dtype=F32)
        X[np.arange(b), np.arange(b)] = 1
        cols = np.arange(b)
        for r in range(1, b):
            acc = np.zeros(b, dtype=F32)
            for t in range(r):
                upd = fmaf(-S[r, t], X[t, :], acc)
                acc = np.where(cols <= t, upd, acc)
            X[r, :] = np.where(cols < r, acc, X[r, :])
        # Y = U^{-1}: Y[c,c] = 1/U[c,c]; rows r < c: (-sum_{t=c}^{r+1} U[r,t] Y[t,c]) / U[r,r], t descending
        Y = np.zeros((b, b), dtype=F32)
        Y[np.arange(b), np.arange(b)] = F32(1) / np.diag(S)
        for r in range(b - 2, -1, -1):
            acc = np.zeros(b, dtype=F32)
            for t in range(b - 1, r, -1):
                upd = fmaf(S[r, t], Y[t, :], acc)
                acc = np.where(cols >= t, upd, acc)
            Y[r, :] = np.where(cols > r, (-acc) / S[r, r], Y[r, :])
        self.Linv[k // BASE] = self.st(X.astype(F64))
        self.Uinv[k // BASE] = self.st(Y.astype(F64))

    def row_panel(self, k: int, b: int, c0: int, c1: int):
        M = self.M
        for s0 in range(k, k + b, BASE):
            bs = min(BASE, k + b - s0)
            li = self.Linv[s0 // BASE][:bs, :bs].astype(F32)
            wk = s0 - k
            acc = np.zeros((bs, c1 - c0), dtype=F32)
            if wk:
                W = np.zeros((bs, wk), dtype=F32)
                for t in range(bs):
                    W = fmaf(li[:, t][:, None], M[s0 + t, k:k + wk].astype(F32)[None, :], W)
                W = self.st((-W).astype(F64)).astype(F32)
                for q in range(wk):
                    acc = fmaf(W[:, q][:, None], M[k + q, c0:c1].astype(F32)[None, :], acc)
            for t in range(bs):
                acc = fmaf(li[:, t][:, None], M[s0 + t, c0:c1].astype(F32)[None, :], acc)
            M[s0:s0 + bs, c0:c1] = self.st(acc.astype(F64))

    def col_panel(self, k: int, b: int, r0: int, r1: int):
        M = self.M
        for s0 in range(k, k + b, BASE):
            bs = min(BASE, k + b - s0)
            ui = self.Uinv[s0 // BASE][:bs, :bs].astype(F32)
            zk = s0 - k
            acc = np.zeros((r1 - r0, bs), dtype=F32)
            if zk:
                Z = np.zeros((zk, bs), dtype=F32)
                for t in range(bs):
                    Z = fmaf(M[k:k + zk, s0 + t].astype(F32)[:, None], ui[t, :][None, :], Z)
                Z = self.st((-Z).astype(F64)).astype(F32)
                for q in range(zk):
                    acc = fmaf(M[r0:r1, k + q].astype(F32)[:, None], Z[q, :][None, :], acc)
            for t in range(bs):
                acc = fmaf(M[r0:r1, s0 + t].astype(F32)[:, None], ui[t, :][None, :], acc)
            M[r0:r1, s0:s0 + bs] = self.st(acc.astype(F64))

    def schur(self, k: int, b: int, e: int, top: bool):
        M = self.M
        m = e - (k + b)
        if m <= 0:
            return
        L = M[k + b:e, k:k + b]
        U = M[k:k + b, k + b:e]
        C = M[k + b:e, k + b:e].astype(F32)
        if top and self.fp8:
            acc = self.fp8_product(L, U)
        else:
            acc = np.zeros((m, m), dtype=F32)
            for p in range(b):
                acc = fmaf(L[:, p].astype(F32)[:, None], U[p, :].astype(F32)[None, :], acc)
        M[k + b:e, k + b:e] = (C - acc).astype(F64) if (top and self.trail32) else self.st((C - acc).astype(F64))

    @staticmethod
    def fp8_product(L, U) -> np.ndarray:
        """Per 128 x 128 tile (rows of L / columns of U, 128-deep slices g):
        s = fl32(amax / 448) (1 for a zero tile), q = E4M3(fl32(x / s)); per
        slice the exact E4M3 products accumulate in fp32, and the slices fold
        as acc = fma(acc_g, fl32(sL sU), acc), g ascending."""
        m, b = L.shape
        ng = -(-b // BASE)
        nt = -(-m // BASE)
        qL = np.zeros((m, b), dtype=F32)
        qU = np.zeros((b, m), dtype=F32)
        sL = np.ones((nt, ng), dtype=F32)
        sU = np.ones((ng, nt), dtype=F32)
        for a in range(nt):
            for g in range(ng):
                ri, pj = slice(a * BASE, min(m, (a + 1) * BASE)), slice(g * BASE, min(b, (g + 1) * BASE))
                for isL in (True, False):
                    T = (L[ri, pj] if isL else U[pj, ri]).astype(F32)
                    amax = np.abs(T).max()
                    sc = F32(1) if amax == 0 else F32(amax) / F32(448)
                    q = e4m3((T / sc).astype(F64)).astype(F32)
                    if isL:
                        qL[ri, pj] = q
                        sL[a, g] = sc
                    else:
                        qU[pj, ri] = q
                        sU[g, a] = sc
        rows = np.arange(m) // BASE
        acc = np.zeros((m, m), dtype=F32)
        for g in range(ng):
            ag = np.zeros((m, m), dtype=F32)
            for p in range(g * BASE, min(b, (g + 1) * BASE)):
                ag = fmaf(qL[:, p][:, None], qU[p, :][None, :], ag)
            sc = (sL[rows, g][:, None] * sU[g, rows][None, :]).astype(F32)
            acc = fmaf(ag, sc, acc)
        return acc

    def lu_range(self, k0: int, size: int, NB: int, top: bool):
        e = k0 + size
        for k in range(k0, e, NB):
            b = min(NB, e - k)
            if top and self.trail32:    # the block column and row take their one rounding to storage
                self.M[k:e, k:k + b] = self.st(self.M[k:e, k:k + b])
                self.M[k:k + b, k + b:e] = self.st(self.M[k:k + b, k + b:e])
            if b <= BASE:
                self.getrf_base(k, b)
            else:
                self.lu_range(k, b, BASE, False)
            if k + b >= e:
                break
            self.row_panel(k, b, k + b, e)
            self.col_panel(k, b, k + b, e)
            self.schur(k, b, e, top)


def method_lu(A, nb: int, fp8_update: bool = False, store=bf16, trail32: bool = False) -> np.ndarray:
    return MethodLU(A, nb, fp8_update, store, trail32).run()
