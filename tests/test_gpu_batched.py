"""GPU parity of the batched entry points (hpmxp_factor_batched with grouped
kernels, hpmxp_solve_ir_batched in lockstep) through the C interface.

The grouped launches compute every tile exactly as the single-system launches
at depth 128 do, so each system's factors are bit-identical to hpmxp_factor's
(nb = 128, no look-ahead at these sizes), and on the SIMT engine bit-identical
to the oracle's.  The lockstep refinement runs each system's kernels in the
same order as hpmxp_solve_ir, so x and the iteration counts are identical too;
against the oracle x is within 1e-10."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2509_19618_gb300 import api, capi  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
SIZES = [1, 100, 128, 129, 300, 1000, 2049, 256, 777]


def systems(sizes, seed0=70, nrhs=None):
    As, bs = [], []
    for q, n in enumerate(sizes):
        k = nrhs[q] if nrhs else 1
        A, b = api.generate(n, seed=seed0 + q, nrhs=k, device=DEV)
        As.append(A)
        bs.append(b)
    return As, bs


@pytest.mark.parametrize("prec", [capi.BF16, capi.FP16])
def test_factor_batched_equals_single_system_factor(prec):
    As, _ = systems(SIZES)
    LUs, per = api.factor_batched(As, prec)
    torch.cuda.synchronize()
    assert per == [capi.OK] * len(As)
    for A, LU in zip(As, LUs):
        one = api.factor(A, prec, 128)
        torch.cuda.synchronize()
        assert torch.equal(LU.view(), one.view()), A.rows


def test_factor_batched_simt_engine_bit_exact_vs_oracle(monkeypatch):
    monkeypatch.setenv("HPMXP_GEMM_ENGINE", "simt")
    sizes = [1, 129, 300, 700]
    As, _ = systems(sizes, seed0=90)
    LUs, per = api.factor_batched(As, capi.BF16)
    torch.cuda.synchronize()
    for q, n in enumerate(sizes):
        A_o, _ = oracle.generate(n, 90 + q)
        LU_o, _ = oracle.factor(A_o, oracle.BF16, 128)
        got = LUs[q].view().float().double().cpu().numpy()
        assert np.array_equal(got, LU_o), n


def test_factor_batched_reports_each_breakdown():
    sizes = [200, 300, 150]
    As, _ = systems(sizes, seed0=5)
    As[1].view()[0, 0] = 0.0
    LUs, per = api.factor_batched(As, capi.BF16, check=False)
    assert per == [capi.OK, capi.EBREAKDOWN, capi.OK]


@pytest.mark.parametrize("pp", [0, 1])
def test_solve_ir_batched_equals_single_system_solves(pp):
    sizes = [300, 1000, 2049, 128, 700]
    nrhs = [1, 3, 2, 1, 8]
    As, bs = systems(sizes, seed0=40, nrhs=nrhs)
    LUs, _ = api.factor_batched(As, capi.BF16)
    p = api.ir_params(precond_fp32=pp, inner_tol=1e-5 if pp else 1e-12)
    xs, infos, st = api.solve_ir_batched(As, LUs, bs, capi.BF16, p)
    torch.cuda.synchronize()
    assert st == capi.OK
    for q in range(len(sizes)):
        x1, info1, st1 = api.solve_ir(As[q], LUs[q], bs[q], capi.BF16, p)
        torch.cuda.synchronize()
        assert st1 == capi.OK
        assert torch.equal(xs[q].view(), x1.view()), sizes[q]
        assert [i["iters"] for i in infos[q]] == [i["iters"] for i in info1]
        sr = api.residual(As[q], xs[q], bs[q])
        assert np.all(sr < 16.0)


def test_solve_ir_batched_against_oracle():
    sizes = [257, 1024, 1500]
    As, bs = systems(sizes, seed0=11, nrhs=[2, 1, 1])
    LUs, _ = api.factor_batched(As, capi.BF16)
    xs, infos, st = api.solve_ir_batched(As, LUs, bs, capi.BF16)
    torch.cuda.synchronize()
    assert st == capi.OK
    for q, n in enumerate(sizes):
        A_o, b_o = oracle.generate(n, 11 + q, nrhs=bs[q].cols)
        LU_o, _ = oracle.factor(A_o, oracle.BF16, 128)
        X_o, info_o, rc = oracle.solve_ir(A_o, LU_o, b_o)
        xg = xs[q].view().cpu().numpy()
        for c in range(bs[q].cols):
            assert np.abs(xg[:, c] - X_o[:, c]).max() <= 1e-10 * np.abs(X_o[:, c]).max()
            assert abs(infos[q][c]["iters"] - info_o[c]["iters"]) <= 1


def test_batched_rejects_bad_problems():
    As, bs = systems([100])
    LU = api.ColMajor.empty(100, 100, torch.bfloat16, DEV)
    p = api._problem(As[0], LU)
    p.ldlu = 101   # not a multiple of 8
    ws = api.workspace(1 << 20, DEV)
    st, _ = capi.hpmxp_factor_batched([p], capi.BF16, ws.data_ptr(), ws.numel(), api.stream_handle())
    assert st == capi.EINVAL
    st, _ = capi.hpmxp_factor_batched([api._problem(As[0], LU)], capi.FP8_E4M3, ws.data_ptr(), ws.numel(),
                                      api.stream_handle())
    assert st == capi.EINVAL
