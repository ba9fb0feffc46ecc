"""The bounded device waits' failure path, made to run out on purpose.

A short wait budget (hpmxp_test_set_wait_budget) makes the preconditioner's
CTAs give up on blocks their peers have not published yet, and the tensor-core
GEMM's pipeline give up on stages that have not filled yet.  Nothing is
missing and nothing faults: the waits simply run out.  Each call must then
return HPMXP_ETIMEOUT (or set the timeout bit of its status word), and the
next call on the same stream with the default budget must give the right
answer again (the GPU context is intact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from inputs import vectors  # noqa: E402
from paper_2509_19618_gb300 import api, capi  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
SHORT = (1, 0)   # one re-poll, no time: a wait gives up unless its data is already there


class short_budget:
    def __enter__(self):
        assert capi.hpmxp_test_set_wait_budget(*SHORT) == capi.OK

    def __exit__(self, *a):
        assert capi.hpmxp_test_set_wait_budget(0, 0) == capi.OK


def test_wait_budget_arguments():
    assert capi.hpmxp_test_set_wait_budget(0, 5) == capi.EINVAL
    assert capi.hpmxp_test_set_wait_budget(-1, 0) == capi.EINVAL
    assert capi.hpmxp_test_set_wait_budget(1, 3_000_000_000) == capi.EINVAL
    assert capi.hpmxp_test_set_wait_budget(0, 0) == capi.OK


@pytest.mark.parametrize("fp32", [0, 1])
def test_precond_wait_runs_out_then_recovers(fp32):
    n, k = 4096, 2
    A_o, _ = oracle.generate(n, 9)
    LU_o, _ = oracle.factor(A_o, oracle.BF16, 128)
    LU = api.ColMajor.from_tensor(torch.from_numpy(LU_o), DEV, dtype=torch.bfloat16)
    V = vectors(n, k, 21)
    v = api.ColMajor.from_tensor(torch.from_numpy(V), DEV)
    ws = api.workspace(capi.hpmxp_solve_workspace(n, k, 1), DEV)

    def apply():
        z = api.ColMajor.empty(n, k, torch.float64, DEV)
        st = capi.hpmxp_test_precond(n, LU.ptr, LU.ld, capi.BF16, v.ptr, v.ld, z.ptr, z.ld, k, fp32,
                                     ws.data_ptr(), ws.numel(), api.stream_handle())
        torch.cuda.synchronize()
        return st, z

    with short_budget():
        st, _ = apply()
    assert st == capi.ETIMEOUT
    st, z = apply()
    assert st == capi.OK
    got = z.view().cpu().numpy()
    for c in range(k):
        want = oracle.precond(LU_o, V[:, c], prec=fp32)
        tol = 1e-5 if fp32 else 1e-13
        assert np.abs(got[:, c] - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("M,N,K", [(2048, 2048, 512), (1024, 768, 128)])
def test_gemm_wait_runs_out_then_recovers(M, N, K):
    g = np.random.default_rng(M + K)
    bf = lambda x: oracle.round_to(x, oracle.BF16)  # noqa: E731
    A = bf(g.uniform(-1, 1, (M, K)))
    B = bf(g.uniform(-1, 1, (N, K)))
    C0 = bf(g.uniform(-64, 64, (M, N)))
    tA = torch.from_numpy(A).to(DEV, torch.bfloat16).contiguous()
    tB = torch.from_numpy(B).to(DEV, torch.bfloat16).contiguous()
    status = torch.zeros(1, dtype=torch.int32, device=DEV)

    def run():
        C = api.ColMajor.from_tensor(torch.from_numpy(C0), DEV, dtype=torch.bfloat16)
        status.zero_()
        st = capi.hpmxp_test_gemm(M, N, K, tA.data_ptr(), K, tB.data_ptr(), K, C.ptr, C.ld, None, 0, 0, 1.0, 0, 0,
                                  None, 0, None, 0, 0, status.data_ptr(), api.stream_handle())
        torch.cuda.synchronize()
        return st, int(status.item()), C

    with short_budget():
        st, word, _ = run()
    assert st == capi.OK and word == 1        # the timeout bit, nothing else
    st, word, C = run()
    assert st == capi.OK and word == 0
    got = C.view().float().double().cpu().numpy()
    want = C0 - A @ B.T
    ulp = np.spacing(np.abs(bf(want)).astype(np.float32)).astype(np.float64) * 2**16
    assert np.all(np.abs(got - want) <= ulp + 1e-5 * np.abs(A).sum(1)[:, None].max())


def test_gemm_fp8_wait_runs_out_then_recovers():
    # E4M3 operands, four 128-deep slices: the per-slice accumulator waits
    M, N, K = 1024, 1024, 512
    g = np.random.default_rng(5)
    codes = lambda r, c: (g.integers(0, 0x60, size=(r, c), dtype=np.uint8)  # noqa: E731
                          | (g.integers(0, 2, size=(r, c), dtype=np.uint8) << 7))
    qa, qb = codes(M, K), codes(N, K)
    sa = np.ones((M // 128, K // 128), np.float32)
    sb = np.ones((N // 128, K // 128), np.float32)
    C0 = oracle.round_to(g.uniform(-64, 64, (M, N)), oracle.BF16)
    tA, tB = torch.from_numpy(qa).to(DEV), torch.from_numpy(qb).to(DEV)
    tsa, tsb = torch.from_numpy(sa).to(DEV), torch.from_numpy(sb).to(DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)

    def run(eng):
        C = api.ColMajor.from_tensor(torch.from_numpy(C0), DEV, dtype=torch.bfloat16)
        status.zero_()
        st = capi.hpmxp_test_gemm(M, N, K, tA.data_ptr(), K, tB.data_ptr(), K, C.ptr, C.ld, None, 0, 0, 1.0, 0, 1,
                                  tsa.data_ptr(), K // 128, tsb.data_ptr(), K // 128, eng, status.data_ptr(),
                                  api.stream_handle())
        torch.cuda.synchronize()
        return st, int(status.item()), C.view().float().double().cpu().numpy()

    with short_budget():
        st, word, _ = run(0)
    assert st == capi.OK and word == 1        # the timeout bit, nothing else
    st, word, got = run(0)
    assert st == capi.OK and word == 0
    st, word, simt = run(1)
    assert st == capi.OK and word == 0
    assert np.all(np.abs(got - simt) <= 2.0**-7 * np.abs(simt) + 0.5)


def test_solve_reports_timeout_then_recovers():
    n = 2048
    A, b = api.generate(n, seed=11, device=DEV)
    s = api.Solver(n, 1, capi.BF16, nb=256, device=DEV)
    with short_budget():
        with pytest.raises(capi.HpmxpError) as e:
            s.factor(A)
        assert e.value.status == capi.ETIMEOUT
    s.factor(A)
    assert s.factor_status == capi.OK
    with short_budget():
        with pytest.raises(capi.HpmxpError) as e:
            s.solve(A, b)
        assert e.value.status == capi.ETIMEOUT
    x, info, st = s.solve(A, b)
    torch.cuda.synchronize()
    assert st == capi.OK and api.residual(A, x, b)[0] < 16.0
