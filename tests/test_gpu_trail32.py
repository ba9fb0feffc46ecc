"""GPU parity of the 32-bit trailing matrix variant (Fig. 1 with fp32 storage
of the matrix being updated: HPMXP_BF16_TRAIL32 / HPMXP_FP16_TRAIL32) and of
the GEMM engines' fp32-C subtract mode it uses, through the C interface.

The SIMT engine keeps the oracle's accumulation order: bit-exact.  The
tensor-core engine: the factor tolerance u_low (and 8 n u_low), the fp32 C
product within fp32 rounding of the exact product."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2509_19618_gb300 import api, capi  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
FMT = {capi.BF16_TRAIL32: oracle.BF16, capi.FP16_TRAIL32: oracle.FP16}
U_LOW = {capi.BF16_TRAIL32: 2.0**-8, capi.FP16_TRAIL32: 2.0**-11}


def to_np(m):
    v = m.view()
    if v.dtype in (torch.bfloat16, torch.float16):
        v = v.float()
    return v.double().cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 128, 128), (200, 333, 256), (1000, 700, 512), (2000, 5000, 256)])
@pytest.mark.parametrize("eng", [0, 1])
def test_gemm_fp32_c(M, N, K, eng):
    g = np.random.default_rng(M + N + K)
    bf = lambda x: oracle.round_to(x, oracle.BF16)  # noqa: E731
    A = bf(g.uniform(-1, 1, (M, K)))
    B = bf(g.uniform(-1, 1, (N, K)))
    C0 = g.uniform(-64, 64, (M, N)).astype(np.float32).astype(np.float64)
    tA = torch.from_numpy(A).to(DEV, torch.bfloat16).contiguous()
    tB = torch.from_numpy(B).to(DEV, torch.bfloat16).contiguous()
    C = api.ColMajor.from_tensor(torch.from_numpy(C0), DEV, dtype=torch.float32, align=4)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = capi.hpmxp_test_gemm(M, N, K, tA.data_ptr(), K, tB.data_ptr(), K, C.ptr, C.ld, None, 0, 2, 1.0, 0, 0,
                              None, 0, None, 0, eng, status.data_ptr(), api.stream_handle())
    assert st == capi.OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = C.view().double().cpu().numpy()
    want = C0 - A @ B.T
    # fp32 accumulation of K exact products, one fp32 subtraction
    bound = (K + 2) * 2.0**-24 * (np.abs(A) @ np.abs(B).T + np.abs(C0))
    assert np.all(np.abs(got - want) <= bound)


def test_gemm_fp32_c_rejects_row_copy():
    st = capi.hpmxp_test_gemm(128, 128, 128, 16, 128, 16, 128, 16, 128, 16, 128, 2, 1.0, 0, 0,
                              None, 0, None, 0, 0, 16, api.stream_handle())
    assert st == capi.EINVAL


@pytest.mark.parametrize("n,nb", [(300, 128), (700, 256), (1031, 512), (1300, 256)])
@pytest.mark.parametrize("prec", [capi.BF16_TRAIL32, capi.FP16_TRAIL32])
def test_factor_trail32_simt_bit_exact(n, nb, prec, monkeypatch):
    monkeypatch.setenv("HPMXP_GEMM_ENGINE", "simt")
    A_o, _ = oracle.generate(n, 60 + n)
    A = api.ColMajor.from_tensor(torch.from_numpy(A_o), DEV)
    LU = api.factor(A, prec, nb)
    torch.cuda.synchronize()
    LU_o, rc = oracle.factor(A_o, FMT[prec], nb, trail32=True)
    assert rc == 0
    assert LU.view().dtype == (torch.float16 if prec == capi.FP16_TRAIL32 else torch.bfloat16)
    assert np.array_equal(to_np(LU), LU_o)


@pytest.mark.parametrize("n,nb", [(1031, 128), (2048, 512), (3000, 256)])
@pytest.mark.parametrize("prec", [capi.BF16_TRAIL32, capi.FP16_TRAIL32])
def test_factor_trail32_tensor_cores_within_tolerance(n, nb, prec):
    A_o, _ = oracle.generate(n, 61 + n)
    A = api.ColMajor.from_tensor(torch.from_numpy(A_o), DEV)
    LU = api.factor(A, prec, nb)
    torch.cuda.synchronize()
    LU_o, _ = oracle.factor(A_o, FMT[prec], nb, trail32=True)
    got = to_np(LU)
    rel = np.linalg.norm(got - LU_o) / np.linalg.norm(LU_o)
    assert rel <= 8 * n * U_LOW[prec] and rel <= U_LOW[prec]
    L, U = oracle.split_lu(got)
    assert np.linalg.norm(L @ U - A_o) / np.linalg.norm(A_o) <= 2 * U_LOW[prec]


@pytest.mark.parametrize("n,nb,prec,k", [(1024, 256, capi.BF16_TRAIL32, 2), (2049, 512, capi.FP16_TRAIL32, 1)])
def test_solve_trail32_against_oracle(n, nb, prec, k):
    A, b = api.generate(n, seed=n + 5, nrhs=k, device=DEV)
    LU = api.factor(A, prec, nb)
    x, info, st = api.solve_ir(A, LU, b, prec)
    torch.cuda.synchronize()
    sr = api.residual(A, x, b)
    A_o, b_o = oracle.generate(n, n + 5, nrhs=k)
    LU_o, _ = oracle.factor(A_o, FMT[prec], nb, trail32=True)
    X_o, info_o, rc = oracle.solve_ir(A_o, LU_o, b_o)
    assert st == capi.OK and rc == 0
    xg = to_np(x)
    for c in range(k):
        assert sr[c] < 16.0
        assert np.abs(xg[:, c] - X_o[:, c]).max() <= 1e-10 * np.abs(X_o[:, c]).max()
        assert abs(info[c]["iters"] - info_o[c]["iters"]) <= 1


def test_full_size_trail32_solve_n32768():
    n = 32768
    A, b = api.generate(n, seed=1, device=DEV)
    s = api.Solver(n, 1, capi.BF16_TRAIL32, nb=512, device=DEV,
                   params=api.ir_params(precond_fp32=1, inner_tol=1e-5))
    x, info, st = s(A, b)
    torch.cuda.synchronize()
    assert st == capi.OK and api.residual(A, x, b)[0] < 16.0, info
    del A, b, s
    torch.cuda.empty_cache()
