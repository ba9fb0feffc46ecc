"""GPU parity of balancing and scaling (hpmxp_balance, hpmxp_factor_scaled,
hpmxp_solve_ir_scaled) against the oracle, through the C interface.

The scales are maxima and powers of two: bit-exact.  The factors of the
balanced matrix: bit-exact on the SIMT engine, within the factor tolerance on
the tensor cores.  The refined x: within 1e-10 of the oracle's, and for BF16
the same bits as the unbalanced solve on the GPU itself (powers of two commute
with every rounding of the path)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2509_19618_gb300 import api, capi  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
ORC_FMT = {capi.BF16: oracle.BF16, capi.FP16: oracle.FP16, capi.FP8_E4M3: oracle.BF16}
U_LOW = {capi.BF16: 2.0**-8, capi.FP16: 2.0**-11, capi.FP8_E4M3: 2.0**-8}


def to_np(m):
    v = m.view()
    if v.dtype in (torch.bfloat16, torch.float16):
        v = v.float()
    return v.double().cpu().numpy()


def system(n, seed, margin=1.0, nrhs=1, distort=True):
    A_o, b_o = oracle.generate(n, seed, margin=margin, nrhs=nrhs)
    if distort and n > 20:
        A_o[:, 7] *= 2.0**-9      # uneven column and row magnitudes
        A_o[11, :] *= 2.0**12
    A = api.ColMajor.from_tensor(torch.from_numpy(A_o), DEV)
    b = api.ColMajor.from_tensor(torch.from_numpy(b_o), DEV)
    return A, b, A_o, b_o


@pytest.mark.parametrize("n", [1, 3, 300, 1000, 4099])
@pytest.mark.parametrize("prec", [capi.BF16, capi.FP16])
def test_balance_bit_exact(n, prec):
    A, _, A_o, _ = system(n, 30 + n)
    rs, cs = api.balance(A, prec)
    torch.cuda.synchronize()
    rs_o, cs_o = oracle.balance(A_o, ORC_FMT[prec])
    assert np.array_equal(rs.cpu().numpy(), rs_o) and np.array_equal(cs.cpu().numpy(), cs_o)


def test_balance_zero_and_nonfinite_lines_get_scale_one():
    n = 256
    A_o, _ = oracle.generate(n, 3)
    A_o[5, :] = 0.0
    A_o[:, 9] = 0.0
    A_o[20, 30] = np.inf
    A = api.ColMajor.from_tensor(torch.from_numpy(A_o), DEV)
    rs, cs = api.balance(A, capi.BF16)
    rs_o, cs_o = oracle.balance(A_o, oracle.BF16)
    assert np.array_equal(rs.cpu().numpy(), rs_o) and np.array_equal(cs.cpu().numpy(), cs_o)
    assert rs_o[5] == 1.0 and cs_o[9] == 1.0 and rs_o[20] == 1.0


@pytest.mark.parametrize("n,nb", [(300, 128), (700, 256), (1031, 512)])
@pytest.mark.parametrize("prec", [capi.BF16, capi.FP16])
def test_factor_scaled_simt_bit_exact(n, nb, prec, monkeypatch):
    monkeypatch.setenv("HPMXP_GEMM_ENGINE", "simt")
    A, _, A_o, _ = system(n, 5)
    sc = api.balance(A, prec)
    LU = api.factor(A, prec, nb, scales=sc)
    torch.cuda.synchronize()
    rs_o, cs_o = oracle.balance(A_o, ORC_FMT[prec])
    LU_o, rc = oracle.factor(A_o, ORC_FMT[prec], nb, rs=rs_o, cs=cs_o)
    assert rc == 0 and np.array_equal(to_np(LU), LU_o)


@pytest.mark.parametrize("n,nb,prec", [(1000, 256, capi.BF16), (2048, 512, capi.FP16), (1500, 512, capi.FP8_E4M3)])
def test_factor_scaled_tensor_cores_within_tolerance(n, nb, prec):
    A, _, A_o, _ = system(n, 6)
    sc = api.balance(A, prec)
    LU = api.factor(A, prec, nb, scales=sc)
    torch.cuda.synchronize()
    rs_o, cs_o = oracle.balance(A_o, ORC_FMT[prec])
    LU_o, _ = oracle.factor(A_o, ORC_FMT[prec], nb, rs=rs_o, cs=cs_o,
                            fmt_update=oracle.E4M3 if prec == capi.FP8_E4M3 else None)
    got = to_np(LU)
    assert np.linalg.norm(got - LU_o) / np.linalg.norm(LU_o) <= U_LOW[prec]


@pytest.mark.parametrize("n,nb,prec,k,pp", [(300, 128, capi.BF16, 1, 0), (1024, 256, capi.BF16, 3, 1),
                                            (2049, 512, capi.FP16, 2, 0), (1500, 512, capi.FP8_E4M3, 1, 1)])
def test_solve_scaled_against_oracle(n, nb, prec, k, pp):
    A, b, A_o, b_o = system(n, 7, nrhs=k)
    sc = api.balance(A, prec)
    LU = api.factor(A, prec, nb, scales=sc)
    p = api.ir_params(precond_fp32=pp, inner_tol=1e-5 if pp else 1e-12)
    x, info, st = api.solve_ir(A, LU, b, prec, p, scales=sc)
    torch.cuda.synchronize()
    sr = api.residual(A, x, b)
    rs_o, cs_o = oracle.balance(A_o, ORC_FMT[prec])
    LU_o, _ = oracle.factor(A_o, ORC_FMT[prec], nb, rs=rs_o, cs=cs_o,
                            fmt_update=oracle.E4M3 if prec == capi.FP8_E4M3 else None)
    X_o, info_o, rc = oracle.solve_ir(A_o, LU_o, b_o, precond_prec=pp, inner_tol=1e-5 if pp else 1e-12,
                                      rs=rs_o, cs=cs_o)
    assert st == capi.OK and rc == 0
    xg = to_np(x)
    # both x have a scaled residual below 16, i.e. a normwise backward error
    # below 16 n eps; two such solutions differ by at most 2 (16 n eps) kappa
    # relative (kappa_inf of the distorted system, computed here), and by no
    # more than 1e-10 relative for the well-conditioned generated systems
    kappa = np.linalg.norm(A_o, np.inf) * np.linalg.norm(np.linalg.inv(A_o), np.inf)
    tol = max(1e-10, 2 * 16 * n * 2.0**-53 * kappa)
    for c in range(k):
        assert sr[c] < 16.0
        assert np.abs(xg[:, c] - X_o[:, c]).max() <= tol * np.abs(X_o[:, c]).max()
        assert abs(info[c]["iters"] - info_o[c]["iters"]) <= 1


@pytest.mark.parametrize("pp", [0, 1])
def test_bf16_balanced_solve_equals_unbalanced_on_gpu(pp):
    n = 2048
    A, b, _, _ = system(n, 8, nrhs=2)
    p = api.ir_params(precond_fp32=pp, inner_tol=1e-5 if pp else 1e-12)
    outs = []
    for bal in (False, True):
        s = api.Solver(n, 2, capi.BF16, nb=256, device=DEV, params=p, balance=bal)
        x, info, st = s(A, b)
        torch.cuda.synchronize()
        assert st == capi.OK
        outs.append((x.view().clone(), [i["iters"] for i in info]))
    assert torch.equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_fp16_out_of_range_system_solves_only_balanced():
    n = 1000
    A, b, A_o, b_o = system(n, 9, margin=1e5, distort=False)
    with pytest.raises(capi.HpmxpError) as e:
        api.factor(A, capi.FP16, 256)
    assert e.value.status == capi.EBREAKDOWN
    s = api.Solver(n, 1, capi.FP16, nb=256, device=DEV, balance=True)
    x, info, st = s(A, b)
    torch.cuda.synchronize()
    assert st == capi.OK and api.residual(A, x, b)[0] < 16.0


def test_full_size_balanced_solve_n32768():
    n = 32768
    A, b = api.generate(n, seed=1, device=DEV)
    s = api.Solver(n, 1, capi.BF16, nb=512, device=DEV, balance=True,
                   params=api.ir_params(precond_fp32=1, inner_tol=1e-5))
    x, info, st = s(A, b)
    torch.cuda.synchronize()
    assert st == capi.OK and api.residual(A, x, b)[0] < 16.0, info
    del A, b, s
    torch.cuda.empty_cache()


def test_scaled_entry_points_reject_one_scale():
    n = 64
    A, b, _, _ = system(n, 1)
    rs, cs = api.balance(A)
    LU = api.ColMajor.empty(n, n, torch.bfloat16, DEV)
    ws = api.workspace(capi.hpmxp_factor_workspace(n, capi.BF16, 128), DEV)
    assert capi.hpmxp_factor_scaled(n, A.ptr, A.ld, capi.BF16, 128, rs.data_ptr(), None, LU.ptr, LU.ld,
                                    ws.data_ptr(), ws.numel(), api.stream_handle()) == capi.EINVAL
    assert capi.hpmxp_balance(n, A.ptr, A.ld, capi.BF16, rs.data_ptr(), rs.data_ptr(),
                              api.stream_handle()) == capi.EINVAL
