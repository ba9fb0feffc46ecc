"""GPU parity of the fp64 LU without pivoting used by the study of section
"Experimental Results" (Figs. 2-4), and the study's qualitative claims.

hpmxp_lu_f64 follows the plain order of Fig. 1 with block width 64 in fp64,
which is exactly the oracle's plain reading in fp64 (pinned against Doolittle
in the oracle tests): bit-exact.  Its solve against the oracle's fp64
substitution: within 1e-13 relative on the well-conditioned systems."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_2509_19618_gb300 import api, capi, study  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("n", [1, 63, 64, 65, 300, 1000])
@pytest.mark.parametrize("mode,margin", [(oracle.DOMINANT, 1.0), (oracle.SQRTN, 1.0), (oracle.NONE, 1.0),
                                         (oracle.DEPARTURE, 0.9)])
def test_lu_f64_bit_exact(n, mode, margin):
    A_o, _ = oracle.generate(n, 50 + n, margin=margin, mode=mode)
    A = api.ColMajor.from_tensor(torch.from_numpy(A_o), DEV)
    LU, st = study.lu_f64(A)
    torch.cuda.synchronize()
    LU_o, rc = oracle.factor_plain(A_o, oracle.FP64, 64)
    assert st == (capi.OK if rc == 0 else capi.EBREAKDOWN)
    got = LU.view().cpu().numpy()
    both_finite = np.isfinite(LU_o)
    assert np.array_equal(got[both_finite], LU_o[both_finite])


def test_lu_f64_zero_pivot_is_breakdown():
    A_o, _ = oracle.generate(100, 2)
    A_o[0, 0] = 0.0
    A = api.ColMajor.from_tensor(torch.from_numpy(A_o), DEV)
    _, st = study.lu_f64(A)
    assert st == capi.EBREAKDOWN


@pytest.mark.parametrize("n,k", [(1, 1), (200, 1), (1000, 3)])
def test_lu_solve_f64_against_oracle(n, k):
    A_o, b_o = oracle.generate(n, 7, nrhs=k)
    A = api.ColMajor.from_tensor(torch.from_numpy(A_o), DEV)
    b = api.ColMajor.from_tensor(torch.from_numpy(b_o), DEV)
    LU, st = study.lu_f64(A)
    x = study.lu_solve_f64(LU, b)
    torch.cuda.synchronize()
    LU_o, _ = oracle.factor_plain(A_o, oracle.FP64, 64)
    got = x.view().cpu().numpy()
    for c in range(k):
        want = oracle.precond(LU_o, b_o[:, c], prec=0)
        assert np.abs(got[:, c] - want).max() <= 1e-13 * np.abs(want).max()


def test_residual_vector_against_oracle():
    n, k = 777, 2
    A_o, b_o = oracle.generate(n, 3, nrhs=k)
    X = np.asfortranarray(np.random.default_rng(4).uniform(-1, 1, (n, k)))
    A = api.ColMajor.from_tensor(torch.from_numpy(A_o), DEV)
    b = api.ColMajor.from_tensor(torch.from_numpy(b_o), DEV)
    x = api.ColMajor.from_tensor(torch.from_numpy(X), DEV)
    r = study.residual_vector(A, x, b).view().cpu().numpy()
    for c in range(k):
        want = oracle.residual_vec(A_o, X[:, c], b_o[:, c])
        assert np.abs(r[:, c] - want).max() <= 2 * n * 2.0**-53 * (np.abs(A_o).sum(1).max() * 1.0 + 1.0)


def test_study_reproduces_the_papers_qualitative_claims():
    """Section "Experimental Results": on unscaled uniform (-1, 1) matrices the
    GEPP pivots stay below about sqrt(n) and the largest one falls late in the
    factorization; without pivoting the residual norms grow by orders of
    magnitude; with the sqrt(n) diagonal scaling the unpivoted LU is as
    accurate as GEPP."""
    n = 2048
    raw = [study.run_case(n, s, "none") for s in (1, 2)]
    for rec in raw:
        assert rec["gepp"]["max_pivot"] <= 1.5 * math.sqrt(n)
        assert rec["gepp"]["max_pivot_pos"] >= 0.5
        for p in ("1", "2", "inf"):
            # "not <=" also accepts a non-finite backward error (catastrophic growth)
            assert not (rec["nopiv"][f"backward_{p}"] <= 10 * rec["gepp"][f"backward_{p}"])
    scaled = study.run_case(n, 1, "sqrtn")
    assert scaled["nopiv_status"] == "OK"
    for p in ("1", "2", "inf"):
        assert scaled["nopiv"][f"backward_{p}"] <= 10 * max(scaled["gepp"][f"backward_{p}"], 1.0)
