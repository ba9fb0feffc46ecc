"""The factorization's schedule knobs (hpmxp_set_tuning) and the autotuner,
through the C interface.

The knobs move work between SMs, tiles and streams; they do not change which
products are summed into an entry or in what order (each step's update of an
entry is one fp32-accumulated product over the same K range, rounded once).
So the factors must be bit-identical under every setting, and the autotuner's
choice must be one of its candidates and applied."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_19618_gb300 import api, autotune, capi  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(autouse=True)
def restore_tuning():
    old = capi.hpmxp_get_tuning()
    yield
    assert capi.hpmxp_set_tuning(**old) == capi.OK


def factors(A, prec, nb):
    LU = api.factor(A, prec, nb)
    torch.cuda.synchronize(DEV)
    return LU.view().float().cpu().numpy() if LU.view().dtype != torch.float32 else LU.view().cpu().numpy()


@pytest.mark.parametrize("prec", [capi.BF16, capi.FP16])
def test_schedule_knobs_keep_factors_bit_identical(prec):
    n, nb = 3000, 256
    A, _ = api.generate(n, seed=11, device=DEV)
    assert capi.hpmxp_set_tuning(0, 0, 0) == capi.OK
    ref = factors(A, prec, nb)
    # look-ahead forced on at this order (threshold 128), with 4 and 40 reserved SMs, both tile heights
    for tile, reserve in ((256, 4), (256, 40), (128, 4), (128, 40)):
        assert capi.hpmxp_set_tuning(tile, reserve, 128) == capi.OK
        got = factors(A, prec, nb)
        assert np.array_equal(got, ref), (tile, reserve)


def test_autotune_applies_a_candidate(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    n = 2048
    A, _ = api.generate(n, seed=3, device=DEV)
    choice = autotune.tune(n, capi.BF16, A, device=DEV)
    sms = torch.cuda.get_device_properties(DEV).multi_processor_count
    assert choice in autotune.candidates(n, capi.BF16, sms)
    t = capi.hpmxp_get_tuning()
    assert (t["gemm_tile"], t["reserve_sms"]) == (choice.gemm_tile, choice.reserve_sms)
    # the second call recalls the cached choice without searching
    monkeypatch.setattr(autotune, "_time", lambda *a, **k: pytest.fail("searched again"))
    assert autotune.tune(n, capi.BF16, A, device=DEV) == choice


@pytest.mark.parametrize("budget", [1, 7, 40])
def test_sm_budget_keeps_results_bit_identical(budget):
    """A smaller persistent GEMM grid and a smaller cooperative preconditioner
    grid (each CTA then owns more block rows) change neither the factors nor x:
    every block row still receives its terms in the same order."""
    n, k, nb = 3000, 3, 128
    A, b = api.generate(n, seed=21, nrhs=k, device=DEV)
    p = api.ir_params(precond_fp32=1, inner_tol=1e-5)
    outs = []
    for sm in (0, budget):
        assert capi.hpmxp_set_tuning(0, 0, 0, sm) == capi.OK
        LU = api.factor(A, capi.BF16, nb)
        x, infos, st = api.solve_ir(A, LU, b, capi.BF16, p)
        torch.cuda.synchronize(DEV)
        assert st == capi.OK
        outs.append((LU.view().float().cpu().numpy(), x.view().cpu().numpy(), [i["iters"] for i in infos]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


@pytest.mark.parametrize("prec", [capi.BF16, capi.FP16, capi.FP8_E4M3])
def test_lookahead_with_balancing_bit_identical(prec):
    """The four-stream look-ahead (forced on at this order) and the plain
    schedule give the same factors of the balanced matrix."""
    n, nb = 2600, 512
    A, _ = api.generate(n, seed=31, device=DEV)
    scales = api.balance(A, prec)
    outs = []
    for overlap in (0, 128):   # 0: the built-in threshold (8192) keeps this order plain
        assert capi.hpmxp_set_tuning(0, 0, overlap) == capi.OK
        LU = api.factor(A, prec, nb, scales=scales)
        torch.cuda.synchronize(DEV)
        outs.append(LU.view().float().cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
