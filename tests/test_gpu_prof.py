"""The measurement support the benchmark's roofline rests on: the GEMM
launches' own execution spans (hpmxp_prof_read_device) against the CUDA-event
intervals around them (hpmxp_prof_read), through the C interface."""
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_19618_gb300 import api, capi  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_gemm_device_spans_within_event_intervals():
    n = 3000
    A, b = api.generate(n, seed=4, device=DEV)
    api.factor(A, capi.BF16, 256)   # warm
    torch.cuda.synchronize(DEV)
    capi.hpmxp_prof_reset()
    capi.hpmxp_prof_enable(True)
    try:
        api.factor(A, capi.BF16, 256)
        torch.cuda.synchronize(DEV)
    finally:
        capi.hpmxp_prof_enable(False)
    for kind in (capi.PROF_GEMM, capi.PROF_GEMM_STORE):
        ev = capi.hpmxp_prof_read(kind)
        dv = capi.hpmxp_prof_read_device(kind)
        assert ev["launches"] > 0
        # every profiled GEMM launch stamped its span
        assert dv["launches"] == ev["launches"]
        # a launch runs inside the events recorded around it on its stream
        assert 0.0 < dv["ms"] <= ev["ms"] * 1.001 + 1e-3
    # kinds that do not stamp report nothing; a bad kind is refused
    assert capi.hpmxp_prof_read_device(capi.PROF_GETRF)["launches"] == 0
    with pytest.raises(capi.HpmxpError):
        capi.hpmxp_prof_read_device(99)
    capi.hpmxp_prof_reset()
    assert capi.hpmxp_prof_read_device(capi.PROF_GEMM) == dict(ms=0.0, launches=0)
