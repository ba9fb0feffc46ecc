"""Host-side checks of the C interface (no GPU needed): the library builds for
sm_103a, loads, exports every symbol include/*.h declares, and rejects bad
arguments before touching the device."""
import ctypes

import pytest

from paper_2509_19618_gb300 import capi


@pytest.fixture(scope="module")
def lib():
    return capi.load()


def test_exports_every_declared_symbol(lib):
    names = capi.declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(8):
        assert capi.status_string(s)
    assert capi.status_string(99) == "unknown status"


def test_workspace_sizes(lib):
    assert capi.hpmxp_generate_workspace(1000) >= 16 * 1000
    assert capi.hpmxp_factor_workspace(1000, capi.BF16, 128) > 0
    assert capi.hpmxp_factor_workspace(1000, capi.BF16, 100) == 0
    assert capi.hpmxp_factor_workspace(1000, 7, 128) == 0
    assert capi.hpmxp_factor_workspace(4096, capi.FP8_E4M3, 512) > capi.hpmxp_factor_workspace(4096, capi.BF16, 512)
    assert capi.hpmxp_solve_workspace(1000, 1, 30) > 0
    assert capi.hpmxp_solve_workspace(1000, 9, 30) == 0
    assert capi.hpmxp_solve_workspace(1000, 1, 65) == 0
    assert capi.hpmxp_residual_workspace(1000, 2) > 0


def test_default_params(lib):
    p = capi.hpmxp_ir_params_default()
    assert (p.restart, p.max_iters, p.accept, p.precond_fp32) == (30, 50, 16.0, 0)
    assert p.inner_tol == 1e-12 and p.theta == 0.1


def test_invalid_arguments_rejected_on_host(lib):
    fake = 4096  # never dereferenced: validation fails first
    assert capi.hpmxp_generate(0, 1, 1.0, 0, fake, 1, fake, 1, 1, fake, 1 << 20, None) == capi.EINVAL
    assert capi.hpmxp_generate(10, 1, 1.0, 5, fake, 10, fake, 10, 1, fake, 1 << 20, None) == capi.EINVAL
    assert capi.hpmxp_generate(10, 1, 1.0, 0, fake, 9, fake, 10, 1, fake, 1 << 20, None) == capi.EINVAL
    assert capi.hpmxp_generate(10, 1, 1.0, 0, fake, 10, fake, 10, 1, fake, 8, None) == capi.ENOMEM
    # ldlu must be a multiple of 8, nb one of 128/256/512
    assert capi.hpmxp_factor(100, fake, 100, capi.BF16, 128, fake, 100, fake, 1 << 30, None) == capi.EINVAL
    assert capi.hpmxp_factor(100, fake, 100, capi.BF16, 64, fake, 104, fake, 1 << 30, None) == capi.EINVAL
    assert capi.hpmxp_factor(100, fake, 100, capi.BF16, 128, fake, 104, fake, 16, None) == capi.ENOMEM
    p = capi.hpmxp_ir_params_default()
    p.restart = 0
    info = (capi.IRInfo * 1)()
    assert capi.hpmxp_solve_ir(100, fake, 100, fake, 104, 0, fake, 100, fake, 100, 1, p, info, fake, 1 << 30,
                               None) == capi.EINVAL
    assert capi.hpmxp_solve_ir(100, fake, 100, fake, 104, 0, fake, 100, fake, 100, 9, None, info, fake, 1 << 30,
                               None) == capi.EINVAL
    out = (ctypes.c_double * 1)()
    assert capi.hpmxp_residual(100, fake, 99, fake, 100, fake, 100, 1, ctypes.addressof(out), fake, 1 << 30,
                               None) == capi.EINVAL
    assert capi.hpmxp_test_gemm(128, 128, 100, fake, 128, fake, 128, fake, 128, None, 0, 0, 1.0, 0, 0, None, 0,
                                None, 0, 0, fake, None) == capi.EINVAL


def test_library_is_sm103a_build():
    from paper_2509_19618_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert _build.LIB.startswith(_build.PKG)   # in-tree


def test_python_modules_import():
    import importlib
    for m in ("paper_2509_19618_gb300.api", "paper_2509_19618_gb300.autotune", "bench"):
        importlib.import_module(m)


def test_schedule_tuning_set_get(lib):
    old = capi.hpmxp_get_tuning()
    try:
        assert capi.hpmxp_set_tuning(128, 20, 4096, 40) == capi.OK
        want = dict(gemm_tile=128, reserve_sms=20, overlap_min=4096, sm_budget=40)
        assert capi.hpmxp_get_tuning() == want
        # tile heights other than 0/128/256, negative counts and a nonzero reserved field are
        # refused and change nothing
        for bad in ((64, 0, 0), (512, 0, 0), (0, -1, 0), (0, 0, -5), (0, 5000, 0), (0, 0, 0, -1), (0, 0, 0, 0, 1)):
            assert capi.hpmxp_set_tuning(*bad) == capi.EINVAL
        assert capi.hpmxp_get_tuning() == want
    finally:
        assert capi.hpmxp_set_tuning(**old) == capi.OK


def test_autotune_search_space():
    from paper_2509_19618_gb300 import autotune
    sms = 152
    big = autotune.candidates(32768, capi.BF16, sms)
    # nb x tile x reserve where the look-ahead schedule runs
    assert len(big) == 3 * 2 * 3
    assert {c.reserve_sms for c in big} == {max(4, sms // d) for d in autotune.RESERVE_DIVISORS}
    assert {c.gemm_tile for c in big} == {128, 256}
    # below the look-ahead threshold the reserve has no effect and is not searched
    small = autotune.candidates(4096, capi.BF16, sms)
    assert len(small) == 3 * 2 and {c.reserve_sms for c in small} == {0}
    # the fp32-trailing variants run without look-ahead
    assert {c.reserve_sms for c in autotune.candidates(32768, capi.BF16_TRAIL32, sms)} == {0}
    # FP8 products stay on one tile height
    assert {c.gemm_tile for c in autotune.candidates(32768, capi.FP8_E4M3, sms)} == {0}
    # nb larger than the matrix is skipped (below 128 the smallest depth stays)
    assert {c.nb for c in autotune.candidates(200, capi.BF16, sms)} == {128}


def test_prof_read_device_on_host(lib):
    # nothing recorded: zeros, no device access; a bad kind is refused
    assert capi.hpmxp_prof_read_device(capi.PROF_GEMM) == dict(ms=0.0, launches=0)
    with pytest.raises(capi.HpmxpError):
        capi.hpmxp_prof_read_device(-1)
