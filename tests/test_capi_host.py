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
