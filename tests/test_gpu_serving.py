"""Serving through the request executor (include/hpmxp_serve.h), on the GPU:
requests that run side by side on several streams give bit-for-bit the x of
the same request run alone, and the x of the plain C-interface path
(hpmxp_generate + hpmxp_factor + hpmxp_solve_ir); admission by arena size
lets every request through even when only one fits at a time."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2509_19618_gb300 import api, capi, serve  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _specs(count=20, seed=77):
    return serve.request_stream(count, rate=0.0, stream_seed=seed, n_min=200, n_max=1100)


def _xs(specs):
    return {s.id: torch.full((s.nrhs, (s.n + 7) // 8 * 8), float("nan"), dtype=torch.float64, device=DEV)
            for s in specs}


def _check_valid(comps):
    for c in comps:
        assert c["status"] == capi.OK, c
        assert all(i["scaled_resid"] < 16.0 for i in c["info"]), c


@pytest.fixture(scope="module")
def mixed():
    specs = _specs()
    xs = _xs(specs)
    with serve.Executor(workers=6, arena_bytes=1 << 30, device=DEV) as ex:
        comps = serve.run_stream(ex, specs, xs=xs)
    torch.cuda.synchronize()
    return specs, xs, comps


def test_mixed_requests_all_valid(mixed):
    specs, xs, comps = mixed
    assert [c["id"] for c in comps] == [s.id for s in specs]
    _check_valid(comps)
    for s in specs:
        assert torch.isfinite(xs[s.id][:, : s.n]).all()


def test_mixed_equals_one_at_a_time(mixed):
    specs, xs, comps = mixed
    xs1 = _xs(specs)
    with serve.Executor(workers=1, arena_bytes=1 << 30, device=DEV) as ex:
        comps1 = serve.run_stream(ex, specs, xs=xs1, one_at_a_time=True)
    torch.cuda.synchronize()
    _check_valid(comps1)
    for s, c, c1 in zip(specs, comps, comps1):
        assert torch.equal(xs[s.id][:, : s.n], xs1[s.id][:, : s.n]), s
        assert [i["iters"] for i in c["info"]] == [i["iters"] for i in c1["info"]]
        assert [i["scaled_resid"] for i in c["info"]] == [i["scaled_resid"] for i in c1["info"]]


def test_mixed_equals_plain_c_interface_path(mixed):
    specs, xs, comps = mixed
    for s in specs[:5]:
        A, b = api.generate(s.n, seed=s.seed, margin=1.0, nrhs=s.nrhs, device=DEV)
        solver = api.Solver(s.n, s.nrhs, capi.BF16, nb=128, device=DEV)
        x, infos, st = solver(A, b)
        assert st == capi.OK
        assert torch.equal(x.view(), xs[s.id][:, : s.n].t()), s


def test_arena_that_fits_one_request_serves_all(mixed):
    specs, xs, comps = mixed
    big = max(capi.hpmxp_request_footprint(serve.make_request(s)) for s in specs)
    xs2 = _xs(specs)
    with serve.Executor(workers=4, arena_bytes=(big * 3) // 2 // 256 * 256 + 256, device=DEV) as ex:
        comps2 = serve.run_stream(ex, specs, xs=xs2)
    torch.cuda.synchronize()
    _check_valid(comps2)
    for s in specs:
        assert torch.equal(xs[s.id][:, : s.n], xs2[s.id][:, : s.n]), s


def test_request_larger_than_arena_is_refused():
    with serve.Executor(workers=1, arena_bytes=1 << 20, device=DEV) as ex:
        with pytest.raises(capi.HpmxpError) as e:
            ex.submit(serve.make_request(serve.Spec(0, 1000, 1, 1, 0.0)))
        assert e.value.status == capi.ENOMEM


def test_open_loop_stream_with_arrivals():
    specs = serve.request_stream(30, rate=2000.0, stream_seed=5, n_min=256, n_max=2048)
    with serve.Executor(workers=4, arena_bytes=2 << 30, device=DEV) as ex:
        comps = serve.run_stream(ex, specs)
    _check_valid(comps)
    summ = serve.summarize(specs, comps)
    assert summ["valid"] and summ["requests"] == 30 and summ["p99_ms"] >= summ["p50_ms"] > 0


def test_batched_executor_equals_plain_executor(mixed):
    """Batch mode (grouped factorization, lockstep refinement, several requests
    per worker at once) gives bit-for-bit the x of the plain executor: every
    request here has n < 4096, so both factor at depth 128 with the same tiles."""
    specs, xs, comps = mixed
    xsb = _xs(specs)
    with serve.Executor(workers=2, arena_bytes=1 << 30, device=DEV, batch=8) as ex:
        compsb = serve.run_stream(ex, specs, xs=xsb)
    torch.cuda.synchronize()
    _check_valid(compsb)
    for s, c, cb in zip(specs, comps, compsb):
        assert torch.equal(xs[s.id][:, : s.n], xsb[s.id][:, : s.n]), s
        assert [i["iters"] for i in c["info"]] == [i["iters"] for i in cb["info"]]


def test_batched_executor_with_an_arena_for_one_request():
    specs = _specs(count=6, seed=3)
    xs = _xs(specs)
    big = max(capi.hpmxp_request_footprint(serve.make_request(s)) for s in specs)
    with serve.Executor(workers=2, arena_bytes=int(big * 1.6), device=DEV, batch=8) as ex:
        comps = serve.run_stream(ex, specs, xs=xs)
    _check_valid(comps)
