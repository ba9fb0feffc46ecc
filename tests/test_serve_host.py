"""Host-side checks of the serving layer (no GPU): the executor's arena
allocator, request footprints and validation, and the request stream."""
import math

import numpy as np
import pytest

from paper_2509_19618_gb300 import capi, serve

KB = 1024


def test_arena_first_fit_alignment_and_exhaustion():
    r = capi.hpmxp_test_arena(4 * KB, [1, 300, 256, 3 * KB + 1, 3 * KB])
    assert r[0] == 0                 # rounded up to one 256-byte block
    assert r[1] == 256               # 300 -> 512 bytes
    assert r[2] == 768
    assert r[3] == -1                # 1 KB used: 3 KB + 1 does not fit
    assert r[4] == KB                # exactly 3 KB does
    r = capi.hpmxp_test_arena(4 * KB, [4 * KB, 1])
    assert r == [0, -1]


def test_arena_release_coalesces_and_first_fit_reuses_holes():
    # a b c d of 1 KB; free b and c (merge), free a (merge with b+c): a 3 KB hole at 0
    ops = [KB, KB, KB, KB, -2, -3, -1, 3 * KB, 256]
    r = capi.hpmxp_test_arena(4 * KB, ops)
    assert r[:4] == [0, KB, 2 * KB, 3 * KB]
    assert r[4] == KB and r[5] == 2 * KB and r[6] == 3 * KB     # free bytes after each release
    assert r[7] == 0                                            # one block spanning the merged hole
    assert r[8] == -1                                           # and now nothing is left


def test_arena_release_in_any_order_restores_everything():
    rng = np.random.default_rng(5)
    sizes = [int(s) for s in rng.integers(1, 3000, size=12)]
    ops = sizes + [-(k + 1) for k in rng.permutation(12)]
    r = capi.hpmxp_test_arena(64 * KB, ops)
    assert all(o >= 0 and o % 256 == 0 for o in r[:12])
    spans = sorted((r[k], r[k] + -(-sizes[k] // 256) * 256) for k in range(12))
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))      # no overlap
    assert r[-1] == 64 * KB
    # after everything is free, the whole arena is one block again
    assert capi.hpmxp_test_arena(64 * KB, ops + [64 * KB])[-1] == 0


def _req(n, nrhs=1, **kw):
    spec = serve.Spec(0, n, nrhs, 1, 0.0)
    return serve.make_request(spec, **kw)


def test_footprint_covers_buffers_and_grows():
    f1 = capi.hpmxp_request_footprint(_req(1000))
    assert f1 >= 10 * 1000 * 1000          # 8 n^2 (A) + 2 n^2 (LU)
    assert capi.hpmxp_request_footprint(_req(2000)) > 3.2 * f1   # 10 n^2 grows 4x; fixed parts do not
    assert capi.hpmxp_request_footprint(_req(1000, 8)) > f1
    assert capi.hpmxp_request_footprint(_req(1000, 9)) == 0    # nrhs above 8
    assert capi.hpmxp_request_footprint(_req(0)) == 0
    bad = _req(1000)
    bad.prec = 9
    assert capi.hpmxp_request_footprint(bad) == 0
    bad = _req(1000)
    bad.nb = 64
    assert capi.hpmxp_request_footprint(bad) == 0


def test_splitmix64_published_values():
    # SplitMix64 seeded with 0: its first outputs, as published with the generator
    assert serve.splitmix64(0) == 0xE220A8397B1DCDAF
    assert serve.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def test_request_stream_distribution():
    specs = serve.request_stream(4000, rate=1000.0, stream_seed=2509)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 256 and ns.max() <= 8192
    # log-uniform: log n has mean (ln 256 + ln 8192) / 2 and standard deviation ln(32)/sqrt(12)
    ln = np.log(ns + 0.5)
    assert abs(ln.mean() - (math.log(256) + math.log(8192)) / 2) < 0.05
    assert abs(ln.std() - math.log(32) / math.sqrt(12)) < 0.05
    nr = np.array([s.nrhs for s in specs])
    assert set(nr.tolist()) == set(range(1, 9))
    gaps = np.diff([s.arrival for s in specs])
    assert abs(gaps.mean() - 1e-3) < 1e-4 and np.all(gaps >= 0)
    assert specs[7].seed == serve.splitmix64(2509 ^ 7)
    assert serve.request_stream(10, 1000.0, 2509) == serve.request_stream(10, 1000.0, 2509)
