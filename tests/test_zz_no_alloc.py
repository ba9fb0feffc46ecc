"""hpmxp_generate_noalloc, the generator entry point that takes no workspace.

It exists for callers that cannot give the library scratch memory (all device
memory held by their own pool, or no cudaMalloc/cudaFree allowed around the
call because those synchronize the device).  Its row sums live in a fixed
array inside the library that every call reuses, so these tests check, through
the C interface, that back-to-back calls give exactly what hpmxp_generate gives
(the generator is integer work: bit-exact), i.e. that the array is cleared at
the start of each call, and that sizes above the array's 131072 rows are
refused before anything runs.

The file name sorts last so that a run stopping at its first failure has run
every other test before these.
"""
import numpy as np
import pytest

from paper_2509_19618_gb300 import capi

MAX_ROWS = 1 << 17


def test_noalloc_rejects_sizes_above_the_fixed_array():
    fake = 4096   # never dereferenced: the size check comes first
    assert capi.hpmxp_generate_noalloc(MAX_ROWS + 1, 1, 1.0, capi.DIAG_DOMINANT, fake, MAX_ROWS + 1, fake,
                                       MAX_ROWS + 1, 1, None) == capi.ENOMEM
    assert capi.hpmxp_generate_noalloc(0, 1, 1.0, capi.DIAG_DOMINANT, fake, 1, fake, 1, 1, None) == capi.EINVAL
    assert capi.hpmxp_generate_noalloc(10, 1, 1.0, 7, fake, 10, fake, 10, 1, None) == capi.EINVAL
    assert capi.hpmxp_generate_noalloc(10, 1, 1.0, capi.DIAG_DOMINANT, fake, 9, fake, 10, 1, None) == capi.EINVAL


def _buffers(torch, n, nrhs, dev):
    ld = (n + 7) // 8 * 8
    A = torch.full((n, ld), float("nan"), dtype=torch.float64, device=dev)
    b = torch.full((max(nrhs, 1), ld), float("nan"), dtype=torch.float64, device=dev)
    return A, b, ld


def _with_workspace(torch, n, seed, margin, mode, nrhs, dev):
    A, b, ld = _buffers(torch, n, nrhs, dev)
    ws = torch.empty(capi.hpmxp_generate_workspace(n), dtype=torch.uint8, device=dev)
    st = capi.hpmxp_generate(n, seed, margin, mode, A.data_ptr(), ld, b.data_ptr(), ld, nrhs, ws.data_ptr(),
                             ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert st == capi.OK, capi.status_string(st)
    torch.cuda.synchronize()
    return A[:, :n].cpu().numpy(), b[:nrhs, :n].cpu().numpy()


def _noalloc(torch, n, seed, margin, mode, nrhs, dev):
    A, b, ld = _buffers(torch, n, nrhs, dev)
    st = capi.hpmxp_generate_noalloc(n, seed, margin, mode, A.data_ptr(), ld, b.data_ptr(), ld, nrhs,
                                     torch.cuda.current_stream().cuda_stream)
    assert st == capi.OK, capi.status_string(st)
    torch.cuda.synchronize()
    return A[:, :n].cpu().numpy(), b[:nrhs, :n].cpu().numpy()


# (n, seed, margin, diag, nrhs) for two calls in a row.  The first call leaves
# larger row sums behind than the second needs; a second call that did not
# clear them would get wrong diagonals.
CASES = [
    [(1500, 11, 1.0, capi.DIAG_DOMINANT, 2), (1000, 12, 1.5, capi.DIAG_DOMINANT, 1)],
    [(777, 3, 1.0, capi.DIAG_DOMINANT, 1), (777, 3, 1.0, capi.DIAG_DOMINANT, 1)],
    [(4100, 5, 2.0, capi.DIAG_SQRTN, 0), (129, 6, 1.0, capi.DIAG_DOMINANT, 3)],
]


@pytest.mark.gpu
@pytest.mark.parametrize("calls", CASES)
def test_noalloc_matches_generate_on_two_calls_in_a_row(calls):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dev = torch.device("cuda:0")
    got = [_noalloc(torch, *c, dev) for c in calls]          # back to back, nothing in between
    for c, (A, b) in zip(calls, got):
        A_ref, b_ref = _with_workspace(torch, *c, dev)
        assert np.array_equal(A, A_ref), c
        assert np.array_equal(b, b_ref), c
        assert np.all(np.isfinite(A))
