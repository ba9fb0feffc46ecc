"""api.HostBuffer: page-locked host memory over a huge-page-advised mapping.

The CPU test replaces the CUDA runtime's register / unregister calls with a
recorder; the GPU test copies through a real registered buffer."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_19618_gb300 import api  # noqa: E402


class _FakeRuntime:
    def __init__(self, fail=False):
        self.calls = []
        self.fail = fail

    def cudaHostRegister(self, ptr, size, flags):
        self.calls.append(("register", ptr, size, flags))
        return 1 if self.fail else 0

    def cudaHostUnregister(self, ptr):
        self.calls.append(("unregister", ptr))
        return 0


def test_host_buffer_registers_whole_mapping_and_unregisters(monkeypatch):
    rt = _FakeRuntime()
    monkeypatch.setattr(torch.cuda, "cudart", lambda: rt)
    hb = api.HostBuffer((7, 130))
    t = hb.tensor
    assert t.shape == (7, 130) and t.dtype == torch.float64 and t.device.type == "cpu"
    assert bool((t == 0).all())
    t[3, 5] = 2.5
    assert float(hb.tensor.view(-1)[3 * 130 + 5]) == 2.5
    ptr = t.data_ptr()
    assert rt.calls == [("register", ptr, 7 * 130 * 8, 0)]
    del t
    hb.close()
    assert rt.calls[-1] == ("unregister", ptr) and hb.tensor is None
    hb.close()   # idempotent
    assert len(rt.calls) == 2


def test_host_buffer_rejects_empty_shape(monkeypatch):
    rt = _FakeRuntime()
    monkeypatch.setattr(torch.cuda, "cudart", lambda: rt)
    with pytest.raises(ValueError):
        api.HostBuffer((0, 5))
    assert rt.calls == []


def test_host_buffer_register_failure_raises(monkeypatch):
    monkeypatch.setattr(torch.cuda, "cudart", lambda: _FakeRuntime(fail=True))
    with pytest.raises(RuntimeError):
        api.HostBuffer((4, 4))


@pytest.mark.gpu
def test_host_buffer_round_trip_on_device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dev = torch.device("cuda:0")
    hb = api.HostBuffer((256, 1000))
    src = torch.from_numpy(np.random.default_rng(3).standard_normal((256, 1000)))
    hb.tensor.copy_(src)
    d = torch.empty((256, 1000), dtype=torch.float64, device=dev)
    d.copy_(hb.tensor, non_blocking=True)
    back = torch.empty_like(src)
    torch.cuda.synchronize()
    back.copy_(d)
    assert torch.equal(back, src)
    hb.close()
