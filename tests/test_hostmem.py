"""Host buffers for the host-input path (paper_1401_7494_gb300.hostmem), on the CPU with a stand-in for
the CUDA runtime's registration calls."""
import gc

import numpy as np
import pytest
import torch

from paper_1401_7494_gb300 import hostmem


class FakeCudart:
    def __init__(self):
        self.registered = {}
        self.unregistered = []

    def cudaHostRegister(self, ptr, size, flags):
        self.registered[ptr] = size
        return 0

    def cudaHostUnregister(self, ptr):
        self.unregistered.append(ptr)
        return 0


@pytest.fixture
def fake(monkeypatch):
    f = FakeCudart()
    monkeypatch.setattr(torch.cuda, "cudart", lambda: f)
    return f


@pytest.mark.parametrize("shape,dtype", [((3, 5, 7), torch.float32), ((1000,), torch.float16), ((2, 3), torch.bfloat16)])
def test_buffer_is_aligned_registered_and_zero(fake, shape, dtype):
    t = hostmem.pinned_empty(shape, dtype)
    assert tuple(t.shape) == shape and t.dtype == dtype and t.is_contiguous()
    hp = hostmem.huge_page_bytes()
    assert t.data_ptr() % hp == 0
    assert t.data_ptr() in fake.registered
    assert fake.registered[t.data_ptr()] >= t.numel() * t.element_size()
    assert torch.count_nonzero(t) == 0
    t.fill_(3)
    assert float(t.float().sum()) == 3 * t.numel()


def test_large_buffers_take_whole_huge_pages(fake, monkeypatch):
    monkeypatch.setattr(hostmem, "huge_page_bytes", lambda: 1 << 20)
    monkeypatch.setattr(hostmem, "huge_pages_enabled", lambda: True)
    t = hostmem.pinned_empty((300, 1024), torch.float32)          # 1.17 MiB: two 1 MiB pages
    assert t.data_ptr() % (1 << 20) == 0 and fake.registered[t.data_ptr()] == 2 << 20
    small = hostmem.pinned_empty((1000,), torch.float32)          # far below a quarter page: base pages
    assert fake.registered[small.data_ptr()] == 4000


def test_buffer_lives_while_any_view_does(fake):
    t = hostmem.pinned_empty((4, 1024), torch.float32)
    addr = t.data_ptr()
    view = t[2:]
    view.fill_(1.5)
    del t
    gc.collect()
    assert addr not in fake.unregistered             # the view still uses the memory
    assert float(view.sum()) == 1.5 * view.numel()
    del view
    gc.collect()
    assert addr in fake.unregistered                 # released with the last tensor


def test_numpy_interop(fake):
    t = hostmem.pinned_empty((6, 8), torch.float32)
    a = t.numpy()
    a[:] = np.arange(48, dtype=np.float32).reshape(6, 8)
    assert float(t[5, 7]) == 47.0


def test_a_chunk_left_in_base_pages_is_mapped_again(fake, monkeypatch):
    """A huge page that comes back in base pages is mapped again (up to `tries` times); the others once."""
    monkeypatch.setattr(hostmem, "huge_page_bytes", lambda: 1 << 20)
    monkeypatch.setattr(hostmem, "huge_pages_enabled", lambda: True)
    calls = []
    real_map = hostmem._map_chunk
    got = {"huge": 0}

    def map_chunk(libc, addr, n):
        real_map(libc, addr, n)
        calls.append(addr)
        # the second chunk gets its huge page only on the third attempt
        idx = sorted(set(calls)).index(addr)
        if idx != 1 or calls.count(addr) >= 3:
            got["huge"] += n
    monkeypatch.setattr(hostmem, "_map_chunk", map_chunk)
    monkeypatch.setattr(hostmem, "_huge_bytes", lambda lo, hi: got["huge"])
    t = hostmem.pinned_empty((3, 1 << 18), torch.float32, tries=3)      # 3 MiB: three chunks
    base = t.data_ptr()
    assert calls == [base, base + (1 << 20), base + (1 << 20), base + (1 << 20), base + (2 << 20)]
    assert torch.count_nonzero(t) == 0


def _locked_bytes(addr: int) -> int:
    """The Locked: bytes of the mapping of this process that contains addr (/proc/self/smaps)."""
    cur = None
    for line in open("/proc/self/smaps").read().splitlines():
        parts = line.split()
        if parts and "-" in parts[0] and ":" not in parts[0]:
            lo, hi = (int(x, 16) for x in parts[0].split("-"))
            cur = lo <= addr < hi
        elif cur and parts and parts[0] == "Locked:":
            return int(parts[1]) * 1024
    return 0


def test_buffer_is_locked_where_the_limit_allows(fake):
    """Buffers are mlock-ed before registration (out of the reclaim scans); a lock limit smaller than the
    buffer leaves it unlocked but usable."""
    import resource
    soft, _ = resource.getrlimit(resource.RLIMIT_MEMLOCK)
    t = hostmem.pinned_empty((1024,), torch.float32)
    if soft == resource.RLIM_INFINITY or soft >= 64 * 1024:
        assert _locked_bytes(t.data_ptr()) >= t.numel() * t.element_size()
    t[:] = 1.0
    assert float(t.sum()) == 1024.0


def test_deferred_registration(fake):
    """register=False leaves the buffer unregistered until finish(), which keeps its contents, registers it
    once and refuses tensors that do not come from pinned_empty."""
    t = hostmem.pinned_empty((4096,), torch.float32, register=False)
    assert t.data_ptr() not in fake.registered
    t[:] = torch.arange(4096, dtype=torch.float32)
    assert hostmem.finish(t) is t
    assert t.data_ptr() in fake.registered and fake.registered[t.data_ptr()] >= 4096 * 4
    assert torch.equal(t, torch.arange(4096, dtype=torch.float32))
    n = len(fake.registered)
    hostmem.finish(t)
    assert len(fake.registered) == n
    with pytest.raises(ValueError):
        hostmem.finish(torch.zeros(4))
