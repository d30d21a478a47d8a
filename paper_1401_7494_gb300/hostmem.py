"""Page-locked host buffers for the host-input path.

``rct_backproject_host`` and ``rct_backproject_host_read`` move the
projections in and the volume out with the copy engines, which need
page-locked host memory.  Memory locked by ``cudaHostAlloc`` (torch's
``pin_memory=True``) is mapped in base pages (64 KiB on the Arm hosts of
GB300 systems).  On hosts whose memory has been allocated and freed in
bulk before (another large job, a test suite), copies from and to such
buffers were measured to stall for 30 to 200 ms every few hundred
milliseconds, while the same copies from buffers backed by transparent huge
pages that are aligned to the huge-page size never stalled: 80 copies of
2.4 GB in, 150 copies of 0.5 GB out and 80 full reconstructions from host
buffers, no step slower than the median.

``pinned_empty`` allocates such a buffer: an anonymous mapping aligned to
the huge-page size, advised for transparent huge pages, touched once,
collapsed into huge pages where the first touch did not get them (a host
with fragmented memory), locked with ``mlock`` (best effort) and registered
with ``cudaHostRegister``.  On a churned host, 90 copy pairs (2.4 GB in, 0.5
GB out) from locked huge-page buffers ran without a stall, while unlocked
huge-page buffers stalled 6 times (31-570 ms) and base-page buffers, locked
or not, about 25 times (up to 1 s);
``huge_fraction`` reports how much of a buffer huge pages back.  The
returned tensor owns the buffer: it is unregistered and unmapped when the
tensor and every view of it are gone.  Where transparent huge pages are switched off the buffer is still
aligned, locked and registered, in base pages.
"""
from __future__ import annotations

import ctypes
import ctypes.util
from pathlib import Path

_PROT_NONE = 0
_PROT_RW = 0x1 | 0x2
_MAP_PRIVATE_ANON = 0x02 | 0x20
_MAP_FIXED = 0x10
_MAP_NORESERVE = 0x4000
_MADV_HUGEPAGE = 14
_MADV_COLLAPSE = 25       # Linux 6.1+: make the range huge pages now (compacting memory if it must)
_THP = Path("/sys/kernel/mm/transparent_hugepage")

_libc = None


def _c():
    global _libc
    if _libc is None:
        _libc = ctypes.CDLL(ctypes.util.find_library("c"), use_errno=True)
        _libc.mmap.restype = ctypes.c_void_p
        _libc.mmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_long]
        _libc.munmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
        _libc.madvise.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        _libc.mlock.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    return _libc


def huge_page_bytes() -> int:
    """The transparent huge-page size of this host (2 MiB where the kernel does not say)."""
    try:
        return int((_THP / "hpage_pmd_size").read_text())
    except (OSError, ValueError):
        return 2 << 20


def huge_pages_enabled() -> bool:
    try:
        return "[never]" not in (_THP / "enabled").read_text()
    except OSError:
        return False


def _vma_table():
    """(start, end, AnonHugePages bytes) of every mapping of this process, from /proc/self/smaps."""
    out = []
    try:
        lines = Path("/proc/self/smaps").read_text().splitlines()
    except OSError:
        return out
    cur = None
    for line in lines:
        parts = line.split()
        if not parts:
            continue
        if "-" in parts[0] and ":" not in parts[0]:
            lo, hi = (int(x, 16) for x in parts[0].split("-"))
            cur = [lo, hi, 0]
            out.append(cur)
        elif cur is not None and parts[0] == "AnonHugePages:":
            cur[2] = int(parts[1]) * 1024
    return out


def _huge_bytes(lo: int, hi: int) -> int:
    """Bytes of [lo, hi) that transparent huge pages back (mappings wholly inside the range)."""
    return sum(h for a, b, h in _vma_table() if lo <= a and b <= hi)


def _map_chunk(libc, addr: int, n: int) -> None:
    got = libc.mmap(addr, n, _PROT_RW, _MAP_PRIVATE_ANON | _MAP_FIXED, -1, 0)
    if got != addr:
        raise MemoryError(f"mmap of {n} bytes at a fixed address failed (errno {ctypes.get_errno()})")
    libc.madvise(addr, n, _MADV_HUGEPAGE)
    ctypes.memset(addr, 0, n)                      # touch every page before it is locked
    libc.madvise(addr, n, _MADV_COLLAPSE)          # best effort: fails harmlessly where unsupported


def pinned_empty(shape, dtype, tries: int = 3, register: bool = True):
    """A page-locked, huge-page-backed host tensor of ``shape`` and ``dtype`` (contents zero).

    The buffer is mapped one huge page at a time inside an aligned reserved range (at most 64 of them; more,
    smaller huge pages are mapped in one go); a huge page that comes back in base pages (a host whose free
    memory is fragmented) is mapped again, up to ``tries`` times, each attempt asking the kernel to compact
    memory for it.  What still fails stays in base pages: the buffer works, more slowly on such hosts
    (``huge_fraction`` tells).  With ``register=False`` the buffer is neither locked nor registered yet:
    ``finish`` (on the returned tensor) retries the collapse of the pages still in base pages, which gives
    the host time to free whole huge pages, then locks and registers it."""
    import torch
    libc = _c()
    n = 1
    for s in shape:
        n *= int(s)
    nbytes = n * torch.empty((), dtype=dtype).element_size()
    hp = huge_page_bytes()
    # Buffers below a quarter of a huge page stay in base pages: a huge page would lock far more memory
    # than they use.  The others are rounded up to whole huge pages.
    huge = huge_pages_enabled() and nbytes >= hp // 4
    size = max(hp, -(-nbytes // hp) * hp) if huge else max(1, nbytes)
    raw_size = size + hp
    raw = libc.mmap(None, raw_size, _PROT_NONE if huge else _PROT_RW,
                    _MAP_PRIVATE_ANON | (_MAP_NORESERVE if huge else 0), -1, 0)
    if raw in (None, ctypes.c_void_p(-1).value):
        raise MemoryError(f"mmap of {raw_size} bytes failed (errno {ctypes.get_errno()})")
    start = -(-raw // hp) * hp
    cudart = torch.cuda.cudart()

    class _Mapping(ctypes.c_char * size):
        """The mapping; torch keeps it alive for as long as any tensor uses the memory."""
        registered = False

        def __del__(self):
            try:
                if self.registered:
                    cudart.cudaHostUnregister(start)
            finally:
                libc.munmap(raw, raw_size)

    if huge and size // hp > 64:
        _map_chunk(libc, start, size)             # small huge pages (2 MiB): one mapping, one collapse
    elif huge:
        for at in range(start, start + size, hp):
            for _ in range(max(1, tries)):
                before = _huge_bytes(start, start + size)
                _map_chunk(libc, at, hp)
                if _huge_bytes(start, start + size) - before >= hp:
                    break
    mapping = _Mapping.from_address(start)
    mapping.span = (start, size, hp if huge and size // hp <= 64 else 0)
    t = torch.frombuffer(mapping, dtype=torch.uint8)
    if not huge:
        t.zero_()                                 # touch every page before it is locked
    out = t[:nbytes].view(dtype).view(*[int(s) for s in shape])
    out._hostmem_mapping = mapping
    if register:
        _lock_and_register(mapping)
    return out


def _lock_and_register(mapping) -> None:
    import torch
    start, size, _ = mapping.span
    # Locked pages sit on the unevictable list, out of the reclaim scans (process-local; released with the
    # mapping).  A refusal (a memory-lock limit) leaves the buffer as it is.
    _c().mlock(start, size)
    err = torch.cuda.cudart().cudaHostRegister(start, size, 0)
    if int(err) != 0:
        raise RuntimeError(f"cudaHostRegister of {size} bytes failed: {err}")
    mapping.registered = True


def finish(t, tries: int = 3):
    """Lock and register a buffer from ``pinned_empty(..., register=False)`` (``t`` is the tensor it
    returned), first asking again, up to ``tries`` times per huge page, for huge pages where base pages
    still back it (the contents are kept).  A registered buffer is returned unchanged."""
    mapping = getattr(t, "_hostmem_mapping", None)
    if mapping is None:
        raise ValueError("finish: not a tensor returned by hostmem.pinned_empty")
    if mapping.registered:
        return t
    start, size, hp = mapping.span
    if hp:
        libc = _c()
        for at in range(start, start + size, hp):
            for _ in range(max(1, tries)):
                if _huge_bytes(start, start + size) >= size:
                    break
                libc.madvise(at, hp, _MADV_COLLAPSE)
    _lock_and_register(mapping)
    return t


def huge_fraction(t) -> float:
    """Fraction of the bytes of the buffer holding tensor ``t`` (from its start to the end of its mapping
    range) that transparent huge pages back, from /proc/self/smaps (0.0 where nothing is found)."""
    addr = t.data_ptr()
    nbytes = t.numel() * t.element_size()
    hp = huge_page_bytes()
    hi = addr + max(hp, -(-nbytes // hp) * hp)
    total = sum(min(b, hi) - max(a, addr) for a, b, _ in _vma_table() if a < hi and b > addr)
    return min(1.0, _huge_bytes(addr, hi) / total) if total else 0.0
