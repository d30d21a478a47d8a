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
with fragmented memory), and registered with ``cudaHostRegister``;
``huge_fraction`` reports how much of a buffer huge pages back.  The returned tensor owns the buffer:
it is unregistered and unmapped when the tensor and every view of it are
gone.  Where transparent huge pages are switched off the buffer is still
aligned, locked and registered, in base pages.
"""
from __future__ import annotations

import ctypes
import ctypes.util
from pathlib import Path

_PROT_RW = 0x1 | 0x2
_MAP_PRIVATE_ANON = 0x02 | 0x20
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


def pinned_empty(shape, dtype):
    """A page-locked, huge-page-backed host tensor of ``shape`` and ``dtype`` (contents zero)."""
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
    raw = libc.mmap(None, raw_size, _PROT_RW, _MAP_PRIVATE_ANON, -1, 0)
    if raw in (None, ctypes.c_void_p(-1).value):
        raise MemoryError(f"mmap of {raw_size} bytes failed (errno {ctypes.get_errno()})")
    start = -(-raw // hp) * hp
    if huge:
        libc.madvise(start, size, _MADV_HUGEPAGE)
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

    mapping = _Mapping.from_address(start)
    t = torch.frombuffer(mapping, dtype=torch.uint8)
    t.zero_()                                     # touch every page before it is locked
    if huge:
        libc.madvise(start, size, _MADV_COLLAPSE)  # best effort: fails harmlessly where unsupported
    err = cudart.cudaHostRegister(start, size, 0)
    if int(err) != 0:
        raise RuntimeError(f"cudaHostRegister of {size} bytes failed: {err}")
    mapping.registered = True
    return t[:nbytes].view(dtype).view(*[int(s) for s in shape])


def huge_fraction(t) -> float:
    """Fraction of the memory mapping that holds tensor ``t`` which transparent huge pages back (from
    /proc/self/smaps; 0.0 where the mapping is not found)."""
    addr = t.data_ptr()
    try:
        lines = Path("/proc/self/smaps").read_text().splitlines()
    except OSError:
        return 0.0
    inside = False
    size = huge = 0
    for line in lines:
        head = line.split()[0] if line.split() else ""
        if "-" in head and ":" not in head:
            lo, hi = (int(x, 16) for x in head.split("-"))
            inside = lo <= addr < hi
            continue
        if inside and line.startswith("Size:"):
            size = int(line.split()[1])
        elif inside and line.startswith("AnonHugePages:"):
            huge = int(line.split()[1])
            break
    return huge / size if size else 0.0
