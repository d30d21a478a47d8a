"""Continuous-batching reconstruction server.

Requests (one scan each: volume size L, a scan protocol -- a calibrated set
of view matrices -- and a projection storage mode) arrive over time; each
request's projections arrive in chunks of ``chunk_views`` views.  The
scheduler keeps the GPU busy with many requests at once:

* admission is by device-memory footprint: a request is admitted when an
  execution slot is free and its slot's bytes fit in the budget (first fit in
  arrival order, so small requests are not stuck behind a large one that does
  not fit yet); idle cached slots are evicted (least recently used) to make
  room;
* every admitted request has its own CUDA stream, so chunks of different
  requests overlap on the device, and its volume stays resident in HBM;
* each chunk pass (staging copies + the backprojection kernel, plus the FP16
  conversion in FP16 mode, plus the cosine weight and ramp filter when the
  request sends raw line integrals) is replayed from a CUDA graph captured
  once per slot and chunk index; slots are reused by later requests of the
  same shape, so graphs are captured once and replayed many times;
* deadlines are enforced on the host (a request that is not complete in time
  is reported as a timeout); no device code waits on anything.

The per-voxel summation order depends only on the view order and the views
per pass K, never on which other requests run at the same time, so a
request's volume is bitwise identical alone and in the mix.

The ``Scheduler`` is pure host logic over an ``Executor`` interface; the
``GpuExecutor`` drives the C ABI (``rct``).  Tests drive the scheduler with a
fake executor on the CPU.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Callable, Protocol

import numpy as np


@dataclass
class Protocol_:
    """A calibrated scan protocol: detector size and one 3x4 matrix per view; for requests that send
    raw line integrals, the filter geometry (source-detector distance and pixel pitch in mm, one
    principal point (u0, v0) per view)."""
    name: str
    det_w: int
    det_h: int
    matrices: np.ndarray          # (n_views, 3, 4) float64
    sdd: float | None = None
    pitch: float | None = None
    principal: np.ndarray | None = None   # (n_views, 2)


@dataclass
class Request:
    rid: int
    L: int
    protocol: str
    n_views: int
    arrival: float                 # seconds from the start of the run
    mode: str = "f32"              # projection storage: "f32" or "f16"
    chunk_views: int = 16
    chunk_interval: float = 0.0    # seconds between chunk arrivals (detector frame rate)
    deadline: float | None = None  # seconds from arrival; None = no deadline
    origin: tuple = None
    spacing: tuple = None
    raw: bool = False              # chunks are raw line integrals: weighted and filtered on the device

    @property
    def n_chunks(self) -> int:
        return -(-self.n_views // self.chunk_views)

    def chunk_arrival(self, c: int) -> float:
        return self.arrival + c * self.chunk_interval

    def chunk_range(self, c: int) -> tuple[int, int]:
        a = c * self.chunk_views
        return a, min(self.n_views, a + self.chunk_views)

    @property
    def updates(self) -> int:
        return self.L ** 3 * self.n_views


@dataclass
class Result:
    rid: int
    status: str                    # ok | timeout | rejected | error
    arrival: float
    admitted: float | None = None
    completed: float | None = None
    message: str = ""
    volume: object = None

    @property
    def time_to_volume(self) -> float | None:
        if self.completed is None:
            return None
        return self.completed - self.arrival


class Executor(Protocol):
    def footprint(self, req: Request) -> int: ...
    def open(self, req: Request): ...                  # returns a handle; may raise MemoryError
    def submit_chunk(self, handle, c: int) -> None: ...
    def seal(self, handle) -> None: ...                  # all chunks submitted
    def done(self, handle) -> bool: ...                  # sealed work finished on the device
    def finish(self, handle, keep_volume: bool): ...    # returns the volume (or None); releases the request
    def abandon(self, handle) -> None: ...               # deadline passed: release once the device is done
    def evict_idle(self, need_bytes: int) -> int: ...   # free cached idle slots; returns bytes freed
    def cached_bytes(self) -> int: ...                   # bytes held by idle cached slots
    def reusable(self, req: Request) -> bool: ...        # an idle cached slot fits this request


@dataclass
class _Active:
    req: Request
    handle: object
    footprint: int
    next_chunk: int = 0
    sealed: bool = False


class Scheduler:
    """Host-side continuous batching over an Executor (see module docstring)."""

    def __init__(self, executor: Executor, hbm_budget: int, max_active: int = 32,
                 clock: Callable[[], float] = time.perf_counter, sleep: Callable[[float], None] = time.sleep,
                 keep_volumes: bool = False, idle_sleep: float = 2e-4):
        self.ex = executor
        self.budget = int(hbm_budget)
        self.max_active = max_active
        self.clock = clock
        self.sleep = sleep
        self.keep_volumes = keep_volumes
        self.idle_sleep = idle_sleep
        self.log: list[tuple] = []      # (time, event, rid)

    def run(self, requests: list[Request]) -> list[Result]:
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: list[Request] = []
        active: dict[int, _Active] = {}
        abandoned: list[_Active] = []
        results: dict[int, Result] = {}
        used = 0                                       # bytes held by active requests
        t0 = self.clock()

        while pending or waiting or active or abandoned:
            now = self.clock() - t0
            progressed = False
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                waiting.append(r)
                results[r.rid] = Result(r.rid, "waiting", r.arrival)
                self.log.append((now, "arrive", r.rid))

            # admission: first fit in arrival order
            for r in list(waiting):
                if len(active) >= self.max_active:
                    break
                fp = self.ex.footprint(r)
                if fp > self.budget:
                    waiting.remove(r)
                    results[r.rid].status, results[r.rid].message = "rejected", "footprint exceeds the budget"
                    self.log.append((now, "reject", r.rid))
                    continue
                if not self.ex.reusable(r):            # a reused slot's bytes are already counted
                    free = self.budget - used - self.ex.cached_bytes()
                    if fp > free:
                        free += self.ex.evict_idle(fp - free)
                    if fp > free:
                        continue
                try:
                    h = self.ex.open(r)
                except (MemoryError, ValueError) as e:       # allocation failed, or the request is unservable
                    waiting.remove(r)
                    what = "allocation failed" if isinstance(e, MemoryError) else "cannot serve"
                    results[r.rid].status, results[r.rid].message = "error", f"{what}: {e}"
                    self.log.append((now, "error", r.rid))
                    continue
                waiting.remove(r)
                active[r.rid] = _Active(r, h, fp)
                used += fp
                results[r.rid].admitted = now
                self.log.append((now, "admit", r.rid))
                progressed = True

            # chunk submission, completion, deadlines
            for rid, a in list(active.items()):
                r = a.req
                while a.next_chunk < r.n_chunks and r.chunk_arrival(a.next_chunk) <= now:
                    self.ex.submit_chunk(a.handle, a.next_chunk)
                    a.next_chunk += 1
                    progressed = True
                if not a.sealed and a.next_chunk == r.n_chunks:
                    self.ex.seal(a.handle)
                    a.sealed = True
                if a.sealed and self.ex.done(a.handle):
                    vol = self.ex.finish(a.handle, self.keep_volumes)
                    res = results[rid]
                    res.completed = self.clock() - t0
                    late = r.deadline is not None and res.time_to_volume > r.deadline
                    res.status = "timeout" if late else "ok"
                    res.volume = vol if not late else None
                    del active[rid]
                    used -= a.footprint
                    self.log.append((res.completed, "done", rid))
                    progressed = True
                elif r.deadline is not None and now - r.arrival > r.deadline:
                    self.ex.abandon(a.handle)
                    results[rid].status, results[rid].message = "timeout", "deadline passed"
                    del active[rid]
                    abandoned.append(a)
                    self.log.append((now, "timeout", rid))
                    progressed = True
            for a in list(abandoned):                  # memory returns once the device is done
                if self.ex.done(a.handle):
                    self.ex.finish(a.handle, False)
                    used -= a.footprint
                    abandoned.remove(a)
            # deadlines of requests still waiting for admission
            for r in list(waiting):
                if r.deadline is not None and now - r.arrival > r.deadline:
                    waiting.remove(r)
                    results[r.rid].status, results[r.rid].message = "timeout", "not admitted before the deadline"
                    self.log.append((now, "timeout", r.rid))
            if not progressed:
                self.sleep(self.idle_sleep)
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]


def summarize(results: list[Result], requests: list[Request], wall_s: float) -> dict:
    ok = [r for r in results if r.status == "ok"]
    ttv = np.array([r.time_to_volume for r in ok]) if ok else np.array([np.nan])
    by_id = {q.rid: q for q in requests}
    updates = sum(by_id[r.rid].updates for r in ok)
    return {"requests": len(results), "ok": len(ok),
            "timeouts": sum(r.status == "timeout" for r in results),
            "rejected": sum(r.status == "rejected" for r in results),
            "errors": sum(r.status == "error" for r in results),
            "p50_ttv_s": float(np.percentile(ttv, 50)), "p99_ttv_s": float(np.percentile(ttv, 99)),
            "mean_ttv_s": float(np.mean(ttv)), "wall_s": wall_s, "gups": updates / wall_s / 1e9}


def poisson_requests(n: int, rate_hz: float, protocols: dict[str, int], *, seed: int = 0,
                     L_choices=(128, 256, 512, 1024), L_weights=(0.4, 0.3, 0.2, 0.1), mode: str = "f32",
                     chunk_views: int = 16, views_per_s: float = 2000.0, deadline: float | None = None,
                     origin_spacing: Callable[[int], tuple] | None = None, raw: bool = False) -> list[Request]:
    """Seeded Poisson arrivals with mixed L and protocols (protocol name -> view count)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    names = sorted(protocols)
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        L = int(rng.choice(L_choices, p=np.asarray(L_weights) / np.sum(L_weights)))
        name = names[int(rng.integers(len(names)))]
        o, s = origin_spacing(L) if origin_spacing else (None, None)
        out.append(Request(i, L, name, protocols[name], t, mode, chunk_views, chunk_views / views_per_s,
                           deadline, o, s, raw))
    return out


# ----------------------------------------------------------------------------- GPU executor

@dataclass
class _Slot:
    key: tuple
    bp: object
    stream: object
    d_chunk: object
    d_half: object
    graphs: list
    footprint: int
    done_event: object = None
    last_used: float = 0.0


@dataclass
class _Handle:
    req: Request
    slot: _Slot
    host: object                   # pinned (n_views, H, W) FP32 projections of the protocol
    abandoned: bool = False


class GpuExecutor:
    """Runs requests through the C ABI with persistent per-shape slots and captured CUDA graphs.

    A slot = one context (resident L^3 volume + staging), one stream, a device
    chunk buffer and one captured graph per chunk index.  ``host_data`` maps
    protocol name -> pinned FP32 host projections (n_views, H, W) that chunks
    are copied from as they "arrive".
    """

    def __init__(self, protocols: dict[str, Protocol_], host_data: dict, *, use_graphs: bool = True,
                 tuning_fn=None, device: int = 0, timeline: bool = False):
        import torch
        from . import rct, tuning
        self.torch = torch
        self.rct = rct
        self.protocols = protocols
        self.host = host_data
        self.use_graphs = use_graphs
        self.tuning_fn = tuning_fn or (lambda L, mode: tuning.lookup(L, mode, "soft"))
        self.device = torch.device("cuda", device)
        self.free_slots: dict[tuple, list[_Slot]] = collections.defaultdict(list)
        self.graph_launches = 0
        self.captures = 0
        # Device timeline (optional): timing events around every chunk's work on its request's stream, so the
        # device intervals of different requests' work can be compared after the run (device_timeline()).
        self.timeline = False
        self._marks: list = []
        self._t0 = None
        if timeline:
            self.start_timeline()

    def start_timeline(self) -> None:
        """Start (or restart) recording the device timeline; earlier records are dropped."""
        torch = self.torch
        torch.cuda.synchronize(self.device)
        self.timeline = True
        self._marks = []
        self._t0 = torch.cuda.Event(enable_timing=True)
        self._t0.record(torch.cuda.current_stream(self.device))

    # -- sizing
    def _key(self, r: Request) -> tuple:
        o = tuple(r.origin) if r.origin is not None else None
        s = tuple(r.spacing) if r.spacing is not None else None
        return (r.L, r.protocol, r.n_views, r.mode, r.chunk_views, o, s, r.raw)

    def footprint(self, r: Request) -> int:
        p = self.protocols[r.protocol]
        t = self.tuning_fn(r.L, r.mode)
        code = self.rct.RCT_PROJ_F16 if r.mode == "f16" else self.rct.RCT_PROJ_F32
        px = p.det_w * p.det_h
        chunk = r.chunk_views * px * 4 + (r.chunk_views * px * 2 if r.mode == "f16" else 0)
        return self.rct.rct_footprint_bytes(r.L, p.det_w, p.det_h, code, t["views_per_pass"], False) + chunk

    def cached_bytes(self) -> int:
        return sum(s.footprint for lst in self.free_slots.values() for s in lst)

    def reusable(self, r: Request) -> bool:
        return bool(self.free_slots.get(self._key(r)))

    def evict_idle(self, need: int) -> int:
        idle = sorted((s for lst in self.free_slots.values() for s in lst), key=lambda s: s.last_used)
        freed = 0
        for s in idle:
            if freed >= need:
                break
            self.free_slots[s.key].remove(s)
            self._destroy(s)
            freed += s.footprint
        return freed

    def _destroy(self, s: _Slot):
        for g in s.graphs:
            self.rct.rct_graph_destroy(g)
        s.graphs = []
        s.bp.close()

    # -- slots
    def _new_slot(self, r: Request) -> _Slot:
        torch, rct = self.torch, self.rct
        p = self.protocols[r.protocol]
        try:
            bp = rct.Backprojector(r.L, p.det_w, p.det_h, r.n_views)
        except rct.RctError as e:
            if e.status == rct.RCT_ENOMEM:
                raise MemoryError(str(e)) from e
            raise
        origin, spacing = r.origin, r.spacing
        if origin is None:
            sp = 256.0 / r.L
            origin, spacing = [-(r.L - 1) / 2.0 * sp] * 3, [sp] * 3
        bp.set_geometry(p.matrices[:r.n_views], origin, spacing)
        code = rct.RCT_PROJ_F16 if r.mode == "f16" else rct.RCT_PROJ_F32
        bp.set_precision(code, rct.RCT_INTERP_SOFT)
        bp.set_tuning(**self.tuning_fn(r.L, r.mode))
        if r.raw:
            if p.sdd is None or p.pitch is None or p.principal is None:
                bp.close()
                raise ValueError(f"protocol {p.name} has no filter geometry for raw projections")
            bp.set_filter(p.sdd, p.pitch, p.principal[:r.n_views])
        rct.rct_prepare(bp.ctx, False)
        stream = torch.cuda.Stream(device=self.device)
        d_chunk = torch.empty((r.chunk_views, p.det_h, p.det_w), dtype=torch.float32, device=self.device)
        d_half = (torch.empty((r.chunk_views, p.det_h, p.det_w), dtype=torch.float16, device=self.device)
                  if r.mode == "f16" else None)
        slot = _Slot(self._key(r), bp, stream, d_chunk, d_half, [], self.footprint(r))
        if self.use_graphs:
            bp.reset(stream)
            for c in range(r.n_chunks):
                rct.rct_graph_begin(stream)
                try:
                    self._chunk_work(slot, r, c)
                finally:
                    g = rct.rct_graph_end(stream)
                slot.graphs.append(g)
                self.captures += 1
        return slot

    def _chunk_work(self, slot: _Slot, r: Request, c: int):
        """The device work of one chunk pass, after its projections are in d_chunk."""
        rct = self.rct
        a, b = r.chunk_range(c)
        n = b - a
        src = slot.d_chunk
        if r.raw:
            # cosine weight + ramp filter; FP16 mode writes the narrowed result directly
            dst, code = ((slot.d_half, rct.RCT_PROJ_F16) if slot.d_half is not None
                         else (slot.d_chunk, rct.RCT_PROJ_F32))
            rct.rct_filter_projections(slot.bp.ctx, slot.d_chunk, dst, code, a, n, slot.stream)
            src = dst
        elif slot.d_half is not None:
            rct.rct_convert_projections(slot.d_chunk, slot.d_half, n * slot.d_chunk[0].numel(),
                                        rct.RCT_PROJ_F16, slot.stream)
            src = slot.d_half
        rct.rct_backproject(slot.bp.ctx, src, a, n, slot.stream)

    def open(self, r: Request) -> _Handle:
        key = self._key(r)
        slot = self.free_slots[key].pop() if self.free_slots[key] else self._new_slot(r)
        if not self.use_graphs:
            slot.bp.reset(slot.stream)
        return _Handle(r, slot, self.host[r.protocol + "/raw" if r.raw else r.protocol])

    def submit_chunk(self, h: _Handle, c: int) -> None:
        torch = self.torch
        a, b = h.req.chunk_range(c)
        s = h.slot
        if self.timeline:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
        with torch.cuda.stream(s.stream):
            s.d_chunk[:b - a].copy_(h.host[a:b], non_blocking=True)
        if self.use_graphs:
            self.rct.rct_graph_launch(s.graphs[c], s.stream)
            self.graph_launches += 1
        else:
            self._chunk_work(s, h.req, c)
        if self.timeline:
            e1.record(s.stream)
            self._marks.append((h.req.rid, c, e0, e1))

    def device_timeline(self) -> list[tuple[int, int, float, float]]:
        """(request id, chunk, start ms, end ms) of every chunk's device work since the executor was made: from
        the moment its stream reached the chunk's copy to the end of its pass (call after the work is done)."""
        self.torch.cuda.synchronize(self.device)
        return [(rid, c, self._t0.elapsed_time(e0), self._t0.elapsed_time(e1)) for rid, c, e0, e1 in self._marks]

    def seal(self, h: _Handle) -> None:
        h.slot.done_event = self.torch.cuda.Event()
        h.slot.done_event.record(h.slot.stream)

    def done(self, h: _Handle) -> bool:
        ev = h.slot.done_event
        return ev is not None and ev.query()

    def finish(self, h: _Handle, keep_volume: bool):
        torch = self.torch
        vol = None
        s = h.slot
        if keep_volume:
            L = h.req.L
            vol = torch.empty((L, L, L), dtype=torch.float32, device=self.device)
            s.bp.read_volume(vol, s.stream)
            s.stream.synchronize()
            vol = vol.cpu()
        s.done_event = None
        s.last_used = time.perf_counter()
        self.free_slots[s.key].append(s)
        return vol

    def abandon(self, h: _Handle) -> None:
        h.abandoned = True
        if h.slot.done_event is None:                # not sealed: mark the end of what was queued
            self.seal(h)

    def close(self):
        for lst in self.free_slots.values():
            for s in lst:
                self._destroy(s)
        self.free_slots.clear()


def overlap_stats(intervals: list[tuple[int, int, float, float]]) -> dict:
    """From (request id, chunk, start, end) device intervals: the time some request's work was in flight, the
    time at least two different requests' work was, and the largest number of requests in flight at once."""
    events = []
    for rid, _, a, b in intervals:
        if b > a:
            events.append((a, 1, rid))
            events.append((b, -1, rid))
    events.sort(key=lambda e: (e[0], e[1]))
    live: dict[int, int] = collections.Counter()
    busy = multi = 0.0
    peak = 0
    last = None
    for t, d, rid in events:
        if last is not None:
            n = sum(1 for v in live.values() if v > 0)
            if n >= 1:
                busy += t - last
            if n >= 2:
                multi += t - last
        live[rid] += d
        peak = max(peak, sum(1 for v in live.values() if v > 0))
        last = t
    return {"busy_ms": busy, "overlap_ms": multi, "overlap_fraction": (multi / busy) if busy else 0.0,
            "peak_requests_in_flight": peak}
