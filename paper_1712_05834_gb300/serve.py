"""Serving P(k) requests with continuous batching over device-resident plans.

A request is one catalog (device-resident positions plus its Nmesh, window
and interlacing) that arrives at some time and wants its power spectrum back.
The server keeps a pool of *slots*.  A slot belongs to one size class (see
``batch.class_key``) and owns a plan with room for ``b`` catalogs and ``C``
objects, a staging buffer of ``C`` objects that the plan paints from, its own
CUDA stream and a completion event.  Meshes, cuFFT plans, bin tables and sort
buffers stay resident between requests.

Continuous batching: each pass of the loop (1) polls the busy slots and
hands back every finished result (pk_result) to its request, (2) gives each
idle slot up to ``b`` waiting requests of its class (FIFO, up to ``C``
objects), copies their positions into the slot's staging buffer and enqueues
one pk_paint_many + pk_compute on the slot's stream.  Requests that arrive
while others are on the GPU join the next batch of their class as soon as a
slot of that class is free, and slots of different classes run on different
streams, so their kernels overlap on the device.  Slots for small meshes get
high-priority streams so that a long job does not hold them back.

Admission by free HBM: a new slot is created only if its estimated device
footprint fits both in the device's free memory (minus a reserve) and in the
server's budget minus what resident slots hold.  To make room, idle slots of
other classes are evicted, least recently used first; a request whose class
cannot get a slot waits in the queue.

Latency of a request = time from its arrival to the moment its result is on
the host.  This module only schedules: every step of the estimator runs in
libpk.so's kernels through the C ABI.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import make_config, pk_compute, pk_destroy, pk_paint_many, pk_plan, pk_result
from .batch import Catalog, class_key


@dataclass
class Request:
    """One P(k) request; ``arrival`` is in seconds from the start of the run."""
    rid: int
    catalog: Catalog
    arrival: float = 0.0
    result: dict | None = None
    t_done: float = float("nan")
    batch_size: int = 0
    tag: str = ""

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def slot_bytes(nmesh: int, interlaced: bool, precision: str, batch: int, capacity: int,
               variant: str = "sort", tile: int = 16) -> int:
    """Estimated device bytes of a slot: meshes, the cuFFT work area (taken as
    one more mesh), sort or atomic buffers, key counts and the staging buffer."""
    nm = 2 if interlaced else 1
    esz = 8 if precision == "f64" else 4
    mesh = batch * nm * nmesh * nmesh * 2 * (nmesh // 2 + 1) * esz
    work = mesh // batch
    if variant == "atomic":
        paint = batch * nm * nmesh ** 3 * 8
    else:
        paint = capacity * 16 + 2 * batch * (nmesh // max(tile, 1)) ** 3 * 27 * 4
    staging = capacity * 16
    return int(mesh + work + paint + staging + (8 << 20))


class _Slot:
    def __init__(self, server, key, batch, capacity, priority):
        import torch
        self.key = key
        self.batch = batch
        self.capacity = capacity
        nmesh, window, interlaced, precision = key[0], key[1], key[2], key[3]
        self.stream = torch.cuda.Stream(priority=priority)
        self.event = torch.cuda.Event()
        width = key[5]
        dtype = torch.float64 if "float64" in key[4] else torch.float32
        self.buf = torch.empty((capacity, width), dtype=dtype, device="cuda")
        self.wbuf = torch.empty((capacity,), dtype=torch.float32, device="cuda") if key[6] else None
        cfg = make_config(nmesh=nmesh, window=window, interlaced=interlaced, batch=batch,
                          capacity=capacity, **server.cfg_kwargs)
        self.plan = pk_plan(cfg, self.stream)
        self.bytes = slot_bytes(nmesh, interlaced, precision, batch, capacity)
        self.busy: list = []
        self.last_used = 0.0

    def start(self, reqs, now_fn):
        """Stage the requests' positions and enqueue paint + compute."""
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())
        offsets = [0]
        with torch.cuda.stream(self.stream):
            for r in reqs:
                a, n = offsets[-1], r.catalog.n
                self.buf[a:a + n].copy_(r.catalog.pos, non_blocking=True)
                if self.wbuf is not None:
                    self.wbuf[a:a + n].copy_(r.catalog.weights, non_blocking=True)
                offsets.append(a + n)
        n = offsets[-1]
        pk_paint_many(self.plan, self.buf[:n], np.asarray(offsets, np.int64),
                      None if self.wbuf is None else self.wbuf[:n])
        pk_compute(self.plan)
        self.event.record(self.stream)
        self.busy = list(reqs)
        for r in reqs:
            r.batch_size = len(reqs)
        self.last_used = now_fn()

    def poll(self, now_fn) -> list:
        """Hand back finished results; returns the finished requests."""
        if not self.busy or not self.event.query():
            return []
        done = self.busy
        for j, r in enumerate(done):
            r.result = pk_result(self.plan, j)
            r.t_done = now_fn()
        self.busy = []
        self.last_used = now_fn()
        return done

    def close(self):
        if self.plan:
            self.stream.synchronize()
            pk_destroy(self.plan)
            self.plan = None
        self.buf = None
        self.wbuf = None


class PowerServer:
    """Continuous-batching P(k) server over resident plans (see module doc).

    ``max_batch``: catalogs per slot; ``max_objects``: objects per slot batch;
    ``slots_per_class``: slots a class may hold at once; ``budget_bytes``: HBM
    the server may hold in slots (None: free HBM at start minus ``reserve_bytes``);
    ``large_nmesh``: classes with Nmesh at least this get one catalog per slot,
    sized to the request, and normal-priority streams."""

    def __init__(self, box_size, dk=None, kmin=0.0, kmax=None, nmu=0, poles=(0, 2, 4), precision="f32",
                 compensated=True, subtract_shot=True, max_batch=8, max_objects=16_000_000,
                 slots_per_class=2, budget_bytes=None, reserve_bytes=4 << 30, large_nmesh=512):
        import torch
        self.torch = torch
        self.cfg_kwargs = dict(box_size=box_size, dk=dk, kmin=kmin, kmax=kmax, nmu=nmu, poles=poles,
                               precision=precision, compensated=compensated,
                               subtract_shot=subtract_shot)
        self.precision = precision
        self.max_batch = int(max_batch)
        self.max_objects = int(max_objects)
        self.slots_per_class = int(slots_per_class)
        self.reserve = int(reserve_bytes)
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(budget_bytes) if budget_bytes is not None else max(free - self.reserve, 0)
        self.large_nmesh = int(large_nmesh)
        self.slots: list[_Slot] = []
        self.queue: dict = collections.OrderedDict()     # class key -> deque of requests
        self.t0 = time.perf_counter()
        self.evictions = 0
        self.slots_made = 0
        self.peak_bytes = 0

    # ---- bookkeeping ----
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def held_bytes(self) -> int:
        return sum(s.bytes for s in self.slots)

    def submit(self, req: Request):
        self.queue.setdefault(class_key(req.catalog, self.precision), collections.deque()).append(req)

    def pending(self) -> int:
        return sum(len(q) for q in self.queue.values()) + sum(len(s.busy) for s in self.slots)

    # ---- admission ----
    def _slot_shape(self, key, head: Request):
        if key[0] >= self.large_nmesh:
            return 1, max(head.catalog.n, 1)
        return self.max_batch, max(self.max_objects, head.catalog.n)

    def _admit(self, key, head: Request):
        """A new slot for `key` if HBM allows (evicting idle slots of other
        classes, least recently used first), else None."""
        batch, cap = self._slot_shape(key, head)
        need = slot_bytes(key[0], key[2], key[3], batch, cap)
        idle_other = sorted((s for s in self.slots if not s.busy and s.key != key), key=lambda s: s.last_used)
        while True:
            free, _ = self.torch.cuda.mem_get_info()
            if need <= self.budget - self.held_bytes() and need <= free - self.reserve:
                break
            if not idle_other:
                return None
            victim = idle_other.pop(0)
            victim.close()
            self.slots.remove(victim)
            self.evictions += 1
            self.torch.cuda.empty_cache()
        prio = 0 if key[0] >= self.large_nmesh else -1
        slot = _Slot(self, key, batch, cap, prio)
        self.slots.append(slot)
        self.slots_made += 1
        self.peak_bytes = max(self.peak_bytes, self.held_bytes())
        return slot

    def _dispatch(self) -> int:
        started = 0
        for key, q in self.queue.items():
            while q:
                n0 = q[0].catalog.n
                slot = next((s for s in self.slots if s.key == key and not s.busy and s.capacity >= n0), None)
                if slot is None:
                    same = [s for s in self.slots if s.key == key]
                    if len(same) >= self.slots_per_class:
                        small = [s for s in same if not s.busy and s.capacity < n0]
                        if not small:
                            break
                        small[0].close()                 # too small for this request: rebuild
                        self.slots.remove(small[0])
                        self.evictions += 1
                    slot = self._admit(key, q[0])
                    if slot is None:
                        break
                take, n = [], 0
                while q and len(take) < slot.batch and n + q[0].catalog.n <= slot.capacity:
                    n += q[0].catalog.n
                    take.append(q.popleft())
                if not take:
                    break
                slot.start(take, self.now)
                started += 1
        return started

    def step(self) -> list:
        """Poll finished work, then start every batch that can start."""
        done = []
        for s in self.slots:
            done += s.poll(self.now)
        started = self._dispatch()
        if not started and not done and any(self.queue.values()) and not any(s.busy for s in self.slots):
            key = next(k for k, q in self.queue.items() if q)
            raise RuntimeError("request of class %s cannot be admitted: the HBM budget (%d bytes) is "
                               "too small for its slot" % (key, self.budget))
        return done

    # ---- runs ----
    def run(self, requests, realtime: bool = True, idle_sleep: float = 50e-6) -> list:
        """Serve `requests` (sorted by arrival).  With realtime=True a request
        is submitted once the wall clock passes its arrival; otherwise all are
        submitted at once (arrival 0, saturated throughput)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        if not realtime:
            for r in reqs:
                r.arrival = 0.0
        self.t0 = time.perf_counter()
        k = 0
        while k < len(reqs) or self.pending():
            t = self.now()
            while k < len(reqs) and reqs[k].arrival <= t:
                self.submit(reqs[k])
                k += 1
            done = self.step()
            if not done and k < len(reqs):
                wait = reqs[k].arrival - self.now()
                if wait > 0:
                    time.sleep(min(idle_sleep, wait))
        return reqs

    def close(self):
        for s in self.slots:
            s.close()
        self.slots = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def plain_serve(requests, box_size, realtime: bool = True, **cfg_kwargs) -> list:
    """The one-at-a-time path: requests in arrival order, each painted,
    transformed, binned and read back alone (pk_paint / pk_compute / pk_result)
    on a resident batch-1 plan of its class before the next one starts."""
    import torch
    reqs = sorted(requests, key=lambda r: r.arrival)
    if not realtime:
        for r in reqs:
            r.arrival = 0.0
    plans = {}
    stream = torch.cuda.current_stream()
    try:
        t0 = time.perf_counter()
        for r in reqs:
            while realtime and time.perf_counter() - t0 < r.arrival:
                pass
            key = class_key(r.catalog, cfg_kwargs.get("precision", "f32"))
            if key not in plans:
                cfg = make_config(box_size=box_size, nmesh=key[0], window=key[1], interlaced=key[2],
                                  **cfg_kwargs)
                plans[key] = pk_plan(cfg, stream)
            from . import pk_paint
            pk_paint(plans[key], r.catalog.pos, r.catalog.weights)
            pk_compute(plans[key])
            r.result = pk_result(plans[key], 0)
            r.t_done = time.perf_counter() - t0
            r.batch_size = 1
    finally:
        for p in plans.values():
            pk_destroy(p)
    return reqs


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def latency_summary(reqs) -> dict:
    """p50 / p99 / mean / max latency (ms), served P(k)/s over the run, mean
    batch size; per tag as well when the requests carry tags."""
    lat = np.array([r.latency for r in reqs]) * 1e3
    t_end = max(r.t_done for r in reqs)
    t_begin = min(r.arrival for r in reqs)
    out = {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
           "max_ms": float(lat.max()), "pk_per_s": len(reqs) / max(t_end - t_begin, 1e-9),
           "mean_batch": float(np.mean([r.batch_size for r in reqs]))}
    tags = sorted({r.tag for r in reqs if r.tag})
    for t in tags:
        lt = np.array([r.latency for r in reqs if r.tag == t]) * 1e3
        out["by_tag"] = out.get("by_tag", {})
        out["by_tag"][t] = {"requests": int(lt.size), "p50_ms": float(np.percentile(lt, 50)),
                            "p99_ms": float(np.percentile(lt, 99)), "max_ms": float(lt.max())}
    return out
