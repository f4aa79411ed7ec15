"""Power spectra of many catalogs at once: size classes, an autotuner, CUDA graphs.

Covariance estimates need P(k) of hundreds of mock catalogs of uneven size
(the paper's log-normal mocks, Sec. 3.2).  Evaluating them one at a time pays
every launch and every small-grid tail once per mock.  Here the mocks are
grouped into size classes -- one class per (Nmesh, window, interlacing, mesh
precision, position layout, weighted or not) -- and each class is ONE plan
whose batch holds all of its catalogs, back to back in one device buffer:

  * one pk_paint_many per class: one count / scan / scatter / tile-paint
    launch set (or one atomic-paint launch and one conversion launch) over
    every catalog of the class;
  * one batched cuFFT call over every mesh of the class;
  * one bin launch (persistent CTAs, a fixed share per catalog), one reduce
    and one finalize launch over every catalog of the class.

The whole sequence for all classes is captured once into a CUDA graph on the
runner's stream and replayed per evaluation; the graph re-reads the position
buffers in place, so refilling them with new mocks and replaying evaluates the
new mocks.  Classes are independent: with ``streams`` > 1 their plans are
spread over that many CUDA streams (largest classes first, each to the
least-loaded stream), forked from and joined back into the runner's stream,
so the graph holds parallel branches and one class's kernels fill the SMs
another leaves idle (grid tails, small reduce / scan / finalize launches).  The autotuner picks, per class, the paint variant (tile sort or
direct atomics) and the tile edge by timing every candidate on the class's own
catalogs; results do not depend on the choice (both variants paint the same
int64 fixed-point cells up to one rounding of each deposit).

This module is host-side scheduling only: every step of the estimator runs in
libpk.so's kernels through the C ABI.  torch provides device memory, streams,
events and graph capture.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import (PkError, make_config, pk_compute, pk_destroy, pk_launch_count, pk_paint_many,
               pk_plan, pk_result)

# Window support span in cells on the meshes painted (both, if interlaced):
# the tile edge must be at least this (a tile's objects reach one neighbour).
_SPAN = {(2, False): 1, (2, True): 2, (3, False): 3, (3, True): 3, (4, False): 3, (4, True): 4}
_WINDOW_P = {"cic": 2, "tsc": 3, "pcs": 4}
TILE_CHOICES = (8, 12, 16, 24)


@dataclass
class Catalog:
    """One catalog: positions (n, 3) float32/float64 or (n, 4) float32 xyzw on
    the device, optional float32 weights (n,), and its mesh options."""
    pos: object
    nmesh: int
    window: str = "cic"
    interlaced: bool = False
    weights: object = None

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def class_key(cat: Catalog, precision: str = "f32") -> tuple:
    """Size class of a catalog: catalogs of one class share a plan."""
    return (int(cat.nmesh), str(cat.window), bool(cat.interlaced), precision,
            str(cat.pos.dtype), int(cat.pos.shape[1]), cat.weights is not None)


def group_classes(catalogs, precision: str = "f32") -> dict:
    """Class key -> indices of its catalogs, classes and members in input order."""
    groups: dict = {}
    for i, c in enumerate(catalogs):
        groups.setdefault(class_key(c, precision), []).append(i)
    return groups


def tile_candidates(nmesh: int, window: str, interlaced: bool) -> list:
    """Tile edges the tile-sort paint accepts for this mesh and window."""
    span = _SPAN[(_WINDOW_P[window], bool(interlaced))]
    return [t for t in TILE_CHOICES if t >= span and nmesh % t == 0]


def paint_candidates(nmesh: int, window: str, interlaced: bool) -> list:
    """(variant, tile) pairs the autotuner times; tile 0 = the library's choice."""
    cands = [("sort", t) for t in tile_candidates(nmesh, window, interlaced)]
    if not cands:
        cands = [("sort", 0)]
    return cands + [("atomic", 0)]


def tune_key(key: tuple, mean_objects: float) -> str:
    """Autotuner cache key: the size class plus log2 of the mean catalog size
    (the best variant depends on the objects per cell)."""
    nmesh, window, interlaced, precision, dtype, width, weighted = key
    return "N%d-%s-%s-%s-%s%d-%s-n2^%d" % (nmesh, window, "il" if interlaced else "noil", precision,
                                           dtype.replace("torch.", ""), width,
                                           "w" if weighted else "unit",
                                           int(round(math.log2(max(mean_objects, 1.0)))))


def assign_streams(loads, nstreams: int) -> list:
    """Stream index of each class: largest load first, each to the stream
    with the least load so far (ties: the lower index)."""
    where = [0] * len(loads)
    total = [0] * max(int(nstreams), 1)
    for k in sorted(range(len(loads)), key=lambda k: (-loads[k], k)):
        s = min(range(len(total)), key=lambda j: (total[j], j))
        where[k] = s
        total[s] += loads[k]
    return where


class Autotuner:
    """Times each (paint variant, tile edge) candidate on a sample of a class's
    catalogs and keeps the fastest per tune_key.  The cache can be saved to and
    loaded from a JSON file so later runs skip the timing."""

    def __init__(self, path: str | None = None, sample: int = 16, repeats: int = 3):
        self.path = path
        self.sample = int(sample)
        self.repeats = int(repeats)
        self.cache: dict = {}
        self.timings: dict = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = {k: tuple(v) for k, v in json.load(f).items()}

    def save(self):
        if self.path:
            with open(self.path, "w") as f:
                json.dump({k: list(v) for k, v in self.cache.items()}, f, indent=1, sort_keys=True)

    def choose(self, key: tuple, cfg_kwargs: dict, pos, offsets, weights, stream) -> tuple:
        """Best (variant, tile) for this class, timing candidates if not cached."""
        import torch
        offsets = np.asarray(offsets, dtype=np.int64)
        nitems = len(offsets) - 1
        tk = tune_key(key, offsets[-1] / max(nitems, 1))
        if tk in self.cache:
            return self.cache[tk]
        m = min(nitems, self.sample)
        off = offsets[: m + 1]
        sub = pos[: int(off[-1])]
        wsub = None if weights is None else weights[: int(off[-1])]
        nmesh, window, interlaced = key[0], key[1], key[2]
        times = {}
        for variant, tile in paint_candidates(nmesh, window, interlaced):
            try:
                cfg = make_config(nmesh=nmesh, window=window, interlaced=interlaced, batch=m,
                                  tile=tile, paint_variant=variant, capacity=int(off[-1]), **cfg_kwargs)
                plan = pk_plan(cfg, stream)
            except PkError:
                continue
            try:
                with torch.cuda.stream(stream):
                    pk_paint_many(plan, sub, off, wsub)                 # warm-up
                    t0 = torch.cuda.Event(enable_timing=True)
                    t1 = torch.cuda.Event(enable_timing=True)
                    t0.record(stream)
                    for _ in range(self.repeats):
                        pk_paint_many(plan, sub, off, wsub)
                    t1.record(stream)
                t1.synchronize()
                times["%s/%d" % (variant, tile)] = t0.elapsed_time(t1) / self.repeats
            finally:
                pk_destroy(plan)
        if not times:
            raise PkError(1, "no paint candidate accepted class %s" % (key,))
        best = min(times, key=times.get)
        variant, tile = best.split("/")
        self.cache[tk] = (variant, int(tile))
        self.timings[tk] = times
        return self.cache[tk]


@dataclass
class _Class:
    key: tuple
    index: list
    offsets: np.ndarray
    pos: object
    weights: object
    choice: tuple
    stream_index: int = 0
    plan: object = None
    results: list = field(default_factory=list)


class BatchPower:
    """P(k) of a fixed set of catalogs, evaluated by size class.

    The catalogs' positions are copied once into one contiguous buffer per
    class (``refill`` copies new catalogs of the same sizes into them).  With
    ``graph=True`` the paint + compute calls of every class are captured into
    one CUDA graph at construction; ``run()`` replays it and returns one result
    dict per catalog (pk_result's fields), in input order."""

    def __init__(self, catalogs, box_size, dk=None, kmin=0.0, kmax=None, nmu=0, poles=(0, 2, 4),
                 precision="f32", compensated=True, subtract_shot=True, tuner: Autotuner | None = None,
                 graph: bool = True, stream=None, streams: int = 1):
        import torch
        if not catalogs:
            raise ValueError("no catalogs")
        if streams < 1:
            raise ValueError("streams must be at least 1")
        self.torch = torch
        self.n = len(catalogs)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.streams = [self.stream] + [torch.cuda.Stream() for _ in range(streams - 1)]
        self.cfg_kwargs = dict(box_size=box_size, dk=dk, kmin=kmin, kmax=kmax, nmu=nmu, poles=poles,
                               precision=precision, compensated=compensated,
                               subtract_shot=subtract_shot)
        self.classes: list[_Class] = []
        self.graph = None
        self.launches_per_run = 0
        self.stream.wait_stream(torch.cuda.current_stream())     # catalogs written on it
        try:
            groups = group_classes(catalogs, precision)
            where = assign_streams([sum(catalogs[i].n for i in idx) for idx in groups.values()],
                                   len(self.streams))
            for (key, idx), si in zip(groups.items(), where):
                sizes = [catalogs[i].n for i in idx]
                offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
                with torch.cuda.stream(self.stream):
                    pos = torch.cat([catalogs[i].pos for i in idx]).contiguous()
                    w = None if not key[6] else torch.cat([catalogs[i].weights for i in idx]).contiguous()
                choice = ("sort", 0)
                if tuner is not None:
                    choice = tuner.choose(key, self.cfg_kwargs, pos, offsets, w, self.stream)
                cfg = make_config(nmesh=key[0], window=key[1], interlaced=key[2], batch=len(idx),
                                  tile=choice[1], paint_variant=choice[0],
                                  capacity=max(int(offsets[-1]), 1), **self.cfg_kwargs)
                c = _Class(key, idx, offsets, pos, w, choice, si)
                c.plan = pk_plan(cfg, self.streams[si])
                self.classes.append(c)
            self.stream.synchronize()
            if graph:
                self._capture()
        except Exception:
            self.close()
            raise

    def _enqueue(self):
        torch = self.torch
        if len(self.streams) > 1:                 # fork: every class stream after the runner's
            fork = torch.cuda.Event()
            fork.record(self.stream)
            for s in self.streams[1:]:
                s.wait_event(fork)
        for c in self.classes:
            pk_paint_many(c.plan, c.pos, c.offsets, c.weights)
            pk_compute(c.plan)
        for s in self.streams[1:]:                # join: the runner's stream after every class
            e = torch.cuda.Event()
            e.record(s)
            self.stream.wait_event(e)

    def _capture(self):
        torch = self.torch
        before = sum(pk_launch_count(c.plan) for c in self.classes)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream, capture_error_mode="thread_local"):
            self._enqueue()
        self.launches_per_run = sum(pk_launch_count(c.plan) for c in self.classes) - before
        self.graph = g

    def refill(self, catalogs):
        """Copy new catalogs (same classes and sizes, same order) into the
        position buffers the plans read."""
        torch = self.torch
        if len(catalogs) != self.n:
            raise ValueError("refill needs as many catalogs as the runner holds")
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for c in self.classes:
                for j, i in enumerate(c.index):
                    cat = catalogs[i]
                    a, b = int(c.offsets[j]), int(c.offsets[j + 1])
                    if cat.n != b - a:
                        raise ValueError("catalog %d has %d objects, the runner holds %d" % (i, cat.n, b - a))
                    c.pos[a:b].copy_(cat.pos)
                    if c.weights is not None:
                        c.weights[a:b].copy_(cat.weights)

    def launch(self):
        """Enqueue one evaluation of every catalog on the runner's stream."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                before = sum(pk_launch_count(c.plan) for c in self.classes)
                self._enqueue()
                self.launches_per_run = sum(pk_launch_count(c.plan) for c in self.classes) - before

    def results(self) -> list:
        """Wait for the last launch and return one result dict per catalog."""
        self.stream.synchronize()
        out = [None] * self.n
        for c in self.classes:
            for j, i in enumerate(c.index):
                out[i] = pk_result(c.plan, j)
        return out

    def run(self) -> list:
        self.launch()
        return self.results()

    def close(self):
        self.graph = None
        for c in self.classes:
            if c.plan:
                pk_destroy(c.plan)
                c.plan = None
        self.classes = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
