"""Power spectra of a stream of catalogs, `depth` plans deep.

Each catalog goes to the next of `depth` plans, each plan on its own CUDA
stream, round robin: pk_paint (for a host catalog, a copy into the plan's
device staging buffer on that stream), pk_compute, and the result read back
once `depth` later catalogs have been queued or the stream ends.  The copy
and the kernels of one catalog thus run while the kernels of the previous
one still occupy the GPU, so catalogs arriving from host memory do not pay
their host-to-device transfer (12 B per object in FP32) on top of the
estimator (Sec. 3.3.1 painting, Sec. 3.4.1 binning: the same plan calls as
one catalog at a time, and the same results).

Host catalogs should sit in pinned memory: a copy from pageable memory
returns only once the driver has staged it, which serializes it with the
host loop.  Every submitted array is kept referenced until its result has
been read (or, for a stream abandoned part way, until its plan's stream has
drained), since an asynchronous copy reads it after pk_paint returns."""
from __future__ import annotations

from collections import deque


def _new_stream():
    import torch
    return torch.cuda.Stream()


class PowerStream:
    """`depth` plans of one configuration, each on its own CUDA stream.

    cfg: a pk_config (make_config) with batch 1.  own_fft: None keeps the
    plan's default transform; True / False selects it (pk_use_own_fft).
    Use as a context manager, or call close()."""

    def __init__(self, cfg, depth: int = 2, own_fft=None):
        from . import pk_destroy, pk_plan, pk_use_own_fft
        if depth < 1:
            raise ValueError("depth must be at least 1")
        self.depth = depth
        self.streams = [_new_stream() for _ in range(depth)]
        self.plans = []
        try:
            for s in self.streams:
                self.plans.append(pk_plan(cfg, s))
                if own_fft is not None:
                    pk_use_own_fft(self.plans[-1], own_fft)
        except BaseException:
            for p in self.plans:
                pk_destroy(p)
            self.plans = []
            raise

    def map(self, catalogs, weights=None):
        """Yield pk_result(plan, 0) of every catalog of the iterable
        `catalogs` (arrays accepted by pk_paint, device or host), in order.
        weights: None, or an iterable of per-catalog weight arrays (or None)
        consumed alongside `catalogs`."""
        from . import pk_compute, pk_paint, pk_result
        if not self.plans:
            raise ValueError("the stream is closed")
        wit = iter(weights) if weights is not None else None
        pending = deque()                        # (plan index, arrays kept alive until read)
        try:
            for k, pos in enumerate(catalogs):
                i = k % self.depth
                if len(pending) == self.depth:
                    j, _ = pending.popleft()     # j == i: the plan about to be reused
                    yield pk_result(self.plans[j], 0)
                w = next(wit) if wit is not None else None
                pk_paint(self.plans[i], pos, w)
                pk_compute(self.plans[i])
                pending.append((i, (pos, w)))
            while pending:
                j, _ = pending[0]
                res = pk_result(self.plans[j], 0)
                pending.popleft()
                yield res
        finally:
            # abandoned (or failed) part way: copies still queued read arrays
            # this frame holds, so let them drain before the frame goes
            for j, _ in pending:
                self.streams[j].synchronize()

    def close(self):
        from . import pk_destroy
        plans, self.plans = self.plans, []
        for p in plans:
            pk_destroy(p)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def power_stream(cfg, catalogs, depth: int = 2, own_fft=None, weights=None):
    """One-shot PowerStream(cfg, depth, own_fft).map(catalogs, weights): the
    plans are made on the first result requested and destroyed at the end."""
    with PowerStream(cfg, depth, own_fft) as ps:
        yield from ps.map(catalogs, weights)
