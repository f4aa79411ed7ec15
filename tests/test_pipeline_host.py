"""Order of the plan calls in pipeline.PowerStream / power_stream (CPU, fake
plan calls): round robin over `depth` plans, results read in submission
order once `depth` later catalogs are queued, every submitted array kept
alive until its result is read (or its stream drained), every plan
destroyed."""
import weakref

import pytest

import paper_1712_05834_gb300 as pk
from paper_1712_05834_gb300 import pipeline


class Cat:
    def __init__(self, k):
        self.k = k


class FakeStream:
    def __init__(self, lib, i):
        self.lib, self.i = lib, i

    def synchronize(self):
        self.lib.log.append(("sync", "P%d" % self.i))


class FakeLib:
    def __init__(self):
        self.log, self.plans, self.destroyed, self.painted, self.nstreams = [], 0, [], {}, 0

    def new_stream(self):
        self.nstreams += 1
        return FakeStream(self, self.nstreams - 1)

    def install(self, monkeypatch):
        monkeypatch.setattr(pipeline, "_new_stream", self.new_stream)
        for name in ("pk_plan", "pk_paint", "pk_compute", "pk_result", "pk_destroy", "pk_use_own_fft"):
            monkeypatch.setattr(pk, name, getattr(self, name))

    def pk_plan(self, cfg, stream):
        self.plans += 1
        return "P%d" % (self.plans - 1)

    def pk_use_own_fft(self, plan, on):
        self.log.append(("own", plan, on))

    def pk_paint(self, plan, pos, w=None):
        self.log.append(("paint", plan, pos.k))
        self.painted[plan] = weakref.ref(pos)

    def pk_compute(self, plan):
        self.log.append(("compute", plan))

    def pk_result(self, plan, item):
        assert item == 0
        ref = self.painted[plan]
        assert ref() is not None, "a catalog was released before its result was read"
        self.log.append(("result", plan, ref().k))
        return ref().k

    def pk_destroy(self, plan):
        self.destroyed.append(plan)


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_round_robin_and_order(monkeypatch, depth):
    f = FakeLib()
    f.install(monkeypatch)
    n = 7
    out = list(pipeline.power_stream(None, (Cat(k) for k in range(n)), depth=depth))
    assert out == list(range(n))
    assert f.plans == depth and sorted(f.destroyed) == sorted("P%d" % i for i in range(depth))
    paints = [e for e in f.log if e[0] == "paint"]
    assert [e[1] for e in paints] == ["P%d" % (k % depth) for k in range(n)]
    # catalog k's result is read just before catalog k + depth is painted
    for k in range(n - depth):
        i_res = f.log.index(("result", "P%d" % (k % depth), k))
        i_next = f.log.index(("paint", "P%d" % (k % depth), k + depth))
        assert i_res == i_next - 1
    # and at most `depth` catalogs are in flight at any time
    inflight = 0
    for e in f.log:
        inflight += e[0] == "paint"
        inflight -= e[0] == "result"
        assert 0 <= inflight <= depth


def test_own_fft_switch_and_weights(monkeypatch):
    f = FakeLib()
    f.install(monkeypatch)
    seen = []
    monkeypatch.setattr(pk, "pk_paint", lambda plan, pos, w=None: (seen.append(w), f.pk_paint(plan, pos)))
    out = list(pipeline.power_stream(None, [Cat(0), Cat(1)], depth=2, own_fft=True, weights=["w0", None]))
    assert out == [0, 1] and seen == ["w0", None]
    assert [e for e in f.log if e[0] == "own"] == [("own", "P0", True), ("own", "P1", True)]


def test_plans_destroyed_when_abandoned(monkeypatch):
    f = FakeLib()
    f.install(monkeypatch)
    g = pipeline.power_stream(None, (Cat(k) for k in range(10)), depth=2)
    assert next(g) == 0
    g.close()
    # catalog 1 was still in flight on P1 (catalog 2 not yet painted): its
    # stream drained first
    assert f.log[-2:] == [("result", "P0", 0), ("sync", "P1")]
    assert sorted(f.destroyed) == ["P0", "P1"]
    with pytest.raises(ValueError):
        pipeline.PowerStream(None, depth=0)


def test_plans_reused_across_maps(monkeypatch):
    f = FakeLib()
    f.install(monkeypatch)
    with pipeline.PowerStream(None, depth=2) as ps:
        assert list(ps.map([Cat(0), Cat(1), Cat(2)])) == [0, 1, 2]
        assert list(ps.map([Cat(3)])) == [3]
        assert f.plans == 2 and not f.destroyed
    assert sorted(f.destroyed) == ["P0", "P1"]
    with pytest.raises(ValueError):
        next(ps.map([Cat(4)]))
