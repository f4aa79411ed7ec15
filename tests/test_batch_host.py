"""Host logic of the batched path that needs no GPU: size classes, autotuner
candidates and cache, and the mock-set generator."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1712_05834_gb300 import batch   # noqa: E402
import synth   # noqa: E402


def _cat(n, nmesh, window, interlaced=False, dtype=torch.float32, weights=False):
    pos = torch.zeros((n, 3), dtype=dtype)
    return batch.Catalog(pos, nmesh, window, interlaced, torch.ones(n) if weights else None)


def test_classes_keep_input_order_and_split_every_option():
    cats = [_cat(5, 128, "cic"), _cat(7, 256, "tsc"), _cat(3, 128, "cic"), _cat(2, 128, "cic", True),
            _cat(4, 128, "cic", dtype=torch.float64), _cat(9, 128, "cic", weights=True), _cat(1, 256, "tsc")]
    g = batch.group_classes(cats)
    assert list(g.values()) == [[0, 2], [1, 6], [3], [4], [5]]
    assert sorted(i for v in g.values() for i in v) == list(range(len(cats)))
    assert batch.class_key(cats[0]) != batch.class_key(cats[0], "f64")


@pytest.mark.parametrize("nmesh,window,il,expect", [
    (128, "cic", False, [8, 16]), (192, "cic", False, [8, 12, 16, 24]), (256, "tsc", False, [8, 16]),
    (192, "pcs", True, [8, 12, 16, 24]), (36, "tsc", False, [12]), (10, "cic", False, []),
])
def test_tile_candidates_divide_the_mesh_and_cover_the_window(nmesh, window, il, expect):
    assert batch.tile_candidates(nmesh, window, il) == expect
    cands = batch.paint_candidates(nmesh, window, il)
    assert cands[-1] == ("atomic", 0)
    assert cands[:-1] == ([("sort", t) for t in expect] or [("sort", 0)])


def test_tune_key_bins_by_log2_of_the_mean_size():
    key = batch.class_key(_cat(1, 192, "tsc"))
    assert batch.tune_key(key, 1.0e6) == batch.tune_key(key, 1.1e6)
    assert batch.tune_key(key, 1.0e6) != batch.tune_key(key, 3.0e6)
    assert batch.tune_key(key, 1.0e6).startswith("N192-tsc-noil-f32-float323-unit-n2^20")


def test_autotuner_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    t = batch.Autotuner(path)
    t.cache["N128-cic"] = ("atomic", 0)
    t.cache["N256-tsc"] = ("sort", 16)
    t.save()
    u = batch.Autotuner(path)
    assert u.cache == {"N128-cic": ("atomic", 0), "N256-tsc": ("sort", 16)}


def test_mock_set_specs_are_seeded_and_follow_their_distributions():
    a = synth.mock_set_specs(256, synth.seed_for(4))
    b = synth.mock_set_specs(256, synth.seed_for(4))
    assert a == b and len(a) == 256
    n = np.array([s["n"] for s in a])
    assert n.min() >= 2e5 and n.max() <= 4e6
    # log-uniform: the mean of log n is the midpoint of the log range (5 sigma)
    mid = 0.5 * (math.log(2e5) + math.log(4e6))
    sd = (math.log(4e6) - math.log(2e5)) / math.sqrt(12 * 256)
    assert abs(np.log(n).mean() - mid) < 5 * sd
    assert {s["nmesh"] for s in a} == {128, 192, 256}
    assert {s["window"] for s in a} == {"cic", "tsc"}
    assert len({s["seed"] for s in a}) == 256


def test_assign_streams_balances_largest_first():
    from paper_1712_05834_gb300.batch import assign_streams
    assert assign_streams([5, 1, 9, 3], 1) == [0, 0, 0, 0]
    # 9 -> s0, 5 -> s1, 3 -> s1 (5 < 9), 1 -> s1 (8 < 9)
    assert assign_streams([5, 1, 9, 3], 2) == [1, 1, 0, 1]
    assert assign_streams([4, 4, 4], 3) == [0, 1, 2]
    assert assign_streams([], 2) == []
    w = assign_streams([7, 7, 2, 2, 2, 2, 2], 2)
    loads = [sum(x for x, s in zip([7, 7, 2, 2, 2, 2, 2], w) if s == k) for k in range(2)]
    assert sorted(loads) == [11, 13]          # greedy, not optimal: 7, 2, 2, 2 / 7, 2, 2
