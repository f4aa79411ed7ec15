"""Host logic of the serving loop that needs no GPU: the slot footprint
estimate, Poisson arrivals and the latency summary."""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_1712_05834_gb300 import serve   # noqa: E402


def test_slot_bytes_counts_meshes_and_buffers():
    one = serve.slot_bytes(256, False, "f32", 1, 1_000_000)
    mesh = 256 * 256 * 2 * 129 * 4
    assert one >= 2 * mesh + 1_000_000 * 36
    assert serve.slot_bytes(256, True, "f32", 1, 1_000_000) > one + mesh
    assert serve.slot_bytes(256, False, "f64", 1, 1_000_000) > one + mesh
    assert serve.slot_bytes(256, False, "f32", 8, 1_000_000) > 8 * mesh
    assert serve.slot_bytes(128, False, "f32", 1, 10, variant="atomic") >= 128 ** 3 * 8


def test_poisson_arrivals_rate_and_order():
    t = serve.poisson_arrivals(20000, 200.0, 1)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 5 * (1 / 200.0) / np.sqrt(20000)
    assert np.array_equal(t, serve.poisson_arrivals(20000, 200.0, 1))


def test_latency_summary():
    reqs = []
    for i in range(100):
        r = serve.Request(i, None, arrival=0.01 * i)
        r.t_done = r.arrival + 0.001 * (i + 1)
        r.batch_size = 1 + i % 3
        reqs.append(r)
    s = serve.latency_summary(reqs)
    assert s["requests"] == 100
    assert s["p50_ms"] == pytest.approx(np.percentile(np.arange(1, 101), 50))
    assert s["p99_ms"] == pytest.approx(np.percentile(np.arange(1, 101), 99))
    assert s["max_ms"] == pytest.approx(100.0)
    assert s["pk_per_s"] == pytest.approx(100 / (0.99 + 0.1))
    assert s["mean_batch"] == pytest.approx(np.mean([1 + i % 3 for i in range(100)]))


def test_latency_summary_by_tag():
    reqs = []
    for i in range(40):
        r = serve.Request(i, None, arrival=0.0, tag="large" if i % 10 == 0 else "pool")
        r.t_done = 0.1 if r.tag == "large" else 0.001
        reqs.append(r)
    s = serve.latency_summary(reqs)
    assert s["by_tag"]["large"]["requests"] == 4 and s["by_tag"]["pool"]["requests"] == 36
    assert s["by_tag"]["large"]["p50_ms"] == pytest.approx(100.0)
    assert s["by_tag"]["pool"]["p99_ms"] == pytest.approx(1.0)
