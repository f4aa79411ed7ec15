"""The multi-process (N > 1) host logic of bench.py on CPU with the gloo
backend, world size 2: the max-over-ranks timing, the barrier, the
whole-job rate of a weak-scaling run, and the reference arm's rule that only
rank 0 runs the oracle."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        bench.barrier(world)
        t = bench.max_over_ranks(1.5 + rank, world)          # rank 1 is the slow one
        out[rank] = (t, bench.job_rate(world, 100, t))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.5, 2 * 100 / 2.5)


def test_job_rate_and_single_rank_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_rate(1, 200, 0.5) == 400.0
    assert bench.job_rate(4, 200, 0.5) == 1600.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_binned_stored_modes_counts_the_modes_in_k_bins():
    """The bench's algorithmic-bytes helper counts stored half-grid modes with
    0 < |k| and a k bin in [0, nk): checked by direct enumeration."""
    import math
    import numpy as np
    import bench
    N, L, dk = 48, 300.0, 0.03
    kF = 2 * math.pi / L
    nk = int(math.floor((math.pi * N / L) / dk))
    f = np.fft.fftfreq(N, 1.0 / N)
    I, J, K = np.meshgrid(f, f, np.arange(N // 2 + 1), indexing="ij")
    m = I * I + J * J + K * K
    b = np.floor(kF * np.sqrt(m) / dk)
    want = int(np.count_nonzero((m > 0) & (b >= 0) & (b < nk)))
    assert bench.binned_stored_modes(N, L, dk) == want
