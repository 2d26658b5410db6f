"""The N > 1 host path of bench.py (replicas): max-over-ranks timing and the whole-job rate, with
two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        # rank r took (r + 1) * 10 ms per step: the job is timed by the slowest rank
        t = bench.max_over_ranks((rank + 1) * 10.0)
        out[rank] = (t, bench.job_rate(1e12, t * 1e-3, ws))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        t, rate = res[r]
        assert t == 20.0
        assert rate == pytest.approx(2 * 1e12 / 0.020 / 1e12)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(2e12, 0.5, 1) == pytest.approx(4.0)
