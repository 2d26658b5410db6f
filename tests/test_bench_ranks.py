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


def _shard_rank(rank, ws, port, out):
    """One rank of the k-sharded build: the oracle's chi0 over this rank's k range (the same sum
    the GPU's rp_build_chi0_kset forms), then the all-reduce of the sharded path."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    from oracle import chi0 as OC, lattice as OL, pair_density as OP
    from synth import make_workload
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        wl = make_workload("micro")
        q = wl.q[0]
        nk = wl.bands.kfrac.shape[0]
        k0, k1 = bench.k_shards(nk, ws)[rank]
        G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
        ks = list(range(k0, k1))
        M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft, k_list=ks)
        part = OC.chi0(M, OC.pair_weights(wl, q, k_list=ks))
        t = torch.from_numpy(part)
        dist.all_reduce(torch.view_as_real(t))
        out[rank] = t.numpy()
    finally:
        dist.destroy_process_group()


def test_k_sharded_sum_equals_unsharded_build():
    """The `--shard k` path of bench.py on two gloo ranks: each rank sums chi0 over its k range and
    one all-reduce forms the whole; the result equals the unsharded sum over the mesh, on both
    ranks.  The shard helpers cover every k point and frequency exactly once."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from oracle import chi0 as OC, lattice as OL, pair_density as OP
    from synth import make_workload
    for n, w in ((8, 2), (1000, 3), (7, 4), (30, 8)):
        cover = np.concatenate([np.arange(a, b) for a, b in bench.k_shards(n, w)])
        assert np.array_equal(cover, np.arange(n))
        cover = np.concatenate([np.arange(a, b) for a, b in bench.f_shards(n, w)])
        assert np.array_equal(cover, np.arange(n))
    wl = make_workload("micro")                  # generated (and cached) before the ranks start
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    q = wl.q[0]
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    full = OC.chi0(M, OC.pair_weights(wl, q))
    for r in range(ws):
        assert np.abs(res[r] - full).max() <= 1e-13 * np.abs(full).max()
