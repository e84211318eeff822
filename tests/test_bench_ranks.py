"""The multi-rank timing of bench.py on CPU (gloo, world size 2).

Every rank counts its own hypergraph; the job's time is the slowest rank's
and its work the sum over ranks, so value = total work / max time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    ms = [120.0, 80.0][rank]           # rank 0 is the slower one
    units = [1.0e12, 3.0e12][rank]
    t, u = bench.reduce_over_ranks(ms, units, 2, "cpu")
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_max_time_and_summed_work_over_two_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (120.0, 4.0e12)
    t, u = res[0]
    assert u / (t / 1000.0) == pytest.approx(4.0e12 / 0.12)


def test_single_rank_is_unchanged():
    import bench
    assert bench.reduce_over_ranks(5.0, 7.0, 1, "cpu") == (5.0, 7.0)


def test_row_partition_covers_every_row_once_and_balances_work():
    import numpy as np
    import bench
    deg = np.random.default_rng(3).zipf(1.6, size=5000).clip(0, 50_000)
    for ws in (1, 2, 3, 8):
        parts = bench.partition_rows(deg, ws)
        allr = np.concatenate(parts)
        assert np.array_equal(np.sort(allr), np.arange(deg.size))
        work = [float((deg[p].astype(float) ** 2).sum()) for p in parts]
        assert max(work) <= 1.25 * (sum(work) / ws) + float(deg.max()) ** 2


def _share_main(rank, port, out):
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    # two ranks' shares of one count, with negative entries as the split
    # decomposition gives them
    share = [np.array([5, -3, 2**40, 0], np.int64), np.array([1, 4, 7, -2], np.int64)][rank]
    out[rank] = bench.reduce_counts(share, 2, "cpu").tolist()
    dist.barrier()
    dist.destroy_process_group()


def test_row_shares_sum_over_two_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_share_main, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == [6, 1, 2**40 + 7, -2]
