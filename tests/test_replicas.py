"""The multi-GPU form of the bench is query replicas: each rank runs its own
slice of the sources on its own copy of the graph, with no collective on the
data path; the whole-job number is total edges over the slowest rank's time.
These tests run that host logic as two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import graphgen as gg
        g = gg.rmat(10, 8, seed=1)
        srcs = bench.rank_sources(g, 4, rank, world)
        everyone = [None] * world
        dist.all_gather_object(everyone, [int(x) for x in srcs])
        t, e, v = bench.combine_ranks(10.0 + rank, 1000.0 * (rank + 1), world, "cpu")
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([t, e, v] + [x for part in everyone for x in part], dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_split_sources_and_combine(tmp_path):
    import torch.multiprocessing as mp
    import graphgen as gg
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    # every rank sees the same whole-job numbers: max time, summed edges
    for r in (r0, r1):
        assert r[0] == 11.0 and r[1] == 3000.0
        assert r[2] == pytest.approx(3000.0 / 0.011 / 1e9)
    # the ranks' sources are disjoint slices of one seeded draw
    got = r0[3:].astype(np.int64)
    assert np.array_equal(got, r1[3:].astype(np.int64))
    g = gg.rmat(10, 8, seed=1)
    want = gg.pick_sources(g, 8, seed=1)
    assert np.array_equal(got, want)
    assert len(set(got[:4]) & set(got[4:])) == 0


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(5.0, 2000.0, 1, "cpu") == (5.0, 2000.0, 2000.0 / 0.005 / 1e9)
