"""The benchmark's several-rank host logic on CPU (gloo, world size 2): each
rank analyses its own seeded batch, and the reported throughput takes the
slowest rank's time over the units all ranks processed."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out_dir: str):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist

    import bench
    import paam_gen

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sy = paam_gen.generate(bench.WORKLOAD, n_sys=200, seed=bench.rank_seed(rank))
    t, chains, systems = bench.reduce_over_ranks(10.0 + rank, sy.n_chain, sy.n_sys, dist, "cpu")
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([t, chains, systems, sy.n_chain, int(sy.T.sum() % (1 << 31))], np.float64))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_shard_and_reduce(tmp_path):
    import numpy as np

    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    # both ranks report the slowest rank's time and the same totals
    assert r0[0] == r1[0] == 11.0
    assert r0[1] == r1[1] == r0[3] + r1[3]
    assert r0[2] == r1[2] == 400
    # the two ranks analysed different systems of the same shape
    assert r0[4] != r1[4]


def test_single_rank_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(3.5, 120, 10, None, "cpu") == (3.5, 120, 10)
    assert bench.rank_seed(0) != bench.rank_seed(1)
