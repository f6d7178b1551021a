"""The multi-GPU path of bench.py on CPU: two gloo ranks each take their own
batch (no shared item) and agree on the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    geoms, runs = bench.rank_workload(rank, 64, 1 << 12)
    keys = sorted((g.C, g.b, g.ways, g.policy, g.seed, r.n_elems, r.stride, r.length)
                  for g, r in zip(geoms, runs))
    t = bench.max_over_ranks(10.0 + rank, world)
    out[rank] = (keys, t, sum(r.length for r in runs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_batches_and_max_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        (k0, t0, a0), (k1, t1, a1) = out[0], out[1]
    assert t0 == t1 == 11.0
    assert len(k0) == len(k1) == 64
    assert not set(k0) & set(k1)  # seeds differ: no item shared between ranks
    assert a0 > 0 and a1 > 0
