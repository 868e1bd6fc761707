"""The bench's multi-process path (one replica of the workload per rank, no collective on the
data path) on CPU ranks with the gloo backend: the max-over-ranks timing reduction and the
whole-job throughput it feeds.  World size 2, rendezvous on 127.0.0.1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # each rank "timed" its own replica; the job time is the slowest rank's
    t = bench.max_over_ranks(dist, 1.0 + rank, "cpu")
    bench.barrier(dist)
    K, steps = 50, 5
    value = world * K * steps / t
    out[rank] = (t, value)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.0, 2 * 50 * 5 / 2.0)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    bench.barrier(None)
