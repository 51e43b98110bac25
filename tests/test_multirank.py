"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): ranks map independent string
networks (weak scaling), the job's time is the slowest rank's, and the value counts every
rank's pairs.  No data-path collective exists: the map shards by network (or pixel range)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth

    w = synth.config(1, seed=1 + rank)                     # the network each rank maps
    ms = 100.0 + 50.0 * rank                               # pretend rank 1 is slower
    mx = bench.max_over_ranks(ms, dist)
    val = bench.weak_scaling_value(w.npix * w.n, 4, world, mx)
    out[rank] = (mx, val, float(w.loop_params[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    pairs = 12 * 512 * 512 * 200000
    assert res[0][1] == pytest.approx(world * pairs * 4 / 0.150)
    assert res[0][2] != res[1][2]                           # independent networks per rank


def test_single_rank_identity():
    import bench

    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.weak_scaling_value(10, 2, 1, 1000.0) == 20.0
