"""The multi-GPU form of the bench is replicas: every rank encodes and
decodes its own stripes, and the only cross-rank operations are a barrier and
the max-reduce of the timings. Checked here with two gloo ranks on the CPU:
disjoint stripe ranges that tile the single-process stream, and the max of
the ranks' times reaching every rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1504_07038_gb300 import inputs
    S, Q, P = 5, 4, 16
    img = inputs.stripes(S, Q, P, first=bench.replica_first_stripe(rank, S))
    t = bench.max_over_ranks(1.5 + rank, dist)
    dist.barrier()
    q.put((rank, img, t))
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    from paper_1504_07038_gb300 import inputs
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict((r, (img, t)) for r, img, t in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = inputs.stripes(10, 4, 16)
    assert np.array_equal(np.concatenate([got[0][0], got[1][0]]), whole)
    assert got[0][1] == got[1][1] == 2.5
