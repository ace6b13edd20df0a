"""The only multi-rank exchange (final best-state merge), on CPU ranks over gloo."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2211_03193_gb300.dist import merge_best
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(100 + rank)
    E = rng.normal(50.0, 5.0, size=7)
    if rank == 1:
        E[3] = -1.0  # the global best lives on rank 1, chain 3
    th = rng.uniform(-np.pi, np.pi, size=(7, 10)).astype(np.float32)
    e, t, r = merge_best(E, th)
    q.put((rank, e, t, r, th[3] if rank == 1 else None))
    dist.barrier()
    dist.destroy_process_group()


def test_merge_best_world_size_two_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    want_theta = out[1][4]
    for rank, e, t, r, _ in out:
        assert e == -1.0 and r == 1
        assert np.array_equal(t, want_theta)


def test_local_best_picks_lowest_chain():
    from paper_2211_03193_gb300.dist import local_best
    E = np.array([3.0, -2.0, 5.0])
    th = np.arange(12, dtype=np.float32).reshape(3, 4)
    e, t = local_best(E, th)
    assert e == -2.0 and np.array_equal(t, th[1])
