"""Host logic of multi-process runs, with two gloo ranks on the CPU (no GPU)."""
import os
import socket

import pytest

from paper_1402_6019_gb300 import replicas


def test_from_env_and_seeds():
    r = replicas.from_env({"RANK": "1", "WORLD_SIZE": "4", "LOCAL_RANK": "1"})
    assert (r.rank, r.world, r.local, r.is_root) == (1, 4, 1, False)
    assert replicas.from_env({}).world == 1
    assert replicas.replica_seed(1402, r) == 1403
    with pytest.raises(ValueError):
        replicas.from_env({"RANK": "4", "WORLD_SIZE": "4"})


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "ran" 100 * (r + 1) sites in 0.5 * (r + 1) seconds
        t, n = replicas.aggregate(0.5 * (rank + 1), 100 * (rank + 1), dist=dist)
        q.put((rank, t, n))
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    # every rank sees the slowest rank's time and the total work
    assert res == [(0, 1.0, 300), (1, 1.0, 300)]
