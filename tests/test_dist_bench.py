"""Host-side logic of the multi-GPU benchmark (independent replicas, one per
rank; the job's time is the slowest rank's), run as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, lr = bench.dist_setup()
    slowest = bench.reduce_max(10.0 * (rank + 1), w)
    q.put((r, w, slowest, bench.rank_seed(1, r)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_max_and_distinct_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 20.0 for r in res)          # every rank sees the slowest rank's time
    assert res[0][3] != res[1][3]                  # independent chains
    assert res[0][3] == 1                          # rank 0 keeps the base seed
