"""The multi-GPU bench path is independent replicas: each rank builds its own
copy of the workload, and rank 0 reports the summed work over the slowest
rank's time.  This checks that aggregation over world_size 2 with the gloo
backend on CPU (no GPU and no data-path collective involved)."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    d = bench.init_dist(w)
    bench.barrier(d)
    t_max = bench.max_over_ranks(d, 1.0 + r)          # rank r "took" 1 + r seconds
    work = bench.sum_over_ranks(d, 1000.0 * (r + 1))  # and built 1000 (r + 1) elements
    q.put((r, w, local, t_max, work))
    d.destroy_process_group()


def test_replica_aggregation_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, world, local, t_max, work) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert t_max == 2.0 and work == 3000.0
