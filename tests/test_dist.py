"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): ranks run
independent replicas (own seeds, no data-path collective); the job time is
the slowest rank's, and the value counts the walker-steps of every rank."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    t = bench.max_over_ranks(100.0 + 50.0 * rank)
    out.put((r, ws, t, bench.replica_seed(3, r)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_seeds():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[2] == 150.0 for x in res)  # the slowest rank's time on both
    assert res[0][3] != res[1][3]  # independent replicas


def test_job_throughput_counts_all_ranks():
    import bench

    assert bench.job_throughput(512, 10, 1000.0, 1) == 5120.0
    assert bench.job_throughput(512, 10, 1000.0, 4) == 4 * 5120.0
    assert bench.max_over_ranks(7.5) == 7.5  # no process group: local value
