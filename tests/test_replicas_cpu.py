"""The multi-GPU bookkeeping of bench.py (replicas, max over ranks, whole-job
throughput), exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_1707_04346_gb300 import replicas

    r, w, local = replicas.setup()
    assert (r, w, local) == (rank, world, rank)
    replicas.barrier(w)
    # rank r took (r + 1) seconds for 100 units: the job is as slow as rank 1
    t = replicas.max_over_ranks(float(r + 1), w)
    out[rank] = (t, replicas.job_throughput(100.0, t, w))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.0, 100.0)


def test_single_rank_is_identity():
    from paper_1707_04346_gb300 import replicas

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert replicas.setup() == (0, 1, 0)
    assert replicas.max_over_ranks(3.5, 1) == 3.5
    assert replicas.job_throughput(10.0, 2.0, 1) == 5.0
