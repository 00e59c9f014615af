"""The N > 1 host path of bench.py on CPU: world_size-2 gloo ranks, each an
independent replica; the job time is the max over ranks and the value counts
the steps of every rank."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    t = bench.job_time_ms(10.0 + 5.0 * rank, ws)   # rank 1 is the slow one
    out[rank] = (t, bench.job_value(t, ws, 4))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_value():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(ws, port, out), nprocs=ws, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == pytest.approx(15.0 / (2 * 4))


def test_single_rank_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(7.5, 1) == 7.5
    assert bench.job_value(8.0, 1, 4) == 2.0
