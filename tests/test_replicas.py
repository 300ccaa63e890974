"""The multi-process path of bench.py (one replica per rank, no data-path
collective) on CPU: two gloo ranks on 127.0.0.1 reduce their step times to
the slowest one and report the whole job's time per mesh."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        step, per_mesh = bench.job_ms(10.0 + 5.0 * rank, ws, dist, "cpu")
        out[rank] = (env, step, per_mesh)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        env, step, per_mesh = res[rank]
        assert env == (ws, rank, rank)
        assert step == 15.0 and per_mesh == 7.5


def test_single_process_needs_no_collective():
    import bench
    assert bench.job_ms(12.5, 1) == (12.5, 12.5)
