"""The multi-GPU path of the bench on CPU: two gloo ranks (replicas, no data
exchange) combine their timings the way `bench.py --gpus N` does under
torchrun -- the slowest rank's time, every rank's events -- and the whole-job
value counts every rank's pixel-frames."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = [12.5, 20.0][rank]
        ev = [1000, 2345][rank]
        dist.barrier()
        q.put((rank, bench.combine_ranks(dist, torch.device("cpu"), ms, ev), bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict()
    for _ in procs:
        rank, combined, env = q.get(timeout=120)
        got[rank] = (combined, env)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        (ms, ev), (ws, r, _) = got[rank]
        assert (ms, ev) == (20.0, 3345)           # slowest rank, all events
        assert (ws, r) == (2, rank)
    # 2 ranks x 1e9 pixel-frames in 20 ms
    assert bench.job_value(10 ** 9, 2, 20.0) == pytest.approx(1e5)


def test_single_process_passes_through():
    assert bench.combine_ranks(None, torch.device("cpu"), 7.0, 11) == (7.0, 11)
    assert bench.job_value(2 * 10 ** 6, 1, 2.0) == pytest.approx(1000.0)
