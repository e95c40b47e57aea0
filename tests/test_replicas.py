"""Replica path of bench.py (one independent problem per GPU, no data-path
collective): the max-over-ranks timing and the whole-job rate, run as two
gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        assert bench._dist() == (ws, rank, rank)
        bench._barrier(ws)
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slower replica
        ms_max = bench._max_over_ranks(ws, ms)
        out[rank] = (ms_max, bench.aggregate_rate(1000, ws, ms_max, 4))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_max_time_and_aggregate():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_max, rate = res[0]
    assert ms_max == 15.0
    # 2 replicas x 1000 units x 4 steps in 15 ms
    assert rate == pytest.approx(2 * 1000 * 4 / 15e-3)
