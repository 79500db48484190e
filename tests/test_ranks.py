"""The benchmark's N > 1 path on CPU: two gloo ranks exercise the barrier,
the max and sum over ranks, and the whole-job (weak scaling) throughput that
`bench.py` reports (all ranks' units over the slowest rank's time)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    assert bench.dist_env() == (ws, rank, rank)
    r = bench.Ranks(ws, backend="gloo", device="cpu")
    r.barrier()
    assert r.max(rank) == ws - 1
    assert r.sum(rank + 1) == ws * (ws + 1) / 2
    # rank i processed 10 units in 0.1 (i + 1) s: the job took 0.1 ws s for 10 ws units
    t, v = r.weak_throughput(10, 0.1 * (rank + 1))
    assert abs(t - 0.1 * ws) < 1e-12 and abs(v - 10 * ws / (0.1 * ws)) < 1e-9
    r.close()


@pytest.mark.parametrize("ws", [2])
def test_ranks_over_gloo(ws):
    mp.spawn(_rank_main, args=(ws, _free_port()), nprocs=ws, join=True)


def test_single_rank_world_needs_no_process_group():
    r = bench.Ranks(1, backend="gloo", device="cpu")
    assert r.dist is None and r.max(3.5) == 3.5 and r.sum(2) == 2.0
    assert r.weak_throughput(20, 0.5) == (0.5, 40.0)
    r.close()
