"""The multi-rank host logic of the benchmark on CPU (gloo, two ranks)."""

import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1712_09624_gb300 import dist as D
    from paper_1712_09624_gb300 import workload as W
    r, w, lr = D.rank_info()
    secs = 0.5 + rank  # rank 1 is the slowest
    slowest = D.max_over_ranks(secs)
    seed = D.rank_seed(7, r)
    keys = W.make_keys(seed, W.STREAM_INSERT_KEYS, 4)
    out[rank] = (r, w, lr, slowest, D.job_throughput(1000, 10, slowest, w), keys.tobytes())
    torch.distributed.destroy_process_group()


def test_two_ranks_reduce_time_and_draw_disjoint_workloads():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:3] == (0, 2, 0) and res[1][:3] == (1, 2, 1)
    assert res[0][3] == res[1][3] == pytest.approx(1.5)
    assert res[0][4] == pytest.approx(2 * 1000 * 10 / 1.5)
    assert res[0][5] != res[1][5]


def test_single_process_passthrough():
    from paper_1712_09624_gb300 import dist as D
    assert D.max_over_ranks(0.25) == 0.25
    assert D.rank_seed(3, 0) == 3
