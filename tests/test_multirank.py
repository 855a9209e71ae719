"""The multi-process timing path of bench.py (one replica per rank, max over
ranks) on CPU ranks with the gloo backend, world size 2."""
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


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = [120.0, 150.0][rank]          # rank 1 is the slow one
    ms_max, value = bench.combine_ranks(ms, nbytes=3_000_000_000, steps=10, ws=ws)
    bench._barrier(ws)
    q.put((rank, ms_max, value))
    dist.destroy_process_group()


def test_weak_scaling_value_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, ms_max, value in res:
        assert ms_max == 150.0
        assert value == pytest.approx(3e9 * 2 * 10 / 0.150 / 1e9)
