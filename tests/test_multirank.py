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


# ------------------------------------------------------------------ sharding
# The multi-GPU path (one slice of the input per rank, then a merge): the
# slices' results come from the oracle here (CPU ranks have no GPU), and the
# merged result must equal the oracle's result for the whole input.

def _merge_rank(rank, ws, port, q, text, px, xy):
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1309_0215_gb300 import multi, WORDCOUNT, HIST_RGB8, LINREG_I8
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    lo, hi = multi.shard_bounds(WORDCOUNT, len(text), ws, rank, multi.reader(text))
    merged = multi.merge_wordcount(oracle.wordcount(text[lo:hi]))
    lo, hi = multi.shard_bounds(HIST_RGB8, len(px), ws, rank)
    h = torch.from_numpy(oracle.hist_rgb8(np.frombuffer(px[lo:hi], dtype=np.uint8)).astype(np.int64))
    multi.allreduce_sum(h)
    lo, hi = multi.shard_bounds(LINREG_I8, len(xy), ws, rank)
    r = torch.from_numpy(oracle.linreg_i8(np.frombuffer(xy[lo:hi], dtype=np.int8)).astype(np.int64))
    multi.allreduce_sum(r)
    q.put((rank, merged, h.numpy().tobytes(), r.numpy().tobytes()))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_jobs_merge_to_the_whole_input_result(ws):
    import numpy as np
    import oracle
    import synth
    text, _, _ = synth.wc_text(1 << 20, nwords=4000, seed=synth.SEED_BASE + 31)
    text = text.tobytes()
    px = synth.hist_rgb8(100_001, seed=synth.SEED_BASE + 32).tobytes()
    xy = synth.linreg_i8(50_001, seed=synth.SEED_BASE + 33).tobytes()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_merge_rank, args=(r, ws, port, q, text, px, xy)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert res[0][1] == oracle.wordcount(text)
    assert all(r[1] is None for r in res[1:])
    h_ref = oracle.hist_rgb8(np.frombuffer(px, dtype=np.uint8)).astype(np.int64).tobytes()
    r_ref = oracle.linreg_i8(np.frombuffer(xy, dtype=np.int8)).astype(np.int64).tobytes()
    for r in res:
        assert r[2] == h_ref and r[3] == r_ref


def _merge_keys_rank(rank, ws, port, q, keys, seq):
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1309_0215_gb300 import multi, HIST_U32, BLOOM_DNA
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    lo, hi = multi.shard_bounds(HIST_U32, len(keys), ws, rank)
    h = oracle.hist_u32(np.frombuffer(keys[lo:hi], dtype=np.uint32), 5000)
    ht = torch.from_numpy(h.view(np.int64).copy())
    multi.allreduce_sum(ht)
    lo, hi = multi.shard_bounds(BLOOM_DNA, len(seq), ws, rank, kmer=32)
    bt = torch.from_numpy(oracle.bloom_dna(seq[lo:hi], 32, 100_003, 7))
    multi.allreduce_or(bt)
    q.put((rank, ht.numpy().tobytes(), bt.numpy().tobytes()))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_keys_and_bloom_merge_to_the_whole_input_result(ws):
    """Large-key histogram slices summed with one all-reduce, Bloom-filter
    slices (each owning the windows that start in it) ORed, against the
    oracle on the whole input."""
    import numpy as np
    import oracle
    import synth
    keys = synth.keys_u32(40_001, 6000, seed=synth.SEED_BASE + 34).tobytes()
    seq = synth.dna(30_011, seed=synth.SEED_BASE + 35, n_runs=20, max_run=40).tobytes()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_merge_keys_rank, args=(r, ws, port, q, keys, seq)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    h_ref = oracle.hist_u32(np.frombuffer(keys, dtype=np.uint32), 5000).tobytes()
    b_ref = oracle.bloom_dna(seq, 32, 100_003, 7).tobytes()
    for r in res:
        assert r[1] == h_ref and r[2] == b_ref


def test_bloom_shards_hold_every_window_once():
    """Each window start belongs to exactly one slice, and that slice holds
    the whole window (brute force over small inputs and world sizes)."""
    from paper_1309_0215_gb300 import multi, BLOOM_DNA
    for n, L in ((1000, 32), (97, 5), (10, 16), (64, 1)):
        for ws in (1, 2, 3, 7):
            b = [multi.shard_bounds(BLOOM_DNA, n, ws, r, kmer=L) for r in range(ws)]
            for p in range(0, n - L + 1):
                inside = [r for r, (lo, hi) in enumerate(b) if lo <= p and p + L <= hi]
                assert len(inside) == 1, (n, L, ws, p, inside)


def test_shard_bounds_never_cut_a_token():
    import oracle
    from paper_1309_0215_gb300 import multi, WORDCOUNT
    text = b"ab cd  efg h" + b"x" * 5000 + b" tail\n"
    for ws in (1, 2, 3, 5, 8):
        b = [multi.shard_bounds(WORDCOUNT, len(text), ws, r, multi.reader(text)) for r in range(ws)]
        assert b[0][0] == 0 and b[-1][1] == len(text)
        assert all(b[i][1] == b[i + 1][0] for i in range(ws - 1))
        # every slice after the first starts with whitespace (or is empty / at the end)
        assert all(lo == hi or text[lo:lo + 1] in (b" ", b"\n") for lo, hi in b[1:])
        assert multi.merge_wordcount_local([oracle.wordcount(text[lo:hi]) for lo, hi in b]) == oracle.wordcount(text)
