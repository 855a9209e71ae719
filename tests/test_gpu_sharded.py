"""The multi-GPU path on one GPU: the input cut into slices as ranks would
take it, each slice run by the CUDA library, the results merged with the
host-side partition / reduce / k-way merge (the same steps as the
all-to-all merge across ranks), compared with the oracle on the whole input."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 5])
def test_sharded_wordcount_equals_whole_input(mr, world):
    import torch
    from paper_1309_0215_gb300 import multi
    text, _, _ = synth.wc_text(8 << 20, seed=synth.SEED_BASE + 41)
    d = torch.from_numpy(text).cuda()
    read = multi.reader(d)
    blobs = []
    for r in range(world):
        lo, hi = multi.shard_bounds(mr.WORDCOUNT, d.numel(), world, r, read)
        blobs.append(mr.wordcount(d[lo:hi].clone()))
    assert multi.merge_wordcount_local(blobs) == oracle.wordcount(text)


def test_sharded_arrays_equal_whole_input(mr):
    import torch
    from paper_1309_0215_gb300 import multi
    px = synth.hist_rgb8(3_000_001, seed=synth.SEED_BASE + 42)
    xy = synth.linreg_i8(2_000_001, seed=synth.SEED_BASE + 43)
    dp, dx = torch.from_numpy(px).cuda(), torch.from_numpy(xy).cuda()
    h = np.zeros(768, dtype=np.uint64)
    s = np.zeros(5, dtype=np.int64)
    for r in range(3):
        lo, hi = multi.shard_bounds(mr.HIST_RGB8, dp.numel(), 3, r)
        h += np.asarray(mr.hist_rgb8(dp[lo:hi]), dtype=np.uint64)
        lo, hi = multi.shard_bounds(mr.LINREG_I8, dx.numel(), 3, r)
        s += np.asarray(mr.linreg_i8(dx[lo:hi]), dtype=np.int64)
    assert np.array_equal(h, oracle.hist_rgb8(px).astype(np.uint64))
    assert s.tolist() == oracle.linreg_i8(xy).tolist()


def test_sharded_keys_and_bloom_equal_whole_input(mr):
    """Large-key histogram and Bloom filter over three slices each (the Bloom
    slices overlapping by a window less a base), merged by sum and OR."""
    import torch
    from paper_1309_0215_gb300 import multi
    keys = synth.keys_u32(3_000_001, 1 << 20, seed=synth.SEED_BASE + 44)
    seq = synth.dna(2_000_003, seed=synth.SEED_BASE + 45, n_runs=200, max_run=100)
    dk, ds = torch.from_numpy(keys).cuda(), torch.from_numpy(seq).cuda()
    h = np.zeros((1 << 20) + 1, dtype=np.uint64)
    blooms = []
    for r in range(3):
        lo, hi = multi.shard_bounds(mr.HIST_U32, dk.numel() * 4, 3, r)
        h += mr.hist_u32(dk[lo // 4:hi // 4], 1 << 20)
        lo, hi = multi.shard_bounds(mr.BLOOM_DNA, ds.numel(), 3, r, kmer=32)
        blooms.append(mr.bloom_dna(ds[lo:hi], 32, 20_000_003, 7))
    assert np.array_equal(h, oracle.hist_u32(keys, 1 << 20))
    assert np.array_equal(multi.merge_bloom_local(blooms), oracle.bloom_dna(seq, 32, 20_000_003, 7))
