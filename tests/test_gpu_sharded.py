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
