"""GPU parity: pipelined map/reduce word count (mapper warps hand cache
misses to reducer warps through shared-memory rings, Sec. III-D).  Results
must equal the oracle and the direct path byte for byte."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nbytes,nwords", [(16 << 20, 50_000), (3 << 20, 500), (1 << 20, 200_000)])
def test_pipelined_matches_oracle_and_direct(mr, nbytes, nwords):
    import torch
    text, _, _ = synth.wc_text(nbytes, nwords=nwords, seed=nbytes + nwords)
    d = torch.from_numpy(text).cuda()
    got = mr.wordcount(d, pipelined=True)
    assert got == mr.wordcount(d)
    assert got == oracle.wordcount(text)


def test_pipelined_edges(mr):
    raws = [b"", b"a", b" \n ", b"x y x", b"hot " * 50000, b" ".join(b"%x" % i for i in range(300_000)),
            b"long_token_" * 3000 + b" z",
            b"prefix_shared_by_long_keys_aaaa prefix_shared_by_long_keys_aaab " * 1000]
    for r in raws:
        assert mr.wordcount(r, pipelined=True) == oracle.wordcount(r), r[:30]
