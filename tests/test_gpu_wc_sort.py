"""GPU parity: the word-count output sort when keys tie on the radix sort's
words (job/count and the first 8 key bytes).

Distinct words that share their first 8 bytes and their count form one tie
run after the key sort.  Runs of up to 32 are ordered by one thread, runs of
up to 2048 by one CTA's bitonic sort, and longer runs by one CTA's merge sort
each; every path must give the oracle's bytes, also with long keys (> 15
bytes) whose first 16 bytes agree, with several long runs in one job, and
inside a batch.
Record capacities up to 2^17 (automatic tables, slots=0) take the sample
sort of compact keys, up to 2^20 the block sort + merge passes (slots=2^18),
from 2^20 on the radix sort (slots=2^20).  A batch whose tables each hold at
most 2^17 slots, and more than 2^17 together, is sorted job by job (the
segmented sample sort: one sample, splitter set and bucket range per job)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _text(nwords: int, prefix: bytes, reps: int, seed: int) -> bytes:
    rng = np.random.default_rng(seed)
    words = [prefix + b"%05d" % i for i in range(nwords)]
    toks = [w for w in words for _ in range(reps)]
    rng.shuffle(toks)
    return b" ".join(toks) + b"\n"


@pytest.mark.parametrize("slots", [0, 1 << 18, 1 << 20])
@pytest.mark.parametrize("nwords", [2, 5, 32, 33, 700, 2048, 2049, 5000])
def test_tie_runs_short_prefix(mr, nwords, slots):
    raw = _text(nwords, b"abcdefgh", 3, nwords) + b" zz yy zz"
    assert mr.wordcount(raw, wc_slots=slots) == oracle.wordcount(raw)


@pytest.mark.parametrize("slots", [0, 1 << 18, 1 << 20])
@pytest.mark.parametrize("nwords", [7, 300, 3000])
def test_tie_runs_long_keys(mr, nwords, slots):
    raw = _text(nwords, b"prefix_shared_by_long_keys_", 2, nwords)
    assert mr.wordcount(raw, wc_slots=slots) == oracle.wordcount(raw)


@pytest.mark.parametrize("slots", [0, 1 << 18, 1 << 20])
def test_several_huge_tie_runs(mr, slots):
    """Runs of 2049..20000 records (one to four merge passes), three of them
    in one job (counts 1, 2 and 3 keep them apart), plus short runs."""
    rng = np.random.default_rng(5)
    toks = []
    for reps, n, pre in ((1, 20000, b"hugehuge"), (2, 4097, b"bigbigbi"), (3, 2049, b"midmidmi")):
        toks += [pre + b"%06d" % i for i in range(n) for _ in range(reps)]
    toks += [b"x", b"y", b"x"]
    rng.shuffle(toks)
    raw = b" ".join(toks) + b"\n"
    assert mr.wordcount(raw, wc_slots=slots) == oracle.wordcount(raw)


def test_radix_path_on_wordcount_text(mr):
    import synth
    text, _, _ = synth.wc_text(4 << 20, nwords=30000, seed=9)
    assert mr.wordcount(text, wc_slots=1 << 20) == oracle.wordcount(text)


@pytest.mark.parametrize("slots", [0, 1 << 16, 1 << 18])
def test_tie_runs_in_a_batch(mr, slots):
    import torch
    raws = [_text(40, b"qqqqqqqq", 2, 1), _text(2500, b"rrrrrrrr", 1, 2), b"a b a", _text(900, b"ssssssss_", 4, 3)]
    c = mr.Context()
    ids = [c.add_job(mr.WORDCOUNT, torch.frombuffer(bytearray(r), dtype=torch.uint8).cuda(), wc_slots=slots)
           for r in raws]
    c.run(mr.RUN_BATCHED)
    for j, r in zip(ids, raws):
        assert c.fetch(j) == oracle.wordcount(r)
    c.close()


def test_segmented_sort_many_jobs(mr):
    """The segmented sample sort over 260 jobs: jobs without records (empty,
    whitespace only) between others, one-word jobs, tie runs and long keys
    inside jobs, and slices of Zipf text up to 4 MiB (up to ~500 buckets in
    a job; tiles of the count and scatter passes that span several jobs)."""
    import torch
    import synth
    text, _, _ = synth.wc_text(8 << 20, nwords=50000, seed=41)
    rng = np.random.default_rng(42)
    raws = []
    for i in range(260):
        r = i % 13
        if r == 0:
            raws.append(b"")
        elif r == 1:
            raws.append(b"solo")
        elif r == 2:
            raws.append(b"  \n\t ")
        elif r == 3:
            raws.append(_text(300 + i, b"tietieti", 2, i))
        elif r == 4:
            raws.append(_text(50, b"prefix_shared_by_long_keys_", 3, i))
        else:
            n = int(np.exp(rng.uniform(np.log(100), np.log(4 << 20))))
            off = int(rng.integers(0, text.size - n))
            raws.append(text[off: off + n].tobytes())
    c = mr.Context(autotune=False)
    bufs = [torch.frombuffer(bytearray(r), dtype=torch.uint8).cuda() if r
            else torch.zeros(0, dtype=torch.uint8, device="cuda") for r in raws]
    ids = [c.add_job(mr.WORDCOUNT, b) for b in bufs]
    c.run(mr.RUN_BATCHED)
    for j, r in zip(ids, raws):
        assert c.fetch(j) == oracle.wordcount(r)
    c.rerun()
    for j, r in zip(ids, raws):
        assert c.fetch(j) == oracle.wordcount(r)
    c.close()


@pytest.mark.parametrize("live", [0, 1, 2])
def test_segmented_sort_mostly_empty_jobs(mr, live):
    """A batch large enough for the segmented sort (48 tables of 4096 slots)
    whose jobs hold no words at all (whitespace only, empty), except `live`
    of them: zero records, a single job's records, two jobs far apart."""
    import torch
    raws = [b"" if i % 2 else b" \n " * (i + 1) for i in range(48)]
    if live >= 1:
        raws[7] = b"alpha beta alpha gamma"
    if live >= 2:
        raws[40] = _text(500, b"zzzzzzzz", 3, 40)
    c = mr.Context()
    bufs = [torch.frombuffer(bytearray(r), dtype=torch.uint8).cuda() if r
            else torch.zeros(0, dtype=torch.uint8, device="cuda") for r in raws]
    ids = [c.add_job(mr.WORDCOUNT, b) for b in bufs]
    c.run(mr.RUN_BATCHED)
    for j, r in zip(ids, raws):
        assert c.fetch(j) == oracle.wordcount(r)
    c.close()


@pytest.mark.parametrize("slots", [1024, 2048])
def test_batch_of_small_pinned_tables(mr, slots):
    """300 jobs with caller-sized tables of 1024 slots (the smallest table,
    one compaction block) or 2048, merged by the segmented sort; a table
    below 1024 slots is refused at mr_add_job."""
    import torch
    c0 = mr.Context()
    with pytest.raises(mr.MRError):
        c0.add_job(mr.WORDCOUNT, torch.zeros(8, dtype=torch.uint8, device="cuda"), wc_slots=512)
    c0.close()
    rng = np.random.default_rng(slots)
    raws = []
    for i in range(300):
        nw = int(rng.integers(0, 300))
        raws.append(_text(nw, b"w%03d_" % (i % 17), int(rng.integers(1, 4)), i) if nw else b"")
    c = mr.Context()
    bufs = [torch.frombuffer(bytearray(r), dtype=torch.uint8).cuda() if r
            else torch.zeros(0, dtype=torch.uint8, device="cuda") for r in raws]
    ids = [c.add_job(mr.WORDCOUNT, b, wc_slots=slots) for b in bufs]
    c.run(mr.RUN_BATCHED)
    for j, r in zip(ids, raws):
        assert c.fetch(j) == oracle.wordcount(r)
    c.close()


def test_rerun_after_a_table_regrows(mr):
    """A batch sorted by the segmented sort whose one job overflows its
    automatic table (2^17 slots, 200,000 distinct words): the fetch regrows
    that table and re-runs the job; mr_rerun then re-captures the batch with
    the grown table (now too large for the segmented sort, so the batch takes
    the comparison sort), and every job still equals the oracle."""
    import torch
    import synth
    text, _, _ = synth.wc_text(6 << 20, nwords=50000, seed=91)
    raws = [b" ".join(b"%x" % i for i in range(200_000))]
    rng = np.random.default_rng(92)
    for _ in range(40):
        n = int(rng.integers(1 << 10, 1 << 20))
        off = int(rng.integers(0, text.size - n))
        raws.append(text[off: off + n].tobytes())
    c = mr.Context()
    bufs = [torch.frombuffer(bytearray(r), dtype=torch.uint8).cuda() for r in raws]
    ids = [c.add_job(mr.WORDCOUNT, b) for b in bufs]
    c.run(mr.RUN_BATCHED)
    exp = [oracle.wordcount(r) for r in raws]
    assert [c.fetch(j) for j in ids] == exp
    c.rerun()
    assert [c.fetch(j) for j in ids] == exp
    c.close()
