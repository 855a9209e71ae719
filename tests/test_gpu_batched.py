"""GPU parity: batched mode (one persistent launch for many jobs, one merge +
sort for all word-count jobs, replayed from a captured CUDA graph).

Every job of a mixed batch must equal the oracle bit for bit, and equal the
same job run alone (plain mode)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _mixed_jobs(seed, njobs, max_bytes):
    rng = np.random.default_rng(seed)
    text_pool, _, _ = synth.wc_text(max(max_bytes, 1 << 20) * 2, nwords=20000, seed=seed)
    px_pool = synth.hist_rgb8(max(max_bytes, 3 << 20) // 3 * 2, seed=seed + 1)
    xy_pool = synth.linreg_i8(max(max_bytes, 2 << 20) // 2 * 2, seed=seed + 2)
    jobs = []
    for i in range(njobs):
        size = int(np.exp(rng.uniform(np.log(64), np.log(max_bytes))))
        kind = rng.choice(3, p=[0.5, 0.3, 0.2])
        if kind == 0:
            off = int(rng.integers(0, text_pool.size - size))
            jobs.append((0, text_pool[off: off + size]))
        elif kind == 1:
            size -= size % 3
            off = 3 * int(rng.integers(0, (px_pool.size - size) // 3))
            jobs.append((1, px_pool[off: off + size]))
        else:
            size -= size % 2
            off = 2 * int(rng.integers(0, (xy_pool.size - size) // 2))
            jobs.append((2, xy_pool[off: off + size]))
    return jobs


def _expect(kind, data):
    if kind == 0:
        return oracle.wordcount(data)
    if kind == 1:
        return oracle.hist_rgb8(data).tobytes()
    return oracle.linreg_i8(data).tobytes()


@pytest.mark.parametrize("autotune", [False, True])
def test_batched_mixed_jobs_equal_oracle_and_plain(mr, autotune):
    import torch
    jobs = _mixed_jobs(11, 120, 3 << 20)
    kinds = {0: mr.WORDCOUNT, 1: mr.HIST_RGB8, 2: mr.LINREG_I8}
    dev = [torch.from_numpy(np.ascontiguousarray(d)).cuda() for _, d in jobs]
    c = mr.Context(autotune=autotune)
    ids = [c.add_job(kinds[k], t) for (k, _), t in zip(jobs, dev)]
    c.run(mr.RUN_BATCHED)
    got = [c.fetch(j) for j in ids]
    for (k, d), g in zip(jobs, got):
        assert g == _expect(k, d)
    # replay of the captured graph gives the same bytes
    c.rerun()
    assert [c.fetch(j) for j in ids] == got
    if autotune:
        assert c.tuning()["tuned"]
    # plain mode, one launch sequence per job, gives the same bytes
    ids2 = [c.add_job(kinds[k], t) for (k, _), t in zip(jobs, dev)]
    c.run(mr.RUN_PLAIN)
    assert [c.fetch(j) for j in ids2] == got
    c.close()


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_jobs_on_unaligned_slices(mr, mode):
    """Jobs that are views at arbitrary byte offsets of one device buffer (as
    a caller slicing a resident pool passes them): the kernels stream them
    from their first 16-byte aligned address, with the head and the tail
    done bytewise.  Sizes span one tile to many; regression offsets are odd
    and even (an odd-aligned input keeps bytewise pair loads)."""
    import torch
    rng = np.random.default_rng(31)
    text, _, _ = synth.wc_text(12 << 20, nwords=20000, seed=32)
    px = synth.hist_rgb8(4 << 20, seed=33)
    xy = synth.linreg_i8(3 << 20, seed=34)
    pools = [torch.from_numpy(a).cuda() for a in (text, px, xy)]
    hosts = [text, px, xy]
    kinds = {0: mr.WORDCOUNT, 1: mr.HIST_RGB8, 2: mr.LINREG_I8}
    jobs = []
    for i in range(48):
        k = i % 3
        size = int(rng.integers(1000, 3 << 20)) if i % 4 else int(rng.integers(1, 700))
        size -= size % (1, 3, 2)[k]
        off = int(rng.integers(0, hosts[k].size - size))
        jobs.append((k, off, size))
    c = mr.Context(autotune=False)
    ids = [c.add_job(kinds[k], pools[k][off: off + n]) for k, off, n in jobs]
    c.run(mr.RUN_BATCHED if mode == "batched" else mr.RUN_PLAIN)
    for (k, off, n), j in zip(jobs, ids):
        assert c.fetch(j) == _expect(k, hosts[k][off: off + n]), (k, off, n)
    c.close()


def test_concurrent_run_equals_oracle(mr):
    """MR_RUN_CONCURRENT: the jobs of a run (array, word-count, key-histogram,
    Bloom and k-means kinds) on forked streams; each result equals the
    oracle's, and work enqueued after the run on the context stream sees all
    of them (a second concurrent run over the same inputs gives equal bytes)."""
    import torch
    jobs = _mixed_jobs(23, 30, 2 << 20)
    kinds = {0: mr.WORDCOUNT, 1: mr.HIST_RGB8, 2: mr.LINREG_I8}
    dev = [torch.from_numpy(np.ascontiguousarray(d)).cuda() for _, d in jobs]
    keys = synth.keys_u32(1_000_003, 70_000, seed=24)
    seq = synth.dna(300_000, seed=25)
    x, _, _ = synth.kmeans_points(4000, 16, 8, seed=26)
    init = synth.kmeans_init(x, 8, seed=27)
    c = mr.Context()
    for rep in range(2):
        ids = [c.add_job(kinds[k], t) for (k, _), t in zip(jobs, dev)]
        jk = c.add_job(mr.HIST_U32, keys, hist_bins=65_000)
        jb = c.add_job(mr.BLOOM_DNA, seq, bloom_kmer=21, bloom_bits=1_000_003, bloom_hashes=4)
        jm = c.add_job(mr.KMEANS_F32, x, km_dims=16, km_k=8, km_iters=2, km_init=init)
        c.run(mr.RUN_CONCURRENT)
        for (k, d), j in zip(jobs, ids):
            assert c.fetch(j) == _expect(k, d)
        assert np.array_equal(np.frombuffer(c.fetch(jk), dtype=np.uint64), oracle.hist_u32(keys, 65_000))
        assert np.array_equal(np.frombuffer(c.fetch(jb), dtype=np.uint8), oracle.bloom_dna(seq, 21, 1_000_003, 4))
        cent, assign, _ = mr.split_kmeans_result(c.fetch(jm), 4000, 16, 8)
        _, a_ref = oracle.kmeans(x, init, 2)
        assert np.array_equal(assign, a_ref)
        for j in ids + [jk, jb, jm]:
            c.release(j)
    c.close()


def test_batched_edge_jobs(mr):
    """Empty inputs, one-byte jobs, unaligned device pointers, a hot key and
    jobs whose automatic table overflows inside the batch (re-run at fetch)."""
    import torch
    raw = [b"", b"a", b"x y x", b"hot " * 20000, b" ".join(b"%x" % i for i in range(200_000)),
           b"prefix_shared_by_long_keys_aaaa prefix_shared_by_long_keys_aaab " * 100]
    c = mr.Context()
    ids, exp = [], []
    for i, r in enumerate(raw):
        buf = torch.zeros(len(r) + 8, dtype=torch.uint8, device="cuda")
        if r:
            buf[i % 5: i % 5 + len(r)] = torch.frombuffer(bytearray(r), dtype=torch.uint8).cuda()
        ids.append(c.add_job(mr.WORDCOUNT, buf[i % 5: i % 5 + len(r)]))
        exp.append(oracle.wordcount(r))
    px = synth.hist_rgb8(1001, seed=4)
    for off in (0, 1, 3):
        buf = torch.zeros(px.size + 16, dtype=torch.uint8, device="cuda")
        buf[off: off + px.size] = torch.from_numpy(px).cuda()
        ids.append(c.add_job(mr.HIST_RGB8, buf[off: off + px.size]))
        exp.append(oracle.hist_rgb8(px).tobytes())
    for n in (0, 2, 30):
        xy = synth.linreg_i8(n // 2, seed=n)
        ids.append(c.add_job(mr.LINREG_I8, xy))
        exp.append(oracle.linreg_i8(xy).tobytes())
    c.run(mr.RUN_BATCHED)
    assert [c.fetch(j) for j in ids] == exp
    c.close()


@pytest.mark.parametrize("njobs", [2, 5, 8, 9])
def test_concurrent_array_jobs_fused_equal_oracle(mr, njobs):
    """Two to eight shared-memory histograms and regressions in one
    MR_RUN_CONCURRENT run take one fused launch (nine fall back to one launch
    sequence per job): unaligned slices, ragged lengths, an empty job and a
    tiny one; every result equals the oracle's, in two runs on one context."""
    import torch
    rng = np.random.default_rng(70 + njobs)
    px = synth.hist_rgb8(2_000_003, seed=71)
    xy = synth.linreg_i8(1_500_001, seed=72)
    dp, dx = torch.from_numpy(px).cuda(), torch.from_numpy(xy).cuda()
    specs = []
    for i in range(njobs):
        if i % 2 == 0:
            n = 3 * int(rng.integers(0, 2_000_000 - 2)) if i else 0
            off = 3 * int(rng.integers(0, 2))
            specs.append((mr.HIST_RGB8, px[off: off + n], dp[off: off + n]))
        else:
            n = 2 * int(rng.integers(1, 1_500_000 - 5)) if i != 3 else 2
            off = 2 * int(rng.integers(0, 3)) + 1  # odd byte offsets: unaligned pairs
            specs.append((mr.LINREG_I8, xy[off: off + n], dx[off: off + n]))
    c = mr.Context()
    for rep in range(2):
        ids = [c.add_job(k, d) for k, _, d in specs]
        c.run(mr.RUN_CONCURRENT)
        for (k, h, _), j in zip(specs, ids):
            got = np.frombuffer(c.fetch(j), dtype=np.uint64 if k == mr.HIST_RGB8 else np.int64)
            exp = oracle.hist_rgb8(h).astype(np.uint64) if k == mr.HIST_RGB8 else oracle.linreg_i8(h).astype(np.int64)
            assert np.array_equal(got, exp), (k, len(h))
            c.release(j)
    c.close()
