"""GPU parity: large-key histogram and Bloom-filter build against the oracle.

Both are integer/bit work, so every result must equal the oracle's bytes.
Cases cover the three containers of the histogram (shared-memory local
arrays of one CTA, local arrays spread over a thread-block cluster, the global
array), key ranges from 1 bin to 16M bins, out-of-range keys,
skewed keys, ragged lengths and unaligned device pointers; for the Bloom
filter, window lengths 1..32, filter sizes that are not powers of two, runs
of non-ACGT bytes and sequences shorter than one window; plus the full-size
workloads (256M keys over 16M bins; 30M windows into 300M bits)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _dev(a, offset_bytes=0):
    """Device copy of a uint8/uint32 array starting offset_bytes into a buffer."""
    import torch
    raw = np.array(a, copy=True, order="C").view(np.uint8)  # a writable copy for torch
    buf = torch.zeros(raw.size + offset_bytes + 16, dtype=torch.uint8, device="cuda")
    if raw.size:
        buf[offset_bytes: offset_bytes + raw.size] = torch.from_numpy(raw).cuda()
    return buf[offset_bytes: offset_bytes + raw.size]


@pytest.mark.parametrize("nbins", [1, 100, 4096, 20000, 1 << 20, 1 << 24])
@pytest.mark.parametrize("container", ["auto", "smem", "global"])
def test_hist_u32_matches_oracle(mr, nbins, container):
    cmap = {"auto": mr.C_AUTO, "smem": mr.C_SMEM_ARRAY, "global": mr.C_GLOBAL_ARRAY}
    if container == "smem" and nbins > 40000:
        pytest.skip("local arrays of this many bins do not fit one CTA")
    n = 3_000_001  # ragged: not a multiple of any tile
    keys = synth.keys_u32(n, nbins + nbins // 8 + 1, seed=nbins)  # about 1 key in 9 out of range
    got = mr.hist_u32(_dev(keys), nbins, container=cmap[container])
    assert np.array_equal(got, oracle.hist_u32(keys, nbins))


def _cluster_max_bins():
    import torch
    return 8 * (torch.cuda.get_device_properties(0).shared_memory_per_block_optin // 4) - 1


@pytest.mark.parametrize("nbins", [1, 7, 8, 40, 70_000, 300_000, "max"])
def test_hist_u32_cluster_container(mr, nbins):
    """Local arrays spread over a thread-block cluster's distributed shared
    memory (a container the caller picks): slice boundaries, the out-of-range
    bin and the largest bin count the cluster holds, against the oracle and
    against the automatically chosen container."""
    if nbins == "max":
        nbins = _cluster_max_bins()
    n = 2_000_003
    keys = synth.keys_u32(n, nbins + nbins // 8 + 1, seed=nbins + 5)
    got = mr.hist_u32(_dev(keys), nbins, container=mr.C_CLUSTER_ARRAY)
    assert np.array_equal(got, oracle.hist_u32(keys, nbins))
    if nbins > 60_000:
        assert np.array_equal(mr.hist_u32(_dev(keys), nbins), got)  # C_AUTO


def test_hist_u32_cluster_container_skewed_unaligned_and_bad_args(mr):
    sk = synth.keys_u32(3_000_001, 200_000, skewed=True, seed=8)
    got = mr.hist_u32(_dev(sk, 4), 200_000, container=mr.C_CLUSTER_ARRAY)
    assert np.array_equal(got, oracle.hist_u32(sk, 200_000))
    c = mr.Context()
    keys = synth.keys_u32(1000, 100, seed=2)
    with pytest.raises(mr.MRError):
        c.add_job(mr.HIST_U32, keys, hist_bins=_cluster_max_bins() + 1, container=mr.C_CLUSTER_ARRAY)
    with pytest.raises(mr.MRError):
        c.add_job(mr.HIST_RGB8, np.zeros(30, dtype=np.uint8), container=mr.C_CLUSTER_ARRAY)
    with pytest.raises(mr.MRError):
        c.add_job(mr.WORDCOUNT, b"a b", container=mr.C_CLUSTER_ARRAY)
    c.close()


@pytest.mark.parametrize("offset", [4, 8, 12])
def test_hist_u32_unaligned_and_tiny(mr, offset):
    for n in (0, 1, 3, 5, 33, 1000):
        keys = synth.keys_u32(n, 50, seed=n + offset)
        for c in (mr.C_SMEM_ARRAY, mr.C_GLOBAL_ARRAY):
            got = mr.hist_u32(_dev(keys, offset), 40, container=c)
            assert np.array_equal(got, oracle.hist_u32(keys, 40)), (n, offset, c)


def test_hist_u32_skewed_and_constant(mr):
    sk = synth.keys_u32(5_000_000, 1 << 24, skewed=True, seed=3)
    for c in (mr.C_GLOBAL_ARRAY, mr.C_AUTO):
        assert np.array_equal(mr.hist_u32(_dev(sk), 1 << 24, container=c), oracle.hist_u32(sk, 1 << 24))
    const = np.full(2_000_003, 77, dtype=np.uint32)
    for c in (mr.C_SMEM_ARRAY, mr.C_GLOBAL_ARRAY):
        got = mr.hist_u32(_dev(const), 1000, container=c)
        assert got[77] == const.size and int(got.sum()) == const.size


def test_hist_u32_host_input_and_bad_args(mr):
    keys = synth.keys_u32(100_000, 5000, seed=1)
    assert np.array_equal(mr.hist_u32(keys, 5000), oracle.hist_u32(keys, 5000))
    c = mr.Context()
    with pytest.raises(mr.MRError):
        c.add_job(mr.HIST_U32, keys, hist_bins=0)
    with pytest.raises(mr.MRError):
        c.add_job(mr.HIST_U32, keys.view(np.uint8)[:7], hist_bins=10)  # not whole keys
    with pytest.raises(mr.MRError):
        c.add_job(mr.HIST_U32, keys, hist_bins=1 << 24, container=mr.C_SMEM_ARRAY)
    c.close()


def test_hist_u32_full_size(mr):
    """The paper's Histogram: 256M keys over 16M bins (global array in L2)."""
    keys = synth.keys_u32(256 << 20, 1 << 24)
    got = mr.hist_u32(_dev(keys), 1 << 24)
    assert int(got.sum()) == keys.size
    assert np.array_equal(got, oracle.hist_u32(keys, 1 << 24))


@pytest.mark.parametrize("L", [1, 5, 16, 31, 32])
@pytest.mark.parametrize("m,h", [(2, 1), (97, 3), (1_000_003, 7), (1 << 22, 32)])
def test_bloom_matches_oracle(mr, L, m, h):
    seq = synth.dna(200_000 + L, seed=L, n_runs=20, max_run=300)
    got = mr.bloom_dna(_dev(seq), L, m, h)
    assert np.array_equal(got, oracle.bloom_dna(seq, L, m, h))


@pytest.mark.parametrize("offset", [1, 3, 7])
def test_bloom_edges(mr, offset):
    cases = [b"", b"ACG", b"ACGT", b"ACGTNACGTN", b"acgtACGTACGTACGT", b"A" * 100, b"ACGT\n" * 50,
             bytes(synth.dna(8192 * 3 + 17, seed=offset))]
    for raw in cases:
        seq = np.frombuffer(raw, dtype=np.uint8)
        for L in (4, 32):
            got = mr.bloom_dna(_dev(seq, offset), L, 10_007, 5)
            assert np.array_equal(got, oracle.bloom_dna(raw, L, 10_007, 5)), (raw[:20], L)


def test_bloom_full_size(mr):
    """The paper's Bloom Filter build: 30M k-mers into 300M bits, 7 hashes."""
    L = 32
    seq = synth.dna(30_000_000 + L - 1)
    got = mr.bloom_dna(_dev(seq), L, 300_000_000, 7)
    assert np.array_equal(got, oracle.bloom_dna(seq, L, 300_000_000, 7))
