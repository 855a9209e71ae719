"""GPU parity: word count (hash container + device sort), bit-exact vs the oracle.

The result is a byte string in the layout of include/mr.h; parity means the
GPU bytes equal the oracle's bytes (same records, same order, same keys)."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _dev(data: bytes, offset=0):
    import torch
    raw = np.frombuffer(bytes(data), dtype=np.uint8)
    buf = torch.zeros(raw.size + offset + 16, dtype=torch.uint8, device="cuda")
    if raw.size:
        buf[offset: offset + raw.size] = torch.from_numpy(raw.copy()).cuda()
    return buf[offset: offset + raw.size]


@pytest.mark.parametrize("name", ["wc_tiny.txt", "wc_edge.bin"])
def test_wc_golden_files(mr, name):
    text = open(os.path.join(GOLDEN, name), "rb").read()
    assert mr.wordcount(_dev(text)) == oracle.wordcount(text)


@pytest.mark.parametrize("text", [
    b"", b" ", b"a", b"a ", b" a", b"x y x y x", b"ab abc ab abd abc", b"\x80 \x7f \x80",
    b"tie1 tie2 tie1 tie2", b"\x00\x00 \x00", b"a\rb\x0bc\x0cd\te\nf g",
])
def test_wc_small_cases(mr, text):
    assert mr.wordcount(_dev(text)) == oracle.wordcount(text)


def test_wc_random_alphabets(mr):
    rng = np.random.default_rng(5)
    alphabet = np.frombuffer(b"ab \n\t\x00\xffc", dtype=np.uint8)
    for n in [1, 31, 511, 512, 513, 575, 576, 577, 5000, 100_000]:
        text = alphabet[rng.integers(0, len(alphabet), n)].tobytes()
        assert mr.wordcount(_dev(text)) == oracle.wordcount(text), n


def test_wc_tokens_straddle_segments_and_long_keys(mr):
    rng = np.random.default_rng(9)
    parts = []
    for _ in range(3000):
        L = int(rng.choice([1, 5, 15, 16, 17, 40, 511, 600, 1300]))
        stem = b"prefix_shared_by_many_keys_" if L > 30 else b""
        body = bytes(rng.integers(97, 100, L).astype(np.uint8))
        parts.append(stem + body)
    parts += [parts[3]] * 50 + [parts[7]] * 20
    rng.shuffle(parts)
    text = b" ".join(parts) + b"x"  # no trailing delimiter
    for off in (0, 1, 7):
        assert mr.wordcount(_dev(text, off)) == oracle.wordcount(text)


@pytest.mark.slow
def test_wc_large_input_path_edge_content(mr):
    """Aligned inputs from 32 MiB take the CTA-table map kernel (a shared
    table per CTA, batched global inserts, segments loaded ahead).  80 MiB of
    adversarial content: tokens of 1..40 bytes and a few of 600 and 1300
    (so keys straddle 512- and 1024-byte boundaries and long keys are
    compared byte by byte), every whitespace byte as a separator, token bytes
    including 0x00 and bytes >= 0x80 (keys whose first 8 bytes are all zero
    never enter the CTA tables), a hot key and a long shared-prefix family;
    aligned (the CTA kernel) and one byte in (the per-warp kernel)."""
    rng = np.random.default_rng(21)
    vocab = []
    for i in range(6000):
        w = np.array([10, 10, 10, 10, 10, 10, 10, 5, 5, 5, 4.98, .01, .01])
        L = int(rng.choice([1, 2, 3, 7, 8, 9, 15, 16, 17, 24, 40, 600, 1300], p=w / w.sum()))
        if i % 7 == 0:  # NUL-led keys, some all NUL
            b = bytes(L) if i % 14 == 0 else b"\x00" * min(L, 8) + bytes(rng.integers(97, 123, max(0, L - 8)).astype(np.uint8))
        else:
            b = bytes(rng.choice(np.frombuffer(b"abcxyz\x01\x7f\x80\xfe\xff", dtype=np.uint8), L))
        vocab.append(b[:L] if len(b) >= L else b + b"q" * (L - len(b)))
    vocab += [b"prefix_shared_by_many_keys_" + bytes([97 + (i % 26)]) * (10 + i % 30) for i in range(200)]
    ws = [b" ", b"\n", b"\t", b"\r", b"\x0b", b"\x0c", b"  ", b" \n\t"]
    ranks = rng.zipf(1.3, 3_000_000) % len(vocab)
    seps = rng.integers(0, len(ws), ranks.size)
    chunks = []
    total = 0
    for r, s in zip(ranks, seps):
        chunks.append(vocab[r])
        chunks.append(ws[s])
        total += len(vocab[r]) + len(ws[s])
        if total >= (80 << 20):
            break
    text = b"".join(chunks)
    while len(text) < (80 << 20):
        text = text + text[: (80 << 20) - len(text)]
    text = text[: 80 << 20]
    exp = oracle.wordcount(text)
    for off in (0, 1):
        assert mr.wordcount(_dev(text, off)) == exp, off


def test_wc_hot_key_contention(mr):
    text = b"hot " * 500_000 + b"cold hot\n" * 1000
    assert mr.wordcount(_dev(text)) == oracle.wordcount(text)


def test_wc_pinned_table_overflow_reports(mr):
    text = b" ".join(b"w%d" % i for i in range(5000))
    c = mr.Context()
    j = c.add_job(mr.WORDCOUNT, _dev(text), wc_slots=1024)
    c.run()
    with pytest.raises(mr.MRError) as e:
        c.fetch(j)
    assert e.value.status == mr.MR_EOVERFLOW
    c.release(j)
    c.close()


def test_wc_automatic_table_regrows(mr):
    # ~4-byte distinct tokens: far more keys than the automatic estimate
    text = b" ".join(b"%x" % i for i in range(400_000))
    assert mr.wordcount(_dev(text)) == oracle.wordcount(text)


def test_wc_host_input(mr):
    text, _, _ = synth.wc_text(1 << 20, nwords=3000)
    assert mr.wordcount(text.tobytes()) == oracle.wordcount(text)


def test_wc_zipf_16MiB_bit_exact(mr):
    """The word-count workload: 16 MiB Zipf(1) text over 50,000 words."""
    import torch
    text, ranks, vocab = synth.wc_text(16 << 20)
    got = mr.wordcount(torch.from_numpy(text).cuda())
    ref = oracle.wordcount(text)
    assert got == ref
    recs = oracle.parse_wordcount(got)
    assert sum(c for _, c in recs) == len(ranks)


def test_wc_zipf_40MiB_cta_kernel_bit_exact(mr):
    """40 MiB of Zipf text (16-byte aligned): just above the size from which
    the CTA-table map kernel runs."""
    text, ranks, _ = synth.wc_text(40 << 20, seed=synth.SEED_BASE + 12)
    got = mr.wordcount(_dev(text))
    assert got == oracle.wordcount(text)
    assert sum(c for _, c in oracle.parse_wordcount(got)) == len(ranks)


_BIG = {}


@pytest.mark.slow
@pytest.mark.parametrize("path", ["cta", "warp", "pipelined"])
def test_wc_zipf_320MiB_bit_exact(mr, path):
    """320 MiB of the same generator's text through each large-input map
    path: the CTA-table kernel (16-byte-aligned input); the per-warp-cache
    kernel (the same text one byte into its buffer), past the size at which
    every warp (5 CTAs x 8 warps per SM, 64 segments of 512 bytes between
    hot-key cache merges: ~199 MB per launch) merges its cache into the
    global table in mid-stream and then re-learns the hot keys; and the
    pipelined mapper/reducer kernel, whose mappers do the same."""
    if not _BIG:
        text, ranks, _ = synth.wc_text(320 << 20, seed=synth.SEED_BASE + 11)
        _BIG.update(text=text, ntok=len(ranks), exp=oracle.wordcount(text))
    text = _BIG["text"]
    d = _dev(text, 1 if path == "warp" else 0)
    got = mr.wordcount(d, pipelined=path == "pipelined")
    assert got == _BIG["exp"]
    recs = oracle.parse_wordcount(got)
    assert sum(c for _, c in recs) == _BIG["ntok"]


@pytest.mark.parametrize("torch_alloc", [False, True])
def test_contexts_release_their_memory(mr, torch_alloc):
    """Without allocator hooks a context allocates from a pool of its own that
    keeps freed memory for reuse, and destroying the context hands it back;
    with torch's caching allocator the blocks go back to torch's cache and
    are reused.  Either way, creating, using and closing contexts in a loop
    leaves the device's free memory where it was."""
    import torch
    text, _, _ = synth.wc_text(4 << 20, seed=77)
    dev = torch.from_numpy(text).cuda()
    exp = oracle.wordcount(text)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(12):
        c = mr.Context(use_torch_allocator=torch_alloc)
        for _ in range(3):
            j = c.add_job(mr.WORDCOUNT, dev)
            c.run(mr.RUN_PLAIN)
            assert c.fetch(j) == exp
            c.release(j)
        c.close()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20), (free0, free1)
