"""GPU parity: SIMD string hashing (SIMDH-Padding, SIMDH-Stream and the wide
variant) against the oracle's FNV-1a 64 of every word-count token.  Hashes
are integers: every method must equal the oracle bit for bit, on the
word-count text, on long and one-byte tokens, and on unaligned text."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _run(mr, raw: bytes, offset: int = 0):
    import torch
    off, ln, h = oracle.token_hashes(raw)
    buf = torch.zeros(len(raw) + offset + 8, dtype=torch.uint8, device="cuda")
    if raw:
        buf[offset: offset + len(raw)] = torch.frombuffer(bytearray(raw), dtype=torch.uint8).cuda()
    text = buf[offset: offset + len(raw)]
    d_off = torch.from_numpy(off.astype(np.int32)).cuda()
    d_len = torch.from_numpy(ln.astype(np.int32)).cuda()
    exp = h.view(np.int64)
    for m in (mr.SIMDH_PADDING, mr.SIMDH_STREAM, mr.SIMDH_WIDE):
        got = mr.simdh_hash(text, d_off, d_len, m).cpu().numpy()
        assert np.array_equal(got, exp), m


def test_simdh_wordcount_text(mr):
    text, _, _ = synth.wc_text(2 << 20, nwords=20000)
    _run(mr, bytes(text))


@pytest.mark.parametrize("offset", [0, 1, 2, 3])
def test_simdh_edges_and_alignment(mr, offset):
    rng = np.random.default_rng(offset)
    parts = []
    for _ in range(3000):
        L = int(rng.choice([1, 2, 3, 4, 5, 15, 16, 17, 63, 200]))
        parts.append(bytes(rng.integers(33, 127, size=L, dtype=np.uint8)))
    raw = b" ".join(parts) + b"\n" + bytes(range(0x80, 0x100)) + b" x"
    _run(mr, raw, offset)
    _run(mr, b"", offset)
    _run(mr, b"a", offset)
