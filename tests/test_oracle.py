"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: hand-counted golden
fixtures, an independent brute force (Python ``bytes.split`` + ``Counter``),
the generator's own record of what it emitted, closed forms, exact rational
nearest-centroid search and conservation invariants.  Each check is chosen so
that a plausible slip in the oracle (a dropped last token, a wrong delimiter
set, a signed byte compare, a reversed tie-break, a transposed channel, a
dropped dimension, a wrong tie rule) fails at least one test.
"""
import collections
import math
import os
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------- word count
def _serialize(pairs):
    """Serialize [(key, count)] in the oracle's result layout."""
    n = len(pairs)
    kb = sum(len(k) for k, _ in pairs)
    out = [struct.pack("<QQ", n, kb)]
    off = 0
    for k, c in pairs:
        out.append(struct.pack("<QQQ", c, off, len(k)))
        off += len(k)
    out.extend(k for k, _ in pairs)
    return b"".join(out)


def _brute_wordcount(text: bytes):
    # bytes.split() with no argument splits on exactly the six ASCII
    # whitespace bytes; Python compares bytes as unsigned values.
    cnt = collections.Counter(text.split())
    return sorted(cnt.items(), key=lambda kv: (-kv[1], kv[0]))


def _read_expected(name, hexkeys=False):
    pairs = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        c, k = line.rstrip("\n").split("\t")
        pairs.append((bytes.fromhex(k) if hexkeys else k.encode(), int(c)))
    return pairs


def test_wc_golden_tiny():
    text = open(os.path.join(GOLDEN, "wc_tiny.txt"), "rb").read()
    assert oracle.parse_wordcount(oracle.wordcount(text)) == _read_expected("wc_tiny.expected")


def test_wc_golden_edge_bytes():
    text = open(os.path.join(GOLDEN, "wc_edge.bin"), "rb").read()
    assert oracle.parse_wordcount(oracle.wordcount(text)) == _read_expected("wc_edge.expected", hexkeys=True)


@pytest.mark.parametrize("text", [
    b"", b" ", b"\n\n\t ", b"a", b"a ", b" a", b"word", b"x y x y x",
    b"ab abc ab abd abc", b"\x80 \x7f \x80", b"Aa aA aa AA",
    b"tie1 tie2 tie1 tie2", b"\x00\x00 \x00", b"a\rb\x0bc\x0cd\te\nf g",
])
def test_wc_brute_force_small(text):
    assert oracle.wordcount(text) == _serialize(_brute_wordcount(text))


def test_wc_brute_force_random():
    rng = np.random.default_rng(7)
    alphabet = np.frombuffer(b"ab \n\t\x00\xffc", dtype=np.uint8)
    for n in [1, 2, 3, 17, 100, 1000, 5000]:
        for _ in range(5):
            text = alphabet[rng.integers(0, len(alphabet), n)].tobytes()
            assert oracle.wordcount(text) == _serialize(_brute_wordcount(text))


def test_wc_generator_ground_truth():
    text, ranks, vocab = synth.wc_text(1 << 20, nwords=5000)
    got = dict(oracle.parse_wordcount(oracle.wordcount(text)))
    emitted = np.bincount(ranks, minlength=len(vocab))
    expect = {vocab[r]: int(c) for r, c in enumerate(emitted) if c}
    assert got == expect
    # Σ count = number of tokens, counted by a separate scan of token starts
    t = np.frombuffer(text.tobytes(), dtype=np.uint8)
    ws = np.isin(t, np.frombuffer(b" \t\n\v\f\r", dtype=np.uint8))
    starts = (~ws) & np.concatenate([[True], ws[:-1]])
    assert sum(got.values()) == int(starts.sum()) == len(ranks)


def test_wc_output_sorted_and_unique():
    text, _, _ = synth.wc_text(1 << 18, nwords=2000)
    recs = oracle.parse_wordcount(oracle.wordcount(text))
    keys = [k for k, _ in recs]
    assert len(set(keys)) == len(keys)
    for (k1, c1), (k2, c2) in zip(recs, recs[1:]):
        assert c1 > c2 or (c1 == c2 and k1 < k2)


# ------------------------------------------------------------------ histogram
def test_hist_bincount_and_invariants():
    px = synth.hist_rgb8(100_003)
    bins = oracle.hist_rgb8(px)
    for c in range(3):
        ref = np.bincount(px[c::3], minlength=256).astype(np.uint64)
        assert np.array_equal(bins[c * 256:(c + 1) * 256], ref)
        assert int(bins[c * 256:(c + 1) * 256].sum()) == 100_003
    assert int(bins.sum()) == 3 * 100_003


def test_hist_channels_not_transposed():
    px = np.tile(np.array([1, 2, 3], dtype=np.uint8), 1000)
    bins = oracle.hist_rgb8(px)
    expect = np.zeros(768, dtype=np.uint64)
    expect[0 * 256 + 1] = expect[1 * 256 + 2] = expect[2 * 256 + 3] = 1000
    assert np.array_equal(bins, expect)


def test_hist_constant_empty_and_bad_length():
    bins = oracle.hist_rgb8(np.full(3 * 777, 255, dtype=np.uint8))
    assert bins[255] == bins[511] == bins[767] == 777 and bins.sum() == 3 * 777
    assert oracle.hist_rgb8(np.zeros(0, dtype=np.uint8)).sum() == 0
    with pytest.raises(ValueError):
        oracle.hist_rgb8(np.zeros(4, dtype=np.uint8))


# ---------------------------------------------------------- linear regression
def test_linreg_hand_computed():
    # pairs (1,3), (-2,-5), (127,-128), worked by hand
    xy = np.array([1, 3, -2, -5, 127, -128], dtype=np.int8)
    assert oracle.linreg_i8(xy).tolist() == [126, -130, 16134, 16418, -16243]


@pytest.mark.parametrize("k", [1, 3, 1000])
def test_linreg_closed_form_full_range(k):
    x = np.tile(np.arange(-128, 128, dtype=np.int64), k)
    y = -1 - x  # bitwise not, also spans -128..127
    xy = np.empty(2 * x.size, dtype=np.int8)
    xy[0::2] = x
    xy[1::2] = y
    sq = sum(i * i for i in range(-128, 128))  # 1,398,016
    # Σy = Σ(-1-x) = -256k + 128k; Σxy = -Σx - Σx²
    assert oracle.linreg_i8(xy).tolist() == [-128 * k, -128 * k, k * sq, k * sq, 128 * k - k * sq]


def test_linreg_brute_force_and_errors():
    xy = synth.linreg_i8(50_001)
    xs = [int(v) for v in xy[0::2]]
    ys = [int(v) for v in xy[1::2]]
    expect = [sum(xs), sum(ys), sum(a * a for a in xs), sum(b * b for b in ys), sum(a * b for a, b in zip(xs, ys))]
    assert oracle.linreg_i8(xy).tolist() == expect
    assert oracle.linreg_i8(np.zeros(0, dtype=np.int8)).tolist() == [0] * 5
    with pytest.raises(ValueError):
        oracle.linreg_i8(np.zeros(3, dtype=np.int8))
    ext = np.full(2 * 999, -128, dtype=np.int8)
    assert oracle.linreg_i8(ext).tolist() == [-128 * 999, -128 * 999, 16384 * 999, 16384 * 999, 16384 * 999]


# -------------------------------------------------------------------- k-means
def _exact_assign(x, c):
    """Exact nearest centroid with rational arithmetic; lowest index on ties.
    Returns (assignment, exact relative margin between best and runner-up)."""
    out, margins = [], []
    cf = [[Fraction(float(v)) for v in row] for row in c]
    for row in x:
        xf = [Fraction(float(v)) for v in row]
        ds = [sum((a - b) ** 2 for a, b in zip(xf, cr)) for cr in cf]
        best = min(range(len(ds)), key=lambda i: (ds[i], i))
        out.append(best)
        rest = [d for i, d in enumerate(ds) if i != best]
        margins.append(float((min(rest) - ds[best]) / max(ds[best], Fraction(1))) if rest else 1.0)
    return np.array(out), np.array(margins)


def test_kmeans_assign_exact_rational():
    rng = np.random.default_rng(3)
    x = rng.normal(0, 3, size=(60, 5)).astype(np.float32)
    c = rng.normal(0, 3, size=(7, 5)).astype(np.float32)
    c[5] = c[2]  # an exact tie: the lower index must win
    a = oracle.kmeans_assign(x, c)
    ex, margin = _exact_assign(x, c)
    safe = margin > 1e-12
    assert np.array_equal(a[safe], ex[safe])
    assert not np.any(a == 5)


def test_kmeans_assign_every_dimension_counts():
    # points differ from the centroids in one coordinate only; dropping any
    # coordinate (or mixing up point and centroid index) changes the answer
    d, k = 6, 6
    c = np.zeros((k, d), dtype=np.float32)
    for j in range(k):
        c[j, j] = 10.0
    x = np.zeros((d, d), dtype=np.float32)
    for j in range(d):
        x[j, j] = 9.0
    assert oracle.kmeans_assign(x, c).tolist() == list(range(d))


def test_kmeans_k1_is_global_mean():
    x, _, _ = synth.kmeans_points(5000, 8, 4)
    c0 = x[:1].copy()
    c1, a = oracle.kmeans(x, c0, 1)
    assert np.all(a == 0)
    exact = np.array([math.fsum(x[:, j].astype(np.float64)) / x.shape[0] for j in range(8)])
    np.testing.assert_allclose(c1[0], exact.astype(np.float32), rtol=2e-7, atol=1e-7)


def test_kmeans_separated_converges_in_one_iteration():
    x, comp, means = synth.kmeans_points(20_000, 16, 12, lo=-100, hi=100, sigma=0.5)
    init = means.astype(np.float32)
    c1, a = oracle.kmeans(x, init, 1)
    assert np.array_equal(a, comp)
    for k in range(12):
        pts = x[comp == k].astype(np.float64)
        exact = np.array([math.fsum(pts[:, j]) / len(pts) for j in range(16)], dtype=np.float32)
        np.testing.assert_allclose(c1[k], exact, rtol=2e-7, atol=1e-6)
    c2, a2 = oracle.kmeans(x, init, 3)
    assert np.array_equal(a2, comp)
    np.testing.assert_array_equal(c2, c1)


def test_kmeans_empty_cluster_keeps_centroid():
    x, _, _ = synth.kmeans_points(2000, 4, 3)
    init = np.concatenate([x[:3], np.full((1, 4), 1e6, dtype=np.float32)])
    c, _ = oracle.kmeans(x, init, 2)
    assert np.array_equal(c[3], init[3])


def test_kmeans_loop_is_assign_then_update():
    x, _, _ = synth.kmeans_points(3000, 8, 16)
    init = synth.kmeans_init(x, 16)
    cur = init
    for _ in range(3):
        a = oracle.kmeans_assign(x, cur)
        cur, counts = oracle.kmeans_update(x, a, cur)
        assert int(counts.sum()) == x.shape[0]
    c3, a3 = oracle.kmeans(x, init, 3)
    assert np.array_equal(c3, cur) and np.array_equal(a3, a)


# ----------------------------------------------------------- large-key histogram

def test_hist_u32_brute_force_tiny():
    rng = np.random.default_rng(7)
    for nbins in (1, 5, 64):
        keys = rng.integers(0, nbins + 3, size=500).astype(np.uint32)  # some keys out of range
        got = oracle.hist_u32(keys, nbins)
        exp = [0] * (nbins + 1)
        for k in keys.tolist():
            exp[k if k < nbins else nbins] += 1
        assert got.tolist() == exp


def test_hist_u32_equals_bincount_and_conserves():
    keys = synth.keys_u32(1 << 20, 1 << 16)
    got = oracle.hist_u32(keys, 1 << 16)
    assert np.array_equal(got[:-1], np.bincount(keys, minlength=1 << 16).astype(np.uint64))
    assert got[-1] == 0 and int(got.sum()) == keys.size
    sk = synth.keys_u32(1 << 20, 1 << 16, skewed=True)
    g2 = oracle.hist_u32(sk, 1 << 16)
    assert np.array_equal(g2[:-1], np.bincount(sk, minlength=1 << 16).astype(np.uint64))


def test_hist_u32_constant_and_extreme_keys():
    keys = np.full(1000, 123, dtype=np.uint32)
    got = oracle.hist_u32(keys, 200)
    assert got[123] == 1000 and int(got.sum()) == 1000
    ext = np.array([0, 2 ** 32 - 1, 9, 10, 2 ** 31], dtype=np.uint32)
    got = oracle.hist_u32(ext, 10)
    assert got.tolist() == [1] + [0] * 8 + [1] + [3]
    assert oracle.hist_u32(np.zeros(0, dtype=np.uint32), 4).tolist() == [0] * 5


# ----------------------------------------------------------------- Bloom filter

def test_mix64_is_splitmix64_output_function():
    # SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) seeded with 1234567: its
    # first five outputs, as published with the generator's reference
    # implementations; next() adds the golden gamma and then mixes.
    gamma = 0x9E3779B97F4A7C15
    st, outs = 1234567, []
    for _ in range(5):
        st = (st + gamma) % 2 ** 64
        outs.append(oracle.mix64(st))
    assert outs == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                    4593380528125082431, 16408922859458223821]
    assert oracle.mix64(gamma) == 0xE220A8397B1DCDAF  # seed 0, first output


def _windows(seq: bytes, L: int):
    return [seq[i:i + L] for i in range(len(seq) - L + 1)]


def test_bloom_window_codes_are_base4_numbers():
    seq = bytes(synth.dna(300, seed=11))
    for L in (1, 7, 31, 32):
        codes = [int(w.translate(bytes.maketrans(b"ACGT", b"0123")), 4) for w in _windows(seq, L)]
        assert np.array_equal(oracle.bloom_dna(seq, L, 1000, 3), oracle.bloom_codes(codes, 1000, 3))


def test_bloom_skips_windows_with_other_bytes():
    a, b = bytes(synth.dna(200, seed=1)), bytes(synth.dna(150, seed=2))
    L, m, h = 16, 4099, 5
    for sep in (b"N", b"\n", b"a", b"NNNN"):
        got = oracle.bloom_dna(a + sep + b, L, m, h)
        assert np.array_equal(got, oracle.bloom_dna(a, L, m, h) | oracle.bloom_dna(b, L, m, h))
    assert not oracle.bloom_dna(b"ACGTNACGTN", 5, m, h).any()  # no complete window
    assert not oracle.bloom_dna(b"ACG", 4, m, h).any()         # shorter than one window


def test_bloom_is_union_of_single_windows():
    seq = bytes(synth.dna(120, seed=3))
    L, m, h = 9, 977, 4
    acc = np.zeros((m + 7) // 8, dtype=np.uint8)
    for w in _windows(seq, L):
        acc |= oracle.bloom_dna(w, L, m, h)
    assert np.array_equal(oracle.bloom_dna(seq, L, m, h), acc)


def test_bloom_bit_positions_of_one_element():
    m, h = 1_000_003, 7
    for code in (0, 1, 12345, 2 ** 64 - 1):
        a = oracle.mix64(code) % m
        b = 1 + oracle.mix64(code ^ 0x9E3779B97F4A7C15) % (m - 1)
        pos = {(a + i * b) % m for i in range(h)}
        bits = np.unpackbits(oracle.bloom_codes([code], m, h), bitorder="little")[:m]
        assert set(np.flatnonzero(bits).tolist()) == pos


def test_bloom_fill_matches_expectation_and_no_false_negatives():
    m, h, n = 1 << 20, 7, 100_000
    codes = np.unique(synth.keys_u32(n + 5000, 2 ** 32 - 1, seed=9).astype(np.uint64) * 7919)[:n]
    bits = np.unpackbits(oracle.bloom_codes(codes, m, h), bitorder="little")[:m]
    # fill of an ideal filter: m (1 - (1 - 1/m)^(h n)), binomial-like spread
    p = 1 - (1 - 1 / m) ** (h * codes.size)
    assert abs(bits.sum() - m * p) < 6 * math.sqrt(m * p * (1 - p))
    for c in codes[:200].tolist():
        one = np.unpackbits(oracle.bloom_codes([c], m, h), bitorder="little")[:m]
        assert np.all(bits[one == 1] == 1)


# ------------------------------------------------------------- string hashing

def test_fnv1a64_published_vectors():
    # FNV-1a 64 test vectors published with the FNV reference code
    assert oracle.fnv1a64(b"") == 0xCBF29CE484222325
    assert oracle.fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert oracle.fnv1a64(b"foobar") == 0x85944171F73967E8


def test_token_hashes_follow_the_tokens():
    import re
    text = bytes(synth.wc_text(200_000, nwords=3000)[0]) + b"\x00\xff x\ty\v\fz\r\n" + b"q" * 40
    off, ln, h = oracle.token_hashes(text)
    spans = [(m.start(), m.end()) for m in re.finditer(rb"[^ \t\n\v\f\r]+", text)]
    assert [(int(a), int(a + b)) for a, b in zip(off, ln)] == spans
    for i in (0, 1, len(spans) // 2, len(spans) - 1):
        a, b = spans[i]
        assert int(h[i]) == oracle.fnv1a64(text[a:b])
    assert oracle.token_hashes(b"")[0].size == 0 and oracle.token_hashes(b" \n ")[0].size == 0
