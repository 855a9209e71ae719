"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's own data sets (word-count text, image histogram, ...) are not
available, so every job runs on inputs produced here.  This module only
produces inputs: it holds none of the map/reduce arithmetic, and it is the one
piece of code that both the oracle and the CUDA path consume.

Recipes:

* word count: 50,000 distinct lowercase words of length 3..12 (letters uniform
  on a..z, duplicates rejected), drawn Zipf(s=1) by rank; single spaces, a
  newline after every 8..20 words; the buffer is filled up to a word boundary
  and padded with newlines to exactly ``nbytes``.
* RGB histogram: per pixel, 70% three uniform bytes, else one of 8 colour
  clusters with channel value clamp(round(centre + 12 N(0,1)), 0, 255).
* linear regression: int8 pairs, x uniform on [-40, 40],
  y = clamp(3x + round(4 N(0,1)), -128, 127), stored x0 y0 x1 y1 ...
* k-means: 256-component Gaussian mixture, means uniform in [-10, 10]^d,
  unit variance, FP32; K initial centroids are K distinct sampled points.
* large-key histogram: u32 keys uniform on [0, 2^24) (or a skewed variant).
* Bloom filter: uniform A/C/G/T bases, optionally with runs of N.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 0x5EED0


def build(force: bool = False) -> str:
    """Compile the generator library next to its source (gcc, a second or two)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, u32, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_void_p)
            lib.synth_hist_rgb8.argtypes = [u64, u64, dbl, u32, dbl, vp, i32]
            lib.synth_linreg_i8.argtypes = [u64, u64, i32, i32, i32, dbl, vp, i32]
            lib.synth_kmeans_f32.argtypes = [u64, u64, u32, u32, dbl, dbl, dbl, vp, vp, vp, i32]
            lib.synth_sample_distinct.argtypes = [u64, u32, u32, vp, vp]
            lib.synth_wc_candidates.argtypes = [u64, u64, u32, u32, u32, vp, vp]
            lib.synth_wc_text.argtypes = [u64, vp, vp, vp, u32, vp, u64, u32, u32, vp, vp, u64]
            lib.synth_wc_text.restype = ctypes.c_int64
            lib.synth_keys_u32.argtypes = [u64, u64, u32, i32, vp, i32]
            lib.synth_dna.argtypes = [u64, u64, u32, u32, vp, i32]
            _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def hist_rgb8(n_pixels: int, seed: int = SEED_BASE + 1, p_uniform: float = 0.7,
              n_clusters: int = 8, sigma: float = 12.0, out: np.ndarray | None = None) -> np.ndarray:
    """Interleaved RGB8 bytes, length 3 * n_pixels."""
    if out is None:
        out = np.empty(3 * n_pixels, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size >= 3 * n_pixels and out.flags.c_contiguous
    rc = _L().synth_hist_rgb8(seed, n_pixels, p_uniform, n_clusters, sigma, _p(out), _threads())
    if rc:
        raise ValueError("synth_hist_rgb8 failed")
    return out[: 3 * n_pixels]


def linreg_i8(n_pairs: int, seed: int = SEED_BASE + 2, xmin: int = -40, xmax: int = 40,
              slope: int = 3, sigma: float = 4.0, out: np.ndarray | None = None) -> np.ndarray:
    """Interleaved int8 (x, y) pairs, length 2 * n_pairs."""
    if out is None:
        out = np.empty(2 * n_pairs, dtype=np.int8)
    assert out.dtype == np.int8 and out.size >= 2 * n_pairs and out.flags.c_contiguous
    rc = _L().synth_linreg_i8(seed, n_pairs, xmin, xmax, slope, sigma, _p(out), _threads())
    if rc:
        raise ValueError("synth_linreg_i8 failed")
    return out[: 2 * n_pairs]


def kmeans_points(n: int, d: int = 64, ncomp: int = 256, seed: int = SEED_BASE + 3,
                  lo: float = -10.0, hi: float = 10.0, sigma: float = 1.0):
    """(X float32 [n, d], component int32 [n], means float64 [ncomp, d])."""
    x = np.empty((n, d), dtype=np.float32)
    comp = np.empty(n, dtype=np.int32)
    means = np.empty((ncomp, d), dtype=np.float64)
    rc = _L().synth_kmeans_f32(seed, n, d, ncomp, lo, hi, sigma, _p(x), _p(comp), _p(means), _threads())
    if rc:
        raise ValueError("synth_kmeans_f32 failed")
    return x, comp, means


def keys_u32(n: int, nbins: int = 1 << 24, seed: int = SEED_BASE + 5, skewed: bool = False,
             out: np.ndarray | None = None) -> np.ndarray:
    """u32 keys in [0, nbins): uniform, or skewed (rank density ~ 1/(rank + 1),
    ranks spread over the key range by a fixed bijection)."""
    if out is None:
        out = np.empty(n, dtype=np.uint32)
    assert out.dtype == np.uint32 and out.size >= n and out.flags.c_contiguous
    if _L().synth_keys_u32(seed, n, nbins, 1 if skewed else 0, _p(out), _threads()):
        raise ValueError("synth_keys_u32 failed")
    return out[:n]


def dna(n: int, seed: int = SEED_BASE + 6, n_runs: int = 0, max_run: int = 1000,
        out: np.ndarray | None = None) -> np.ndarray:
    """ASCII DNA bases (uniform A/C/G/T), with n_runs runs of 'N' written over it."""
    if out is None:
        out = np.empty(n, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size >= n and out.flags.c_contiguous
    if _L().synth_dna(seed, n, n_runs, max_run, _p(out), _threads()):
        raise ValueError("synth_dna failed")
    return out[:n]


def sample_distinct(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices of [0, n) (partial Fisher-Yates)."""
    scratch = np.empty(n, dtype=np.uint32)
    out = np.empty(k, dtype=np.uint32)
    if _L().synth_sample_distinct(seed, n, k, _p(scratch), _p(out)):
        raise ValueError("k > n")
    return out


def kmeans_init(x: np.ndarray, k: int, seed: int = SEED_BASE + 4) -> np.ndarray:
    """K initial centroids: K distinct points of x (float32 [k, d])."""
    idx = sample_distinct(x.shape[0], k, seed)
    return np.ascontiguousarray(x[idx.astype(np.int64)])


def wc_vocab(nwords: int = 50_000, seed: int = SEED_BASE, minlen: int = 3, maxlen: int = 12):
    """Distinct random lowercase words, in generation order (rank r = index r)."""
    words: list[bytes] = []
    seen: set[bytes] = set()
    stream = 0
    batch = 65536
    while len(words) < nwords:
        buf = np.empty(batch * maxlen, dtype=np.uint8)
        lens = np.empty(batch, dtype=np.uint32)
        if _L().synth_wc_candidates(seed, stream, batch, minlen, maxlen, _p(buf), _p(lens)):
            raise ValueError("bad vocabulary parameters")
        raw = buf.tobytes()
        for i in range(batch):
            w = raw[i * maxlen: i * maxlen + int(lens[i])]
            if w not in seen:
                seen.add(w)
                words.append(w)
                if len(words) == nwords:
                    break
        stream += 1
    return words


def zipf_cdf(nwords: int, s: float = 1.0) -> np.ndarray:
    w = 1.0 / np.arange(1, nwords + 1, dtype=np.float64) ** s
    cdf = np.cumsum(w) / w.sum()
    cdf[-1] = 1.0
    return cdf


def wc_text(nbytes: int = 16 << 20, seed: int = SEED_BASE, nwords: int = 50_000,
            nl_min: int = 8, nl_max: int = 20, vocab: list[bytes] | None = None,
            want_ranks: bool = True):
    """(text uint8 [nbytes], ranks uint32 [ntokens] or None, vocab list[bytes])."""
    if vocab is None:
        vocab = wc_vocab(nwords, seed)
    vlen = np.array([len(w) for w in vocab], dtype=np.uint32)
    voff = np.zeros(len(vocab), dtype=np.uint64)
    voff[1:] = np.cumsum(vlen[:-1], dtype=np.uint64)
    vbytes = np.frombuffer(b"".join(vocab), dtype=np.uint8).copy()
    cdf = zipf_cdf(len(vocab))
    out = np.empty(nbytes, dtype=np.uint8)
    cap = nbytes // 2 + 1
    ranks = np.empty(cap, dtype=np.uint32) if want_ranks else None
    n = _L().synth_wc_text(seed, _p(vbytes), _p(voff), _p(vlen), len(vocab), _p(cdf), nbytes,
                           nl_min, nl_max, _p(out), _p(ranks) if want_ranks else None, cap)
    if n < 0:
        raise ValueError("synth_wc_text failed")
    return out, (ranks[:n].copy() if want_ranks else None), vocab
