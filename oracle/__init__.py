"""CPU oracle — TEST INFRASTRUCTURE ONLY.

A plain serial C++ restatement of every job's map/reduce (see oracle.cpp for
the citations).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package; the CUDA library never calls it and shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
            lib.oracle_wordcount.argtypes = [vp, u64, vp, u64, ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_hist_rgb8.argtypes = [vp, u64, vp]
            lib.oracle_linreg_i8.argtypes = [vp, u64, vp]
            lib.oracle_kmeans_assign.argtypes = [vp, u64, u32, vp, u32, vp, vp]
            lib.oracle_kmeans_update.argtypes = [vp, u64, u32, vp, u32, vp, vp, vp]
            lib.oracle_kmeans.argtypes = [vp, u64, u32, vp, u32, u32, vp, vp]
            lib.oracle_hist_u32.argtypes = [vp, u64, u32, vp]
            lib.oracle_mix64.argtypes = [u64]
            lib.oracle_mix64.restype = u64
            lib.oracle_bloom_dna.argtypes = [vp, u64, u32, u64, u32, vp]
            lib.oracle_bloom_codes.argtypes = [vp, u64, u64, u32, vp]
            lib.oracle_fnv1a64.argtypes = [vp, u64]
            lib.oracle_fnv1a64.restype = u64
            lib.oracle_token_hashes.argtypes = [vp, u64, vp, vp, vp, u64, ctypes.POINTER(ctypes.c_uint64)]
            _lib = lib
    return _lib


def _buf(a) -> tuple[np.ndarray, int]:
    a = np.ascontiguousarray(a)
    return a, (a.ctypes.data if a.size else 0)


def wordcount(text) -> bytes:
    """Serialized word-count result (layout in oracle.cpp)."""
    t = np.frombuffer(bytes(text), dtype=np.uint8) if isinstance(text, (bytes, bytearray)) else np.ascontiguousarray(text, dtype=np.uint8)
    t, p = _buf(t)
    need = ctypes.c_uint64(0)
    rc = _L().oracle_wordcount(p, t.size, None, 0, ctypes.byref(need))
    if rc:
        raise ValueError("oracle_wordcount: %d" % rc)
    out = np.empty(need.value, dtype=np.uint8)
    rc = _L().oracle_wordcount(p, t.size, out.ctypes.data, out.size, ctypes.byref(need))
    if rc:
        raise ValueError("oracle_wordcount: %d" % rc)
    return out.tobytes()


def hist_rgb8(px) -> np.ndarray:
    px, p = _buf(np.asarray(px, dtype=np.uint8))
    bins = np.zeros(768, dtype=np.uint64)
    if _L().oracle_hist_rgb8(p, px.size, bins.ctypes.data):
        raise ValueError("input length must be a multiple of 3")
    return bins


def linreg_i8(xy) -> np.ndarray:
    xy, p = _buf(np.asarray(xy, dtype=np.int8))
    sums = np.zeros(5, dtype=np.int64)
    if _L().oracle_linreg_i8(p, xy.size, sums.ctypes.data):
        raise ValueError("input length must be even")
    return sums


def hist_u32(keys, nbins: int) -> np.ndarray:
    """u64[nbins + 1]: counts of each key < nbins, then the out-of-range count."""
    k, p = _buf(np.asarray(keys, dtype=np.uint32))
    out = np.zeros(nbins + 1, dtype=np.uint64)
    if _L().oracle_hist_u32(p, k.size, nbins, out.ctypes.data):
        raise ValueError("oracle_hist_u32")
    return out


def mix64(z: int) -> int:
    return int(_L().oracle_mix64(ctypes.c_uint64(z & (2 ** 64 - 1))))


def bloom_dna(seq, L: int, m: int, h: int) -> np.ndarray:
    """Bloom filter bits (ceil(m/8) bytes) of every all-ACGT window of length L."""
    s, p = _buf(np.frombuffer(seq, dtype=np.uint8) if isinstance(seq, (bytes, bytearray))
                else np.asarray(seq, dtype=np.uint8))
    out = np.zeros((m + 7) // 8, dtype=np.uint8)
    if _L().oracle_bloom_dna(p, s.size, L, m, h, out.ctypes.data):
        raise ValueError("oracle_bloom_dna")
    return out


def bloom_codes(codes, m: int, h: int) -> np.ndarray:
    c, p = _buf(np.asarray(codes, dtype=np.uint64))
    out = np.zeros((m + 7) // 8, dtype=np.uint8)
    if _L().oracle_bloom_codes(p, c.size, m, h, out.ctypes.data):
        raise ValueError("oracle_bloom_codes")
    return out


def fnv1a64(data: bytes) -> int:
    buf = np.frombuffer(bytes(data), dtype=np.uint8)
    return int(_L().oracle_fnv1a64(buf.ctypes.data if buf.size else None, buf.size))


def token_hashes(text):
    """(offsets u64, lengths u64, FNV-1a 64 hashes u64) of the word-count tokens, in order."""
    t, p = _buf(np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray))
                else np.asarray(text, dtype=np.uint8))
    cnt = ctypes.c_uint64()
    if _L().oracle_token_hashes(p, t.size, None, None, None, 0, ctypes.byref(cnt)):
        raise ValueError("oracle_token_hashes")
    n = cnt.value
    off, ln, h = (np.zeros(n, dtype=np.uint64) for _ in range(3))
    if _L().oracle_token_hashes(p, t.size, off.ctypes.data, ln.ctypes.data, h.ctypes.data, n, ctypes.byref(cnt)):
        raise ValueError("oracle_token_hashes")
    return off, ln, h


def kmeans_assign(x, c, want_dmin: bool = False):
    x, px = _buf(np.asarray(x, dtype=np.float32))
    c, pc = _buf(np.asarray(c, dtype=np.float32))
    n, d = x.shape
    k = c.shape[0]
    a = np.empty(n, dtype=np.int32)
    dmin = np.empty(n, dtype=np.float64) if want_dmin else None
    if _L().oracle_kmeans_assign(px, n, d, pc, k, a.ctypes.data, dmin.ctypes.data if want_dmin else None):
        raise ValueError("oracle_kmeans_assign")
    return (a, dmin) if want_dmin else a


def kmeans_update(x, assign, c_prev):
    x, px = _buf(np.asarray(x, dtype=np.float32))
    a, pa = _buf(np.asarray(assign, dtype=np.int32))
    cp, pcp = _buf(np.asarray(c_prev, dtype=np.float32))
    n, d = x.shape
    k = cp.shape[0]
    cn = np.empty_like(cp)
    counts = np.empty(k, dtype=np.uint64)
    if _L().oracle_kmeans_update(px, n, d, pa, k, pcp, cn.ctypes.data, counts.ctypes.data):
        raise ValueError("oracle_kmeans_update")
    return cn, counts


def kmeans(x, init, iters: int):
    x, px = _buf(np.asarray(x, dtype=np.float32))
    c0, pc = _buf(np.asarray(init, dtype=np.float32))
    n, d = x.shape
    k = c0.shape[0]
    cout = np.empty_like(c0)
    a = np.zeros(n, dtype=np.int32)
    if _L().oracle_kmeans(px, n, d, pc, k, iters, cout.ctypes.data, a.ctypes.data):
        raise ValueError("oracle_kmeans")
    return cout, a


def parse_wordcount(blob: bytes):
    """Decode the serialized word-count layout into [(key bytes, count), ...]."""
    n, kb = np.frombuffer(blob[:16], dtype=np.uint64)
    n = int(n)
    rec = np.frombuffer(blob[16:16 + 24 * n], dtype=np.uint64).reshape(n, 3)
    keys = blob[16 + 24 * n:]
    assert len(keys) == int(kb)
    return [(keys[int(o):int(o) + int(l)], int(c)) for c, o, l in rec]
