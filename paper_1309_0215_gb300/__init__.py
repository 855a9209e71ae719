"""GB300 fused map-and-reduce — Python binding of ``libmrgb.so``.

This module only marshals arguments for the C ABI declared in
``include/mr.h``; every step of every job (map, combine, reduce, merge, sort)
runs in the library's CUDA kernels.  PyTorch supplies device memory (through
its caching allocator, passed to the library as allocation hooks) and
streams.  There is no CPU path: if the library is missing or no GPU is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from ._build import LIB as _LIB_PATH, build as _build_lib, up_to_date as _up_to_date

# ---------------------------------------------------------------- constants
MR_OK, MR_EINVAL, MR_ENOMEM, MR_ECUDA, MR_EOVERFLOW, MR_ETIMEOUT, MR_EBUDGET, MR_ENOTREADY, MR_ENOJOB = range(9)
WORDCOUNT, HIST_RGB8, LINREG_I8, KMEANS_F32, HIST_U32, BLOOM_DNA = range(6)
C_AUTO, C_SMEM_ARRAY, C_GLOBAL_ARRAY, C_HASH, C_CLUSTER_ARRAY = range(5)
RUN_PLAIN, RUN_BATCHED, RUN_CONCURRENT = range(3)
KM_FP32, KM_BF16_TC, KM_BF16X1_TC = range(3)

# every entry point declared in include/mr.h
EXPORTS = ("mr_create", "mr_destroy", "mr_add_job", "mr_run", "mr_fetch", "mr_result_device", "mr_release",
           "mr_submit", "mr_poll", "mr_sync", "mr_bytes_in_use", "mr_job_elapsed_ms", "mr_job_kernel_ms",
           "mr_kernel_launches",
           "mr_status_str", "mr_last_error", "mr_wordcount_noalloc", "mr_rerun", "mr_get_tuning", "mr_simdh_hash",
           "mr_set_option")
SIMDH_PADDING, SIMDH_STREAM, SIMDH_WIDE = range(3)
NOALLOC_WC_SLOTS = 131072
FLAG_TIMING = 1
FLAG_AUTOTUNE = 2
# diagnostic options (mr_set_option)
OPT_WAIT_POLLS, OPT_KM_GRID_CAP, OPT_KM_STOP_COPIES = range(3)
OPT_DEFAULT = 2 ** 64 - 1


class MRError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__("%s failed: %s%s" % (what, _status_str(status), (" [%s]" % detail) if detail else ""))


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class _Config(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("hbm_budget", ctypes.c_uint64), ("alloc", _ALLOC_FN), ("free", _FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("arr_tile", ctypes.c_uint64), ("wc_tile", ctypes.c_uint64), ("hist_global_below", ctypes.c_uint64),
                ("best_ms", ctypes.c_float), ("tuned", ctypes.c_uint32)]


class _JobDesc(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("kind", ctypes.c_int), ("input", ctypes.c_void_p),
                ("input_bytes", ctypes.c_uint64), ("input_on_device", ctypes.c_int), ("container", ctypes.c_int),
                ("km_dims", ctypes.c_uint32), ("km_k", ctypes.c_uint32), ("km_iters", ctypes.c_uint32),
                ("km_init", ctypes.c_void_p), ("km_precision", ctypes.c_uint32), ("wc_slots", ctypes.c_uint64),
                ("hist_bins", ctypes.c_uint32), ("bloom_kmer", ctypes.c_uint32), ("bloom_hashes", ctypes.c_uint32),
                ("bloom_bits", ctypes.c_uint64), ("wc_pipelined", ctypes.c_uint32)]


_lib = None
_lib_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile libmrgb.so for sm_103a (in-tree) and load it."""
    path = _build_lib(force=force)
    load()
    return path


def load():
    """Load the built library; raises if it has not been built."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libmrgb.so is not built: call paper_1309_0215_gb300.build() first")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, u64 = ctypes.c_void_p, ctypes.c_uint64
        st = ctypes.c_int
        lib.mr_create.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(vp)]
        lib.mr_create.restype = st
        lib.mr_destroy.argtypes = [vp]
        lib.mr_destroy.restype = None
        lib.mr_add_job.argtypes = [vp, ctypes.POINTER(_JobDesc), ctypes.POINTER(u64)]
        lib.mr_add_job.restype = st
        lib.mr_submit.argtypes = [vp, ctypes.POINTER(_JobDesc), ctypes.POINTER(u64)]
        lib.mr_submit.restype = st
        lib.mr_run.argtypes = [vp, ctypes.c_int]
        lib.mr_run.restype = st
        lib.mr_fetch.argtypes = [vp, u64, vp, u64, ctypes.POINTER(u64)]
        lib.mr_fetch.restype = st
        lib.mr_result_device.argtypes = [vp, u64, ctypes.POINTER(vp), ctypes.POINTER(u64)]
        lib.mr_result_device.restype = st
        lib.mr_release.argtypes = [vp, u64]
        lib.mr_release.restype = st
        lib.mr_poll.argtypes = [vp, u64]
        lib.mr_poll.restype = st
        lib.mr_sync.argtypes = [vp]
        lib.mr_sync.restype = st
        lib.mr_bytes_in_use.argtypes = [vp]
        lib.mr_bytes_in_use.restype = u64
        lib.mr_set_option.argtypes = [vp, ctypes.c_int, u64]
        lib.mr_set_option.restype = st
        lib.mr_job_elapsed_ms.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_float)]
        lib.mr_job_elapsed_ms.restype = st
        lib.mr_job_kernel_ms.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint32)]
        lib.mr_job_kernel_ms.restype = st
        lib.mr_kernel_launches.argtypes = [vp]
        lib.mr_kernel_launches.restype = u64
        lib.mr_rerun.argtypes = [vp]
        lib.mr_rerun.restype = st
        lib.mr_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        lib.mr_get_tuning.restype = st
        lib.mr_wordcount_noalloc.argtypes = [vp, u64, vp, u64, ctypes.POINTER(u64), vp]
        lib.mr_wordcount_noalloc.restype = st
        lib.mr_simdh_hash.argtypes = [vp, u64, vp, vp, u64, ctypes.c_int, vp, vp]
        lib.mr_simdh_hash.restype = st
        lib.mr_status_str.argtypes = [ctypes.c_int]
        lib.mr_status_str.restype = ctypes.c_char_p
        lib.mr_last_error.argtypes = []
        lib.mr_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _status_str(s: int) -> str:
    try:
        return load().mr_status_str(s).decode()
    except Exception:
        return "status %d" % s


def _check(status: int, what: str):
    if status != MR_OK:
        detail = ""
        if status == MR_ECUDA:
            detail = load().mr_last_error().decode(errors="replace")
        raise MRError(status, what, detail)


def _as_input(data):
    """Return (address, nbytes, on_device, keepalive) for a tensor / array / bytes."""
    try:
        import torch
        if isinstance(data, torch.Tensor):
            if not data.is_contiguous():
                data = data.contiguous()
            return data.data_ptr(), data.numel() * data.element_size(), bool(data.is_cuda), data
    except ImportError:  # pragma: no cover
        pass
    if isinstance(data, (bytes, bytearray, memoryview)):
        arr = np.frombuffer(bytes(data), dtype=np.uint8)
    else:
        arr = np.ascontiguousarray(data)
    return (arr.ctypes.data if arr.size else None), arr.nbytes, False, arr


class Context:
    """One library context: a device, a stream and the jobs queued on it."""

    def __init__(self, device: Optional[int] = None, stream=None, hbm_budget: int = 0,
                 use_torch_allocator: bool = True, timing: bool = False, autotune: bool = False,
                 allocator=None):
        """allocator: optional (alloc, free) pair of Python callables used as
        the library's device allocator hooks in place of torch's caching
        allocator: alloc(nbytes) returns a device address or 0 on failure,
        free(address) releases one."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the map/reduce library runs only on the GPU")
        self._lib = load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        cfg = _Config()
        cfg.struct_size = ctypes.sizeof(_Config)
        cfg.device = self.device
        cfg.cuda_stream = ctypes.c_void_p(stream.cuda_stream)
        cfg.hbm_budget = int(hbm_budget)
        cfg.flags = (FLAG_TIMING if timing else 0) | (FLAG_AUTOTUNE if autotune else 0)
        self._cb = None
        if allocator is not None:
            u_alloc, u_free = allocator

            def _alloc(_user, n):
                try:
                    return u_alloc(int(n)) or None
                except Exception:
                    return None

            def _free(_user, p):
                u_free(p)

            self._cb = (_ALLOC_FN(_alloc), _FREE_FN(_free))
            cfg.alloc, cfg.free = self._cb
        elif use_torch_allocator:
            dev, sptr = self.device, stream.cuda_stream

            def _alloc(_user, n):
                try:
                    return torch.cuda.caching_allocator_alloc(int(n), dev, sptr)
                except Exception:
                    return None

            def _free(_user, p):
                torch.cuda.caching_allocator_delete(p)

            self._cb = (_ALLOC_FN(_alloc), _FREE_FN(_free))
            cfg.alloc, cfg.free = self._cb
        self._h = ctypes.c_void_p()
        _check(self._lib.mr_create(ctypes.byref(cfg), ctypes.byref(self._h)), "mr_create")
        self._keep = {}

    # ------------------------------------------------------------------ jobs
    def _desc(self, kind, data, container, km_dims, km_k, km_iters, km_init, km_precision, wc_slots,
              hist_bins=0, bloom_kmer=0, bloom_hashes=0, bloom_bits=0, wc_pipelined=0):
        addr, nbytes, on_dev, keep = _as_input(data)
        d = _JobDesc()
        d.struct_size = ctypes.sizeof(_JobDesc)
        d.kind = int(kind)
        d.input = addr
        d.input_bytes = nbytes
        d.input_on_device = int(on_dev)
        d.container = int(container)
        d.km_dims, d.km_k, d.km_iters = int(km_dims), int(km_k), int(km_iters)
        keep_init = None
        if km_init is not None:
            iaddr, _, ion_dev, keep_init = _as_input(km_init)
            if ion_dev != on_dev:
                raise ValueError("km_init must live in the same memory space as the input")
            d.km_init = iaddr
        d.km_precision = int(km_precision)
        d.wc_slots = int(wc_slots)
        d.hist_bins = int(hist_bins)
        d.bloom_kmer, d.bloom_hashes, d.bloom_bits = int(bloom_kmer), int(bloom_hashes), int(bloom_bits)
        d.wc_pipelined = int(wc_pipelined)
        return d, (keep, keep_init) if on_dev else None

    def add_job(self, kind, data, container=C_AUTO, km_dims=0, km_k=0, km_iters=0, km_init=None,
            km_precision=KM_FP32, wc_slots=0, **params) -> int:
        """params: hist_bins (large-key histogram); bloom_kmer, bloom_hashes,
        bloom_bits (Bloom filter); wc_pipelined (word count)."""
        d, keep = self._desc(kind, data, container, km_dims, km_k, km_iters, km_init, km_precision, wc_slots,
                             **params)
        jid = ctypes.c_uint64()
        _check(self._lib.mr_add_job(self._h, ctypes.byref(d), ctypes.byref(jid)), "mr_add_job")
        if keep is not None:
            self._keep[jid.value] = keep  # device inputs are borrowed until release
        return jid.value

    def submit(self, kind, data, container=C_AUTO, km_dims=0, km_k=0, km_iters=0, km_init=None,
            km_precision=KM_FP32, wc_slots=0, **params) -> int:
        """params: hist_bins (large-key histogram); bloom_kmer, bloom_hashes,
        bloom_bits (Bloom filter); wc_pipelined (word count)."""
        d, keep = self._desc(kind, data, container, km_dims, km_k, km_iters, km_init, km_precision, wc_slots,
                             **params)
        jid = ctypes.c_uint64()
        _check(self._lib.mr_submit(self._h, ctypes.byref(d), ctypes.byref(jid)), "mr_submit")
        if keep is not None:
            self._keep[jid.value] = keep
        return jid.value

    def run(self, mode=RUN_PLAIN):
        _check(self._lib.mr_run(self._h, int(mode)), "mr_run")

    def fetch(self, job: int) -> bytes:
        need = ctypes.c_uint64()
        _check(self._lib.mr_fetch(self._h, job, None, 0, ctypes.byref(need)), "mr_fetch(size)")
        buf = np.empty(max(int(need.value), 1), dtype=np.uint8)
        _check(self._lib.mr_fetch(self._h, job, buf.ctypes.data, buf.nbytes, ctypes.byref(need)), "mr_fetch")
        return buf[: int(need.value)].tobytes()

    def fetch_into(self, job: int, buf: np.ndarray) -> int:
        need = ctypes.c_uint64()
        _check(self._lib.mr_fetch(self._h, job, buf.ctypes.data, buf.nbytes, ctypes.byref(need)), "mr_fetch")
        return int(need.value)

    def result_device(self, job: int):
        p, n = ctypes.c_void_p(), ctypes.c_uint64()
        _check(self._lib.mr_result_device(self._h, job, ctypes.byref(p), ctypes.byref(n)), "mr_result_device")
        return p.value, n.value

    def poll(self, job: int) -> bool:
        s = self._lib.mr_poll(self._h, job)
        if s == MR_ENOTREADY:
            return False
        _check(s, "mr_poll")
        return True

    def release(self, job: int):
        _check(self._lib.mr_release(self._h, job), "mr_release")
        self._keep.pop(job, None)

    def sync(self):
        _check(self._lib.mr_sync(self._h), "mr_sync")

    def rerun(self):
        """Re-run the last batched mr_run in place (relaunches its CUDA graph)."""
        _check(self._lib.mr_rerun(self._h), "mr_rerun")

    def tuning(self) -> dict:
        t = Tuning()
        _check(self._lib.mr_get_tuning(self._h, ctypes.byref(t)), "mr_get_tuning")
        return {"arr_tile": t.arr_tile, "wc_tile": t.wc_tile, "hist_global_below": t.hist_global_below,
                "best_ms": t.best_ms, "tuned": bool(t.tuned)}

    def elapsed_ms(self, job: int) -> float:
        ms = ctypes.c_float()
        _check(self._lib.mr_job_elapsed_ms(self._h, job, ctypes.byref(ms)), "mr_job_elapsed_ms")
        return float(ms.value)

    def kernel_ms(self, job: int):
        """(summed ms, launches) of the job's main-kernel launches (timing contexts, plain jobs)."""
        ms, n = ctypes.c_float(), ctypes.c_uint32()
        _check(self._lib.mr_job_kernel_ms(self._h, job, ctypes.byref(ms), ctypes.byref(n)), "mr_job_kernel_ms")
        return float(ms.value), int(n.value)

    def set_option(self, opt: int, value: int):
        """Diagnostic option (OPT_*; include/mr.h mr_option) for jobs launched from now on."""
        _check(self._lib.mr_set_option(self._h, int(opt), int(value)), "mr_set_option")

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.mr_kernel_launches(self._h))

    @property
    def bytes_in_use(self) -> int:
        return int(self._lib.mr_bytes_in_use(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.mr_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ----------------------------------------------------------- one-shot helpers
_default = {}


def _ctx() -> Context:
    import torch
    dev = torch.cuda.current_device()
    c = _default.get(dev)
    if c is None:
        c = _default[dev] = Context(dev)
    return c


def _one(kind, data, **kw) -> bytes:
    c = _ctx()
    j = c.add_job(kind, data, **kw)
    c.run()
    try:
        return c.fetch(j)
    finally:
        c.release(j)


def wordcount(text, wc_slots: int = 0, pipelined: bool = False) -> bytes:
    """Word count; returns the serialized result (see include/mr.h)."""
    return _one(WORDCOUNT, text, wc_slots=wc_slots, wc_pipelined=int(pipelined))


def hist_rgb8(px, container=C_AUTO) -> np.ndarray:
    return np.frombuffer(_one(HIST_RGB8, px, container=container), dtype=np.uint64).copy()


def linreg_i8(xy) -> np.ndarray:
    return np.frombuffer(_one(LINREG_I8, xy), dtype=np.int64).copy()


def simdh_hash(text, tok_off, tok_len, method: int = SIMDH_STREAM, out=None, stream=None):
    """FNV-1a 64 of each token (device tensors: text uint8, tok_off / tok_len
    int32 or uint32 views); returns the uint64 hashes as an int64 device
    tensor (launched on `stream`, default: torch's current stream)."""
    import torch
    lib = load()
    ntok = int(tok_off.numel())
    if out is None:
        out = torch.empty(ntok, dtype=torch.int64, device=text.device)
    s = stream if stream is not None else torch.cuda.current_stream(text.device)
    st = lib.mr_simdh_hash(text.data_ptr() if text.numel() else None, int(text.numel()),
                           tok_off.data_ptr() if ntok else None, tok_len.data_ptr() if ntok else None, ntok,
                           int(method), out.data_ptr() if ntok else None, ctypes.c_void_p(s.cuda_stream))
    _check(st, "mr_simdh_hash")
    return out


def hist_u32(keys, nbins: int, container=C_AUTO) -> np.ndarray:
    """uint64 [nbins + 1]: count of each key < nbins, then the out-of-range count."""
    return np.frombuffer(_one(HIST_U32, keys, container=container, hist_bins=nbins), dtype=np.uint64).copy()


def bloom_dna(seq, kmer: int, bits: int, hashes: int) -> np.ndarray:
    """Bloom-filter bytes (ceil(bits / 8)) of every all-ACGT window of kmer bases."""
    raw = _one(BLOOM_DNA, seq, bloom_kmer=kmer, bloom_bits=bits, bloom_hashes=hashes)
    return np.frombuffer(raw, dtype=np.uint8).copy()


def kmeans(x, init, iters: int, precision: int = KM_FP32):
    """(centroids float32 [K, D], assignments int32 [N], stats uint64 [4])."""
    n, d = x.shape
    k = init.shape[0]
    raw = _one(KMEANS_F32, x, km_dims=d, km_k=k, km_iters=iters, km_init=init, km_precision=precision)
    return split_kmeans_result(raw, n, d, k)


def split_kmeans_result(raw: bytes, n: int, d: int, k: int):
    """Decode the k-means result layout: f32 [K*D] | i32 [N] | pad to 8 | u64 [4]."""
    cb = k * d * 4
    cent = np.frombuffer(raw[:cb], dtype=np.float32).reshape(k, d).copy()
    assign = np.frombuffer(raw[cb: cb + 4 * n], dtype=np.int32).copy()
    off = (cb + 4 * n + 7) & ~7
    stats = np.frombuffer(raw[off: off + 32], dtype=np.uint64).copy()
    return cent, assign, stats
