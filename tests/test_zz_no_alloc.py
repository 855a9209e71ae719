"""mr_wordcount_noalloc: word count for callers that cannot allocate device
memory (for example a host program that reserves the GPU's memory for its own
pool, or a latency-critical loop that cannot afford cudaMalloc's implicit
synchronisation).  Its scratch is a fixed device array inside the library.

Called through the C ABI and compared, byte for byte, with the regular
word-count entry point (mr_add_job / mr_run / mr_fetch) and with the CPU
oracle on two calls in a row
with different inputs, so a second call cannot pass on the first call's left-
over table contents.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _call(mr, d_in, cap_extra=0):
    import torch
    lib = mr.load()
    n = d_in.numel()
    cap = 16 + 24 * mr.NOALLOC_WC_SLOTS + n + cap_extra
    d_out = torch.empty(max(cap, 1), dtype=torch.uint8, device="cuda")
    nbytes = ctypes.c_uint64(0)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.mr_wordcount_noalloc(d_in.data_ptr() if n else None, n, d_out.data_ptr(), cap, ctypes.byref(nbytes),
                                  ctypes.c_void_p(stream))
    return st, d_out, nbytes.value


def test_noalloc_matches_regular_entry_point_twice(mr):
    import torch
    inputs = [synth.wc_text(1 << 20, nwords=5000, seed=123)[0],
              synth.wc_text(3 << 19, nwords=20000, seed=456)[0]]
    for text in inputs:
        d_in = torch.from_numpy(text).cuda()
        expect = mr.wordcount(d_in)
        st, d_out, nbytes = _call(mr, d_in)
        assert st == mr.MR_OK
        assert nbytes == len(expect)
        got = d_out[:nbytes].cpu().numpy().tobytes()
        assert got == expect
        # and with the CPU oracle, so that code both entry points share
        # (the merge and sort after the map pass) is checked independently
        assert got == oracle.wordcount(text)


def test_noalloc_rejects_small_output_and_reports_overflow(mr):
    import torch
    d_in = torch.from_numpy(np.frombuffer(b"a b c", dtype=np.uint8).copy()).cuda()
    st, _, _ = _call(mr, d_in, cap_extra=-1)
    assert st == mr.MR_EINVAL
    many = b" ".join(b"%x" % i for i in range(300_000))  # more distinct words than the table holds
    d_many = torch.from_numpy(np.frombuffer(many, dtype=np.uint8).copy()).cuda()
    st, _, _ = _call(mr, d_many)
    assert st == mr.MR_EOVERFLOW
    # the next call still works: each call clears the shared scratch first
    text = synth.wc_text(1 << 18, nwords=1000, seed=9)[0]
    d_t = torch.from_numpy(text).cuda()
    st, d_out, nbytes = _call(mr, d_t)
    assert st == mr.MR_OK
    assert d_out[:nbytes].cpu().numpy().tobytes() == mr.wordcount(d_t)
