"""GPU: failure paths, made to happen on the host or by a wait that nothing
satisfies — never by a GPU fault.

* Bounded device waits: with the context's wait limit set to 0 polls (or a
  tensor-core pass whose bulk-copy thread stops staging tiles, so the waits
  behind the missing tiles run out while earlier tiles are still in flight),
  the kernel gives up, drains what it started, frees its tensor memory and
  reports; mr_fetch returns MR_ETIMEOUT.  A normal job on the same context
  afterwards must still equal the oracle, so the context stays usable.
* Allocation failure: an allocator hook that returns NULL gives MR_ENOMEM,
  frees whatever the call had already taken, and a failed run leaves its jobs
  pending for the next run.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel_err(c, ref):
    num = np.linalg.norm(c.astype(np.float64) - ref.astype(np.float64), axis=1)
    den = np.maximum(np.linalg.norm(ref.astype(np.float64), axis=1), 1.0)
    return float((num / den).max())


def _km_job(mr, ctx, x, init, iters, precision):
    import torch
    n, d = x.shape
    return ctx.add_job(mr.KMEANS_F32, torch.from_numpy(x).cuda(), km_dims=d, km_k=init.shape[0], km_iters=iters,
                       km_init=torch.from_numpy(init).cuda(), km_precision=precision)


def _fetch_status(mr, ctx, j):
    try:
        return mr.MR_OK, ctx.fetch(j)
    except mr.MRError as e:
        return e.status, None


def _km_check(mr, ctx, x, init, iters, precision):
    c_ref, a_ref = oracle.kmeans(x, init, iters)
    j = _km_job(mr, ctx, x, init, iters, precision)
    ctx.run()
    c, a, st = mr.split_kmeans_result(ctx.fetch(j), x.shape[0], x.shape[1], init.shape[0])
    ctx.release(j)
    assert np.array_equal(a, a_ref)
    assert _rel_err(c, c_ref) <= TOL
    assert int(st[3]) == 0


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_kmeans_wait_gives_up_then_context_recovers(mr, precision):
    """0 polls: the first bounded wait of the pipelined kernels gives up (the
    tensor-core pass for precision 1 and 2; for 0 the bulk-copy update, which
    runs for D > 64 with rows of a multiple of 4 floats: D <= 64 takes the
    window-sorted update)."""
    d = 96 if precision == 0 else 64
    x, _, _ = synth.kmeans_points(12_000, d, 64, seed=61 + precision)
    init = synth.kmeans_init(x, 64, seed=62)
    ctx = mr.Context()
    ctx.set_option(mr.OPT_WAIT_POLLS, 0)
    j = _km_job(mr, ctx, x, init, 2, precision)
    ctx.run()
    st, _ = _fetch_status(mr, ctx, j)
    assert st == mr.MR_ETIMEOUT
    ctx.release(j)
    ctx.set_option(mr.OPT_WAIT_POLLS, mr.OPT_DEFAULT)
    _km_check(mr, ctx, x, init, 2, precision)
    ctx.close()


def test_kmeans_fp32_window_path_has_no_waits(mr):
    """The FP32 pass and the window-sorted update (D <= 64) wait on nothing,
    so a wait limit of 0 polls changes nothing there: the job completes and
    equals the oracle."""
    x, _, _ = synth.kmeans_points(12_000, 48, 64, seed=64)
    init = synth.kmeans_init(x, 64, seed=62)
    ctx = mr.Context()
    ctx.set_option(mr.OPT_WAIT_POLLS, 0)
    _km_check(mr, ctx, x, init, 2, 0)
    ctx.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_kmeans_tensor_core_timeout_with_work_in_flight(mr, precision):
    """The bulk-copy thread of every CTA stops after 5 of its ~40 tiles: the
    converters' wait for tile 5 runs out while the MMAs and epilogue of the
    earlier tiles are still running; the CTA must drain them before it frees
    TMEM.  Then the same context computes the job correctly."""
    x, _, _ = synth.kmeans_points(20_000, 64, 256, seed=63)
    init = synth.kmeans_init(x, 256, seed=64)
    ctx = mr.Context()
    ctx.set_option(mr.OPT_KM_GRID_CAP, 4)
    ctx.set_option(mr.OPT_KM_STOP_COPIES, 5)
    ctx.set_option(mr.OPT_WAIT_POLLS, 1 << 14)
    j = _km_job(mr, ctx, x, init, 2, precision)
    ctx.run()
    st, _ = _fetch_status(mr, ctx, j)
    assert st == mr.MR_ETIMEOUT
    ctx.release(j)
    ctx.set_option(mr.OPT_KM_STOP_COPIES, 0)
    ctx.set_option(mr.OPT_WAIT_POLLS, mr.OPT_DEFAULT)
    _km_check(mr, ctx, x, init, 2, precision)   # still capped: many tiles per CTA
    ctx.close()


def test_pipelined_wordcount_wait_gives_up_then_recovers(mr):
    import torch
    text, _, _ = synth.wc_text(2 << 20, nwords=20000, seed=65)
    d = torch.from_numpy(text).cuda()
    ctx = mr.Context()
    ctx.set_option(mr.OPT_WAIT_POLLS, 0)
    j = ctx.add_job(mr.WORDCOUNT, d, wc_pipelined=1)
    ctx.run()
    st, _ = _fetch_status(mr, ctx, j)
    assert st == mr.MR_ETIMEOUT
    ctx.release(j)
    ctx.set_option(mr.OPT_WAIT_POLLS, mr.OPT_DEFAULT)
    j = ctx.add_job(mr.WORDCOUNT, d, wc_pipelined=1)
    ctx.run()
    assert ctx.fetch(j) == oracle.wordcount(text)
    ctx.release(j)
    ctx.close()


def test_set_option_rejects_bad_values(mr):
    ctx = mr.Context()
    for opt, val in ((7, 1), (mr.OPT_WAIT_POLLS, (1 << 40) + 1), (mr.OPT_KM_GRID_CAP, 1 << 32)):
        with pytest.raises(mr.MRError) as e:
            ctx.set_option(opt, val)
        assert e.value.status == mr.MR_EINVAL
    ctx.close()


class _Alloc:
    """Device allocator hooks (torch's caching allocator underneath) that fail
    once `fail_after` allocations have been made; tracks what is live."""

    def __init__(self):
        import torch
        self.dev = torch.cuda.current_device()
        self.stream = torch.cuda.current_stream().cuda_stream
        self.calls = 0
        self.fail_after = None
        self.live = {}

    def alloc(self, n):
        import torch
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            return 0
        p = torch.cuda.caching_allocator_alloc(n, self.dev, self.stream)
        self.live[p] = n
        return p

    def free(self, p):
        import torch
        self.live.pop(p)
        torch.cuda.caching_allocator_delete(p)


def test_allocation_failure_gives_enomem_without_leaks(mr):
    """Every allocation point of mr_add_job fails once (host inputs: the input
    copy, then the job's slab): MR_ENOMEM, nothing held afterwards."""
    text, _, _ = synth.wc_text(1 << 20, nwords=3000, seed=66)
    x, _, _ = synth.kmeans_points(4000, 16, 8, seed=67)
    init = synth.kmeans_init(x, 8, seed=68)
    px = synth.hist_rgb8(30_001, seed=69)
    cases = [
        (mr.WORDCOUNT, text, {}, lambda got: got == oracle.wordcount(text)),
        (mr.KMEANS_F32, x, dict(km_dims=16, km_k=8, km_iters=2, km_init=init),
         lambda got: np.array_equal(mr.split_kmeans_result(got, 4000, 16, 8)[1], oracle.kmeans(x, init, 2)[1])),
        (mr.HIST_RGB8, px, {}, lambda got: got == oracle.hist_rgb8(px).tobytes()),
    ]
    al = _Alloc()
    ctx = mr.Context(allocator=(al.alloc, al.free))
    for kind, data, kw, ok in cases:
        for k in range(2):
            base_live, base_bytes = dict(al.live), ctx.bytes_in_use
            al.fail_after = al.calls + k
            try:
                j = ctx.add_job(kind, data, **kw)
            except mr.MRError as e:
                assert e.status == mr.MR_ENOMEM
                assert al.live == base_live and ctx.bytes_in_use == base_bytes
                continue
            al.fail_after = None
            ctx.run()
            assert ok(ctx.fetch(j))
            ctx.release(j)
        al.fail_after = None
        j = ctx.add_job(kind, data, **kw)
        ctx.run()
        assert ok(ctx.fetch(j))
        ctx.release(j)
    assert ctx.bytes_in_use == 0
    ctx.close()
    assert al.live == {}


def test_batched_run_allocation_failure_keeps_jobs_pending(mr):
    """The batch's scratch cannot be allocated: mr_run returns MR_ENOMEM, the
    jobs stay pending, and the next mr_run computes them."""
    import torch
    text, _, _ = synth.wc_text(1 << 20, nwords=3000, seed=70)
    px = synth.hist_rgb8(50_000, seed=71)
    xy = synth.linreg_i8(40_000, seed=72)
    al = _Alloc()
    ctx = mr.Context(allocator=(al.alloc, al.free))
    ids = [ctx.add_job(mr.WORDCOUNT, torch.from_numpy(text).cuda()),
           ctx.add_job(mr.HIST_RGB8, torch.from_numpy(px).cuda()),
           ctx.add_job(mr.LINREG_I8, torch.from_numpy(xy).cuda())]
    al.fail_after = al.calls
    with pytest.raises(mr.MRError) as e:
        ctx.run(mr.RUN_BATCHED)
    assert e.value.status == mr.MR_ENOMEM
    assert not ctx.poll(ids[0])
    al.fail_after = None
    ctx.run(mr.RUN_BATCHED)
    assert ctx.fetch(ids[0]) == oracle.wordcount(text)
    assert ctx.fetch(ids[1]) == oracle.hist_rgb8(px).tobytes()
    assert ctx.fetch(ids[2]) == oracle.linreg_i8(xy).tobytes()
    for j in ids:
        ctx.release(j)
    ctx.close()
    assert al.live == {}
