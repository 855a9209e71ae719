"""GPU parity: k-means (array container keyed by cluster id).

Assignments must equal the FP64 oracle's exactly; centroids must be within
1e-5 relative (per centroid, ||c - c64|| / max(||c64||, 1)) of the oracle's.
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(mr, x, init, iters, precision=0, on_device=True):
    if on_device:
        return mr.kmeans(_dev(x), _dev(init), iters, precision)
    return mr.kmeans(x, init, iters, precision)


def _assign_all(x, c):
    """The oracle's FP64 assignment of every point, computed serially on row
    slices by a pool of host threads (the oracle call releases the GIL)."""
    import concurrent.futures as cf
    import os
    nth = max(1, min(32, os.cpu_count() or 1))
    step = (x.shape[0] + nth - 1) // nth
    parts = [x[i: i + step] for i in range(0, x.shape[0], step)]
    with cf.ThreadPoolExecutor(nth) as ex:
        return np.concatenate(list(ex.map(lambda p: oracle.kmeans_assign(p, c), parts)))


def _run_ctx(mr, ctx, dx, cur, iters, precision):
    n, d = dx.shape
    j = ctx.add_job(mr.KMEANS_F32, dx, km_dims=d, km_k=cur.shape[0], km_iters=iters, km_init=_dev(cur),
                    km_precision=precision)
    ctx.run()
    out = mr.split_kmeans_result(ctx.fetch(j), n, d, cur.shape[0])
    ctx.release(j)
    return out


@pytest.mark.parametrize("n,d,k,iters", [
    (20_000, 64, 256, 3),   # the workload's shape, reduced N
    (5_001, 37, 50, 2),     # ragged dims / tiles
    (3_000, 100, 20, 2),    # D > 64: chunked dimensions
    (4_000, 16, 300, 2),    # K > 256: chunked centroids
    (6_000, 128, 260, 2),   # K*D sums too large for shared memory: the sorted update
    (9_001, 64, 300, 2),    # window-sorted update with K not a multiple of 32
    (5_000, 64, 1, 2),      # window-sorted update, one cluster
    (6_000, 8, 3_000, 2),   # K x D sums fit, but not beside the window buffers: the row-pipelined update
    (3_001, 67, 20, 2),     # D > 64 and not a multiple of 4: the plain local-array update
    (777, 3, 1, 2),         # K = 1: the global mean
    (64, 8, 64, 1),         # every point its own centroid
])
def test_kmeans_fp32_vs_oracle(mr, n, d, k, iters):
    x, _, _ = synth.kmeans_points(n, d, max(1, min(k, 256)), seed=n + d + k)
    init = synth.kmeans_init(x, k, seed=n)
    c_ref, a_ref = oracle.kmeans(x, init, iters)
    c, a, stats = _run(mr, x, init, iters)
    assert np.array_equal(a, a_ref)
    assert _rel_err(c, c_ref) <= TOL
    assert int(stats[2]) == iters


@pytest.mark.parametrize("precision", [0, 1])
def test_kmeans_points_not_16_byte_aligned(mr, precision):
    """Points 4 bytes into a buffer: no bulk copies and no 8-byte loads; the
    window-sorted update reads them with 4-byte loads."""
    import torch
    x, _, _ = synth.kmeans_points(5000, 64, 32, seed=51)
    init = synth.kmeans_init(x, 32, seed=52)
    buf = torch.zeros(x.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(x.ravel()).cuda()
    c_ref, a_ref = oracle.kmeans(x, init, 3)
    c, a, stats = mr.kmeans(buf[1:].view(5000, 64), _dev(init), 3, precision)
    assert np.array_equal(a, a_ref)
    assert _rel_err(c, c_ref) <= TOL


def test_kmeans_host_inputs(mr):
    x, _, _ = synth.kmeans_points(4096, 32, 64, seed=5)
    init = synth.kmeans_init(x, 64, seed=6)
    c_ref, a_ref = oracle.kmeans(x, init, 2)
    c, a, _ = _run(mr, x, init, 2, on_device=False)
    assert np.array_equal(a, a_ref) and _rel_err(c, c_ref) <= TOL


def test_kmeans_exact_ties_take_lowest_index(mr):
    x, _, _ = synth.kmeans_points(6000, 8, 16, seed=21)
    init = synth.kmeans_init(x, 16, seed=22)
    init[9] = init[4]     # duplicate centroid: index 4 must win every tie
    init[15] = init[0]
    c_ref, a_ref = oracle.kmeans(x, init, 1)
    c, a, stats = _run(mr, x, init, 1)
    assert np.array_equal(a, a_ref)
    assert not np.any(a == 9) and not np.any(a == 15)
    assert int(stats[1]) > 0  # the tied points were re-checked in FP64
    assert _rel_err(c, c_ref) <= TOL


@pytest.mark.parametrize("precision,d", [(0, 64), (1, 64), (0, 8)])
def test_kmeans_all_centroids_tied(mr, precision, d):
    """Every centroid the same point: every distance ties, every point goes
    to the FP64 stage with all 256 centroids as candidates (in chunks of the
    stage's product scratch: 128 at D = 64, 256 at D = 8), and index 0 wins
    every tie, as in the definition."""
    x, _, _ = synth.kmeans_points(3000, d, 16, seed=81 + d)
    init = np.repeat(x[7:8], 256, axis=0)
    a_ref = oracle.kmeans_assign(x, init)
    c_ref, _ = oracle.kmeans_update(x, a_ref, init)
    c, a, st = _run(mr, x, init, 1, precision)
    assert np.array_equal(a, a_ref) and not np.any(a)
    assert int(st[1]) >= 2999  # (a point equal to the centroid may be decided earlier)
    assert _rel_err(c, c_ref) <= TOL


def test_kmeans_empty_cluster_keeps_centroid(mr):
    x, _, _ = synth.kmeans_points(3000, 4, 3, seed=31)
    init = np.concatenate([x[:3], np.full((1, 4), 1e4, dtype=np.float32)])
    c_ref, a_ref = oracle.kmeans(x, init, 3)
    c, a, _ = _run(mr, x, init, 3)
    assert np.array_equal(a, a_ref)
    assert np.array_equal(c[3], init[3])
    assert _rel_err(c, c_ref) <= TOL


def test_kmeans_teacher_forced_iterations(mr):
    """Each GPU iteration, started from the oracle's centroids, reproduces the
    oracle's assignment exactly and its update within tolerance."""
    x, _, _ = synth.kmeans_points(30_000, 64, 256, seed=41)
    cur = synth.kmeans_init(x, 256, seed=42)
    for _ in range(4):
        a_ref = oracle.kmeans_assign(x, cur)
        c_ref, _ = oracle.kmeans_update(x, a_ref, cur)
        c, a, _ = _run(mr, x, cur, 1)
        assert np.array_equal(a, a_ref)
        assert _rel_err(c, c_ref) <= TOL
        cur = c_ref


def test_kmeans_rejects_bad_args(mr):
    x = np.zeros((10, 4), dtype=np.float32)
    with pytest.raises(mr.MRError):
        mr.kmeans(x, np.zeros((2, 4), dtype=np.float32), 0)
    c = mr.Context()
    with pytest.raises(mr.MRError):
        c.add_job(mr.KMEANS_F32, x, km_dims=3, km_k=2, km_iters=1, km_init=np.zeros((2, 3), dtype=np.float32))
    c.close()


@pytest.mark.slow
def test_kmeans_full_size_fp32(mr):
    """4M x 64 points, K = 256, 10 iterations: determinism across a split run;
    the tenth iteration's assignment of EVERY point equals the FP64 oracle's
    on the GPU's ninth centroids, for the FP32 path and both tensor-core
    paths (whose persistent CTAs run ~216 tiles each here); and the final
    update equals the oracle's FP64 update within tolerance."""
    import torch
    x, _, _ = synth.kmeans_points(4 << 20, 64, 256)
    init = synth.kmeans_init(x, 256)
    dx = torch.from_numpy(x).cuda()
    c10, a10, _ = mr.kmeans(dx, _dev(init), 10)
    c9, _, _ = mr.kmeans(dx, _dev(init), 9)
    c10b, a10b, _ = mr.kmeans(dx, _dev(c9), 1)
    assert np.array_equal(c10, c10b) and np.array_equal(a10, a10b)
    a_ref = _assign_all(x, c9)
    assert np.array_equal(a10, a_ref)
    for precision in (1, 2):
        _, a_tc, st = mr.kmeans(dx, _dev(c9), 1, precision)
        assert np.array_equal(a_tc, a_ref), precision
        assert int(st[3]) == 0
    c_upd, _ = oracle.kmeans_update(x, a10, c9)
    assert _rel_err(c10, c_upd) <= TOL


@pytest.mark.parametrize("precision,d", [(0, 64), (1, 64), (2, 64), (1, 21)])
def test_kmeans_many_tiles_per_cta_teacher_forced(mr, precision, d):
    """The persistent kernels capped at 4 CTAs: each tensor-core CTA runs ~39
    tiles of 128 points (its copy ring, operand stages, TMEM accumulators and
    key hand-off all wrap many times; D = 21: the converters' own row loads),
    each FP32 CTA ~78 tiles of 64, and each update
    CTA its ~5,000 points in two windows.  Every assignment of every
    iteration, started from the oracle's centroids, equals the oracle's."""
    x, _, _ = synth.kmeans_points(20_000, d, 256, seed=45 + precision)
    cur = synth.kmeans_init(x, 256, seed=46)
    dx = _dev(x)
    ctx = mr.Context()
    ctx.set_option(mr.OPT_KM_GRID_CAP, 4)
    for _ in range(3):
        a_ref = oracle.kmeans_assign(x, cur)
        c_ref, _ = oracle.kmeans_update(x, a_ref, cur)
        c, a, st = _run_ctx(mr, ctx, dx, cur, 1, precision)
        assert np.array_equal(a, a_ref)
        assert _rel_err(c, c_ref) <= TOL
        assert int(st[3]) == 0
        cur = c_ref
    ctx.close()


@pytest.mark.parametrize("d,k", [(64, 256), (64, 17), (64, 380), (48, 256), (37, 17), (33, 100), (8, 64), (1, 5)])
def test_kmeans_window_update_many_windows(mr, d, k):
    """The update for D <= 64 sorts each window of 8,192 points (4,096 when
    the K x D sums leave too little shared memory: K = 380 at D = 64) by
    cluster and sums runs in registers (lanes past D idle).  Two CTAs of
    10,001 points each: a full window and a ragged one (4,096: two full and a
    ragged third), so the window loop, the per-window histogram and scatter
    and the run flushes across windows are all exercised, against the
    oracle's update from the same assignment."""
    import torch
    x, _, _ = synth.kmeans_points(20_002, d, min(k, 64), seed=71 + k + d)
    dx = torch.from_numpy(x).cuda()
    cur = synth.kmeans_init(x, k, seed=72)
    ctx = mr.Context()
    ctx.set_option(mr.OPT_KM_GRID_CAP, 2)
    for _ in range(2):
        a_ref = oracle.kmeans_assign(x, cur)
        c_ref, _ = oracle.kmeans_update(x, a_ref, cur)
        c, a, st = _run_ctx(mr, ctx, dx, cur, 1, 0)
        assert np.array_equal(a, a_ref)
        assert _rel_err(c, c_ref) <= TOL
        cur = c_ref
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_kmeans_eight_tiles_per_cta_natural_grid(mr, precision):
    """152 x 8 x 128 points at the default grid (one tensor-core CTA per SM):
    every CTA runs 8 tiles, past the two-deep rings' first reuse.  All points
    against the oracle, teacher-forced for two iterations."""
    import torch
    n = torch.cuda.get_device_properties(0).multi_processor_count * 8 * 128
    x, _, _ = synth.kmeans_points(n, 64, 256, seed=47)
    cur = synth.kmeans_init(x, 256, seed=48)
    dx = _dev(x)
    ctx = mr.Context()
    for _ in range(2):
        a_ref = _assign_all(x, cur)
        c_ref, _ = oracle.kmeans_update(x, a_ref, cur)
        c, a, st = _run_ctx(mr, ctx, dx, cur, 1, precision)
        assert np.array_equal(a, a_ref)
        assert _rel_err(c, c_ref) <= TOL
        cur = c_ref
    ctx.close()


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("n,d,k,iters", [
    (20_000, 64, 256, 3),   # the workload's shape, reduced N
    (5_001, 37, 50, 2),     # D < 64 (zero-padded), K not a multiple of 16
    (777, 3, 1, 2),         # K = 1
    (300, 64, 16, 1),       # fewer points than one CTA per SM
    (641, 1, 4, 2),         # D = 1, a last tile of one point
    (2_050, 48, 40, 2),     # D a multiple of 16 below 64
    (6_000, 64, 136, 2),    # 144 columns: the last epilogue quarter idle, the third partly masked
    (6_000, 20, 200, 2),    # 208 columns
])
def test_kmeans_bf16_tensor_core_vs_oracle(mr, precision, n, d, k, iters):
    x, _, _ = synth.kmeans_points(n, d, max(1, min(k, 256)), seed=n + d + k + 7)
    init = synth.kmeans_init(x, k, seed=n + 1)
    c_ref, a_ref = oracle.kmeans(x, init, iters)
    c, a, stats = _run(mr, x, init, iters, precision=precision)
    assert np.array_equal(a, a_ref)
    assert _rel_err(c, c_ref) <= TOL
    assert int(stats[3]) == 0


def test_kmeans_bf16_teacher_forced(mr):
    x, _, _ = synth.kmeans_points(30_000, 64, 256, seed=43)
    cur = synth.kmeans_init(x, 256, seed=44)
    for _ in range(3):
        a_ref = oracle.kmeans_assign(x, cur)
        c_ref, _ = oracle.kmeans_update(x, a_ref, cur)
        c, a, stats = _run(mr, x, cur, 1, precision=1)
        assert np.array_equal(a, a_ref)
        assert _rel_err(c, c_ref) <= TOL
        cur = c_ref


@pytest.mark.slow
def test_kmeans_full_size_bf16_matches_fp32_path(mr):
    """4M x 64, K = 256, 10 iterations: the tensor-core path gives the same
    assignments and centroids as the FP32 path (both equal the FP64 argmin
    each iteration, and the integer sums make the update deterministic)."""
    import torch
    x, _, _ = synth.kmeans_points(4 << 20, 64, 256)
    init = synth.kmeans_init(x, 256)
    dx = torch.from_numpy(x).cuda()
    c32, a32, _ = mr.kmeans(dx, _dev(init), 10, 0)
    c16, a16, st = mr.kmeans(dx, _dev(init), 10, 1)
    assert np.array_equal(a16, a32)
    assert np.array_equal(c16, c32)
    assert int(st[3]) == 0
