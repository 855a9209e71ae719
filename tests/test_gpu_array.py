"""GPU parity: RGB histogram and int8 regression sums, bit-exact vs the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _dev(arr, offset=0):
    """Copy a numpy array to the GPU starting `offset` bytes into a buffer."""
    import torch
    raw = np.frombuffer(arr.tobytes(), dtype=np.uint8)
    buf = torch.empty(raw.size + offset + 16, dtype=torch.uint8, device="cuda")
    buf[offset: offset + raw.size] = torch.from_numpy(raw.copy()).cuda()
    return buf[offset: offset + raw.size]


@pytest.mark.parametrize("npix", [0, 1, 2, 7, 511, 512, 513, 4096 + 5, 1 << 16, 1_000_003])
def test_hist_small_and_ragged(mr, npix):
    px = synth.hist_rgb8(npix, seed=100 + npix)
    got = mr.hist_rgb8(_dev(px))
    assert np.array_equal(got, oracle.hist_rgb8(px))


@pytest.mark.parametrize("offset", [1, 2, 3, 5, 8, 15])
def test_hist_unaligned_device_pointer(mr, offset):
    px = synth.hist_rgb8(200_001, seed=7)
    assert np.array_equal(mr.hist_rgb8(_dev(px, offset)), oracle.hist_rgb8(px))


def test_hist_host_input_and_skew(mr):
    px = np.full(3 * 300_000, 200, dtype=np.uint8)  # every emit hits one bin per channel
    got = mr.hist_rgb8(px)
    assert np.array_equal(got, oracle.hist_rgb8(px))
    px2 = np.tile(np.array([0, 128, 255], dtype=np.uint8), 123_457)
    assert np.array_equal(mr.hist_rgb8(_dev(px2)), oracle.hist_rgb8(px2))


@pytest.mark.parametrize("npix", [1, 1000, 1 << 18])
def test_hist_global_array_container(mr, npix):
    px = synth.hist_rgb8(npix, seed=3)
    got = mr.hist_rgb8(_dev(px), container=mr.C_GLOBAL_ARRAY)
    assert np.array_equal(got, oracle.hist_rgb8(px))


def test_hist_rejects_bad_length(mr):
    with pytest.raises(mr.MRError) as e:
        mr.hist_rgb8(np.zeros(4, dtype=np.uint8))
    assert e.value.status == mr.MR_EINVAL


@pytest.mark.slow
def test_hist_full_size_1_5GiB(mr):
    """512M pixels (1,610,612,736 bytes), the histogram workload's full size."""
    import torch
    px = synth.hist_rgb8(512 << 20)
    d = torch.from_numpy(px).cuda()
    got = mr.hist_rgb8(d)
    ref = oracle.hist_rgb8(px)
    assert np.array_equal(got, ref)
    assert int(got.sum()) == 3 * (512 << 20)


@pytest.mark.parametrize("npairs", [0, 1, 7, 8, 9, 4095, 65536 + 3, 1_000_001])
def test_linreg_small_and_ragged(mr, npairs):
    xy = synth.linreg_i8(npairs, seed=200 + npairs)
    assert mr.linreg_i8(_dev(xy)).tolist() == oracle.linreg_i8(xy).tolist()


@pytest.mark.parametrize("offset", [1, 2, 6, 14])
def test_linreg_unaligned_device_pointer(mr, offset):
    xy = synth.linreg_i8(100_003, seed=9)
    assert mr.linreg_i8(_dev(xy, offset)).tolist() == oracle.linreg_i8(xy).tolist()


def test_linreg_extremes(mr):
    xy = np.full(2 * 3_000_001, -128, dtype=np.int8)
    assert mr.linreg_i8(_dev(xy)).tolist() == oracle.linreg_i8(xy).tolist()
    x = np.tile(np.arange(-128, 128, dtype=np.int16), 5000)
    xy2 = np.empty(2 * x.size, dtype=np.int8)
    xy2[0::2] = x
    xy2[1::2] = 127 - (x + 128)
    assert mr.linreg_i8(xy2).tolist() == oracle.linreg_i8(xy2).tolist()


@pytest.mark.slow
def test_linreg_full_size_256M_pairs(mr):
    import torch
    xy = synth.linreg_i8(256 << 20)
    got = mr.linreg_i8(torch.from_numpy(xy).cuda())
    assert got.tolist() == oracle.linreg_i8(xy).tolist()


def test_context_jobs_plain_sequence(mr):
    """Several jobs of different kinds in one mr_run, fetched in any order."""
    c = mr.Context()
    px = synth.hist_rgb8(77_777, seed=11)
    xy = synth.linreg_i8(55_555, seed=12)
    j1 = c.add_job(mr.HIST_RGB8, _dev(px))
    j2 = c.add_job(mr.LINREG_I8, xy)
    j3 = c.add_job(mr.HIST_RGB8, px)
    c.run()
    assert np.frombuffer(c.fetch(j2), dtype=np.int64).tolist() == oracle.linreg_i8(xy).tolist()
    ref = oracle.hist_rgb8(px)
    assert np.array_equal(np.frombuffer(c.fetch(j3), dtype=np.uint64), ref)
    assert np.array_equal(np.frombuffer(c.fetch(j1), dtype=np.uint64), ref)
    for j in (j1, j2, j3):
        c.release(j)
    with pytest.raises(mr.MRError):
        c.fetch(j1)
    c.close()


def test_main_kernel_timing(mr):
    """mr_job_kernel_ms: one timed launch per counting job, one per k-means
    iteration, and the summed launch time within the job's own time."""
    c = mr.Context(timing=True)
    px = synth.hist_rgb8(3_000_000, seed=13)
    x, _, _ = synth.kmeans_points(20_000, 64, 16, seed=14)
    init = synth.kmeans_init(x, 16, seed=15)
    text, _, _ = synth.wc_text(1 << 20, seed=16, want_ranks=False)
    jh = c.add_job(mr.HIST_RGB8, _dev(px))
    jl = c.add_job(mr.LINREG_I8, synth.linreg_i8(100_000, seed=17))
    jk = c.add_job(mr.KMEANS_F32, x, km_dims=64, km_k=16, km_iters=3, km_init=init, km_precision=mr.KM_BF16_TC)
    jw = c.add_job(mr.WORDCOUNT, text)
    c.run()
    for j, launches in ((jh, 1), (jl, 1), (jk, 3), (jw, 1)):
        ms, n = c.kernel_ms(j)
        assert n == launches
        assert 0.0 < ms <= c.elapsed_ms(j) * 1.01
    assert np.array_equal(np.frombuffer(c.fetch(jh), dtype=np.uint64), oracle.hist_rgb8(px))
    c.close()
    plain = mr.Context()  # no timing: refused
    j = plain.add_job(mr.HIST_RGB8, px)
    plain.run()
    with pytest.raises(mr.MRError):
        plain.kernel_ms(j)
    plain.close()
    batched = mr.Context(timing=True)  # the batched launch is shared by its jobs: refused
    j = batched.add_job(mr.HIST_RGB8, px)
    batched.run(mr.RUN_BATCHED)
    with pytest.raises(mr.MRError):
        batched.kernel_ms(j)
    batched.close()
