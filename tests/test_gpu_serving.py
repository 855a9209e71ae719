"""GPU: serving with continuous batching (mr_submit / mr_poll).

Requests are submitted in waves while earlier ones are still running, so
they are launched in several overlapping micro-batches; each result must be
the same as the same request run alone (bit for bit, k-means included: its
sums are exact integers) and equal the oracle (k-means: the FP64 argmin
assignments exactly, centroids within 1e-5 relative)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _requests(seed):
    rng = np.random.default_rng(seed)
    text, _, _ = synth.wc_text(4 << 20, nwords=8000, seed=seed)
    px = synth.hist_rgb8(1 << 20, seed=seed + 1)
    xy = synth.linreg_i8(1 << 20, seed=seed + 2)
    reqs = []
    for i in range(48):
        kind = i % 4
        n = int(np.exp(rng.uniform(np.log(1024), np.log(2 << 20))))
        if kind == 0:
            o = int(rng.integers(0, text.size - n))
            reqs.append(("wc", text[o: o + n]))
        elif kind == 1:
            n -= n % 3
            o = 3 * int(rng.integers(0, (px.size - n) // 3))
            reqs.append(("hist", px[o: o + n]))
        elif kind == 2:
            n -= n % 2
            o = 2 * int(rng.integers(0, (xy.size - n) // 2))
            reqs.append(("lr", xy[o: o + n]))
        else:
            d = int(rng.integers(8, 65))
            k = int(rng.integers(16, 257))
            npts = int(rng.integers(2000, 20000))
            x, _, _ = synth.kmeans_points(npts, d, 32, seed=seed + i)
            init = synth.kmeans_init(x, k, seed=seed + i)
            reqs.append(("km", (x, init, int(rng.integers(0, 3)))))
    return reqs


def _submit(mr, c, req, plain=False):
    import torch
    kind, data = req
    if kind == "km":
        x, init, prec = data
        args = dict(km_dims=x.shape[1], km_k=init.shape[0], km_iters=3, km_init=torch.from_numpy(init).cuda(),
                    km_precision=prec)
        t = torch.from_numpy(x).cuda()
        mk = mr.KMEANS_F32
    else:
        args = {}
        t = torch.from_numpy(np.ascontiguousarray(data)).cuda()
        mk = {"wc": mr.WORDCOUNT, "hist": mr.HIST_RGB8, "lr": mr.LINREG_I8}[kind]
    if plain:
        j = c.add_job(mk, t, **args)
        c.run(mr.RUN_PLAIN)
        return j
    return c.submit(mk, t, **args)


def test_serving_mix_equals_alone(mr):
    reqs = _requests(3)
    served = mr.Context(hbm_budget=8 << 30)
    ids = []
    for w in range(0, len(reqs), 8):  # waves: later requests arrive while earlier ones run
        ids += [_submit(mr, served, r) for r in reqs[w: w + 8]]
        for j in ids[: w // 2]:
            served.poll(j)
    got = [served.fetch(j) for j in ids]
    alone = mr.Context()
    for r, g in zip(reqs, got):
        j = _submit(mr, alone, r, plain=True)
        assert alone.fetch(j) == g
        alone.release(j)
        kind, data = r
        if kind == "wc":
            assert g == oracle.wordcount(data)
        elif kind == "hist":
            assert g == oracle.hist_rgb8(data).tobytes()
        elif kind == "lr":
            assert g == oracle.linreg_i8(data).tobytes()
        else:  # k-means: FP64 argmin assignments, centroids within 1e-5 of the FP64 means
            x, init, _ = data
            c_ref, a_ref = oracle.kmeans(x, init, 3)
            c, a, st = mr.split_kmeans_result(g, x.shape[0], x.shape[1], init.shape[0])
            assert np.array_equal(a, a_ref)
            num = np.linalg.norm(c.astype(np.float64) - c_ref.astype(np.float64), axis=1)
            assert float((num / np.maximum(np.linalg.norm(c_ref.astype(np.float64), axis=1), 1.0)).max()) <= 1e-5
            assert int(st[3]) == 0
    for j in ids:
        served.release(j)
    assert served.bytes_in_use < (64 << 20)  # only reusable scratch stays
    served.close()
    alone.close()


def test_serving_admission_by_budget(mr):
    import torch
    c = mr.Context(hbm_budget=64 << 20)
    big = torch.zeros(48 << 20, dtype=torch.uint8, device="cuda")
    j1 = c.submit(mr.HIST_RGB8, big[: 30 << 20])  # fits: its container is small
    text, _, _ = synth.wc_text(48 << 20, nwords=1000, seed=5)
    t = torch.from_numpy(text).cuda()
    with pytest.raises(mr.MRError) as e:
        c.submit(mr.WORDCOUNT, t)  # its result buffer alone exceeds the budget
    assert e.value.status == mr.MR_EBUDGET
    assert np.frombuffer(c.fetch(j1), dtype=np.uint64).sum() == 30 << 20
    c.release(j1)
    small = t[: 1 << 20]
    j2 = c.submit(mr.WORDCOUNT, small)
    assert c.fetch(j2) == oracle.wordcount(text[: 1 << 20])
    c.close()
