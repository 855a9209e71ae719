#!/usr/bin/env python
"""Benchmark of the fused map-and-reduce hot path on GB300.

Default workload (one "step"): the array-container job pair — an RGB8
histogram over 1,610,612,736 bytes (512M pixels) and int8 regression sums over
536,870,912 bytes (256M pairs) — run through the C ABI (mr_add_job x2 +
mr_run) on inputs already resident in HBM.  Inputs are larger than L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload arrays|wordcount|kmeans|histkeys|bloom|batched|serving] [--scale S]

Other workloads are for manual measurement; the default line is the contract.
Multi-GPU (torchrun): each rank runs its own replica of the workload on its own
GPU (weak scaling, no data-path collective); the barrier and max-over-ranks
timing follow the contract.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input GB/s per job (% of HBM peak); batched jobs/s and p99 latency vs plain"
HIST_PIXELS = 512 << 20      # 1,610,612,736 bytes
KM_ITERS = 10
LR_PAIRS = 256 << 20         # 536,870,912 bytes
HK_KEYS = 256 << 20          # large-key histogram: 256M u32 keys (1 GiB) ...
HK_BINS = 1 << 24            # ... over 16M bins
BF_ELEMS = 30_000_000        # Bloom filter: 30M k-mers ...
BF_BITS = 300_000_000        # ... into 300M bits ...
BF_KMER, BF_HASHES = 32, 7   # ... 32-base windows, 7 bit positions each


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("bf16_tflops", 1956.4)), float(p.get("bf16_tflops_sustained", 1764.5)), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def _sm_max_mhz() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def source_sha(sources) -> str:
    h = hashlib.sha256()
    for src in sources:
        h.update(open(os.path.join(ROOT, src), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, sources, input_bytes: int):
    """Per-launch DRAM bytes from the committed ncu summary, scaled from the
    input size it was captured at to this launch's input bytes (the traffic
    of these kernels grows in proportion to their input), if the kernel's
    sources are unchanged since the capture (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        if rec.get("source_sha") != source_sha(sources):
            return None
        return int(round(rec["bytes_per_launch"] * input_bytes / rec["input_bytes"]))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            time.sleep(0.12)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_ranks(ms: float, nbytes: int, steps: int, ws: int):
    """Whole-job throughput of weak-scaled replicas: every rank processed
    nbytes per step; the job took the slowest rank's time.  Returns
    (ms_max, value in GB/s)."""
    ms_max = _max_over_ranks(ms, ws)
    return ms_max, nbytes * ws * steps / (ms_max / 1e3) / 1e9


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ workloads
def make_inputs(workload: str, scale: float, rank: int):
    import synth
    if workload == "arrays":
        npix = max(1, int(HIST_PIXELS * scale))
        npairs = max(1, int(LR_PAIRS * scale))
        px = synth.hist_rgb8(npix, seed=synth.SEED_BASE + 1 + 1000 * rank)
        xy = synth.linreg_i8(npairs, seed=synth.SEED_BASE + 2 + 1000 * rank)
        return {"px": px, "xy": xy}
    if workload == "wordcount":
        n = max(1024, int((16 << 20) * scale))
        text, _, _ = synth.wc_text(n, seed=synth.SEED_BASE + 1000 * rank)
        return {"text": text}
    if workload == "kmeans":
        n = max(1024, int((4 << 20) * scale))
        x, _, _ = synth.kmeans_points(n, 64, 256, seed=synth.SEED_BASE + 3 + 1000 * rank)
        init = synth.kmeans_init(x, 256, seed=synth.SEED_BASE + 4 + 1000 * rank)
        return {"x": x, "init": init}
    if workload == "histkeys":
        n = max(1024, int(HK_KEYS * scale))
        return {"keys": synth.keys_u32(n, HK_BINS, seed=synth.SEED_BASE + 5 + 1000 * rank)}
    if workload == "bloom":
        n = max(1024, int(BF_ELEMS * scale)) + BF_KMER - 1
        return {"seq": synth.dna(n, seed=synth.SEED_BASE + 6 + 1000 * rank)}
    raise ValueError(workload)


def workload_config(workload: str, inp, pipelined: bool = False) -> dict:
    if workload == "arrays":
        return {"workload": "rgb8 histogram %d B (%d px) + int8 linreg %d B (%d pairs)" % (
            inp["px"].nbytes, inp["px"].nbytes // 3, inp["xy"].nbytes, inp["xy"].nbytes // 2),
            "inputs": "synthetic, resident in HBM, larger than L2 (no flush needed)",
            "containers": "histogram: shared-memory local arrays; regression: register accumulators"}
    if workload == "kmeans":
        n, d = inp["x"].shape
        return {"workload": "k-means %d x %d FP32 points (%d B), K=%d, %d iterations" % (
            n, d, inp["x"].nbytes, inp["init"].shape[0], KM_ITERS),
            "inputs": "synthetic 256-component Gaussian mixture, resident in HBM, larger than L2"}
    if workload == "histkeys":
        return {"workload": "large-key histogram: %d u32 keys (%d B) uniform over %d bins" % (
            inp["keys"].size, inp["keys"].nbytes, HK_BINS),
            "inputs": "synthetic, resident in HBM, larger than L2 (no flush needed)",
            "containers": "global array (u32 counters, 64 MiB, L2-resident), no local arrays"}
    if workload == "bloom":
        return {"workload": "Bloom-filter build: %d-base windows of %d uniform ACGT bases (%d elements) into %d bits, "
                            "%d hashes" % (BF_KMER, inp["seq"].size, inp["seq"].size - BF_KMER + 1, BF_BITS, BF_HASHES),
                "inputs": "synthetic, resident in HBM; the 37.5 MB filter is L2-resident"}
    return {"workload": "word count %d B Zipf(1) text, 50,000-word vocabulary%s" % (
                inp["text"].nbytes, ", pipelined map/reduce warps" if pipelined else ""),
            "inputs": "synthetic, resident in HBM; 16 MiB fits in L2 (warm)"}


def run_ours(args):
    import numpy as np
    import torch
    import paper_1309_0215_gb300 as mr

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    mr.load()
    hbm_peak, _, _, peak_src = _peaks()

    inp = make_inputs(args.workload, args.scale, rank)
    stream = torch.cuda.Stream()
    ctx = mr.Context(dev, stream=stream, timing=True)
    with torch.cuda.stream(stream):
        dinp = {k: torch.from_numpy(v).cuda() for k, v in inp.items()}
    stream.synchronize()

    if args.workload == "arrays":
        d_px, d_xy = dinp["px"], dinp["xy"]
        total_bytes = d_px.numel() + d_xy.numel()

        def step():
            # two independent jobs run concurrently: the library fuses them
            # into one launch (each CTA takes its share of both inputs)
            a = ctx.add_job(mr.HIST_RGB8, d_px)
            b = ctx.add_job(mr.LINREG_I8, d_xy)
            ctx.run(mr.RUN_CONCURRENT)
            return [a, b]
        dominant = ("array_fused_kernel", ["paper_1309_0215_gb300/csrc/k_array.cu",
                                           "paper_1309_0215_gb300/csrc/dev_array.cuh"], total_bytes)
    elif args.workload == "kmeans":
        d_x, d_i = dinp["x"], dinp["init"]
        total_bytes = d_x.numel() * 4
        nn, dd = d_x.shape
        kk = d_i.shape[0]

        def step():
            a = ctx.add_job(mr.KMEANS_F32, d_x, km_dims=dd, km_k=kk, km_iters=KM_ITERS, km_init=d_i,
                            km_precision=args.precision)
            ctx.run()
            return [a]
        kname = "km_tc_assign_kernel" if args.precision else "km_assign_fp32_kernel"
        dominant = (kname, ["paper_1309_0215_gb300/csrc/k_kmeans_tc.cu" if args.precision else
                            "paper_1309_0215_gb300/csrc/k_kmeans.cu", "paper_1309_0215_gb300/csrc/dev_pipe.cuh"],
                    d_x.numel() * 4)
    elif args.workload == "histkeys":
        d_k = dinp["keys"]
        total_bytes = d_k.numel() * 4

        def step():
            a = ctx.add_job(mr.HIST_U32, d_k, hist_bins=HK_BINS)
            ctx.run()
            return [a]
        dominant = ("hk_global_kernel", ["paper_1309_0215_gb300/csrc/k_keys.cu"], d_k.numel() * 4)
    elif args.workload == "bloom":
        d_s = dinp["seq"]
        total_bytes = d_s.numel()

        def step():
            a = ctx.add_job(mr.BLOOM_DNA, d_s, bloom_kmer=BF_KMER, bloom_bits=BF_BITS, bloom_hashes=BF_HASHES)
            ctx.run()
            return [a]
        dominant = ("bloom_kernel", ["paper_1309_0215_gb300/csrc/k_keys.cu"], d_s.numel())
    else:
        d_t = dinp["text"]
        total_bytes = d_t.numel()

        def step():
            a = ctx.add_job(mr.WORDCOUNT, d_t, wc_pipelined=int(args.pipelined))
            ctx.run()
            return [a]
        # the plain map pass runs the CTA-table kernel from 64 MiB on
        mapk = "wc_pipe_kernel" if args.pipelined else (
            "wc_map_cta_kernel" if d_t.numel() >= (64 << 20) else "wc_map_kernel")
        dominant = (mapk, ["paper_1309_0215_gb300/csrc/k_wordcount.cu",
                           "paper_1309_0215_gb300/csrc/dev_wordcount.cuh"], d_t.numel())

    # Jobs are released RELEASE_LAG steps after they were enqueued, as a
    # serving loop releases its results: the GPU stays that many steps ahead of
    # the host, and the allocator reuses released buffers instead of growing
    # (a fresh device allocation would stall the stream).
    RELEASE_LAG = 3
    job_stats = []

    def retire(js, record):
        if record:
            job_stats.append((ctx.elapsed_ms(js[0]), ctx.kernel_ms(js[0])))
        for j in js:
            ctx.release(j)

    # warm-up, plus a parity spot check of the last warm-up step
    jobs = []
    for _ in range(args.warmup):
        jobs.append(step())
        if len(jobs) > RELEASE_LAG + 1:
            retire(jobs.pop(0), False)
    ctx.sync()
    parity = None
    if args.workload == "arrays":
        import oracle
        got_h, got_l = ctx.fetch(jobs[-1][0]), ctx.fetch(jobs[-1][1])
        bins = np.frombuffer(got_h, dtype=np.uint64)
        assert int(bins.sum()) == 3 * (d_px.numel() // 3), "histogram invariant failed"
        parity = {"histogram_bit_exact_vs_oracle": got_h == oracle.hist_rgb8(inp["px"]).tobytes(),
                  "regression_bit_exact_vs_oracle": got_l == oracle.linreg_i8(inp["xy"]).tobytes()}
        assert all(parity.values()), "arrays step differs from the oracle"
    if args.workload == "histkeys":
        bins = np.frombuffer(ctx.fetch(jobs[-1][0]), dtype=np.uint64)
        assert int(bins.sum()) == d_k.numel() and int(bins[-1]) == 0, "histogram invariant failed"
    for js in jobs:
        for j in js:
            ctx.release(j)

    clocks = ClockSampler(dev)
    clocks.start()
    _barrier(ws)
    torch.cuda.synchronize()
    l0 = ctx.kernel_launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    h0 = time.perf_counter()
    inflight = []
    for _ in range(args.steps):
        inflight.append(step())
        if len(inflight) > RELEASE_LAG:
            retire(inflight.pop(0), True)
    host_ms = (time.perf_counter() - h0) * 1e3 / args.steps  # host time to enqueue (and retire) a step
    ev1.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    clk = clocks.stop()
    launches = ctx.kernel_launches - l0
    ms = ev0.elapsed_time(ev1)
    for js in inflight:
        retire(js, True)
    job_ms = statistics.mean(e for e, _ in job_stats)
    # the dominant kernel's average launch duration (CUDA events around each launch, on its stream)
    kern_ms = sum(t for _, (t, _) in job_stats) / max(1, sum(c for _, (_, c) in job_stats))
    ms_max, value = combine_ranks(ms, total_bytes, args.steps, ws)
    ms_per_step = ms_max / args.steps

    # end to end through the public API: pinned host inputs, H2D + run + D2H every step
    km_stats = None
    if args.workload == "kmeans":
        js = step()
        ctx.sync()
        raw = ctx.fetch(js[0])
        _, _, st = mr.split_kmeans_result(raw, nn, dd, kk)
        km_stats = {"fp32_rechecks": int(st[0]), "fp64_rechecks": int(st[1]), "iterations": int(st[2]),
                    "timeouts": int(st[3]), "ms_per_iteration": round(job_ms / KM_ITERS, 4),
                    "distance_pass_ms": round(kern_ms, 4),
                    "distance_tflops_per_job": round(2.0 * nn * kk * dd * KM_ITERS / (job_ms / 1e3) / 1e12, 2)}
        ctx.release(js[0])
    e2e = None
    if not args.no_e2e and args.workload != "kmeans":
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in inp.items()}
        adders = {"px": lambda t: ctx.add_job(mr.HIST_RGB8, t), "xy": lambda t: ctx.add_job(mr.LINREG_I8, t),
                  "text": lambda t: ctx.add_job(mr.WORDCOUNT, t),
                  "keys": lambda t: ctx.add_job(mr.HIST_U32, t, hist_bins=HK_BINS),
                  "seq": lambda t: ctx.add_job(mr.BLOOM_DNA, t, bloom_kmer=BF_KMER, bloom_bits=BF_BITS,
                                               bloom_hashes=BF_HASHES)}
        out_bytes = {}
        out_pinned = {}  # result buffers in pinned host memory, sized by the first (warm-up) fetch

        def e2e_step():
            ids = [(k, adders[k](t)) for k, t in pinned.items()]
            ctx.run(mr.RUN_CONCURRENT)
            for k, j in ids:
                if k not in out_pinned:
                    nb = len(ctx.fetch(j))
                    out_pinned[k] = torch.empty(max(nb, 1), dtype=torch.uint8).pin_memory()
                    out_bytes[k] = nb
                else:
                    out_bytes[k] = ctx.fetch_into(j, out_pinned[k].numpy())
                ctx.release(j)
        for _ in range(2):
            e2e_step()
        n_e2e = max(1, min(args.steps, 10))
        _barrier(ws)
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        t1 = time.perf_counter()
        el = _max_over_ranks(t1 - t0, ws)
        e2e = {"value": round(total_bytes * ws * n_e2e / el / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": int(total_bytes), "d2h_bytes_per_step": int(sum(out_bytes.values())),
               "steps": n_e2e}

    # per job: each array job's own input GB/s and fraction of the HBM peak,
    # from its kernel time when it runs alone (in the step the two share one
    # fused launch, so the step cannot split the time between them)
    per_job_alone = {}
    if args.workload == "arrays":
        for name, kind, t in (("histogram", mr.HIST_RGB8, d_px), ("regression", mr.LINREG_I8, d_xy)):
            ts = []
            for i in range(8):
                j = ctx.add_job(kind, t)
                ctx.run(mr.RUN_PLAIN)
                ctx.fetch(j)
                if i >= 3:
                    kt, kc = ctx.kernel_ms(j)
                    ts.append(kt / max(1, kc))
                ctx.release(j)
            ms = statistics.median(ts)
            gbs = t.numel() / (ms / 1e3) / 1e9
            per_job_alone[name] = {"bytes": int(t.numel()), "launch_ms": round(ms, 5), "gbs": round(gbs, 1),
                                   "frac": round(gbs / hbm_peak, 4), "measured": "alone (RUN_PLAIN), 5 launches"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and args.workload != "kmeans":
        cpu = cpu_baseline(args.workload, inp)
        cpu["all_cores"] = cpu_all_cores(args.workload, inp)
        cpu["host"] = host_info()

    ctx.close()
    if rank == 0:
        kname, ksrc, kbytes = dominant
        achieved = kbytes / (kern_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": hbm_peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "traffic": _traffic(kname, ksrc, kbytes), "algorithmic_bytes_per_launch": int(kbytes),
                "launch_ms": round(kern_ms, 5), "launches_timed": int(sum(c for _, (_, c) in job_stats))}
        if args.workload == "arrays":
            step_gbs = total_bytes / (ms_per_step / 1e3) / 1e9
            roof["step_achieved"] = round(step_gbs, 1)
            roof["step_frac"] = round(step_gbs / hbm_peak, 4)
            roof["note"] = ("the histogram and regression jobs run as one fused launch; achieved = both "
                            "inputs' bytes per launch; step_achieved = both inputs' bytes per step (with the "
                            "launch gaps)")
        if args.workload == "kmeans":
            # a dense contraction: work is the distance GEMM, not bytes
            if args.precision:
                terms = 3 if args.precision == 1 else 1
                flops = 2.0 * nn * kk * dd * terms
                peak, bound, unit = _peaks()[1], "tensor", "TFLOP/s"
                note = ("BF16 tcgen05 products (%d per distance: x*c split into hi/lo parts) x 2*N*K*D, "
                        "per launch of the distance pass; peak = measured cuBLAS bf16 burst" % terms)
            else:
                flops = 2.0 * nn * kk * dd
                props = torch.cuda.get_device_properties(dev)
                peak = props.multi_processor_count * 128 * 2 * _sm_max_mhz() * 1e6 / 1e12
                bound, unit = "alu", "TFLOP/s"
                note = "FP32 FMA: 2*N*K*D per launch; peak = SMs x 128 FP32 lanes x 2 x max SM clock"
            ach = flops / (kern_ms / 1e3) / 1e12
            roof = {"bound": bound, "kernel": kname, "achieved": round(ach, 1), "peak": round(peak, 1),
                    "peak_source": peak_src if args.precision else "derived", "unit": unit,
                    "frac": round(ach / peak, 4), "traffic": _traffic(kname, ksrc, kbytes),
                    "algorithmic_flops_per_launch": flops, "launch_ms": round(kern_ms, 5),
                    "launches_timed": int(sum(c for _, (_, c) in job_stats)), "note": note}
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/i8 in, u64/i64 exact counts",
            "data": "synthetic (seeded generators shaped like the paper's workloads)",
            "config": workload_config(args.workload, inp, args.pipelined),
            "pct_of_hbm_peak": round(100 * value / ws / hbm_peak, 2),
            "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "host_enqueue_ms_per_step": round(host_ms, 5),
        }
        if args.workload == "histkeys":
            line["updates"] = {"keys_per_s": round(d_k.numel() / (kern_ms / 1e3), 1),
                               "note": "one counter increment per key (atomics after warp combining)"}
        if args.workload == "bloom":
            ne = d_s.numel() - BF_KMER + 1
            line["updates"] = {"elements_per_s": round(ne / (kern_ms / 1e3), 1),
                               "bit_sets_per_s": round(ne * BF_HASHES / (kern_ms / 1e3), 1)}
        if km_stats:
            line["kmeans"] = km_stats
        if parity:
            line["parity"] = parity
        if args.workload == "arrays":
            line["per_job"] = per_job_alone
        if ws == 1 and args.workload == "arrays" and not args.no_extra:
            # the metric's other parts, each on its own configuration, after
            # the headline step (its inputs and context are gone by now)
            del dinp, d_px, d_xy
            torch.cuda.empty_cache()
            line["configs"] = extra_configs(args)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def tokens_of(text):
    """(offsets, lengths) of the word-count tokens (maximal non-whitespace runs), numpy."""
    import numpy as np
    ws = np.isin(text, np.frombuffer(b" \t\n\v\f\r", dtype=np.uint8))
    tok = ~ws
    edge = np.diff(np.concatenate([[False], tok, [False]]).astype(np.int8))
    starts = np.flatnonzero(edge == 1)
    ends = np.flatnonzero(edge == -1)
    return starts.astype(np.int32), (ends - starts).astype(np.int32)


def run_simdh(args):
    """Pure hash computation over the word-count tokens (Sec. III-C, Fig. 10a):
    SIMDH-Padding vs SIMDH-Stream (and the wide variant), tokens/s."""
    import numpy as np
    import torch
    import synth
    import paper_1309_0215_gb300 as mr
    torch.cuda.set_device(0)
    mr.load()
    n = max(1024, int((16 << 20) * args.scale))
    text, _, _ = synth.wc_text(n, seed=synth.SEED_BASE)
    off, ln = tokens_of(text)
    d_text = torch.from_numpy(text).cuda()
    d_off, d_len = torch.from_numpy(off).cuda(), torch.from_numpy(ln).cuda()
    out = torch.empty(off.size, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    names = {mr.SIMDH_PADDING: "padding", mr.SIMDH_STREAM: "stream", mr.SIMDH_WIDE: "wide"}
    ref = None
    for m, name in names.items():
        for _ in range(args.warmup):
            mr.simdh_hash(d_text, d_off, d_len, m, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            mr.simdh_hash(d_text, d_off, d_len, m, out=out)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        h = out.cpu().numpy()
        if ref is None:
            ref = h
        assert np.array_equal(h, ref), "hash methods disagree"
        res[name] = {"ms": round(ms, 5), "tokens_per_s": round(off.size / (ms / 1e3), 1),
                     "bytes_per_s": round(int(ln.sum()) / (ms / 1e3), 1)}
    best = max(res.values(), key=lambda r: r["tokens_per_s"])
    print(json.dumps({
        "metric": METRIC, "value": best["tokens_per_s"], "unit": "tokens/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8 in, u64 FNV-1a out",
        "data": "synthetic (seeded word-count generator)",
        "config": {"workload": "FNV-1a 64 of %d word-count tokens (%d text bytes), pure hash computation" % (
            off.size, n), "inputs": "text and token list resident in HBM (L2-resident at 16 MiB)"},
        "methods": res, "gpu_launches": args.steps * 3}), flush=True)


def batched_specs(njobs: int, seed: int):
    """4,096-job mix: 50% word count, 30% RGB histogram, 20% regression; sizes
    log-uniform on [4 KiB, 64 MiB], rounded down to the kind's record size."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(4096), np.log(64 << 20), njobs)).astype(np.int64)
    kinds = rng.choice(3, size=njobs, p=[0.5, 0.3, 0.2])
    offs = rng.random(njobs)
    out = []
    for k, n, o in zip(kinds, sizes, offs):
        n = int(n) - (int(n) % (1, 3, 2)[k])
        out.append((int(k), n, float(o)))
    return out


def _oracle_result(kind, data):
    import oracle
    if kind == 0:
        return oracle.wordcount(data)
    if kind == 1:
        return oracle.hist_rgb8(data).tobytes()
    return oracle.linreg_i8(data).tobytes()


def batched_eval(scale: float, steps: int, warmup: int, autotune: bool = True, check_all: bool = True) -> dict:
    """Batched jobs/s: the 4,096-job mix in one persistent launch (CUDA graph
    replay) vs the plain one-launch-sequence-per-job path (sequential and on
    four streams).  check_all: every job's result is compared with the
    oracle's, the oracle running serially per job on a pool of host threads."""
    import concurrent.futures as cf
    import numpy as np
    import torch
    import synth
    import paper_1309_0215_gb300 as mr
    njobs = max(8, int(4096 * scale))
    specs = batched_specs(njobs, synth.SEED_BASE + 7)
    pool_text, _, _ = synth.wc_text(256 << 20, seed=synth.SEED_BASE, want_ranks=False)
    pool_px = synth.hist_rgb8(64 << 20, seed=synth.SEED_BASE + 1)
    pool_xy = synth.linreg_i8(64 << 20, seed=synth.SEED_BASE + 2)
    pools_h = [pool_text, pool_px, pool_xy]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pools = [torch.from_numpy(p).cuda() for p in pools_h]
    stream.synchronize()
    kinds = [mr.WORDCOUNT, mr.HIST_RGB8, mr.LINREG_I8]
    rec = (1, 3, 2)

    def slice_of(k, n, o):
        cap = pools[k].numel() - n
        off = int(o * cap) // rec[k] * rec[k]
        return off, pools[k][off: off + n]
    total_bytes = sum(n for _, n, _ in specs)
    ctx = mr.Context(0, stream=stream, autotune=autotune)
    ids = [ctx.add_job(kinds[k], slice_of(k, n, o)[1]) for k, n, o in specs]
    t0 = time.perf_counter()
    ctx.run(mr.RUN_BATCHED)
    ctx.sync()
    t_first = time.perf_counter() - t0
    check = {"jobs_checked": 0, "mismatches": 0}
    if check_all:
        # every job against the oracle: results fetched here (one context is
        # single-threaded), the oracle runs on host threads, a bounded number
        # of results in flight
        nth = max(1, os.cpu_count() or 1)
        t_chk = time.perf_counter()
        bad = []
        with cf.ThreadPoolExecutor(nth) as ex:
            futs = {}
            for i, (k, n, o) in enumerate(specs):
                off, _ = slice_of(k, n, o)
                got = ctx.fetch(ids[i])
                futs[ex.submit(lambda k=k, off=off, n=n, got=got: _oracle_result(k, pools_h[k][off: off + n]) == got)] = i
                if len(futs) >= 4 * nth:
                    done, _ = cf.wait(list(futs), return_when=cf.FIRST_COMPLETED)
                    for f in done:
                        if not f.result():
                            bad.append(futs[f])
                        del futs[f]
            for f, i in futs.items():
                if not f.result():
                    bad.append(i)
        check = {"jobs_checked": njobs, "mismatches": len(bad), "first_mismatches": sorted(bad)[:8],
                 "host_threads": nth, "seconds": round(time.perf_counter() - t_chk, 1)}
    for _ in range(warmup):
        ctx.rerun()
    ctx.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.kernel_launches
    ev0.record(stream)
    for _ in range(steps):
        ctx.rerun()
    ev1.record(stream)
    ev1.synchronize()
    launches = ctx.kernel_launches - l0
    ms = ev0.elapsed_time(ev1) / steps
    # a replay recomputes every result in place: spot-check that it still matches
    small = [i for i, (k, n, o) in enumerate(specs) if n < (1 << 20)][:8]
    for i in small:
        k, n, o = specs[i]
        off, _ = slice_of(k, n, o)
        assert ctx.fetch(ids[i]) == _oracle_result(k, pools_h[k][off: off + n]), "replayed job %d differs" % i
    # plain path: one launch sequence per job, same jobs
    ids2 = [ctx.add_job(kinds[k], slice_of(k, n, o)[1]) for k, n, o in specs]
    ctx.sync()
    ev0.record(stream)
    w0 = time.perf_counter()
    ctx.run(mr.RUN_PLAIN)
    ev1.record(stream)
    ev1.synchronize()
    plain_wall = time.perf_counter() - w0
    plain_ms = ev0.elapsed_time(ev1)
    for i in small:
        assert ctx.fetch(ids2[i]) == ctx.fetch(ids[i])
    for j in ids2:
        ctx.release(j)
    # concurrent plain path: the same launch sequences on four streams
    ids3 = [ctx.add_job(kinds[k], slice_of(k, n, o)[1]) for k, n, o in specs]
    ctx.sync()
    ev0.record(stream)
    w0 = time.perf_counter()
    ctx.run(mr.RUN_CONCURRENT)
    ev1.record(stream)
    ev1.synchronize()
    conc_wall = time.perf_counter() - w0
    conc_ms = ev0.elapsed_time(ev1)
    for i in small:
        assert ctx.fetch(ids3[i]) == ctx.fetch(ids[i])
    tune = ctx.tuning()
    ctx.close()
    hbm_peak = _peaks()[0]
    plain_t = max(plain_ms, 1e3 * plain_wall)
    conc_t = max(conc_ms, 1e3 * conc_wall)
    return {
        "workload": "%d jobs (50%% word count, 30%% RGB histogram, 20%% int8 regression), sizes log-uniform "
                    "4 KiB-64 MiB, %d bytes in total; job inputs are slices of device-resident pools" % (njobs, total_bytes),
        "mode": "one persistent launch + one word-count merge/sort, replayed from a CUDA graph",
        "jobs": njobs, "total_bytes": int(total_bytes), "steps": steps, "warmup": warmup,
        "ms_per_batch": round(ms, 4), "jobs_per_s": round(njobs / (ms / 1e3), 1),
        "aggregate_gbs": round(total_bytes / (ms / 1e3) / 1e9, 2),
        "pct_of_hbm_peak": round(100 * total_bytes / (ms / 1e3) / 1e9 / hbm_peak, 2),
        "plain": {"ms_device": round(plain_ms, 3), "ms_wall": round(1e3 * plain_wall, 3),
                  "jobs_per_s": round(njobs / (plain_t / 1e3), 1)},
        "speedup_vs_plain": round(plain_t / ms, 2),
        "concurrent_plain": {"ms_device": round(conc_ms, 3), "ms_wall": round(1e3 * conc_wall, 3),
                             "jobs_per_s": round(njobs / (conc_t / 1e3), 1)},
        "speedup_vs_concurrent_plain": round(conc_t / ms, 2),
        "first_run_s_incl_autotune": round(t_first, 3), "tuning": tune, "gpu_launches": int(launches),
        "oracle_check": check,
    }


def run_batched(args):
    """Batched jobs/s as its own JSON line."""
    import torch
    import paper_1309_0215_gb300 as mr
    torch.cuda.set_device(0)
    mr.load()
    r = batched_eval(args.scale, args.steps, args.warmup, autotune=not args.no_autotune)
    print(json.dumps({
        "metric": METRIC, "value": r["jobs_per_s"], "unit": "jobs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_batch"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8/i8 in, u64/i64 exact counts",
        "data": "synthetic (seeded generators); job inputs are slices of device-resident pools",
        "config": {"workload": r["workload"], "mode": r["mode"]}, "gpu_launches": r["gpu_launches"],
        "batched": r}), flush=True)


def serving_specs(rate: float, duration: float, seed: int):
    """Poisson arrivals; 25% each of word count, RGB histogram, int8 regression
    and k-means; sizes log-uniform on [1 KiB, 256 MiB] (k-means: D in [8, 64],
    K in [16, 256], N in [64K, 2M] clamped to 256 MiB of points, 10 iterations,
    BF16 tensor-core path)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    n = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    t = t[t < duration]
    out = []
    for a in t:
        kind = int(rng.integers(0, 4))
        if kind < 3:
            size = int(np.exp(rng.uniform(np.log(1024), np.log(256 << 20))))
            size -= size % (1, 3, 2)[kind]
            out.append((float(a), kind, (size, float(rng.random()))))
        else:
            d = int(rng.integers(8, 65))
            k = int(rng.integers(16, 257))
            npts = int(np.exp(rng.uniform(np.log(64 << 10), np.log(2 << 20))))
            npts = min(npts, (256 << 20) // (4 * d))
            out.append((float(a), 3, (npts, d, k, int(rng.integers(0, 2)))))
    return out


def serving_eval(rate: float, duration: float, plain_duration: float) -> dict:
    """Poisson request stream served with continuous batching (mr_submit /
    mr_poll) against an HBM budget, vs a plain server that launches each
    request on arrival; latency = arrival to result in host memory.  The
    plain server gets the arrivals of the trace's first plain_duration
    seconds: it cannot keep up with the offered load, so its queue (and its
    p99) only grows with the length of the run, and a shorter run gives a
    lower bound of its p99 over the whole trace."""
    import collections
    import numpy as np
    import torch
    import synth
    import paper_1309_0215_gb300 as mr
    specs = serving_specs(rate, duration, synth.SEED_BASE + 9)
    pool_text, _, _ = synth.wc_text(256 << 20, seed=synth.SEED_BASE, want_ranks=False)
    pools_h = [pool_text, synth.hist_rgb8((256 << 20) // 3, seed=synth.SEED_BASE + 1),
               synth.linreg_i8(128 << 20, seed=synth.SEED_BASE + 2)]
    kx, _, _ = synth.kmeans_points(2 << 20, 64, 256, seed=synth.SEED_BASE + 3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pools = [torch.from_numpy(p).cuda() for p in pools_h]
        kpool = torch.from_numpy(kx.reshape(-1)).cuda()
    stream.synchronize()
    kinds = [mr.WORDCOUNT, mr.HIST_RGB8, mr.LINREG_I8]

    def submit(ctx, spec, plain):
        kind, p = spec[1], spec[2]
        if kind < 3:
            size, o = p
            pool = pools[kind]
            size = min(size, pool.numel())
            rec = (1, 3, 2)[kind]
            off = int(o * (pool.numel() - size)) // rec * rec
            t, args_ = pool[off: off + size], {}
            mk = kinds[kind]
        else:
            npts, d, k, prec = p
            t = kpool[: npts * d].view(npts, d)
            args_ = dict(km_dims=d, km_k=k, km_iters=10, km_init=t[:k].contiguous(), km_precision=1)
            mk = mr.KMEANS_F32
        if plain:
            j = ctx.add_job(mk, t, **args_)
            ctx.run(mr.RUN_PLAIN)
            return j, t.numel() * t.element_size()
        return ctx.submit(mk, t, **args_), t.numel() * t.element_size()

    def serve(plain, specs):
        ctx = mr.Context(0, stream=stream, hbm_budget=120 << 30)
        waiting = collections.deque()
        inflight = {}
        lat, kinds, nbytes = [], [], 0
        nxt = 0
        t0 = time.perf_counter()
        while nxt < len(specs) or waiting or inflight:
            now = time.perf_counter() - t0
            while nxt < len(specs) and specs[nxt][0] <= now:
                waiting.append(specs[nxt])
                nxt += 1
            while waiting:
                try:
                    j, b = submit(ctx, waiting[0], plain)
                except mr.MRError as e:
                    if e.status != mr.MR_EBUDGET:
                        raise
                    break
                sp = waiting.popleft()
                inflight[j] = (sp[0], b, sp[1])
            for j in list(inflight):
                if ctx.poll(j):
                    ctx.fetch(j)
                    arr, b, kind = inflight.pop(j)
                    lat.append(time.perf_counter() - t0 - arr)
                    kinds.append(kind)
                    nbytes += b
                    ctx.release(j)
        wall = time.perf_counter() - t0
        ctx.close()
        lat, kinds = np.array(lat) * 1e3, np.array(kinds)
        by_kind = {}
        for kind, name in enumerate(("wordcount", "hist_rgb8", "linreg_i8", "kmeans")):
            v = lat[kinds == kind]
            if v.size:
                by_kind[name] = {"requests": int(v.size), "p50_ms": round(float(np.percentile(v, 50)), 3),
                                 "p99_ms": round(float(np.percentile(v, 99)), 3)}
        return {"requests": len(lat), "wall_s": round(wall, 3), "req_per_s": round(len(lat) / wall, 1),
                "gbs": round(nbytes / wall / 1e9, 3), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3), "max_ms": round(float(lat.max()), 3),
                "by_kind": by_kind}

    served = serve(False, specs)
    plain = serve(True, [sp for sp in specs if sp[0] < plain_duration])
    return {
        "workload": "Poisson %.0f req/s, 25%% each word count / histogram / regression / k-means (BF16 tensor-core "
                    "path, 10 iterations), sizes log-uniform 1 KiB-256 MiB, 120 GiB HBM budget" % rate,
        "arrivals_s": duration, "plain_arrivals_s": min(plain_duration, duration),
        "served_continuous_batching": served, "plain_one_launch_per_request": plain,
        "p99_speedup_vs_plain": round(plain["p99_ms"] / served["p99_ms"], 2) if served["p99_ms"] else None,
        "p50_speedup_vs_plain": round(plain["p50_ms"] / served["p50_ms"], 2) if served["p50_ms"] else None,
    }


def run_serving(args):
    """Serving p99 latency as its own JSON line."""
    import torch
    import paper_1309_0215_gb300 as mr
    torch.cuda.set_device(0)
    mr.load()
    r = serving_eval(args.rate, args.duration, args.plain_duration)
    print(json.dumps({
        "metric": METRIC, "value": r["served_continuous_batching"]["p99_ms"], "unit": "ms (p99 latency)",
        "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8/i8/f32 in, exact counts; k-means FP32/BF16 paths",
        "data": "synthetic; request inputs are slices of device-resident pools",
        "config": {"workload": r["workload"] + ", %.1f s of arrivals" % r["arrivals_s"]}, "serving": r}), flush=True)


def host_info() -> dict:
    """Host CPU as the OS reports it: logical CPUs and model name."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def cpu_all_cores(workload, inp) -> dict:
    """The same serial oracle on every host core at once: split-parallel for
    the array jobs (the step's input cut into one slice per thread, each slice
    through the oracle on its own thread, the per-slice bins and sums added),
    job-parallel for word count (each thread runs the oracle on its own copy
    of the job).  ctypes releases the GIL inside the oracle's C++ code."""
    import concurrent.futures as cf
    import numpy as np
    import oracle
    nth = max(1, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(nth) as ex:
        list(ex.map(lambda _: None, range(nth)))  # threads started before timing
        if workload == "arrays":
            px, xy = inp["px"], inp["xy"]
            ps = -(-(px.size // 3) // nth) * 3
            xs = -(-(xy.size // 2) // nth) * 2
            reps = 0
            t0 = time.perf_counter()
            while reps < 3 or time.perf_counter() - t0 < 10.0:  # about 10 s of work
                h = list(ex.map(oracle.hist_rgb8, [px[i: i + ps] for i in range(0, px.size, ps)]))
                r = list(ex.map(oracle.linreg_i8, [xy[i: i + xs] for i in range(0, xy.size, xs)]))
                bins, sums = np.sum(h, axis=0), np.sum(r, axis=0)
                reps += 1
            el = time.perf_counter() - t0
            assert int(bins.sum()) == px.size and sums.shape == (5,)
            nbytes = reps * (px.nbytes + xy.nbytes)
            sample = "%d full steps, each split into %d slices per input" % (reps, nth)
        elif workload == "wordcount":
            t = inp["text"]
            t0 = time.perf_counter()
            list(ex.map(lambda _: oracle.wordcount(t), range(nth)))
            el = time.perf_counter() - t0
            nbytes = t.nbytes * nth
            sample = "%d copies of the %d-byte job, one per thread" % (nth, t.nbytes)
        else:
            return None
    return {"value": round(nbytes / el / 1e9, 4), "unit": "GB/s", "cores": nth, "kind": "oracle",
            "mode": "split-parallel" if workload == "arrays" else "job-parallel", "sample": sample}


def wordcount_eval(steps: int, warmup: int) -> dict:
    """Word count on the 16 MiB Zipf(1) text: device time per job with the
    input warm in L2 (jobs back to back) and cold (a buffer twice the L2 size
    written between jobs, outside the timed job)."""
    import numpy as np
    import torch
    import oracle
    import synth
    import paper_1309_0215_gb300 as mr
    text, _, _ = synth.wc_text(16 << 20, want_ranks=False)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = torch.from_numpy(text).cuda()
        flush = torch.empty(2 * torch.cuda.get_device_properties(0).L2_cache_size, dtype=torch.uint8,
                            device="cuda")
    stream.synchronize()
    hbm_peak = _peaks()[0]
    exp = oracle.wordcount(text)
    ctx = mr.Context(0, stream=stream, timing=True)
    out = {"bytes": int(text.nbytes)}
    for mode in ("warm", "cold"):
        jobs, el, km = [], [], [0.0, 0]
        for i in range(warmup + steps):
            if mode == "cold":
                with torch.cuda.stream(stream):
                    flush.fill_(i & 255)
            j = ctx.add_job(mr.WORDCOUNT, d)
            ctx.run()
            jobs.append(j)
            if len(jobs) > 3:  # release a few jobs behind, as a serving loop does
                old = jobs.pop(0)
                if i - 3 >= warmup:
                    el.append(ctx.elapsed_ms(old))
                    t, c = ctx.kernel_ms(old)
                    km[0] += t
                    km[1] += c
                ctx.release(old)
        ok = ctx.fetch(jobs[-1]) == exp
        for j in jobs:
            el.append(ctx.elapsed_ms(j))
            t, c = ctx.kernel_ms(j)
            km[0] += t
            km[1] += c
            ctx.release(j)
        ms = statistics.median(el)
        out[mode] = {"ms_per_job": round(ms, 4), "gbs": round(text.nbytes / (ms / 1e3) / 1e9, 2),
                     "frac_of_hbm": round(text.nbytes / (ms / 1e3) / 1e9 / hbm_peak, 4),
                     "map_kernel_ms": round(km[0] / max(1, km[1]), 4), "jobs_timed": len(el),
                     "bit_exact_vs_oracle": ok}
    ctx.close()
    out["note"] = ("job = map + combine + global reduce + merge and sort of the ~50K distinct words; "
                   "the 16 MiB input fits in L2, so the job is latency- and launch-bound, not HBM-bound")
    return out


def kmeans_eval(steps: int, warmup: int) -> dict:
    """k-means 4M x 64 FP32 points, K = 256, 10 iterations, on the BF16
    tensor-core paths (three products, one product) and the FP32 path."""
    import numpy as np
    import torch
    import oracle
    import synth
    import paper_1309_0215_gb300 as mr
    x, _, _ = synth.kmeans_points(4 << 20, 64, 256)
    init = synth.kmeans_init(x, 256)
    n, dd = x.shape
    kk = init.shape[0]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dx = torch.from_numpy(x).cuda()
        di = torch.from_numpy(init).cuda()
    stream.synchronize()
    hbm_peak, bf16_peak, _, _ = _peaks()
    fp32_peak = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * _sm_max_mhz() * 1e6 / 1e12
    ctx = mr.Context(0, stream=stream, timing=True)

    def job(prec, iters, init_t):
        return ctx.add_job(mr.KMEANS_F32, dx, km_dims=dd, km_k=kk, km_iters=iters, km_init=init_t,
                           km_precision=prec)
    out = {"workload": "k-means %d x %d FP32 points (%d B), K=%d, %d iterations" % (n, dd, x.nbytes, kk, KM_ITERS)}
    results = {}
    for prec, name in ((1, "bf16_split_tc"), (2, "bf16_single_tc"), (0, "fp32")):
        reps = steps if prec else max(1, steps // 3)
        el, km, raw = [], [0.0, 0], None
        for i in range(warmup + reps):
            j = job(prec, KM_ITERS, di)
            ctx.run()
            if i >= warmup:
                el.append(ctx.elapsed_ms(j))
                t, c = ctx.kernel_ms(j)
                km[0] += t
                km[1] += c
            raw = ctx.fetch(j)
            ctx.release(j)
        c10, a10, st = mr.split_kmeans_result(raw, n, dd, kk)
        results[prec] = (c10, a10)
        it_ms = statistics.median(el) / KM_ITERS
        dk = km[0] / max(1, km[1])
        terms = 3 if prec == 1 else 1
        r = {"ms_per_iteration": round(it_ms, 4), "distance_kernel_ms": round(dk, 4),
             "method_tflops": round(2.0 * n * kk * dd / (dk / 1e3) / 1e12, 1),
             "points_gbs": round(x.nbytes / (dk / 1e3) / 1e9, 1),
             "points_frac_of_hbm": round(x.nbytes / (dk / 1e3) / 1e9 / hbm_peak, 4),
             "fp32_rechecks": int(st[0]), "fp64_rechecks": int(st[1]), "timeouts": int(st[3])}
        if prec:
            tt = 2.0 * n * kk * dd * terms / (dk / 1e3) / 1e12
            r.update({"tensor_products_per_distance": terms, "tensor_tflops": round(tt, 1),
                      "tensor_frac_of_bf16_peak": round(tt / bf16_peak, 4)})
        else:
            r.update({"fp32_frac_of_fma_peak": round(2.0 * n * kk * dd / (dk / 1e3) / 1e12 / fp32_peak, 4)})
        out[name] = r
    # the three paths give identical results (each iteration's assignment is
    # the FP64 argmin, and the update's integer sums make it order-free)
    out["bf16_paths_equal_fp32"] = bool(all(np.array_equal(results[p][0], results[0][0]) and
                                            np.array_equal(results[p][1], results[0][1]) for p in (1, 2)))
    # sampled check of the last iteration against the oracle, on the GPU's ninth centroids
    j = job(1, KM_ITERS - 1, di)
    ctx.run()
    c9, _, _ = mr.split_kmeans_result(ctx.fetch(j), n, dd, kk)
    ctx.release(j)
    rng = np.random.default_rng(0)
    smp = rng.choice(n, 8192, replace=False)
    out["sampled_assignments_equal_oracle"] = bool(np.array_equal(results[1][1][smp],
                                                                  oracle.kmeans_assign(x[smp], c9)))
    c_upd, _ = oracle.kmeans_update(x, results[1][1], c9)
    num = np.linalg.norm(results[1][0].astype(np.float64) - c_upd.astype(np.float64), axis=1)
    out["centroid_rel_err_vs_fp64_update"] = float((num / np.maximum(np.linalg.norm(
        c_upd.astype(np.float64), axis=1), 1.0)).max())
    ctx.close()
    return out


def extra_configs(args) -> dict:
    """The metric's other parts, each on its own configuration; a failure is
    reported in its entry instead of failing the whole run."""
    res = {}
    runs = (("wordcount_16MiB", lambda: wordcount_eval(20, 3)),
            ("kmeans_4Mx64_K256", lambda: kmeans_eval(3, 1)),
            ("batched_4096_jobs", lambda: batched_eval(1.0, 5, 3, autotune=True, check_all=True)),
            ("serving", lambda: serving_eval(2000.0, args.duration, args.plain_duration)))
    for name, fn in runs:
        t0 = time.perf_counter()
        try:
            res[name] = fn()
        except Exception as e:  # reported, not hidden
            res[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        res[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        import torch
        torch.cuda.empty_cache()
    return res



def run_histkeys_sweep(args):
    """Local arrays vs the global array as the key range grows (the GPU form
    of the paper's "eliminating local arrays" experiment, Sec. III-E and its
    evaluation in Sec. IV-B): 256M u32 keys uniform on [0, bins), bins from
    2^10 to 2^28, so the u32 counters go from a few KB (shared memory) past
    the 129 MB L2 into HBM.  Each configuration is timed on its counting
    kernel (CUDA events around every launch); results are checked against
    the count invariant, and at the smallest sizes against the oracle."""
    import numpy as np
    import torch
    import oracle
    import synth
    import paper_1309_0215_gb300 as mr
    torch.cuda.set_device(0)
    mr.load()
    n = max(1 << 20, int(HK_KEYS * args.scale))
    keys = synth.keys_u32(n, 1 << 28, seed=synth.SEED_BASE + 5)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dk = torch.from_numpy(keys.view(np.int32)).cuda()
        dm = torch.empty_like(dk)
    stream.synchronize()
    ctx = mr.Context(0, stream=stream, timing=True)
    smem_max = None
    rows = []
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    for lb in (10, 12, 14, 15, 16, 18, 20, 22, 24, 25, 26, 28):
        bins = 1 << lb
        with torch.cuda.stream(stream):
            torch.bitwise_and(dk, bins - 1, out=dm)
        stream.synchronize()
        for cont, cname in ((mr.C_SMEM_ARRAY, "local arrays (shared memory)"),
                            (mr.C_CLUSTER_ARRAY, "cluster local arrays (distributed shared memory)"),
                            (mr.C_GLOBAL_ARRAY, "global array")):
            try:
                js = []
                for i in range(args.warmup + args.steps):
                    js.append(ctx.add_job(mr.HIST_U32, dm, container=cont, hist_bins=bins))
                    ctx.run()
            except mr.MRError as e:
                if e.status == mr.MR_EINVAL and cont == mr.C_SMEM_ARRAY:
                    smem_max = smem_max or lb
                    continue
                if e.status == mr.MR_EINVAL and cont == mr.C_CLUSTER_ARRAY:
                    continue
                raise
            res = np.frombuffer(ctx.fetch(js[-1]), dtype=np.uint64)
            assert int(res.sum()) == n and int(res[-1]) == 0, "count invariant"
            if lb <= 12:
                assert np.array_equal(res, oracle.hist_u32(keys & (bins - 1), bins)), "oracle"
            t, c = 0.0, 0
            for j in js[args.warmup:]:
                tt, cc = ctx.kernel_ms(j)
                t += tt
                c += cc
            for j in js:
                ctx.release(j)
            ms = t / c
            rows.append({"bins": bins, "counter_bytes": (bins + 1) * 4, "counters_fit_l2": (bins + 1) * 4 <= l2,
                         "container": cname, "launch_ms": round(ms, 4),
                         "keys_per_s": round(n / (ms / 1e3), 1), "key_gbs": round(4 * n / (ms / 1e3) / 1e9, 1)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    ctx.close()
    # where the global array overtakes the local arrays (the largest bin count
    # at which local arrays are still at least as fast), from the rows above
    both = {}
    for r in rows:
        both.setdefault(r["bins"], {})[r["container"].split(" ")[0]] = r["launch_ms"]
    last_local_win = max([b for b, v in both.items() if "local" in v and v["local"] <= v["global"]] or [0])
    last_cluster_win = max([b for b, v in both.items() if "cluster" in v and v["cluster"] <= v["global"]] or [0])
    best = max(rows, key=lambda r: r["keys_per_s"])
    print(json.dumps({
        "metric": METRIC, "value": best["keys_per_s"], "unit": "keys/s (best configuration)", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["launch_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 keys in, u32 counters, u64 out",
        "data": "synthetic: %d u32 keys uniform on [0, bins)" % n,
        "config": {"workload": "large-key histogram container sweep, %d keys, bins 2^10..2^28" % n},
        "l2_bytes": l2, "rows": rows, "local_arrays_fastest_up_to_bins": last_local_win,
        "cluster_arrays_beat_global_up_to_bins": last_cluster_win,
        "local_arrays_rejected_from_bins": 1 << smem_max if smem_max else None}), flush=True)


def cpu_baseline(workload, inp, max_seconds=30.0):
    """The serial oracle timed on this host's cores (1 thread) on the whole
    step's input, or a leading sample of it if that would exceed max_seconds."""
    import oracle
    if workload == "arrays":
        # whole steps, repeated until about 10 s of CPU work (at least 3)
        px, xy = inp["px"], inp["xy"]
        reps = 0
        t0 = time.perf_counter()
        while reps < 3 or time.perf_counter() - t0 < 10.0:
            oracle.hist_rgb8(px)
            oracle.linreg_i8(xy)
            reps += 1
        el = time.perf_counter() - t0
        return {"value": round(reps * (px.nbytes + xy.nbytes) / el / 1e9, 4), "unit": "GB/s", "cores": 1,
                "kind": "oracle", "seconds": round(el, 1),
                "sample": "%d full steps (histogram %d B + regression %d B each), serial C++ oracle" % (
                    reps, px.nbytes, xy.nbytes)}
    if workload == "histkeys":
        k = inp["keys"][: 64 << 20]
        t0 = time.perf_counter()
        oracle.hist_u32(k, HK_BINS)
        el = time.perf_counter() - t0
        return {"value": round(k.nbytes / el / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                "sample": "first %d keys of the step's input, serial C++ oracle" % k.size}
    if workload == "bloom":
        sq = inp["seq"][: 10_000_000]
        t0 = time.perf_counter()
        oracle.bloom_dna(sq, BF_KMER, BF_BITS, BF_HASHES)
        el = time.perf_counter() - t0
        return {"value": round(sq.nbytes / el / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                "sample": "first %d bases of the step's input, serial C++ oracle" % sq.size}
    t = inp["text"]
    t0 = time.perf_counter()
    oracle.wordcount(t)
    el = time.perf_counter() - t0
    return {"value": round(t.nbytes / el / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "one full step: word count %d B, serial C++ oracle" % t.nbytes}


def run_reference(args):
    """The oracle as the reference arm: serial CPU, a bounded sample per step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np
    import oracle
    inp = make_inputs(args.workload, args.scale, 0)
    budget = 120.0
    nsteps = args.steps + args.warmup
    if args.workload == "arrays":
        px, xy = inp["px"], inp["xy"]
        # calibrate the oracle's rate on a small slice
        t0 = time.perf_counter()
        oracle.hist_rgb8(px[: 3 * (1 << 20)])
        oracle.linreg_i8(xy[: 2 * (1 << 19)])
        rate = (3 * (1 << 20) + (1 << 20)) / (time.perf_counter() - t0)
        per_step = min(budget / nsteps * rate, px.nbytes + xy.nbytes)
        frac = per_step / (px.nbytes + xy.nbytes)
        sp = px[: 3 * max(1, int(px.nbytes // 3 * frac))]
        sx = xy[: 2 * max(1, int(xy.nbytes // 2 * frac))]

        def step():
            oracle.hist_rgb8(sp)
            oracle.linreg_i8(sx)
        nbytes = sp.nbytes + sx.nbytes
        sample = "first %d B of the histogram input + first %d B of the regression input per step" % (sp.nbytes, sx.nbytes)
    elif args.workload in ("histkeys", "bloom"):
        a = inp["keys"] if args.workload == "histkeys" else inp["seq"]
        if args.workload == "histkeys":
            def run_on(x):
                oracle.hist_u32(x, HK_BINS)
        else:
            def run_on(x):
                oracle.bloom_dna(x, BF_KMER, BF_BITS, BF_HASHES)
        t0 = time.perf_counter()
        run_on(a[: 1 << 20])
        rate = (1 << 20) / (time.perf_counter() - t0)  # elements per second
        cnt = int(min(budget / nsteps * rate, a.size))
        sa = a[: max(cnt, 64)]

        def step():
            run_on(sa)
        nbytes = sa.nbytes
        sample = "first %d %s of the input per step" % (sa.size, "keys" if args.workload == "histkeys" else "bases")
    else:
        t = inp["text"]
        t0 = time.perf_counter()
        oracle.wordcount(t[: 1 << 20])
        rate = (1 << 20) / (time.perf_counter() - t0)
        n = int(min(budget / nsteps * rate, t.nbytes))
        st = t[:n]

        def step():
            oracle.wordcount(st)
        nbytes = n
        sample = "first %d B of the text per step" % n
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = nbytes * args.steps / el / 1e9
    inp_cfg = workload_config(args.workload, inp)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/i8 in, u64/i64 exact counts",
        "data": "synthetic (seeded generators shaped like the paper's workloads)", "config": inp_cfg,
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["arrays", "wordcount", "kmeans", "histkeys", "bloom", "batched", "serving",
                                           "simdh", "histkeys-sweep"], default="arrays")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean requests per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--plain-duration", type=float, default=20.0,
                    help="serving: seconds of the same arrivals given to the plain server")
    ap.add_argument("--precision", type=int, default=1, help="k-means: 0 FP32, 1 BF16 split, 2 BF16 single")
    ap.add_argument("--scale", type=float, default=1.0, help="input size relative to the full workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="arrays: skip the word-count, k-means, batched and serving configurations")
    ap.add_argument("--no-autotune", action="store_true", help="batched: keep the default tile sizes")
    ap.add_argument("--pipelined", action="store_true", help="word count: pipelined map/reduce warps")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "simdh":
        run_simdh(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "histkeys-sweep":
        run_histkeys_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
