#!/usr/bin/env python
"""Benchmark of the fused map-and-reduce hot path on GB300.

Default workload (one "step"): the array-container job pair — an RGB8
histogram over 1,610,612,736 bytes (512M pixels) and int8 regression sums over
536,870,912 bytes (256M pairs) — run through the C ABI (mr_add_job x2 +
mr_run) on inputs already resident in HBM.  Inputs are larger than L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload arrays|wordcount|kmeans|batched|serving] [--scale S]

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
LR_PAIRS = 256 << 20         # 536,870,912 bytes


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("bf16_tflops", 1956.4)), float(p.get("bf16_tflops_sustained", 1764.5)), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def _traffic(kernel: str, source: str):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel's
    source is unchanged since the capture (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        h = hashlib.sha256(open(os.path.join(ROOT, source), "rb").read()).hexdigest()[:16]
        return rec["bytes_per_launch"] if rec.get("source_sha") == h else None
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
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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
    raise ValueError(workload)


def workload_config(workload: str, inp) -> dict:
    if workload == "arrays":
        return {"workload": "rgb8 histogram %d B (%d px) + int8 linreg %d B (%d pairs)" % (
            inp["px"].nbytes, inp["px"].nbytes // 3, inp["xy"].nbytes, inp["xy"].nbytes // 2),
            "inputs": "synthetic, resident in HBM, larger than L2 (no flush needed)",
            "containers": "histogram: shared-memory local arrays; regression: register accumulators"}
    return {"workload": "word count %d B Zipf(1) text, 50,000-word vocabulary" % inp["text"].nbytes,
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
            a = ctx.add_job(mr.HIST_RGB8, d_px)
            b = ctx.add_job(mr.LINREG_I8, d_xy)
            ctx.run()
            return [a, b]
        dominant = ("hist_smem_kernel", "paper_1309_0215_gb300/csrc/k_array.cu", d_px.numel())
    else:
        d_t = dinp["text"]
        total_bytes = d_t.numel()

        def step():
            a = ctx.add_job(mr.WORDCOUNT, d_t)
            ctx.run()
            return [a]
        dominant = ("wc_map_kernel", "paper_1309_0215_gb300/csrc/k_wordcount.cu", d_t.numel())

    # warm-up, plus a parity spot check of the last warm-up step
    jobs = []
    for _ in range(args.warmup):
        jobs.append(step())
    ctx.sync()
    if args.workload == "arrays":
        bins = np.frombuffer(ctx.fetch(jobs[-1][0]), dtype=np.uint64)
        assert int(bins.sum()) == 3 * (d_px.numel() // 3), "histogram invariant failed"
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
    timed = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    clk = clocks.stop()
    launches = ctx.kernel_launches - l0
    ms = ev0.elapsed_time(ev1)
    dom_ms = statistics.mean(ctx.elapsed_ms(js[0]) for js in timed)
    for js in timed:
        for j in js:
            ctx.release(j)
    ms_max = _max_over_ranks(ms, ws)
    ms_per_step = ms_max / args.steps
    value = total_bytes * ws * args.steps / (ms_max / 1e3) / 1e9

    # end to end through the public API: pinned host inputs, H2D + run + D2H every step
    e2e = None
    if not args.no_e2e:
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in inp.items()}
        kinds = {"px": mr.HIST_RGB8, "xy": mr.LINREG_I8, "text": mr.WORDCOUNT}
        out_bytes = {}

        def e2e_step():
            ids = [(k, ctx.add_job(kinds[k], t)) for k, t in pinned.items()]
            ctx.run()
            for k, j in ids:
                out_bytes[k] = len(ctx.fetch(j))
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

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, inp)

    ctx.close()
    if rank == 0:
        kname, ksrc, kbytes = dominant
        achieved = kbytes / (dom_ms / 1e3) / 1e9
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/i8 in, u64/i64 exact counts",
            "data": "synthetic (seeded generators shaped like the paper's workloads)",
            "config": workload_config(args.workload, inp),
            "pct_of_hbm_peak": round(100 * value / ws / hbm_peak, 2),
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": hbm_peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                         "traffic": _traffic(kname, ksrc),
                         "algorithmic_bytes_per_launch": int(kbytes)},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(workload, inp, max_seconds=30.0):
    """The serial oracle timed on this host's cores (1 thread) on the whole
    step's input, or a leading sample of it if that would exceed max_seconds."""
    import oracle
    if workload == "arrays":
        px, xy = inp["px"], inp["xy"]
        t0 = time.perf_counter()
        oracle.hist_rgb8(px)
        oracle.linreg_i8(xy)
        el = time.perf_counter() - t0
        return {"value": round((px.nbytes + xy.nbytes) / el / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                "sample": "one full step: histogram %d B + regression %d B, serial C++ oracle" % (px.nbytes, xy.nbytes)}
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
    ap.add_argument("--workload", choices=["arrays", "wordcount"], default="arrays")
    ap.add_argument("--scale", type=float, default=1.0, help="input size relative to the full workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
