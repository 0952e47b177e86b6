"""Benchmark of the dedispersion search hot path on GB300.

Workload (default): one beam streamed in 2^17-sample blocks with the overlap
tail carried on the device; 1024 channels over 398-418 MHz, t_samp 51.2 us,
640 DM trials 0-127.8 step 0.2, FP32 samples: N(0,1) noise, 16 dispersed
Gaussian pulses per block (random trial DM 5-120, SNR 8-30, FWHM 0.5-4 ms)
and Poisson narrowband RFI bursts.  A step is one block through every stage:
window assembly (push), statistics and masks (A1-A3), dedispersion (A4-A5),
series statistics and candidate compaction (A6-A7).

Metric: DM-trial.samples/s = sum over beams of ndm x new output samples per
block / time.  Also reported: real-time beams sustained (metric / (ndm /
t_samp)), p50/p99 device time per block, the dominant kernel's roofline, an
end-to-end number through the C ABI from pinned host buffers, and the CPU
oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 it runs under torch.distributed.run: every rank processes
its own beam (independent replicas, no data-path collective).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

NCHAN, F_LO, BW, TSAMP = 1024, 398.0, 20.0, 51.2e-6
BLOCK = 1 << 17
DMS = np.arange(640) * 0.2
NBUF = 3  # distinct synthetic blocks cycled through
PAPER_DERIVED = 6.5e7  # DM-trial.samples/s per GPU derived from the paper's Table 1
# DRAM bytes (read + write) of one dedispersion launch of the stream workload
# (1024 channels, 640 DMs, a steady-state 2^17-sample block), per (sample
# format, kernel shape), measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the launch the benchmark times; shapes without
# such a capture report null.
TRAFFIC_BY_SHAPE = {("f32", 33): 584.843264e6 + 331.993600e6, ("f32", 46): 175.55649461716e9 * 5.406816e-3,
                    ("f32", 55): 192.00875257012e9 * 5.089248e-3, ("f32", 53): 650.720768e6 + 315.274240e6,
                    ("u8", 57): 291.825408e6 + 305.486592e6, ("u8", 43): 284.709888e6 + 299.847936e6}
# shared-memory data-path utilisation (l1tex__data_pipe_lsu_wavefronts as a
# fraction of peak) in the same captures
SMEM_FRAC_BY_SHAPE = {("f32", 46): 0.6806, ("f32", 55): 0.5959, ("f32", 53): 0.7222, ("u8", 57): 0.3859,
                      ("u8", 43): 0.4080}
METRIC = "DM-trial*samples/s per GB300 (real-time beams sustained, p99 block latency alongside)"
WORKLOAD = "stream: 1 beam, 1024 ch 398-418 MHz, 51.2 us, 640 DMs 0-127.8 step 0.2, FP32, 2^17-sample blocks"


def stream_config(overlap, world):
    """The metric's workload, as both arms report it."""
    return {"workload": WORKLOAD, "nchan": NCHAN, "ndm": len(DMS), "block": BLOCK, "overlap": int(overlap),
            "beams_per_gpu": 1, "l2": "inputs larger than L2 (562 MB window per block, 3 distinct blocks cycled)",
            "parallelism": f"replicas x{world}"}


def device_peaks(dev):
    """Add-pipe peak from the device's SM count and the largest SM clock
    (nvidia-smi, else the measured-peaks file, else 2070 MHz), and the measured
    HBM copy bandwidth when the measured-peaks file is present."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, src = None, None
    try:
        out = subprocess.run(["nvidia-smi", f"--id={dev.index or 0}", "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        mhz, src = float(out.stdout.strip().splitlines()[0]), "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pass
    hbm = None
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(mp["hbm_gbs"])
        if mhz is None:
            mhz, src = float(mp["sm_max_mhz"]), "measured peaks sm_max_mhz"
    except (OSError, ValueError, KeyError):
        pass
    if mhz is None:
        mhz, src = 2070.0, "nominal maximum"
    return {"sms": sms, "sm_max_mhz": mhz, "clock_source": src,
            "add_peak_T": sms * 128 * mhz * 1e6 / 1e12, "hbm_GBps": hbm}


def _raw(h):
    """A host block as an array torch can hold: bfloat16 bits as int16,
    complex int16 voltages as one int32 per sample."""
    if h.dtype == np.uint16:
        return h.view(np.int16)
    if h.dtype.names:
        return h.view(np.int32)
    return h


def make_block(seed, delay, max_delay, dtype="f32"):
    """One synthetic block: noise, 16 pulses on random trials, RFI bursts;
    FP32 N(0,1) by default, stored as binary16 / bfloat16, or as 8-bit
    round(N(128, 16)); complex int16 voltages whose power carries the same
    pulses and bursts on a unit envelope."""
    g = synth.rng(seed)
    x = synth.noise(NCHAN, BLOCK, seed) if dtype != "c16" else np.ones((NCHAN, BLOCK), np.float32)
    for _ in range(16):
        d = int(g.integers(min(25, delay.shape[0] - 1), min(601, delay.shape[0])))
        t = int(g.integers(0, BLOCK - int(delay[d].max()) - 200))
        snr = float(g.uniform(8, 30))
        fwhm = float(g.uniform(0.5, 4.0)) * 1e-3 / TSAMP
        synth.add_pulse(x, delay[d].astype(np.float64) + t, fwhm, snr / math.sqrt(NCHAN))
    synth.apply_bursts(x, synth.poisson_bursts(NCHAN, BLOCK, seed + 7))
    if dtype == "f16":
        return synth.to_f16(x)
    if dtype == "bf16":
        return synth.to_bf16_bits(x)
    if dtype == "u8":
        return synth.to_u8(x * 16.0 + 128.0)
    if dtype == "c16":
        return synth.complex_voltage(np.maximum(x, 0.05), seed + 11, sigma=30.0)
    return x


class Clocks:
    """nvidia-smi sampler over the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    world = int(os.environ["WORLD_SIZE"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_window(delays, max_delay):
    x = make_block(999, delays, max_delay)
    return np.ascontiguousarray(np.concatenate([x[:, BLOCK - max_delay:], x], axis=1))  # tail + block


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(delays, max_delay, n_dm_sample=None, threads=None, win=None):
    """The CPU oracle on a bounded sample of the workload: A1-A3 over a full
    streaming window plus A5-A7 for an evenly spread subset of the DM trials
    (at least two trials per thread, so that every thread of the OpenMP loop
    over trials has work), extrapolated linearly in the number of trials to
    all 640."""
    from oracle import oracle as O
    threads = threads or os.cpu_count() or 1
    used = O.set_threads(threads)
    if n_dm_sample is None:
        n_dm_sample = max(32, 2 * used)
    n_dm_sample = min(n_dm_sample, len(DMS))
    if win is None:
        win = cpu_window(delays, max_delay)
    rfi = O.RfiParams()
    t0 = time.perf_counter()
    st = O.bandpass(win, "f32")
    _, cf = O.channel_mask(win, "f32", st, rfi)
    sf = O.spectrum_mask(win, "f32", st, rfi, cf)
    t_rfi = time.perf_counter() - t0
    sel = np.linspace(0, len(DMS) - 1, n_dm_sample).astype(int)
    t1 = time.perf_counter()
    D = O.dedisperse(win, "f32", st, cf, sf, rfi.chunk_width, delays[sel], BLOCK)
    ss = O.series_stats(D)
    O.candidates(D, ss["mu"], ss["sigma"], 5.0)
    t_dm = time.perf_counter() - t1
    total = t_rfi + t_dm * len(DMS) / n_dm_sample
    value = len(DMS) * BLOCK / total
    return {"value": value, "unit": "DM-trial*samples/s", "cores": used, "kind": "oracle",
            "sample": (f"one 1024 x {BLOCK + max_delay} FP32 window: A1-A3 in full ({t_rfi:.2f} s), "
                       f"A5-A7 for {n_dm_sample} of 640 DMs ({t_dm:.2f} s) on {used} threads, extrapolated "
                       "linearly to 640"),
            "extrapolated": True, "seconds": t_rfi + t_dm}


def cpu_baselines(delays, max_delay, win=None):
    """The oracle on all host cores (the reported baseline) and on one thread."""
    win = cpu_window(delays, max_delay) if win is None else win
    allc = cpu_baseline(delays, max_delay, win=win)
    one = cpu_baseline(delays, max_delay, n_dm_sample=8, threads=1, win=win)
    allc.pop("seconds", None)
    allc["single_thread"] = {"value": one["value"], "sample": one["sample"]}
    allc["nproc"] = os.cpu_count()
    allc["cpu_model"] = cpu_model()
    return allc


def run_reference(args):
    """--impl reference: the CPU oracle as it stands on the host cores, on the
    metric's workload (each step a bounded sample of one block, extrapolated
    to the whole block)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    delays, max_delay = O.delay_table(NCHAN, F_LO, BW, TSAMP, DMS)
    vals = []
    win = cpu_window(delays, max_delay)
    r = None
    for k in range(args.warmup + args.steps):
        r = cpu_baseline(delays, max_delay, win=win)
        if k >= args.warmup:
            vals.append(r["value"])
    if not vals:
        r = cpu_baseline(delays, max_delay, win=win)
        vals.append(r["value"])
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DM-trial*samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": len(DMS) * BLOCK / value * 1e3, "ms_per_step_extrapolated": True,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value / PAPER_DERIVED, "dtype": "f64", "data": "synthetic",
            "config": stream_config(max_delay, args.gpus),
            "cpu_baseline": {"value": value, "unit": "DM-trial*samples/s", "cores": r["cores"],
                             "kind": "oracle", "sample": r["sample"], "nproc": os.cpu_count(),
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "DM-trial*samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def dedisp_roof(adds, ms, peaks, packed=False, traffic=None, traffic_note=None):
    """Roofline entry of a dedispersion launch: adds per launch / launch time
    against the add-pipe peak (SMs x 128 lanes x clock); 8-bit data add two
    16-bit lanes per integer add, so their packed peak is twice that."""
    achieved = adds / (ms / 1e3) / 1e12
    peak = peaks["add_peak_T"] * (2 if packed else 1)
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": traffic, "ms_per_launch": ms,
           "peak_note": (f"{peaks['sms']} SMs x 128 lanes x {peaks['sm_max_mhz']:.0f} MHz "
                         f"({peaks['clock_source']})" + (" x 2 sample-adds per packed integer add" if packed
                                                         else "") + "; 1 add counted as 1 op")}
    if packed:
        out["frac_of_scalar_peak"] = achieved / peaks["add_peak_T"]
    if traffic_note:
        out["traffic_note"] = traffic_note
    return out


BATCH_DMS = [320, 320, 640, 640, 960, 960, 1280, 1280]


def run_batch8(args, dtype="f16", steps=20, warmup=3, peaks=None):
    """Config 3: 8 beams, 1024 channels, DM ranges of 320/640/960/1280 trials
    (step 0.2), binary16 storage, 2^17-sample blocks; every stage of all
    beams issued as batched launches replayed from a CUDA graph, the kernel
    shape picked by the batch autotuner.  Inputs generated on the device."""
    import torch
    import paper_1307_5700_gb300 as tp

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks = peaks or device_peaks(dev)
    tp.build()
    stream = torch.cuda.Stream(dev)
    e = tp.tp_engine_create(local, 0, stream.cuda_stream)
    plans, beams, blocks = {}, [], []
    with torch.cuda.stream(stream):
        for i, nd in enumerate(BATCH_DMS):
            if nd not in plans:
                plans[nd] = tp.tp_create_plan(e, NCHAN, F_LO, BW, TSAMP, np.arange(nd) * 0.2, dtype, None, 5.0)
            p = plans[nd]
            beams.append(tp.tp_beam_open(e, p, BLOCK, 1 << 20))
            delays = tp.tp_get_delay_table(p)
            g = synth.rng(3000 + 31 * i + 7 * rank)
            bl = []
            for k in range(2):
                arr = []
                for _ in range(8):
                    d = int(g.integers(min(25, nd - 1), nd))
                    t = int(g.integers(0, BLOCK - int(delays[d].max()) - 200))
                    arr.append((delays[d].astype(np.float64) + t, float(g.uniform(0.5, 4.0)) * 1e-3 / TSAMP,
                                float(g.uniform(8, 30)) / math.sqrt(NCHAN)))
                bl.append(synth.torch_block(NCHAN, BLOCK, 3000 + 31 * i + 7 * rank + k, arr,
                                            rfi_channels=g.integers(0, NCHAN, 8), device=dev, fmt=dtype))
            blocks.append(bl)
    stream.synchronize()
    for b, bl in zip(beams, blocks):
        tp.tp_push_block(e, b, bl[0])
    tp.tp_run_ready(e, use_graph=False)
    # the second block has the steady-state length: tune on it
    for b, bl in zip(beams, blocks):
        tp.tp_push_block(e, b, bl[1])
    if args.shape is None:
        best, shape_ms = tp.tp_autotune_batch(e, reps=1)
    else:
        best, shape_ms = args.shape, np.full(1, -1.0)
        for p in plans.values():
            tp.tp_plan_set_shape(p, best)
    tp.tp_run_ready(e, use_graph=False)
    units_per_step = sum(BATCH_DMS) * BLOCK
    adds = sum(BATCH_DMS) * NCHAN * BLOCK

    def step(k, graph=True):
        for b, bl in zip(beams, blocks):
            tp.tp_push_block(e, b, bl[k % 2])
        if getattr(args, "per_beam", False):
            for b in beams:
                tp.tp_dedisperse(e, b)
                tp.tp_detect(e, b)
        else:
            tp.tp_run_ready(e, use_graph=graph)

    for k in range(warmup):
        step(k)
    stream.synchronize()
    l0 = tp.tp_engine_launches(e)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    t0.record(stream)
    for k in range(steps):
        step(k)
    t1.record(stream)
    stream.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    launches = tp.tp_engine_launches(e) - l0
    # the batched dedispersion launch itself, timed with events on the same
    # launches issued outside the graph
    tp.tp_set_profiling(e, True)
    for k in range(max(3, steps // 4)):
        step(k, graph=False)
    bms, bn = tp.tp_get_batch_times(e)
    tp.tp_set_profiling(e, False)
    ncand = [tp.tp_get_candidates(e, b, 0)[1] for b in beams]
    shapes = {str(nd): int(tp.tp_plan_shapes(p)[0]) for nd, p in plans.items()}
    for b in beams:
        tp.tp_beam_close(e, b)
    for p in plans.values():
        tp.tp_plan_destroy(p)
    tp.tp_engine_destroy(e)
    del blocks
    torch.cuda.empty_cache()
    value = units_per_step * steps * world / (ms / 1e3)
    return {"workload": f"batch: 8 beams x 1024 ch 398-418 MHz, DM trials {BATCH_DMS} step 0.2, {dtype}, "
                        "2^17-sample blocks, every stage batched and replayed from a CUDA graph",
            "value": value, "unit": "DM-trial*samples/s", "dtype": dtype, "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "adds_per_s": adds * steps * world / (ms / 1e3),
            "kernel_shape": int(best), "kernel_shape_per_plan": shapes,
            "autotune_ms": {str(i): round(float(v), 3) for i, v in enumerate(shape_ms) if v >= 0},
            "realtime_beams": value / (len(DMS) / TSAMP),
            "roofline": dedisp_roof(adds, bms / bn, peaks) if bn else None,
            "gpu_launches": int(launches), "candidates_last_block": ncand, "clocks": clk}


# Config 5: the wide band.
WIDE = dict(nbeams=16, nchan=4096, f_lo=1200.0, bw=300.0, ts=64e-6, ndm=2048, block=1 << 18)


def run_wide16(args, steps=3, warmup=2, peaks=None):
    """Config 5: 16 beams x 4096 channels over 1200-1500 MHz, 64 us, DM
    trials 0-2047 step 1, 8-bit samples (exact int32 sums), 2^18-sample
    blocks; 4 dispersed pulses per block and narrowband bursts on 5 % of the
    channels.  One plan, every stage of all beams batched (graph replay),
    the kernel shape tuned on one beam.  Inputs generated on the device."""
    import torch
    import paper_1307_5700_gb300 as tp

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks = peaks or device_peaks(dev)
    tp.build()
    W = WIDE
    stream = torch.cuda.Stream(dev)
    e = tp.tp_engine_create(local, 0, stream.cuda_stream)
    dms = np.arange(W["ndm"]) * 1.0
    plan = tp.tp_create_plan(e, W["nchan"], W["f_lo"], W["bw"], W["ts"], dms, "u8", None, 5.0)
    delays = tp.tp_get_delay_table(plan)
    max_delay = tp.tp_plan_info(plan)["max_delay"]
    beams = [tp.tp_beam_open(e, plan, W["block"], 1 << 20) for _ in range(W["nbeams"])]
    nrfi = int(round(0.05 * W["nchan"]))
    pool = []
    g = synth.rng(5000 + rank)
    with torch.cuda.stream(stream):
        for k in range(4):
            arr = []
            for _ in range(4):
                d = int(g.integers(100, W["ndm"] - 100))
                t = int(g.integers(0, W["block"] - int(delays[d].max()) - 200))
                arr.append((delays[d].astype(np.float64) + t, float(g.uniform(1.0, 4.0)) * 1e-3 / W["ts"],
                            float(g.uniform(10, 30)) / math.sqrt(W["nchan"])))
            pool.append(synth.torch_block(W["nchan"], W["block"], 5000 + 100 * rank + k, arr,
                                          rfi_channels=g.choice(W["nchan"], nrfi, replace=False), device=dev,
                                          fmt="u8"))
    stream.synchronize()

    def push_all(k):
        for i, b in enumerate(beams):
            tp.tp_push_block(e, b, pool[(i + k) % len(pool)])

    push_all(0)
    tp.tp_run_ready(e, use_graph=False)
    push_all(1)
    if args.shape is None:
        # tune on one beam's steady-state block (the plan is shared); the
        # timing runs leave that beam to be processed again
        tp.tp_dedisperse(e, beams[0])
        best, shape_ms = tp.tp_autotune(e, beams[0], reps=1)
    else:
        best, shape_ms = args.shape, np.full(1, -1.0)
        tp.tp_plan_set_shape(plan, best)
    tp.tp_run_ready(e, use_graph=False)
    units_per_step = W["nbeams"] * W["ndm"] * W["block"]
    adds = units_per_step * W["nchan"]
    for k in range(warmup):
        push_all(k)
        tp.tp_run_ready(e, use_graph=True)
    stream.synchronize()
    l0 = tp.tp_engine_launches(e)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    t0.record(stream)
    for k in range(steps):
        push_all(k)
        tp.tp_run_ready(e, use_graph=True)
    t1.record(stream)
    stream.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    launches = tp.tp_engine_launches(e) - l0
    tp.tp_set_profiling(e, True)
    for k in range(2):
        push_all(k)
        tp.tp_run_ready(e, use_graph=False)
    bms, bn = tp.tp_get_batch_times(e)
    tp.tp_set_profiling(e, False)
    ncand = [tp.tp_get_candidates(e, b, 0)[1] for b in beams]
    for b in beams:
        tp.tp_beam_close(e, b)
    tp.tp_plan_destroy(plan)
    tp.tp_engine_destroy(e)
    del pool
    torch.cuda.empty_cache()
    value = units_per_step * steps * world / (ms / 1e3)
    return {"workload": (f"wide band: {W['nbeams']} beams x {W['nchan']} ch 1200-1500 MHz, 64 us, "
                         f"{W['ndm']} DMs 0-2047 step 1, u8 (int32 sums), 2^18-sample blocks, 4 pulses per "
                         "block, bursts on 5 % of the channels, every stage batched and replayed from a CUDA graph"),
            "value": value, "unit": "DM-trial*samples/s", "dtype": "u8", "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "adds_per_s": adds * steps * world / (ms / 1e3),
            "overlap": int(max_delay), "kernel_shape": int(best),
            "autotune_ms": {str(i): round(float(v), 3) for i, v in enumerate(shape_ms) if v >= 0},
            "realtime_beams": value / (W["ndm"] / W["ts"]),
            "roofline": dedisp_roof(adds, bms / bn, peaks, packed=True) if bn else None,
            "gpu_launches": int(launches), "candidates_last_block": ncand, "clocks": clk}


def serve_streams():
    """32 streams: channel counts cycle 256/512/1024/4096 and block lengths
    2^16/2^17/2^18; up to 1024 channels: 398-418 MHz, 51.2 us, 320 DMs step
    0.2; 4096 channels: 1200-1500 MHz, 64 us, 1024 DMs step 1; 8-bit samples
    round(N(128, 16))."""
    out = []
    for i in range(32):
        nchan = (256, 512, 1024, 4096)[i % 4]
        block = 1 << (16 + i % 3)
        if nchan == 4096:
            out.append(dict(nchan=nchan, f_lo=1200.0, bw=300.0, ts=64e-6, dms=np.arange(1024) * 1.0, block=block))
        else:
            out.append(dict(nchan=nchan, f_lo=398.0, bw=20.0, ts=51.2e-6, dms=np.arange(320) * 0.2, block=block))
    return out


def run_serve(args, speedup=None, blocks_per_stream=None):
    """Config 4, the serving loop: Poisson block arrivals on 32 streams (mean
    interval = the block's real-time duration, compressed by ``speedup``),
    HBM admission within --hbm-gb, continuous batching.  Latency = completion
    - arrival of each block, also as a fraction of the block's real-time
    duration."""
    import torch
    import paper_1307_5700_gb300 as tp

    speedup = args.speedup if speedup is None else speedup
    blocks_per_stream = args.blocks_per_stream if blocks_per_stream is None else blocks_per_stream
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    tp.build()
    streams = serve_streams()
    cache = {}
    blocks = []
    for i, st in enumerate(streams):
        key = (st["nchan"], st["block"])
        if key not in cache:
            g = synth.rng(5000 + len(cache))
            xf = g.standard_normal((st["nchan"], st["block"]), dtype=np.float32)
            synth.apply_bursts(xf, synth.poisson_bursts(st["nchan"], st["block"], 6000 + len(cache)))
            host = torch.empty(xf.shape, dtype=torch.uint8, pin_memory=True)
            host.numpy()[...] = synth.to_u8(xf * 16.0 + 128.0)
            cache[key] = host
        blocks.append(cache[key])
    stream = torch.cuda.Stream(dev)
    e = tp.tp_engine_create(local, int(args.hbm_gb * (1 << 30)), stream.cuda_stream)
    srv = tp.tp_server_create(e, nsigma=5.0)
    g = synth.rng(99 + rank)
    for i, st in enumerate(streams):
        sid = tp.tp_server_add_stream(srv, st["nchan"], st["f_lo"], st["bw"], st["ts"], st["dms"], "u8",
                                      st["block"], 1 << 20)
        dur = st["block"] * st["ts"] / speedup          # compressed block duration
        t = float(g.exponential(dur))
        for k in range(blocks_per_stream):
            tp.tp_server_submit(srv, sid, blocks[i], t)
            t += float(g.exponential(dur))
        tp.tp_server_end_stream(srv, sid)
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    w0 = time.perf_counter()
    tp.tp_server_run(srv, time_limit_s=600.0)
    wall = max_over_ranks(time.perf_counter() - w0, world, dev)
    clk = clocks.stop()
    res = tp.tp_server_results(srv)
    launches = tp.tp_engine_launches(e)
    tp.tp_server_destroy(srv)
    tp.tp_engine_destroy(e)
    lat = (res["done_s"] - res["arrival_s"]) * 1e3
    total_units = sum(len(streams[r["stream"]]["dms"]) * streams[r["stream"]]["block"] for r in res)
    rt = [((r["done_s"] - r["arrival_s"]) / (streams[r["stream"]]["block"] * streams[r["stream"]]["ts"]))
          for r in res]
    return {"workload": ("serving: 32 streams, nchan 256/512/1024/4096, blocks 2^16-2^18, u8, Poisson arrivals "
                         f"at {speedup:g}x real time, {blocks_per_stream} blocks/stream, HBM budget "
                         f"{args.hbm_gb:g} GB"),
            "value": total_units * world / wall, "unit": "DM-trial*samples/s", "dtype": "u8",
            "blocks": int(len(res)), "wall_s": wall,
            "p50_block_latency_ms": float(np.percentile(lat, 50)),
            "p99_block_latency_ms": float(np.percentile(lat, 99)),
            "latency_over_block_duration_p50": float(np.percentile(rt, 50)),
            "latency_over_block_duration_p99": float(np.percentile(rt, 99)),
            "arrival_speedup": speedup, "gpu_launches": int(launches), "clocks": clk}


def run_stream(args, dtype, steps, warmup, e2e_on, peaks=None):
    """Config 2, the metric's workload: one beam streamed in 2^17-sample
    blocks (push, A1-A3, A4-A5, A6-A7 per step), device-resident inputs;
    optionally the same end to end through the C ABI from pinned host
    buffers."""
    import torch
    import paper_1307_5700_gb300 as tp

    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks = peaks or device_peaks(dev)
    tp.build()
    stream = torch.cuda.current_stream(dev)
    e = tp.tp_engine_create(local, 0, stream)
    rfi = tp.tp_rfi_defaults()
    if args.fit >= 0:
        rfi.tau_channel = 40.0  # with the fitted bandpass tau_c counts in units of the fit's RMSE
    plan = tp.tp_create_plan(e, NCHAN, F_LO, BW, TSAMP, DMS, dtype, rfi, 5.0)
    if args.median > 1 or args.detrend:
        tp.tp_plan_set_postprocess(plan, args.median, args.detrend)
    if args.fit >= 0:
        tp.tp_plan_set_bandpass_fit(plan, args.fit, 5.0)
    if args.cluster:
        tp.tp_plan_set_clustering(plan)
    delays = tp.tp_get_delay_table(plan)
    max_delay = tp.tp_plan_info(plan)["max_delay"]
    beam = tp.tp_beam_open(e, plan, BLOCK, 1 << 20)

    host = [make_block(2000 + 17 * rank + i, delays, max_delay, dtype) for i in range(NBUF)]
    # device-resident inputs as a producer on the device would leave them:
    # each block in its own buffer, after max_delay columns of headroom that
    # the engine fills with the overlap tail (tp_push_inplace); --copy-push
    # pushes the same blocks by copy instead
    dev_bufs = []
    for h in host:
        t = torch.from_numpy(_raw(h)).to(dev)
        es = t.element_size()
        pitch = max_delay + BLOCK
        pitch += (-pitch * es) % 256 // es
        buf = torch.zeros((NCHAN, pitch), dtype=t.dtype, device=dev)
        buf[:, max_delay:max_delay + BLOCK] = t
        dev_bufs.append(buf)
    dev_blocks = [b[:, max_delay:max_delay + BLOCK].contiguous() for b in dev_bufs] if args.copy_push else None
    pushes = [0]

    def push():
        # consecutive blocks alternate the buffers (the next push copies the
        # tail out of the previous one)
        i = pushes[0] % NBUF
        pushes[0] += 1
        if args.copy_push:
            tp.tp_push_block(e, beam, dev_blocks[i])
        else:
            tp.tp_push_inplace(e, beam, dev_bufs[i], BLOCK)

    # first block of the stream fills the overlap tail; not timed
    push()
    tp.tp_dedisperse(e, beam)
    tp.tp_detect(e, beam)
    tp.tp_get_candidates(e, beam, 0)
    # the second block has the steady-state length (the first yields
    # block - max_delay outputs, a different number of CTA waves): autotune
    # the dedispersion kernel shape on it
    push()
    tp.tp_dedisperse(e, beam)
    if args.shape is None:
        best, shape_ms = tp.tp_autotune(e, beam, reps=2)
        tp.tp_dedisperse(e, beam)
    else:
        best, shape_ms = args.shape, np.full(1, -1.0)
        tp.tp_plan_set_shape(plan, best)
    tune = {str(i): round(float(v), 3) for i, v in enumerate(shape_ms) if v >= 0}
    tp.tp_detect(e, beam)
    tp.tp_get_candidates(e, beam, 0)

    def step(k, starts=None, ends=None):
        if starts is not None:
            starts[k].record(stream)
        push()
        tp.tp_dedisperse(e, beam)
        tp.tp_detect(e, beam)
        if ends is not None:
            ends[k].record(stream)

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize(dev)

    # ---- device-resident timed region -------------------------------------------
    tp.tp_set_profiling(e, True)
    l0 = tp.tp_engine_launches(e)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(steps):
        step(k, starts, ends)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    launches = tp.tp_engine_launches(e) - l0
    ms_local = t_start.elapsed_time(t_end)
    ms = max_over_ranks(ms_local, world, dev)
    stage_ms, nstage = tp.tp_get_stage_times(e, beam)
    tp.tp_set_profiling(e, False)
    per_block = np.array([s.elapsed_time(t) for s, t in zip(starts, ends)])
    last_block = {"detections": int(tp.tp_get_candidates(e, beam, 0)[1])}
    if args.cluster:  # what the clustering worked on (read after the timed region)
        cl, ncl, trunc = tp.tp_get_clusters(e, beam)
        last_block.update(clusters=int(ncl), candidate_clusters=int(np.count_nonzero(cl["flags"] & 1)),
                          broadband_clusters=int(np.count_nonzero(cl["flags"] & 2)), truncated=bool(trunc))
    units = len(DMS) * BLOCK * steps * world
    value = units / (ms / 1e3)

    # roofline of the dominant kernel (dedisperse_kernel, stage A4-A5): its
    # launches timed by the library with CUDA events on the beam's stream
    dd_ms = stage_ms[2] / max(nstage, 1)
    adds = len(DMS) * NCHAN * BLOCK
    traffic = TRAFFIC_BY_SHAPE.get((dtype, int(best)))
    roof = dedisp_roof(adds, dd_ms, peaks, packed=dtype == "u8", traffic=traffic,
                       traffic_note=None if traffic else f"no ncu capture of shape {best} for {dtype} data")
    roof["kernel"] = f"dedisperse_kernel (shape {best})"
    roof["stage_ms_per_block"] = {"push": stage_ms[0] / max(nstage, 1), "a1_a3": stage_ms[1] / max(nstage, 1),
                                  "a4_a5": dd_ms, "a6_a7": stage_ms[3] / max(nstage, 1)}
    # the second roof: each staged sample is read from shared memory once per
    # window that covers it (128 bytes per clock per SM)
    roof["shared_memory"] = {"peak_TBps": peaks["sms"] * 128 * peaks["sm_max_mhz"] * 1e6 / 1e12,
                             "ncu_data_path_frac": SMEM_FRAC_BY_SHAPE.get((dtype, int(best)))}

    # ---- end to end through the C ABI from pinned host buffers -------------------
    e2e = None
    if e2e_on:
        pinned = []
        tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.int16, "u8": torch.uint8,
               "c16": torch.int32}[dtype]
        for h in host:
            t = torch.empty(h.shape, dtype=tdt, pin_memory=True)
            t.numpy()[...] = _raw(h).view(t.numpy().dtype)
            pinned.append(t)
        cand_buf_cap = 1 << 20
        ncand = []
        for k in range(2):
            tp.tp_push_block(e, beam, pinned[k % NBUF])
            tp.tp_dedisperse(e, beam)
            tp.tp_detect(e, beam)
            tp.tp_get_candidates(e, beam, cand_buf_cap)
        # two page-locked result slots: block k's candidates are exported into
        # slot k % 2 on the beam's stream (no host wait), and the host reads
        # block k - 1's slot once block k's work is enqueued
        slots = [(torch.empty(cand_buf_cap * 24, dtype=torch.uint8, pin_memory=True),
                  torch.zeros(1, dtype=torch.int64, pin_memory=True),
                  torch.zeros(1, dtype=torch.int32, pin_memory=True)) for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        # the machine's host -> device copy rate for one block (pinned, 1D; the
        # leg below is bound by it when it exceeds the block's device time)
        probe = torch.empty(pinned[0].numel(), dtype=pinned[0].dtype, device=dev)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        probe.copy_(pinned[0].view(-1), non_blocking=True)
        c0.record(stream)
        for _ in range(3):
            probe.copy_(pinned[0].view(-1), non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        h2d_gbps = 3 * host[0].nbytes / (c0.elapsed_time(c1) / 1e3) / 1e9
        del probe
        tp.tp_set_profiling(e, True)  # per-stage device times of the leg's blocks
        barrier(world)
        torch.cuda.synchronize(dev)
        # double-buffered ingest: block k + 1's host -> device copy runs while
        # block k is processed; every block's copy and its candidates' copy to
        # the host lie inside the timed region
        w0 = time.perf_counter()
        ne2e = max(8, steps)

        def read(k):
            done[k % 2].synchronize()
            out, cnt, st = slots[k % 2]
            n = int(cnt.item())
            if int(st.item()) != 0:
                raise RuntimeError(f"block {k}: status {int(st.item())}")
            ncand.append(n)
            return out[:24 * min(n, cand_buf_cap)]

        for k in range(ne2e):
            tp.tp_prefetch_block(e, beam, pinned[k % NBUF])
            tp.tp_push_prefetched(e, beam)
            tp.tp_dedisperse(e, beam)
            tp.tp_detect(e, beam)
            tp.tp_export_candidates(e, beam, slots[k % 2][0], cand_buf_cap, slots[k % 2][1], slots[k % 2][2])
            done[k % 2].record(stream)
            if k > 0:
                read(k - 1)
        read(ne2e - 1)
        torch.cuda.synchronize(dev)
        w = max_over_ranks(time.perf_counter() - w0, world, dev)
        e2e_stage_ms, e2e_nstage = tp.tp_get_stage_times(e, beam)
        tp.tp_set_profiling(e, False)
        e2e = {"value": len(DMS) * BLOCK * ne2e * world / w, "unit": "DM-trial*samples/s",
               "h2d_bytes_per_step": int(host[0].nbytes),
               "d2h_bytes_per_step": int(8 + 24 * float(np.mean(ncand))), "steps": ne2e,
               "candidates_per_block": float(np.mean(ncand)), "h2d_GBps_measured": h2d_gbps,
               "h2d_ms_per_block": host[0].nbytes / (h2d_gbps * 1e9) * 1e3,
               "wall_ms_per_block": w / ne2e * 1e3,
               "stage_ms_per_block": {n: e2e_stage_ms[i] / max(e2e_nstage, 1)
                                      for i, n in enumerate(("push", "a1_a3", "a4_a5", "a6_a7"))}}

    tp.tp_beam_close(e, beam)
    tp.tp_plan_destroy(plan)
    tp.tp_engine_destroy(e)
    del dev_bufs, dev_blocks
    torch.cuda.empty_cache()
    return {"value": value, "ms": ms, "steps": steps, "warmup": warmup, "dtype": dtype, "best": int(best),
            "tune": tune, "max_delay": int(max_delay), "delays": delays, "world": world, "rank": rank,
            "last_block": last_block, "per_block": per_block, "roofline": roof, "e2e": e2e,
            "launches": int(launches), "clocks": clk, "adds_per_s": adds * steps * world / (ms / 1e3)}


def form_entry(r, fp32_adds_per_s):
    """A `forms` entry of the benchmark line: a reduced-precision or batched
    form with its own throughput, roofline and multiple over the FP32
    single-beam stream (in sample-adds per second, since the configurations
    differ in channels per trial)."""
    r = dict(r)
    r["multiple_over_fp32_adds"] = r["adds_per_s"] / fp32_adds_per_s if fp32_adds_per_s else None
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="stream: skip the other forms (8-bit stream, batch, wide band, serving)")
    ap.add_argument("--dtype", default=None, choices=["f32", "f16", "bf16", "u8", "c16"],
                    help="sample storage format (default: f32 for the metric's stream workload, binary16 for "
                         "batch8)")
    ap.add_argument("--workload", default="stream", choices=["stream", "batch8", "wide16", "serve32"],
                    help="stream: the metric's 1-beam streaming workload (with the other forms); batch8: 8 "
                         "uneven beams batched; wide16: 16 wide-band 8-bit beams; serve32: the serving loop")
    ap.add_argument("--copy-push", action="store_true",
                    help="stream: push the device-resident blocks by copy (tp_push_block) instead of in place")
    ap.add_argument("--per-beam", action="store_true",
                    help="batch8: per-beam dedisperse/detect calls instead of the batched launch")
    ap.add_argument("--speedup", type=float, default=20.0,
                    help="serve32: arrival time compression (20: about two thirds of the GPU's capacity)")
    ap.add_argument("--blocks-per-stream", type=int, default=4, help="serve32: blocks per stream")
    ap.add_argument("--hbm-gb", type=float, default=48.0, help="serve32: engine HBM budget")
    ap.add_argument("--shape", type=int, default=None,
                    help="use this kernel shape instead of autotuning")
    ap.add_argument("--median", type=int, default=1,
                    help="stream: median filter width of the post-processing (odd, 1 = off)")
    ap.add_argument("--detrend", action="store_true", help="stream: detrended detection (post-processing)")
    ap.add_argument("--cluster", action="store_true",
                    help="stream: cluster and classify every block's detections (Sec. 2.3)")
    ap.add_argument("--fit", type=int, default=-1,
                    help="stream: fitted bandpass of this polynomial order (-1 = block mean)")
    args = ap.parse_args()
    if args.dtype is None:
        args.dtype = "f16" if args.workload == "batch8" else "f32"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch8", "wide16", "serve32"):
        if args.workload == "batch8":
            r = run_batch8(args, dtype=args.dtype, steps=args.steps, warmup=max(3, args.warmup))
        elif args.workload == "wide16":
            r = run_wide16(args, steps=args.steps, warmup=max(2, args.warmup))
        else:
            r = run_serve(args)
        if int(os.environ.get("RANK", "0")) == 0:
            line = {"metric": METRIC, "value": r["value"], "unit": r["unit"], "n_gpus": args.gpus,
                    "steps": r.get("steps", r.get("blocks")), "warmup": r.get("warmup", 0),
                    "ms_per_step": r.get("ms_per_step"), "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": r["value"] / PAPER_DERIVED, "dtype": r["dtype"], "data": "synthetic",
                    "config": {"workload": r["workload"]}, **{k: v for k, v in r.items()
                                                            if k not in ("value", "unit", "workload", "dtype")}}
            print(json.dumps(line), flush=True)
        return

    s = run_stream(args, args.dtype, args.steps, args.warmup, not args.no_e2e)
    forms = None
    if not args.no_forms and s["world"] == 1:
        import torch
        peaks = device_peaks(torch.device("cuda", 0))
        forms = {}
        legs = [("stream_u8", lambda: run_stream(args, "u8", args.steps, args.warmup, False, peaks)),
                ("batch8_f16", lambda: run_batch8(args, "f16", max(8, args.steps // 2), 3, peaks)),
                ("wide16_u8", lambda: run_wide16(args, 3, 2, peaks)),
                ("serve32_u8", lambda: run_serve(args))]
        for name, fn in legs:
            try:
                r = fn()
                if name == "stream_u8":
                    r = {"workload": WORKLOAD.replace("FP32", "8-bit (int32 sums)"), "value": r["value"],
                         "unit": "DM-trial*samples/s", "dtype": "u8", "steps": r["steps"],
                         "warmup": r["warmup"], "ms_per_step": r["ms"] / r["steps"], "adds_per_s": r["adds_per_s"],
                         "kernel_shape": r["best"], "autotune_ms": r["tune"],
                         "realtime_beams": r["value"] / (len(DMS) / TSAMP), "roofline": r["roofline"],
                         "p99_block_latency_ms": float(np.percentile(r["per_block"], 99)),
                         "gpu_launches": r["launches"], "clocks": r["clocks"]}
                forms[name] = form_entry(r, s["adds_per_s"]) if "adds_per_s" in r else r
            except Exception as ex:  # a failed leg is reported, the headline still prints
                forms[name] = {"error": f"{type(ex).__name__}: {ex}"}
    if s["rank"] != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and s["world"] == 1 and args.dtype == "f32":
        cpu = cpu_baselines(s["delays"], s["max_delay"])
    dtype = args.dtype
    cfg = stream_config(s["max_delay"], s["world"])
    cfg["push"] = ("copy of each device-resident block (tp_push_block)" if args.copy_push else
                   "in place: each block in its producer's buffer, the overlap tail copied in (tp_push_inplace)")
    if dtype != "f32":
        cfg["workload"] = WORKLOAD.replace("FP32", {"f16": "binary16", "bf16": "bfloat16", "u8": "8-bit",
                                                    "c16": "complex int16 voltages detected as power"}[dtype])
    line = {"metric": METRIC, "value": s["value"], "unit": "DM-trial*samples/s", "n_gpus": s["world"],
            "steps": s["steps"], "warmup": s["warmup"], "ms_per_step": s["ms"] / s["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": s["value"] / PAPER_DERIVED,
            "dtype": dtype, "data": "synthetic", "config": cfg,
            "kernel": {"shape": s["best"], "autotune_ms": s["tune"],
                       "postprocess": {"median_width": args.median, "detrend": bool(args.detrend)},
                       "bandpass_fit_order": args.fit, "clustering": bool(args.cluster),
                       "last_block": s["last_block"]},
            "realtime_beams": s["value"] / (len(DMS) / TSAMP),
            "p50_block_latency_ms": float(np.percentile(s["per_block"], 50)),
            "p99_block_latency_ms": float(np.percentile(s["per_block"], 99)),
            "block_latency_note": "device time per block of the timed stream; serving latency is in forms",
            "block_duration_ms": BLOCK * TSAMP * 1e3,
            "roofline": s["roofline"], "cpu_baseline": cpu, "e2e": s["e2e"], "gpu_launches": s["launches"],
            "clocks": s["clocks"], "forms": forms}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
