"""Throughput benchmark of the receiver hot path on one GB300.

Workload (one step): a continuous DP-QPSK 28 GBd stream of 2^24 symbols per
polarisation (2^25 complex64 samples per polarisation, 10,000 km of
D = 17 ps/(nm km), SNR 10 dB, 100 MHz frequency offset, 100 kHz Wiener
phase noise, random polarisation rotation), pushed in 2^16-symbol blocks
with all receiver state carried across blocks, through the whole chain
(CD/OLS, timing, FO, MIMO + adaptation, BPS, decisions, demap, BER).
Every step starts a fresh stream on the same handle (rx_reset), so the
acquisition of the first frame is inside every step.  Inputs are resident
in HBM and larger than L2 (512 MiB).

Prints one JSON line.  --impl reference times the FP64 oracle on the host
cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# Hardware work queues for concurrent streams (read when the CUDA context is
# created): each receiver runs four CUDA streams, and many receivers share
# the GPU in the serving workloads; with the default 8 queues their kernels
# serialise.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max clock


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [v.strip() for v in line.split(",")]))

    def wait_first(self, timeout=5.0):
        t = time.perf_counter() + timeout
        while self.proc is not None and not self.rows and time.perf_counter() < t:
            time.sleep(0.01)

    def stop(self, t0=None, t1=None):
        """Stops sampling after a short grace period; summary of [t0, t1]."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summary(t0, t1)

    def summary(self, t0=None, t1=None):
        """Summary of the samples taken in [t0, t1] (host perf_counter
        times); when the window is shorter than the sampling period, the
        samples within one period of it."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [(t, r) for t, r in list(self.rows) if len(r) >= 7]
        if t0 is not None:
            inside = [r for t, r in rows if t0 <= t <= t1]
            rows = inside or [r for t, r in rows if t0 - 0.15 <= t <= t1 + 0.15]
        else:
            rows = [r for _, r in rows]
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def profiled_traffic(kernel):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or
    None when the kernel's sources changed since that capture."""
    import hashlib
    try:
        lines = open(os.path.join(ROOT, "profiles", "traffic.txt")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = ln.split()
        if not f or f[0].startswith("#") or f[0] != kernel:
            continue
        h = hashlib.sha256()
        for src in f[3].split(","):
            with open(os.path.join(ROOT, "paper_2108_07001_gb300", "csrc", src), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] != f[4]:
            return None
        return int(f[1]) + int(f[2])
    return None


def workload(stride=1, name=None):
    """The stream workload (default: the 28 GBd 10,000 km stream); stride > 1
    selects the two-stage blind phase search over bps_angles / stride coarse
    angles."""
    from paper_2108_07001_gb300 import workloads
    wl = workloads.STREAMS[name] if name else workloads.DP_QPSK_10000KM_STREAM
    if stride > 1:
        wl = dict(wl, rx=dict(wl["rx"], bps_coarse_stride=stride))
    return wl


def stage_work(wl, n_sym):
    """Algorithmic work per step of each stage (flops or bytes).  One step
    processes n_sym symbols per polarisation = 4 n_sym complex samples."""
    rx = wl["rx"]
    B, T = rx["bps_angles"] // rx.get("bps_coarse_stride", 1), rx["mimo_taps"]
    samples = 4 * n_sym
    return {
        # CD: each complex64 sample read once from the ring, written once
        "cd": ("hbm", samples * 16.0),
        # FIR (2 outputs x 2 inputs x T complex MACs) + gradient (same), 8 flops per CMAC
        "mimo": ("alu", n_sym * 2 * (4 * T) * 8.0),
        # per symbol, polarisation and searched angle: 7.5 flops (the count of the
        # blind phase search's arithmetic: rotation, distance to the nearest
        # point, sliding-window update)
        "bps": ("alu", n_sym * 2 * B * 7.5),
    }


def run_ours(args):
    import torch
    from paper_2108_07001_gb300 import rx

    wl = workload(args.bps_coarse_stride, args.stream)
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    if args.fft_n:  # an FFT size, or -1: the one rx_autotune_fft picks on this GPU
        n = args.fft_n if args.fft_n > 0 else rx.autotune_fft(rx.default_config(**wl["rx"]), frames=4)[0]
        wl = dict(wl, rx=dict(wl["rx"], fft_n=n))
    import rxsim
    t0 = time.time()
    lk = dict(wl["link"])
    if args.symbols:
        lk["n_sym"] = args.symbols
    sim = rxsim.simulate(rxsim.LinkConfig(**lk))
    x = sim["rx"]  # [2, 2^25] complex64
    del sim
    gen_s = time.time() - t0
    n_samp = x.shape[1]
    n_sym = n_samp // 2
    m = 2 * wl["push_syms"]
    nb = n_samp // m
    blocks = np.ascontiguousarray(x.reshape(2, nb, m).transpose(1, 0, 2))  # [nb][2][m]
    del x
    dx = torch.from_numpy(blocks).to(dev)  # resident in HBM
    stream = torch.cuda.current_stream().cuda_stream
    cfg = rx.default_config(**wl["rx"])
    r = rx.Receiver(cfg)                                 # timed for the value
    rp = rx.Receiver(rx.default_config(**wl["rx"], profile=1))  # per-stage CUDA-event timings
    lib = r.lib
    base = dx.data_ptr()
    bbytes = 2 * m * 8
    out_bytes = n_sym * 2 * cfg.modulation // 8
    outbuf = np.empty(out_bytes + 16, dtype=np.uint8)

    # the per-push arguments are built once, so the timed loop is the C-ABI
    # calls themselves (one rx_push_block per 2^16-symbol block)
    push = lib.rx_push_block
    c_stream = ctypes.c_void_p(stream)
    dev_ptrs = [ctypes.c_void_p(base + b * bbytes) for b in range(nb)]

    def step(rr):
        rr.reset()
        h = rr.h
        for p in dev_ptrs:
            rc = push(h, p, m, rx.RX_C64, 1, c_stream)
            if rc:
                raise rx.RxError(rc, lib.rx_last_error().decode())
        rr.end()
        rr.join(stream)

    def timed(rr, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        h0 = time.perf_counter()
        for _ in range(steps):
            step(rr)
        h1 = time.perf_counter()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), h0, h1

    clk = ClockSampler()
    clk.start()
    for rr in (r, rp):
        for _ in range(args.warmup):
            step(rr)
            rr.pull_bytes(outbuf)
    torch.cuda.synchronize()
    clk.wait_first()
    total_ms, host0, host1 = timed(r, args.steps)
    host_t1 = time.perf_counter()
    stats = r.stats()
    before = rp.stage_times()
    prof_ms, _, _ = timed(rp, args.steps)
    after = rp.stage_times()
    # the timed region, and (more samples) the timed and the profiled passes
    # of the same steps together
    clocks = clk.stop(host0, host_t1)
    clocks["both_passes"] = clk.summary(host0, time.perf_counter())
    stage_tot = {k: [after[k][0] - before[k][0], after[k][1] - before[k][1]] for k in rx.STAGES}
    rp.close()
    ms_step = total_ms / args.steps
    samples_step = 2 * n_samp
    bits_step = n_sym * 2 * cfg.modulation
    value = samples_step / (ms_step * 1e-3) / 1e9
    gbps = bits_step / (ms_step * 1e-3) / 1e9

    # roofline of the dominant stage (live stage timings of the timed steps);
    # the FP32 peak is measured on this GPU (scalar and packed-pair FMA)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    fma_tf, fma2_tf = rx.fp32_peak(0)
    alu_peak = max(fma_tf, fma2_tf) or FP32_PEAK_TFLOPS
    work = stage_work(wl, n_sym)
    stages = {}
    for k in ("cd", "mimo", "bps"):
        ms, n = stage_tot[k]
        bound, w = work[k]
        sec = ms * 1e-3 / args.steps
        if bound == "hbm":
            ach = w / sec / 1e9
            peak = hbm_peak or 6800.0
            unit = "GB/s"
        else:
            ach = w / sec / 1e12
            peak = alu_peak
            unit = "TFLOP/s"
        stages[k] = {"bound": bound, "achieved": round(ach, 2), "peak": round(peak, 1), "unit": unit,
                     "frac": round(ach / peak, 4), "ms_per_step": round(ms / args.steps, 3),
                     "launches_per_step": n / args.steps}
    other_ms = {k: round(v[0] / args.steps, 3) for k, v in stage_tot.items() if k not in stages}
    dom = max(stages, key=lambda k: stages[k]["ms_per_step"])
    roof = dict(stages[dom])
    roof["kernel"] = dom
    roof["traffic"] = profiled_traffic("bps2" if dom == "bps" and args.bps_coarse_stride > 1 else dom)
    if roof["traffic"] is not None:
        roof["traffic_unit"] = "bytes per launch (ncu dram read+write, profiles/traffic.txt)"
    roof.pop("launches_per_step", None)
    roof["peak_source"] = ("measured MEASURED_PEAKS.json hbm_gbs" if roof["bound"] == "hbm" and hbm_peak
                           else f"measured on this GPU by rx_fp32_peak: {fma_tf:.1f} TFLOP/s fma.rn.f32, "
                                f"{fma2_tf:.1f} fma.rn.f32x2 (the larger is the peak; derived nominal "
                                f"{FP32_PEAK_TFLOPS:.1f}: 152 SMs x 128 lanes x 2 flops x 2070 MHz)")
    if roof["traffic"] is not None:  # DRAM bytes of one launch over its live duration
        launch_s = roof["ms_per_step"] * 1e-3 / stages[dom]["launches_per_step"]
        roof["dram_gbs"] = round(roof["traffic"] / launch_s / 1e9, 1)
        if hbm_peak:
            roof["dram_frac_of_hbm"] = round(roof["dram_gbs"] / hbm_peak, 4)
    gpu_launches = int(sum(v[1] for v in stage_tot.values()))

    # e2e: the same stream from pinned host memory (taken in stream order
    # without a host wait, on_device = 2 or 3), bits read back
    if not args.e2e:
        return finish(args, wl, cfg, r, value, ms_step, n_sym, gbps, stats, roof, stages, other_ms,
                      gpu_launches, clocks, host0, host1, gen_s, None)
    hx = torch.from_numpy(blocks).pin_memory()
    hbase = hx.data_ptr()
    # Two receivers take the steps in turn, so step k's bits are read back
    # (and its statistics) while step k + 1 already runs, as a continuously
    # streaming application would; every step's input crosses from pinned
    # host memory and every step's bits come back to the host.
    r2 = rx.Receiver(cfg)
    outbufs = [np.empty_like(outbuf), np.empty_like(outbuf)]

    host_ptrs = [ctypes.c_void_p(hbase + b * bbytes) for b in range(nb)]

    def push_host_step(rr, mode):
        rr.reset()
        h = rr.h
        for p in host_ptrs:
            rc = push(h, p, m, rx.RX_C64, mode, c_stream)
            if rc:
                raise rx.RxError(rc, lib.rx_last_error().decode())
        rr.end()

    def read_back(rr, k):
        rr.pull_bytes(outbufs[k % 2], timeout_ms=-1)
        rr.stats()

    def e2e_run(mode):
        push_host_step(r, mode)
        read_back(r, 0)
        torch.cuda.synchronize()
        ke = args.steps
        e0 = time.perf_counter()
        prev = None
        for k in range(ke):
            rr = (r, r2)[k % 2]
            push_host_step(rr, mode)
            if prev is not None:
                read_back(prev, k - 1)
            prev = rr
        read_back(prev, ke - 1)
        torch.cuda.synchronize()
        return (time.perf_counter() - e0) / ke

    # on_device = 2: a copy engine moves each block into a staging slot;
    # on_device = 3: the ingest kernel reads the pinned block itself
    e_times = {mode: e2e_run(mode) for mode in (2, 3)}
    best = min(e_times, key=e_times.get)
    e_s = e_times[best]
    r2.close()
    how = {2: "copied by a copy engine into staging slots in stream order (on_device=2)",
           3: "read by the ingest kernel through the device mapping in stream order (on_device=3)"}
    e2e = {"value": round(samples_step / e_s / 1e9, 3), "unit": "Gsamples/s",
           "h2d_bytes_per_step": int(blocks.nbytes), "d2h_bytes_per_step": int(out_bytes),
           "ms_per_step": round(e_s * 1e3, 2),
           "protocol": "pinned host blocks " + how[best] + "; bits and stats read back every step, overlapped "
                       "with the next step on a second receiver",
           "forms": {f"on_device={mode}": round(samples_step / t / 1e9, 3) for mode, t in e_times.items()}}

    return finish(args, wl, cfg, r, value, ms_step, n_sym, gbps, stats, roof, stages, other_ms,
                  gpu_launches, clocks, host0, host1, gen_s, e2e)


def chain_dram(n_sym, bits_per_sym, ms_step, hbm_peak):
    """Whole-chain DRAM bytes of a step, from the ncu capture in
    profiles/traffic.txt ('chain': every kernel of one 2^20-symbol frame,
    caches not flushed between kernels), scaled to the step's frames,
    beside the algorithmic bytes (complex64 input read once, decided bits
    written once); None once the kernel sources changed since the capture."""
    per_frame = profiled_traffic("chain")
    alg = 4 * n_sym * 8 + n_sym * 2 * bits_per_sym / 8
    out = {"algorithmic_bytes_per_step": int(alg), "source": "profiles/ingest_and_chain_traffic_dp-qpsk-10000km.md"}
    if per_frame is None:
        out["measured_bytes_per_step"] = None
        return out
    meas = per_frame * n_sym / (1 << 20)
    out["measured_bytes_per_step"] = int(meas)
    out["measured_over_algorithmic"] = round(meas / alg, 2)
    out["measured_gbs"] = round(meas / (ms_step * 1e-3) / 1e9, 1)
    if hbm_peak:
        out["measured_frac_of_hbm"] = round(meas / (ms_step * 1e-3) / 1e9 / hbm_peak, 4)
    return out


def finish(args, wl, cfg, r, value, ms_step, n_sym, gbps, stats, roof, stages, other_ms,
           gpu_launches, clocks, host0, host1, gen_s, e2e):
    cpu = cpu_baseline(args.bps_coarse_stride, wl["name"]) if args.cpu_baseline else None
    batched = batched_fp16_summary(measured_peaks().get("hbm_gbs")) if args.batched else None
    qam16 = qam16_summary() if args.batched else None
    serving = serving_summary() if args.batched else None
    line = {
        "metric": "gsamples_per_s", "value": round(value, 3), "unit": "Gsamples/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded link simulator)",
        "config": {"workload": wl["name"], "symbols_per_pol": n_sym, "push_syms": wl["push_syms"],
                   "frame_syms": cfg.frame_syms,
                   "fft_n": cfg.fft_n if cfg.fft_n else "default rule (smallest power of 2 >= 4 x halo)",
                   "fft_n_from": "autotuner" if args.fft_n < 0 else ("given" if args.fft_n else "default rule"),
                   "mimo_taps": cfg.mimo_taps,
                   "bps_angles": cfg.bps_angles, "bps_search": "full" if cfg.bps_coarse_stride == 1 else
                   f"two-stage: {cfg.bps_angles // cfg.bps_coarse_stride} coarse angles + parabolic refinement",
                   "storage": "c64", "input": "resident in HBM, 512 MiB > L2",
                   "l2": "inputs larger than L2"},
        "decoded_gbps": round(gbps, 3),
        "ber": stats["ber"], "bits": stats["bits"], "bit_errors": stats["bit_errors"],
        "cycle_slips": stats["cycle_slips"], "latency_p50_ms": round(stats["latency_p50_ms"], 3),
        "latency_p99_ms": round(stats["latency_p99_ms"], 3),
        "roofline": roof, "stages": stages, "other_stage_ms": other_ms,
        "stage_timing": "per-stage CUDA events on a second, profiled handle over the same timed protocol",
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clocks,
        "batched_fp16": batched, "qam16_fp16": qam16, "serving": serving, "dram": chain_dram(n_sym, cfg.modulation, ms_step, measured_peaks().get("hbm_gbs")),
        "host_launch_s_per_step": round((host1 - host0) / args.steps, 4), "sim_seconds": round(gen_s, 1),
    }
    r.close()
    return line


ORACLE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS")


def workload_by_name(name):
    from paper_2108_07001_gb300 import workloads
    for wl in workloads.ALL:
        if wl["name"] == name:
            return wl
    raise KeyError(name)


def oracle_child(name, n_sym, reps, stride=1):
    """Runs in a child process with one BLAS/OpenMP thread: simulates the
    first n_sym symbols of the named workload's link once (complex64
    samples, as the GPU forms receive them), then times the FP64 oracle on
    them reps times.  Prints {"times": [...], "ber": {...}} as JSON."""
    import rxsim
    from oracle import rx_oracle as O
    from paper_2108_07001_gb300.workloads import oracle_kwargs
    wl = workload_by_name(name)
    lk = dict(wl["link"])
    lk["n_sym"] = n_sym
    lk["out_dtype"] = "c64"
    sim = rxsim.simulate(rxsim.LinkConfig(**lk))
    x = sim["rx"].astype(np.complex128)
    del sim
    kw = oracle_kwargs(wl["rx"])
    if stride > 1:
        kw["bps_coarse_stride"] = stride
    times, res = [], None
    for _ in range(reps):
        t0 = time.perf_counter()
        res = O.Receiver(O.RxConfig(**kw)).run(x)
        times.append(time.perf_counter() - t0)
    b = res["ber"]
    print(json.dumps({"times": times, "ber": {"errors": int(b["errors"]), "bits": int(b["bits"]),
                                              "slips": int(b["slips"]), "ber": float(b["ber"]),
                                              "evm": float(b["evm"])}}), flush=True)


def oracle_run(n_sym, reps, name=None, stride=1):
    """Oracle run times (and the last run's BER counters) on the host cores,
    measured in a fresh single-threaded process (fork+exec, so safe after
    CUDA initialisation)."""
    env = dict(os.environ)
    for k in ORACLE_THREAD_ENV:
        env[k] = "1"
    name = name or workload()["name"]
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", name, str(n_sym), str(reps),
                          str(stride)],
                         env=env, capture_output=True, text=True, check=True, cwd=ROOT)
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_times(n_sym, reps, stride=1):
    return oracle_run(n_sym, reps, stride=stride)["times"]


CPU_BASELINE_SYMS = 1 << 20  # one full frame, acquisition included (10-30 s of one core)


def cpu_baseline(stride=1, name=None):
    t = oracle_run(CPU_BASELINE_SYMS, 1, name, stride)["times"][0]
    v = 4 * CPU_BASELINE_SYMS / t / 1e9
    return {"value": round(v, 6), "unit": "Gsamples/s", "cores": 1, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"first {CPU_BASELINE_SYMS} symbols/pol of the workload (one whole frame incl. "
                      f"acquisition), FP64 numpy oracle, one thread of the host's {os.cpu_count()}, {t:.1f} s"}


REFERENCE_STEP_SYMS = 1 << 18


def run_reference(args):
    wl = workload()
    # ~1.6 s of one core per 2^18-symbol step: smaller samples for long runs,
    # so that the whole run stays within a few minutes
    n_sym = REFERENCE_STEP_SYMS if args.steps + args.warmup <= 40 else REFERENCE_STEP_SYMS // 4
    times = oracle_times(n_sym, args.warmup + args.steps)[args.warmup:]
    t = sum(times) / len(times)
    v = 4 * n_sym / t / 1e9
    return {"impl": "reference", "metric": "gsamples_per_s", "value": round(v, 6), "unit": "Gsamples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded link simulator)",
            "config": {"workload": wl["name"], "sample_symbols_per_pol": n_sym},
            "cpu_baseline": {"value": round(v, 6), "unit": "Gsamples/s", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"first {n_sym} symbols/pol of the workload per step, one thread of the "
                                       f"host's {os.cpu_count()}"},
            "e2e": {"value": round(v, 6), "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_qam16(args):
    """DP-16QAM 32 GBd, 2^22 symbols, 5,000 km, 18 dB: the same complex64
    samples through the FP32-storage path and the FP16-storage path (FP32
    arithmetic), pushed in 2^18-symbol blocks from HBM, against the FP64
    oracle on the same samples: throughput, BER and EVM of each form and
    the EVM penalty of each GPU form over the oracle."""
    import torch
    import rxsim
    from paper_2108_07001_gb300 import rx, workloads
    wl = workloads.DP_16QAM_5000KM
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    lk = dict(wl["link"])
    lk["out_dtype"] = "c64"
    if args.symbols:
        lk["n_sym"] = args.symbols
    x = rxsim.simulate(rxsim.LinkConfig(**lk))["rx"]
    n_samp = x.shape[1]
    n_sym = n_samp // 2
    push_syms = min(1 << 18, n_sym)
    m = 2 * push_syms
    nb = n_samp // m
    blocks = np.ascontiguousarray(x[:, :nb * m].reshape(2, nb, m).transpose(1, 0, 2))
    dx64 = torch.from_numpy(blocks).to(dev)
    dx16 = torch.from_numpy(np.stack([blocks.real, blocks.imag], axis=-1).astype(np.float16)).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    forms = {}
    for form, storage, dtype, data, esz in (("fp32_storage", rx.RX_C64, rx.RX_C64, dx64, 8),
                                            ("fp16_storage", rx.RX_C16, rx.RX_C16, dx16, 4)):
        cfg = rx.default_config(**wl["rx"], storage_dtype=storage, max_block_samples=m)
        r = rx.Receiver(cfg)
        base, bbytes = data.data_ptr(), 2 * m * esz

        def step():
            r.reset()
            for b in range(nb):
                rc = r.lib.rx_push_block(r.h, ctypes.c_void_p(base + b * bbytes), m, dtype, 1, ctypes.c_void_p(stream))
                if rc:
                    raise rx.RxError(rc, r.lib.rx_last_error().decode())
            r.end()
            r.join(stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        st = r.stats()
        forms[form] = {"value": round(2 * n_samp / (ms * 1e-3) / 1e9, 3), "unit": "Gsamples/s",
                       "ms_per_step": round(ms, 3), "ber": st["ber"], "bit_errors": st["bit_errors"],
                       "bits": st["bits"], "cycle_slips": st["cycle_slips"], "evm": st["evm"],
                       "evm_db": round(10 * math.log10(st["evm"]), 3) if st["evm"] > 0 else None}
        r.close()
    orc = oracle_run(n_sym, 1, wl["name"])
    ob = orc["ber"]
    oracle = {"ber": ob["ber"], "bit_errors": ob["errors"], "bits": ob["bits"], "cycle_slips": ob["slips"],
              "evm": ob["evm"], "evm_db": round(10 * math.log10(ob["evm"]), 3), "cores": 1,
              "seconds": round(orc["times"][0], 1)}
    for f in forms.values():
        f["evm_penalty_db"] = round(f["evm_db"] - oracle["evm_db"], 4) if f["evm_db"] is not None else None
    return {"metric": "gsamples_per_s", "value": forms["fp16_storage"]["value"], "unit": "Gsamples/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "workload": "qam16", "dtype": "f16 storage, f32 arithmetic", "data": "synthetic (seeded link simulator)",
            "config": {"workload": wl["name"], "symbols_per_pol": n_sym, "push_syms": push_syms,
                       "mimo_taps": wl["rx"]["mimo_taps"], "bps_angles": wl["rx"]["bps_angles"],
                       "bps_half_window": wl["rx"]["bps_half_window"]},
            "forms": forms, "oracle": oracle, "cpu_baseline": {
                "value": round(4 * n_sym / orc["times"][0] / 1e9, 6), "unit": "Gsamples/s", "cores": 1,
                "kind": "oracle", "sample": f"the whole {n_sym}-symbol stream, FP64 numpy oracle, one thread"}}


KK_BUFFER = 1 << 22        # samples per ADC buffer (the paper's)
KK_BUFFERS_PER_STEP = 16   # 2^26 samples = 128 MiB of codes per step (> L2)


def kk_link(n_samples):
    """The paper's single-polarisation link (1 GBd QPSK, 1 % roll-off, 4 GS/s,
    CSPR 12 dB) over 1,000 km at an optical SNR of 8 dB per 4-sps sample
    (BER ~3e-4 after the chain).  The simulator's output is periodic in its
    length when the tone offset makes a whole number of turns over it, so
    the tone sits 0.515625 GHz from the signal centre (the paper: 0.516
    GHz), 33 x 2^15 turns over 2^23 samples, and a short simulation tiles
    into a continuous stream."""
    import rxsim
    return rxsim.simulate_kk(rxsim.KKLinkConfig(n_sym=n_samples // 4, fiber_len_m=1000e3, cspr_db=12.0,
                                                snr_db=8.0, f_c_hz=0.515625e9, seed=2108, prbs_seed=2108))


def kk_oracle_child(n_samples):
    """Child process (one thread): times the FP64 oracle of the whole KK
    receiver on n_samples codes (the bench's receiver settings)."""
    import rxsim
    from oracle import kk_oracle as K
    d = kk_link(n_samples)
    b2 = rxsim.beta2_from_dispersion(17.0, 1550e-9)
    t0 = time.perf_counter()
    K.kk_receive(d["codes"], d["gain"], d["offset"], d["fs"], d["f_c"], 1024, 1024, 1e9, 0.01, b2, 1000e3, 2, 5e-3,
                 64, 512, n_samples // 4, 8192)
    print(json.dumps({"seconds": time.perf_counter() - t0}), flush=True)


def run_kk(args):
    """The paper's KK receiver (Sec. II) on 2^22-sample buffers of 12-bit ADC
    codes at 4 GS/s: sqrt/log, the 1024-point 100 % overlap-save Hilbert
    transform, field reconstruction and downshift, the static equaliser with
    4 -> 2 sps resampling, the widely-linear DD-LMS and the decisions.  A step
    is 16 buffers (2^26 samples, 2^24 symbols) from HBM to packed bits in HBM
    (the value); the front end alone (codes to the complex64 field) is timed
    beside it and is the roofline's kernel; the end-to-end form takes the
    codes from page-locked host memory and returns the bits to it."""
    import torch
    from paper_2108_07001_gb300 import rx
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    t0 = time.time()
    d = kk_link(2 * KK_BUFFER)
    nbuf = KK_BUFFERS_PER_STEP
    codes = np.tile(d["codes"], nbuf // 2)
    gen_s = time.time() - t0
    n = codes.size
    dc = torch.from_numpy(codes).to(dev)
    out = torch.empty(n, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    fe = rx.KKFrontEnd(fs_hz=d["fs"], f_shift_hz=d["f_c"], adc_gain=d["gain"], adc_offset=d["offset"], fft_n=1024,
                       max_block_samples=KK_BUFFER)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nbuf)]

    def step(profile=False):
        fe.reset()
        pos = 0
        for b in range(nbuf):
            if profile:
                evs[b][0].record()
            pos += fe.push_device(dc.data_ptr() + 2 * b * KK_BUFFER, KK_BUFFER, out.data_ptr() + 8 * pos, n - pos,
                                  stream)
            if profile:
                evs[b][1].record()
        pos += fe.end(out.data_ptr() + 8 * pos, n - pos, stream)
        return pos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler()
    clk.start()
    clk.wait_first()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    h0 = time.perf_counter()
    for _ in range(args.steps):
        assert step() == n
    ev1.record()
    torch.cuda.synchronize()
    h1 = time.perf_counter()
    clocks = clk.stop(h0, h1)
    ms = ev0.elapsed_time(ev1) / args.steps
    value = n / (ms * 1e-3) / 1e9
    # per-push device time (one field launch of 2^22 samples + a carry copy of < 1024 codes)
    push_ms = []
    for _ in range(max(1, min(args.steps, 5))):
        step(profile=True)
        torch.cuda.synchronize()
        push_ms += [a.elapsed_time(b) for a, b in evs]
    launch_s = float(np.mean(push_ms)) * 1e-3
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    alg_bytes = KK_BUFFER * (2 + 8)
    ach = alg_bytes / launch_s / 1e9
    roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": round(hbm_peak, 1), "unit": "GB/s",
            "frac": round(ach / hbm_peak, 4), "kernel": "kk_kernel<1024>",
            "algorithmic_bytes_per_launch": alg_bytes, "launch_us": round(launch_s * 1e6, 2),
            "traffic": profiled_traffic("kk"),
            "peak_source": "measured MEASURED_PEAKS.json hbm_gbs" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s"}
    # parity spot check of the timed output against the oracle (one segment per buffer)
    from oracle import kk_oracle as K
    got = out.cpu().numpy()
    I = K.adc_to_intensity(codes, d["gain"], d["offset"])
    worst = 0.0
    for b in range(nbuf):
        s0 = b * KK_BUFFER + 3 * 512 * (b + 1)
        w0 = s0 - 512
        f = K.kk_field_from_intensity(I[w0:w0 + 1536], 0.5 * d["gain"], 1024, d["f_c"] / d["fs"], t0=w0)
        ref = f[512:1024]
        worst = max(worst, float(np.abs(got[s0:s0 + 512] - ref).max() / np.abs(ref).max()))
    fe.close()
    # the whole receiver: codes -> field -> static equaliser (4 -> 2 sps) -> widely-linear DD-LMS -> bits;
    # one frame of 2^20 symbols per 2^22-sample buffer, the acquisition inside every step
    n_sym = n // 4
    bits = torch.zeros(n_sym * 2 // 8, dtype=torch.uint8, device=dev)
    rcv = rx.KKReceiver(fe=dict(fs_hz=d["fs"], f_shift_hz=d["f_c"], adc_gain=d["gain"], adc_offset=d["offset"],
                                fft_n=1024, max_block_samples=KK_BUFFER),
                        baud_hz=1e9, modulation=2, fiber_len_m=1000e3, rrc_rolloff=0.01, eq_fft_n=1024, mu=5e-3,
                        seg_syms=512, frame_syms=KK_BUFFER // 4, acq_syms=8192)

    def chain_step():
        rcv.reset()
        nb = 0
        for b in range(nbuf):
            nb += rcv.push_device(dc.data_ptr() + 2 * b * KK_BUFFER, KK_BUFFER, bits.data_ptr() + nb // 8,
                                  bits.numel() - nb // 8, stream)
        nb += rcv.end(bits.data_ptr() + nb // 8, bits.numel() - nb // 8, stream)
        return nb

    for _ in range(args.warmup):
        chain_step()
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        assert chain_step() == 2 * n_sym
    ev1.record()
    torch.cuda.synchronize()
    cms = ev0.elapsed_time(ev1) / args.steps
    # end to end: the codes from page-locked host memory (copied in stream
    # order), the bits back to page-locked host memory, every step
    e2e = None
    if args.e2e:
        hc = torch.from_numpy(codes).pin_memory()
        hb = torch.empty(bits.numel(), dtype=torch.uint8).pin_memory()

        def e2e_step():
            rcv.reset()
            nb = 0
            for b in range(nbuf):
                nb += rcv.push_host(hc[b * KK_BUFFER:(b + 1) * KK_BUFFER].numpy(), bits.data_ptr() + nb // 8,
                                    bits.numel() - nb // 8, stream)
            nb += rcv.end(bits.data_ptr() + nb // 8, bits.numel() - nb // 8, stream)
            hb.copy_(bits, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e_s = (time.perf_counter() - e0) / args.steps
        e2e = {"value": round(n / e_s / 1e9, 3), "unit": "Gsamples/s", "h2d_bytes_per_step": 2 * n,
               "d2h_bytes_per_step": int(bits.numel()), "ms_per_step": round(e_s * 1e3, 2),
               "protocol": "codes from page-locked host memory (copied in stream order), the packed bits back "
                           "to page-locked host memory"}
    rcv.close()
    tx = np.tile(d["bits"], nbuf // 2)
    got_bits = np.unpackbits(bits.cpu().numpy())
    a0, e0 = 2 * 8192, got_bits.size - 2 * 64
    ber = float(np.mean(got_bits[a0:e0] != tx[a0:e0]))
    receiver = {"value": round(n / (cms * 1e-3) / 1e9, 3), "unit": "Gsamples/s", "ms_per_step": round(cms, 3),
                "decoded_gbps": round(2 * n_sym / (cms * 1e-3) / 1e9, 3), "ber": ber,
                "x_paper_realtime_rate": round(n / (cms * 1e-3) / 1e9 / 4.0, 1),
                "stages": "KK field, static equaliser 1024-point with 4 -> 2 sps, widely-linear DD-LMS "
                          "(4 taps, 512-symbol segments), decisions, Gray bits; acquisition of 8192 symbols "
                          "inside every step"}
    cpu = None
    if args.cpu_baseline:
        env = dict(os.environ)
        for k in ORACLE_THREAD_ENV:
            env[k] = "1"
        m = KK_BUFFER
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--kk-oracle-child", str(m)], env=env,
                           capture_output=True, text=True, check=True, cwd=ROOT)
        sec = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
        cpu = {"value": round(m / sec / 1e9, 6), "unit": "Gsamples/s", "cores": 1, "kind": "oracle",
               "sample": f"one {m}-sample buffer through the whole receiver, FP64 numpy oracle, one thread, "
                         f"{sec:.1f} s"}
    return {"metric": "gsamples_per_s", "value": receiver["value"], "unit": "Gsamples/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": receiver["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "workload": "kk",
            "dtype": "f32 (int16 codes in, packed bits out)", "receiver": receiver,
            "frontend_only": {"value": round(value, 3), "unit": "Gsamples/s", "ms_per_step": round(ms, 3),
                              "output": "complex64 field"},
            "data": "synthetic (seeded minimum-phase link simulator)",
            "config": {"workload": "kk-frontend-1gbd-4gsps-2^22-buffers", "fft_n": 1024,
                       "buffers_per_step": nbuf, "samples_per_buffer": KK_BUFFER, "cspr_db": 10.0,
                       "input": "resident in HBM, 128 MiB > L2", "l2": "inputs larger than L2"},
            "x_paper_realtime_rate": receiver["x_paper_realtime_rate"], "frontend_max_rel_err_vs_oracle": worst,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            # per receiver step: per buffer the field, its carry, the equaliser, its carry and one DD-LMS
            # frame; the acquisition; at the end the field and the equaliser
            "gpu_launches": (5 * nbuf + 3) * args.steps,
            "clocks": clocks, "sim_seconds": round(gen_s, 1)}


KKB_CHANNELS = 64
KKB_ROUNDS = 64


def run_kk_batch(args):
    """Many KK front ends with small, uneven buffers (low latency): 64
    channels, each round pushing 2^12..2^16 codes per channel (drawn per
    channel and round), as one graph replay per round (rx_kk_batch_push)
    and as one push per channel (rx_kk_push): throughput and host time per
    round."""
    import torch
    from paper_2108_07001_gb300 import rx
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    d = kk_link(1 << 23)
    codes = torch.from_numpy(d["codes"]).to(dev)  # every channel reads its own window of one link
    rng = np.random.default_rng(5)
    sizes = rng.integers(1 << 12, (1 << 16) + 1, (KKB_ROUNDS, KKB_CHANNELS))
    total = int(sizes.sum())
    starts = [int(s) for s in rng.integers(0, (1 << 23) - int(sizes.sum(axis=0).max()), KKB_CHANNELS)]
    cap = int(sizes.sum(axis=0).max()) + 2048
    out = torch.empty((KKB_CHANNELS, cap), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    fcfg = dict(fs_hz=d["fs"], f_shift_hz=d["f_c"], adc_gain=d["gain"], adc_offset=d["offset"], fft_n=1024,
                max_block_samples=1 << 16)
    base = codes.data_ptr()
    obase = out.data_ptr()
    row = cap * 8

    def run(mode):
        fes = [rx.KKFrontEnd(**fcfg) for _ in range(KKB_CHANNELS)]
        batch = rx.KKBatch(fes) if mode == "batch" else None
        pin = list(starts)
        pout = [0] * KKB_CHANNELS
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        h0 = time.perf_counter()
        for r in range(KKB_ROUNDS):
            if batch is not None:
                got = batch.push([base + 2 * pin[c] for c in range(KKB_CHANNELS)], [int(x) for x in sizes[r]],
                                 [obase + c * row + 8 * pout[c] for c in range(KKB_CHANNELS)],
                                 [cap - pout[c] for c in range(KKB_CHANNELS)], stream)
            else:
                got = [fes[c].push_device(base + 2 * pin[c], int(sizes[r, c]), obase + c * row + 8 * pout[c],
                                          cap - pout[c], stream) for c in range(KKB_CHANNELS)]
            for c in range(KKB_CHANNELS):
                pin[c] += int(sizes[r, c])
                pout[c] += got[c]
        h1 = time.perf_counter()
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        res = out[:, :min(pout)].clone()
        if batch is not None:
            batch.close()
        for f in fes:
            f.close()
        return ms, (h1 - h0) * 1e3, res

    forms = {}
    results = {}
    for mode in ("per_channel", "batch"):
        run(mode)  # warm-up
        ms, host_ms, res = run(mode)
        results[mode] = res
        forms[mode] = {"gsamples_s": round(total / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3),
                       "host_ms": round(host_ms, 3), "launches": KKB_ROUNDS * (1 if mode == "batch" else
                                                                                2 * KKB_CHANNELS)}
    same = bool(torch.equal(results["batch"], results["per_channel"]))
    return {"metric": "gsamples_per_s", "value": forms["batch"]["gsamples_s"], "unit": "Gsamples/s", "n_gpus": 1,
            "higher_is_better": True, "workload": "kk_batch", "dtype": "f32 (int16 codes in, c64 field out)",
            "data": "synthetic (seeded minimum-phase link simulator)",
            "config": {"channels": KKB_CHANNELS, "rounds": KKB_ROUNDS, "codes_per_push": "2^12..2^16 per channel",
                       "codes_total": total, "fft_n": 1024},
            "forms": forms, "x_per_channel": round(forms["batch"]["gsamples_s"] / forms["per_channel"]["gsamples_s"], 2),
            "batch_equals_per_channel": same}


def run_kkrx_batch(args):
    """Many whole KK receivers with small, uneven buffers: 64 receivers
    (frames of 2^16 symbols = 65 us of signal, acquisition 4096), each round pushing
    2^12..2^16 codes per receiver, as one batch push per round
    (rx_kkrx_batch_push: a front-end graph, an equaliser graph, the DD-LMS
    of completed frames) and as one push per receiver (rx_kkrx_push), all
    streams ended; throughput, host time, and the bits of both forms."""
    import torch
    from paper_2108_07001_gb300 import rx
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    d = kk_link(1 << 23)
    codes = torch.from_numpy(d["codes"]).to(dev)
    rng = np.random.default_rng(6)
    sizes = rng.integers(1 << 12, (1 << 16) + 1, (KKB_ROUNDS, KKB_CHANNELS))
    per = sizes.sum(axis=0)
    total = int(per.sum())
    # windows start on multiples of 256 samples: whole symbols, and whole turns of the tone offset
    # (33/256 of a turn per sample), so each receiver's downshift matches the link's phase
    starts = [256 * (int(s) // 256) for s in rng.integers(0, (1 << 23) - int(per.max()), KKB_CHANNELS)]
    nbytes = int(per.max()) // 4 * 2 // 8 + 4096
    bits = torch.zeros((KKB_CHANNELS, nbytes), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    base, bbase = codes.data_ptr(), bits.data_ptr()
    fe = dict(fs_hz=d["fs"], f_shift_hz=d["f_c"], adc_gain=d["gain"], adc_offset=d["offset"], fft_n=1024,
              max_block_samples=1 << 16)
    rcfg = dict(baud_hz=1e9, modulation=2, fiber_len_m=1000e3, rrc_rolloff=0.01, eq_fft_n=1024, mu=5e-3, seg_syms=512,
                frame_syms=1 << 16, acq_syms=4096)

    def run(mode):
        rcvs = [rx.KKReceiver(fe=fe, **rcfg) for _ in range(KKB_CHANNELS)]
        batch = rx.KKReceiverBatch(rcvs) if mode == "batch" else None
        pin = list(starts)
        nb = [0] * KKB_CHANNELS
        bits.zero_()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        h0 = time.perf_counter()
        for r in range(KKB_ROUNDS):
            if batch is not None:
                got = batch.push([base + 2 * pin[c] for c in range(KKB_CHANNELS)], [int(x) for x in sizes[r]],
                                 [bbase + c * nbytes + nb[c] // 8 for c in range(KKB_CHANNELS)],
                                 [nbytes - nb[c] // 8 for c in range(KKB_CHANNELS)], stream)
            else:
                got = [rcvs[c].push_device(base + 2 * pin[c], int(sizes[r, c]), bbase + c * nbytes + nb[c] // 8,
                                           nbytes - nb[c] // 8, stream) for c in range(KKB_CHANNELS)]
            for c in range(KKB_CHANNELS):
                pin[c] += int(sizes[r, c])
                nb[c] += got[c]
        if batch is not None:
            batch.close()
        for c in range(KKB_CHANNELS):
            nb[c] += rcvs[c].end(bbase + c * nbytes + nb[c] // 8, nbytes - nb[c] // 8, stream)
        h1 = time.perf_counter()
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        for r_ in rcvs:
            r_.close()
        return ms, (h1 - h0) * 1e3, bits.clone(), nb

    forms, out = {}, {}
    for mode in ("per_channel", "batch"):
        run(mode)  # warm-up
        ms, host_ms, b, nb = run(mode)
        out[mode] = (b, nb)
        forms[mode] = {"gsamples_s": round(total / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 3),
                       "host_ms": round(host_ms, 3)}
    same = bool(torch.equal(out["batch"][0], out["per_channel"][0])) and out["batch"][1] == out["per_channel"][1]
    # BER of channel 0 against the transmitted bits of its window
    sym0 = starts[0] // 4
    tx = np.tile(d["bits"], 2)[2 * sym0:2 * sym0 + out["batch"][1][0]]
    got0 = np.unpackbits(out["batch"][0][0].cpu().numpy())[:out["batch"][1][0]]
    ber0 = float(np.mean(got0[2 * 4096:-256] != tx[2 * 4096:-256]))
    return {"metric": "gsamples_per_s", "value": forms["batch"]["gsamples_s"], "unit": "Gsamples/s", "n_gpus": 1,
            "higher_is_better": True, "workload": "kkrx_batch", "dtype": "f32 (int16 codes in, packed bits out)",
            "data": "synthetic (seeded minimum-phase link simulator)",
            "config": {"receivers": KKB_CHANNELS, "rounds": KKB_ROUNDS, "codes_per_push": "2^12..2^16 per receiver",
                       "codes_total": total, "frame_syms": 1 << 16, "fft_n": 1024, "eq_fft_n": 1024},
            "forms": forms, "x_per_channel": round(forms["batch"]["gsamples_s"] / forms["per_channel"]["gsamples_s"], 2),
            "batch_equals_per_channel": same, "ber_receiver0": ber0}


def combine_replicas(line, world, reduce_max):
    """Whole-job line of N independent replicas: the step time (and the
    end-to-end step time) is the maximum over ranks (reduce_max: list of
    floats -> element-wise max over ranks, a collective every rank calls)
    and the value counts the samples of every rank."""
    e2e = line.get("e2e")
    ms, e2e_ms = reduce_max([float(line["ms_per_step"]), float(e2e["ms_per_step"]) if e2e else 0.0])
    out = dict(line)
    samples = world * 4 * line["config"]["symbols_per_pol"]
    out["n_gpus"] = world
    out["ms_per_step"] = ms
    out["value"] = round(samples / (ms * 1e-3) / 1e9, 3)
    out["config"] = dict(line["config"], parallelism=f"replicas x{world}")
    if e2e:
        out["e2e"] = dict(e2e, ms_per_step=e2e_ms, value=round(samples / (e2e_ms * 1e-3) / 1e9, 3),
                          h2d_bytes_per_step=e2e["h2d_bytes_per_step"] * world,
                          d2h_bytes_per_step=e2e["d2h_bytes_per_step"] * world)
    return out


def shard_streams(costs, world):
    """Streams to ranks, greedy by cost (e.g. Gsamples): the costliest
    stream first, each to the rank with the least cost so far (the lowest
    rank on a tie).  Returns every rank's stream indices, ascending."""
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(o) for o in out]


def combine_shards(part, world, reduce_max, reduce_sum):
    """Whole-job line of a stream-sharded run (every rank ran its own
    streams on its own GPU, no collective on the data path): the wall time
    is the slowest rank's, samples, streams, synced streams, slips and
    launches add up, the BER is the worst stream's.  reduce_max /
    reduce_sum: list of floats -> element-wise max / sum over ranks, a
    collective every rank calls."""
    wall_ms, ber_max = reduce_max([float(part["wall_ms"]), float(part["ber_max"])])
    samples, streams, synced, slips, launches = reduce_sum(
        [float(part["samples"]), float(part["streams"]), float(part["synced_streams"]),
         float(part["cycle_slips"]), float(part["launches"])])
    return {"metric": "gsamples_per_s", "value": round(samples / (wall_ms * 1e-3) / 1e9, 3), "unit": "Gsamples/s",
            "n_gpus": world, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "workload": "batched", "form": part["form"], "dtype": part.get("dtype", "f32"),
            "data": "synthetic (seeded link simulator)", "wall_ms": round(wall_ms, 3),
            "config": {"streams": int(streams), "parallelism": f"streams sharded x{world} (greedy by Gsamples)",
                       "symbols_per_pol_per_stream": part["symbols_per_pol_per_stream"]},
            "synced_streams": int(synced), "cycle_slips": int(slips), "ber_max": ber_max, "launches": int(launches)}


SERVING_STREAMS = 16
SERVING_SYMS = 1 << 21       # symbols per polarisation per stream
SERVING_FRAME = 1 << 18


def serving_streams(n_streams, n_sym):
    """16 channel streams: DP-QPSK and DP-16QAM alternating, baud rates
    28-64 GBd, 10,000 km of D = 17 ps/(nm km), capture blocks of 2^16-2^20
    symbols.  Seeds: 1004 * 1000 + stream index."""
    rng = np.random.default_rng(1004)
    bauds = [28e9, 32e9, 40e9, 48e9, 56e9, 64e9]
    out = []
    for i in range(n_streams):
        qam = i % 2 == 1
        baud = bauds[int(rng.integers(len(bauds)))]
        seed = 1004 * 1000 + i
        link = dict(baud_hz=baud, bits_per_sym=4 if qam else 2, n_sym=n_sym, fiber_len_m=10000e3,
                    snr_db=18.0 if qam else 11.0, prbs_seed=seed, seed=seed, out_dtype="c64")
        rxc = dict(baud_hz=baud, modulation=4 if qam else 2, fiber_len_m=10000e3,
                   mimo_taps=25 if qam else 15, bps_angles=32 if qam else 64, bps_half_window=32 if qam else 16,
                   frame_syms=SERVING_FRAME, prbs_seed=seed, max_block_samples=2 << 20)
        if qam:
            rxc["mu_dd"] = 2e-3
        sizes, left = [], n_sym
        while left:
            m = min(left, 1 << int(rng.integers(16, 21)))
            sizes.append(m)
            left -= m
        out.append((link, rxc, sizes))
    return out


def run_serving(args):
    """The serving layer under load: 16 mixed channel streams (configs as in
    serving_streams) on one GPU.  First the capacity (every block submitted
    at once), then blocks arriving as one Poisson process at 80 % of that
    capacity (arrival order interleaves the streams, each stream's blocks
    in order): sustained throughput and p50/p99 frame latency, for FP32 and
    FP16 sample storage."""
    import torch
    import rxsim
    from paper_2108_07001_gb300 import rx
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    n_sym = args.symbols or SERVING_SYMS
    streams = serving_streams(SERVING_STREAMS, n_sym)
    data = []
    t0 = time.time()
    for link, rxc, sizes in streams:
        x = rxsim.simulate(rxsim.LinkConfig(**link))["rx"]
        blocks, a = [], 0
        for m in sizes:
            blocks.append(torch.from_numpy(np.ascontiguousarray(x[:, 2 * a:2 * (a + m)])).to(dev))
            a += m
        data.append(blocks)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    total_samples = 4 * n_sym * len(streams)
    bits_per_pass = sum(2 * rxc["modulation"] * n_sym for _, rxc, _ in streams)
    order = [(i, j) for j in range(max(len(b) for b in data)) for i in range(len(streams)) if j < len(data[i])]

    def one_pass(storage, arrivals, batch=0):
        with rx.Server(max_streams=64, batch=batch) as srv:
            sids = [srv.open(**dict(rxc, storage_dtype=storage)) for _, rxc, _ in streams]
            t_start = time.perf_counter()
            for k, (i, j) in enumerate(order):
                if arrivals is not None:
                    while time.perf_counter() - t_start < arrivals[k]:
                        pass
                b = data[i][j]
                srv.submit_device(sids[i], b.data_ptr(), b.shape[1], rx.RX_C64)
            for sid in sids:
                srv.end(sid)
            for sid in sids:
                srv.sync(sid, timeout_ms=600000)
            wall = time.perf_counter() - t_start
            st = srv.stats()
            ber = [srv.stream_stats(sid) for sid in sids]
        return wall, st, ber

    forms = {}
    for form, storage, batch in (("fp32_storage", rx.RX_C64, 0), ("fp16_storage", rx.RX_C16, 0),
                                 ("batched_fp32_storage", rx.RX_C64, 1), ("batched_fp16_storage", rx.RX_C16, 1)):
        one_pass(storage, None, batch)  # warm-up
        wall, st, ber = one_pass(storage, None, batch)
        cap = total_samples / wall / 1e9
        rate = 0.8 * cap * 1e9  # samples/s offered
        rng = np.random.default_rng(7)
        sizes = [4 * streams[i][2][j] for i, j in order]
        gaps = rng.exponential(np.asarray(sizes, dtype=np.float64) / rate)
        arrivals = np.cumsum(gaps) - gaps[0]
        wall_l, st_l, ber_l = one_pass(storage, arrivals, batch)
        forms[form] = {
            "capacity_gsamples_s": round(cap, 3),
            "offered_gsamples_s": round(0.8 * cap, 3),
            "sustained_gsamples_s": round(total_samples / wall_l / 1e9, 3),
            "sustained_decoded_gbps": round(bits_per_pass / wall_l / 1e9, 3),
            "latency_p50_ms": round(st_l["latency_p50_ms"], 3), "latency_p99_ms": round(st_l["latency_p99_ms"], 3),
            "latency_max_ms": round(st_l["latency_max_ms"], 3), "latency_samples": st_l["latency_samples"],
            "capacity_latency_p50_ms": round(st["latency_p50_ms"], 3),
            "capacity_latency_p99_ms": round(st["latency_p99_ms"], 3),
            "ber_max": max(b["ber"] for b in ber_l), "cycle_slips": int(sum(b["cycle_slips"] for b in ber_l)),
            "synced_streams": int(sum(b["synced"] for b in ber_l)),
            "mem_gib": round(st_l["mem_in_use_bytes"] / 2 ** 30, 2) if st_l["mem_in_use_bytes"] else None,
            "batch_calls": st_l["batch_calls"],
        }
    return {"metric": "gsamples_per_s", "value": forms["batched_fp16_storage"]["sustained_gsamples_s"],
            "value_form": "batched_fp16_storage", "unit": "Gsamples/s",
            "n_gpus": 1, "higher_is_better": True, "workload": "serving", "dtype": "f32 arithmetic",
            "data": "synthetic (seeded link simulator)",
            "config": {"streams": len(streams), "symbols_per_pol_per_stream": n_sym,
                       "baud_gbd": [s[0]["baud_hz"] / 1e9 for s in streams],
                       "modulation": ["16qam" if s[1]["modulation"] == 4 else "qpsk" for s in streams],
                       "fiber_km": 10000, "blocks": len(order), "block_syms": "2^16..2^20",
                       "frame_syms": SERVING_FRAME, "arrivals": "Poisson at 0.8 x capacity"},
            "forms": forms, "sim_seconds": round(gen_s, 1)}


BATCH_STREAMS = 64
BATCH_SYMS = 1 << 19
BATCH_FRAME = 1 << 16


def batched_streams(n_streams, n_sym):
    """64 independent DP-QPSK streams: 28-64 GBd, 1,000-10,000 km, SNR
    9-14 dB, capture blocks of 2^12-2^18 symbols.  Seeds 1003 * 1000 + i."""
    rng = np.random.default_rng(1003)
    bauds = [28e9, 32e9, 40e9, 48e9, 56e9, 64e9]
    out = []
    for i in range(n_streams):
        baud = bauds[int(rng.integers(len(bauds)))]
        L = float(rng.uniform(1000e3, 10000e3))
        snr = float(rng.uniform(9.0, 14.0))
        seed = 1003 * 1000 + i
        link = dict(baud_hz=baud, bits_per_sym=2, n_sym=n_sym, fiber_len_m=L, snr_db=snr, prbs_seed=seed,
                    seed=seed, out_dtype="c64")
        rxc = dict(baud_hz=baud, modulation=2, fiber_len_m=L, frame_syms=BATCH_FRAME, prbs_seed=seed,
                   max_block_samples=1 << 19)
        sizes, left = [], n_sym
        while left:
            m = min(left, 1 << int(rng.integers(12, 19)))
            sizes.append(m)
            left -= m
        out.append((link, rxc, sizes))
    return out


def load_batched_streams(n_sym, dev, subset=None):
    """The 64 streams of batched_streams (or the listed subset) simulated
    and split into their capture blocks, resident on the device."""
    import torch
    import rxsim
    streams = batched_streams(BATCH_STREAMS, n_sym)
    if subset is not None:
        streams = [streams[i] for i in subset]
    data = []
    for link, rxc, sizes in streams:
        x = rxsim.simulate(rxsim.LinkConfig(**link))["rx"]
        blocks, a = [], 0
        for m in sizes:
            blocks.append(torch.from_numpy(np.ascontiguousarray(x[:, 2 * a:2 * (a + m)])).to(dev))
            a += m
        data.append(blocks)
    torch.cuda.synchronize()
    return streams, data


def serve_pass(streams, data, fft, storage, batch=0):
    """Every block of every stream submitted at once to one server (batch =
    1: batched rounds); wall time from the first submission to the last
    stream's end, server and per-stream statistics."""
    from paper_2108_07001_gb300 import rx
    order = [(i, j) for j in range(max(len(b) for b in data)) for i in range(len(streams)) if j < len(data[i])]
    with rx.Server(max_streams=128, batch=batch) as srv:
        sids = [srv.open(**dict(rxc, fft_n=fft[i], storage_dtype=storage)) for i, (_, rxc, _) in enumerate(streams)]
        t_start = time.perf_counter()
        for i, j in order:
            b = data[i][j]
            srv.submit_device(sids[i], b.data_ptr(), b.shape[1], rx.RX_C64)
        for sid in sids:
            srv.end(sid)
        for sid in sids:
            srv.sync(sid, timeout_ms=600000)
        wall = time.perf_counter() - t_start
        st = srv.stats()
        per = [srv.stream_stats(sid) for sid in sids]
    return wall, st, per


def plain_pass(streams, data):
    """The same streams one after another, each through its own plain
    receiver (FP32 storage, default FFT size) from its first block to its
    last frame, before the next stream starts."""
    import torch
    from paper_2108_07001_gb300 import rx
    cur = torch.cuda.current_stream()
    wall, per = 0.0, []
    for i, (_, rxc, _) in enumerate(streams):
        r = rx.Receiver(**rxc)
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        for b in data[i]:
            r.push_device(b.data_ptr(), b.shape[1], rx.RX_C64, cur.cuda_stream)
        r.end()
        r.join(cur.cuda_stream)
        torch.cuda.synchronize()
        wall += time.perf_counter() - t_start
        per.append(r.stats())
        r.close()
    return wall, per


def batch_pass(streams, data, fft, storage, barrier=None, graph=False):
    """All streams through one rx_batch: round j pushes every stream's j-th
    block in one call (one launch per stage and frame ordinal, or with
    graph one replay of the batch's captured graph), the last call ends
    every stream."""
    import torch
    from paper_2108_07001_gb300 import rx
    cur = torch.cuda.current_stream()
    dev = data[0][0].device
    recs = [rx.Receiver(**dict(rxc, fft_n=fft[i], storage_dtype=storage)) for i, (_, rxc, _) in enumerate(streams)]
    dummy = torch.zeros(16, dtype=torch.complex64, device=dev)
    n_rounds = max(len(b) for b in data)
    with rx.Batch(recs, graph=graph) as batch:
        torch.cuda.synchronize()
        if barrier:
            barrier()
        t_start = time.perf_counter()
        for j in range(n_rounds):
            ptrs = [data[i][j].data_ptr() if j < len(data[i]) else dummy.data_ptr() for i in range(len(streams))]
            ns = [data[i][j].shape[1] if j < len(data[i]) else 0 for i in range(len(streams))]
            batch.push(ptrs, ns, rx.RX_C64, cur.cuda_stream)
        batch.end(cur.cuda_stream)
        host = time.perf_counter() - t_start
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_start
        if barrier:
            barrier()
        info = dict(batch.info(), **{"graph_" + k: v for k, v in batch.graph_info().items()})
    per = [r.stats() for r in recs]
    for r in recs:
        r.close()
    return wall, host, info, per


def stream_summary(per):
    return {"synced_streams": int(sum(p["synced"] for p in per)), "ber_max": max(p["ber"] for p in per),
            "cycle_slips": int(sum(p["cycle_slips"] for p in per))}


def run_batched(args, rank=0, world=1, barrier=None):
    """64 independent streams with uneven capture blocks, every block
    submitted at once: through the serving layer with per-stream pushes
    (FFT size of the default rule (N >= 4 halo), the size the autotuner picks
    per stream, and the latter with FP16 sample storage), through the
    serving layer in batched rounds (FP32 and FP16 storage; FP16 also with
    graph replay), and through one rx_batch (round j pushes every stream's
    j-th block in one call: one launch per stage and frame ordinal,
    pipelined over the batch's four streams, or one replay of the batch's
    captured graph); beside them the plain per-stream chain (one stream at a
    time).  The value is the fastest form."""
    import torch
    from paper_2108_07001_gb300 import rx
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    n_sym = args.symbols or BATCH_SYMS
    subset = None
    if world > 1:  # this rank's shard of the streams (the batched launch alone)
        subset = shard_streams([4.0 * n_sym] * BATCH_STREAMS, world)[rank]
        args.batched_forms = "batch"
    t0 = time.time()
    streams, data = load_batched_streams(n_sym, dev, subset)
    gen_s = time.time() - t0
    t0 = time.time()
    only_batch = args.batched_forms == "batch"
    tuned = [0] * len(streams) if only_batch else \
        [rx.autotune_fft(rx.default_config(**rxc), frames=8)[0] for _, rxc, _ in streams]
    tune_s = time.time() - t0
    total_samples = 4 * n_sym * len(streams)
    n_blocks = sum(len(b) for b in data)
    deflt = [0] * len(streams)

    forms = {}
    if only_batch:  # the batched launch alone (for launch lists)
        batch_pass(streams, data, deflt, rx.RX_C64)
        wall, host, info, per = batch_pass(streams, data, deflt, rx.RX_C64, barrier)
        return dict({"workload": "batched", "form": "batch_default_fft",
                     "gsamples_s": round(total_samples / wall / 1e9, 3),
                     "samples": total_samples, "streams": len(streams), "symbols_per_pol_per_stream": n_sym,
                     "wall_ms": round(wall * 1e3, 1), "host_ms": round(host * 1e3, 1),
                     "host_wait_ms": round(info["wait_ms"], 1), "calls": info["calls"],
                     "launches": info["launches"]}, **stream_summary(per))
    plain_pass(streams, data)
    wall, per = plain_pass(streams, data)
    forms["plain_per_stream"] = dict({"gsamples_s": round(total_samples / wall / 1e9, 3),
                                      "wall_ms": round(wall * 1e3, 1)}, **stream_summary(per))
    for form, fft, storage, batch in (("default_fft", deflt, rx.RX_C64, 0), ("autotuned_fft", tuned, rx.RX_C64, 0),
                                      ("autotuned_fft_fp16_storage", tuned, rx.RX_C16, 0),
                                      ("served_batched_default_fft", deflt, rx.RX_C64, 1),
                                      ("served_batched_default_fft_fp16_storage", deflt, rx.RX_C16, 1),
                                      ("served_batched_graph_default_fft_fp16_storage", deflt, rx.RX_C16, 2)):
        serve_pass(streams, data, fft, storage, batch)
        wall, st, per = serve_pass(streams, data, fft, storage, batch)
        forms[form] = dict({"gsamples_s": round(total_samples / wall / 1e9, 3), "wall_ms": round(wall * 1e3, 1),
                            "latency_p50_ms": round(st["latency_p50_ms"], 3),
                            "latency_p99_ms": round(st["latency_p99_ms"], 3),
                            "mem_gib": round(st["mem_in_use_bytes"] / 2 ** 30, 2) if st["mem_in_use_bytes"] else None,
                            "batch_calls": st["batch_calls"]}, **stream_summary(per))
    for form, fft, storage, graph in (("batch_default_fft", deflt, rx.RX_C64, False),
                                      ("batch_default_fft_fp16_storage", deflt, rx.RX_C16, False),
                                      ("batch_autotuned_fft_fp16_storage", tuned, rx.RX_C16, False),
                                      ("batch_graph_default_fft", deflt, rx.RX_C64, True),
                                      ("batch_graph_default_fft_fp16_storage", deflt, rx.RX_C16, True)):
        batch_pass(streams, data, fft, storage, graph=graph)
        wall, host, info, per = batch_pass(streams, data, fft, storage, graph=graph)
        # block latency of a call (its start on the stream to its bits), the
        # same for every stream the call carried
        forms[form] = dict({"gsamples_s": round(total_samples / wall / 1e9, 3), "wall_ms": round(wall * 1e3, 1),
                            "latency_p50_ms": round(float(np.median([p["latency_p50_ms"] for p in per])), 3),
                            "latency_p99_ms": round(max(p["latency_p99_ms"] for p in per), 3),
                            "host_ms": round(host * 1e3, 1), "host_wait_ms": round(info["wait_ms"], 1),
                            "calls": info["calls"], "launches": info["launches"],
                            "graph_replays": info["graph_replays"], "graph_nodes": info["graph_nodes"],
                            "fft_groups": len(set(fft)) if fft[0] else None}, **stream_summary(per))
    base = forms["plain_per_stream"]["gsamples_s"]
    strong = forms["default_fft"]["gsamples_s"]
    for form in forms:
        if form != "plain_per_stream":
            forms[form]["x_plain_per_stream"] = round(forms[form]["gsamples_s"] / base, 2) if base else None
            forms[form]["x_served_per_stream"] = round(forms[form]["gsamples_s"] / strong, 2) if strong else None
    best = max((f for f in forms if f != "plain_per_stream"), key=lambda f: forms[f]["gsamples_s"])
    return {"metric": "gsamples_per_s", "value": forms[best]["gsamples_s"], "value_form": best,
            "unit": "Gsamples/s",
            "n_gpus": 1, "higher_is_better": True, "workload": "batched", "dtype": "f16 storage, f32 arithmetic",
            "data": "synthetic (seeded link simulator)",
            "config": {"streams": len(streams), "symbols_per_pol_per_stream": n_sym, "blocks": n_blocks,
                       "block_syms": "2^12..2^18", "frame_syms": BATCH_FRAME,
                       "baud_gbd": [s[0]["baud_hz"] / 1e9 for s in streams],
                       "fiber_km": [round(s[0]["fiber_len_m"] / 1e3) for s in streams],
                       "autotuned_fft": tuned, "submission": "every block at once"},
            "forms": forms, "autotune_seconds": round(tune_s, 1), "sim_seconds": round(gen_s, 1)}


def batched_fp16_summary(hbm_peak):
    """The 64-stream workload (batched_streams) through the batched
    FP16-storage serving path (the serving layer in batched rounds), beside
    the plain per-stream FP32 chain (one stream at a time) and the same
    streams served concurrently through plain receivers (per-stream
    pushes, FP32): throughput, ratios, frame latency, worst BER, and the
    chain's algorithmic HBM bytes (complex64 input read once, decided bits
    written once) over the measured HBM bandwidth."""
    import torch
    from paper_2108_07001_gb300 import rx
    t0 = time.time()
    streams, data = load_batched_streams(BATCH_SYMS, torch.device("cuda:0"))
    gen_s = time.time() - t0
    total = 4 * BATCH_SYMS * len(streams)
    deflt = [0] * len(streams)
    plain_pass(streams, data)
    w_plain, per_plain = plain_pass(streams, data)
    serve_pass(streams, data, deflt, rx.RX_C64, 0)
    w_serv, _, per_serv = serve_pass(streams, data, deflt, rx.RX_C64, 0)
    serve_pass(streams, data, deflt, rx.RX_C16, 1)
    w_b, st_b, per_b = serve_pass(streams, data, deflt, rx.RX_C16, 1)
    del data
    torch.cuda.empty_cache()
    v = total / w_b / 1e9
    bytes_per_sample = 8.0 + 2.0 / 8.0 / 2.0  # c64 in; 2 bits per QPSK symbol and polarisation out (1 bit per sample)
    out = {"path": "serving layer, batched rounds (rx_server batch = 1), FP16 sample storage, FP32 arithmetic",
           "streams": len(streams), "symbols_per_pol_per_stream": BATCH_SYMS, "block_syms": "2^12..2^18",
           "gsamples_s": round(v, 3), "decoded_gbps": round(v, 3),
           "latency_p50_ms": round(st_b["latency_p50_ms"], 3), "latency_p99_ms": round(st_b["latency_p99_ms"], 3),
           "batch_calls": st_b["batch_calls"],
           "plain_per_stream_fp32_gsamples_s": round(total / w_plain / 1e9, 3),
           "x_plain_per_stream_fp32": round(w_plain / w_b, 2),
           "served_per_stream_fp32_gsamples_s": round(total / w_serv / 1e9, 3),
           "x_served_per_stream_fp32": round(w_serv / w_b, 2),
           "ber_max": max(p["ber"] for p in per_b), "ber_max_plain_fp32": max(p["ber"] for p in per_plain),
           "synced_streams": int(sum(p["synced"] for p in per_b)),
           "cycle_slips": int(sum(p["cycle_slips"] for p in per_b)),
           "hbm_algorithmic_gbs": round(v * bytes_per_sample, 1),
           "sim_seconds": round(gen_s, 1)}
    if hbm_peak:
        out["hbm_frac"] = round(v * bytes_per_sample / hbm_peak, 4)
    return out


def qam16_summary():
    """The DP-16QAM workload (32 GBd, 5,000 km, 18 dB, 2^22 symbols, 25 taps,
    32 angles) in the default line: FP16 and FP32 sample storage (FP32
    arithmetic), throughput, BER and the EVM penalty of each over the FP64
    oracle on the same samples (run_qam16, fewer timed steps)."""
    r = run_qam16(argparse.Namespace(symbols=0, steps=5, warmup=2))
    f16, f32, o = r["forms"]["fp16_storage"], r["forms"]["fp32_storage"], r["oracle"]
    return {"workload": r["config"]["workload"], "symbols_per_pol": r["config"]["symbols_per_pol"],
            "fp16_storage_gsamples_s": f16["value"], "fp32_storage_gsamples_s": f32["value"],
            "ber_fp16_storage": f16["ber"], "ber_fp32_storage": f32["ber"], "ber_oracle": o["ber"],
            "evm_penalty_db_fp16_storage": f16["evm_penalty_db"], "evm_penalty_db_fp32_storage": f32["evm_penalty_db"],
            "cycle_slips": f16["cycle_slips"] + f32["cycle_slips"], "oracle_cores": o["cores"],
            "oracle_seconds": o["seconds"]}


def serving_summary():
    """The serving workload (16 mixed QPSK/16QAM streams, 28-64 GBd, 10,000
    km, blocks of 2^16-2^20 symbols) in the default line: capacity, then
    Poisson arrivals at 80 % of it, per-stream pushes with FP32 and FP16
    storage and batched rounds with FP16 storage (run_serving)."""
    r = run_serving(argparse.Namespace(symbols=0))
    out = {"streams": r["config"]["streams"], "symbols_per_pol_per_stream": r["config"]["symbols_per_pol_per_stream"],
           "arrivals": r["config"]["arrivals"]}
    for form in ("fp32_storage", "fp16_storage", "batched_fp16_storage"):
        f = r["forms"][form]
        out[form] = {k: f[k] for k in ("capacity_gsamples_s", "sustained_gsamples_s", "sustained_decoded_gbps",
                                       "latency_p50_ms", "latency_p99_ms", "ber_max", "synced_streams",
                                       "cycle_slips")}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)  # ~0.74 s timed on the stream workload
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="stream workload: leave out the sub-records of the other workloads (batched_fp16: 64 "
                         "streams, batched serving; qam16_fp16: DP-16QAM storage forms against the oracle; "
                         "serving: 16 streams under Poisson arrivals)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--symbols", type=int, default=0, help="stream length per pol (default: the workload's 2^24)")
    ap.add_argument("--oracle-child", nargs=4, help=argparse.SUPPRESS)
    ap.add_argument("--kk-oracle-child", type=int, help=argparse.SUPPRESS)
    ap.add_argument("--fft-n", type=int, default=0,
                    help="stream workload: overlap-save FFT size (0: the default rule, -1: the autotuner's pick)")
    ap.add_argument("--batched-forms", default="all", choices=["all", "batch"],
                    help="batched workload: all forms, or the batched launch alone")
    ap.add_argument("--stream", default=None,
                    help="stream workload by name (default dp-qpsk-28gbd-10000km-stream-2^24sym; "
                         "dp-qpsk-64gbd-10000km-stream: 64 GBd, the 32768-point transform)")
    ap.add_argument("--bps-coarse-stride", type=int, default=1,
                    help="stream workload: 4 = two-stage BPS over 16 coarse angles (default 1: all 64)")
    ap.add_argument("--workload", default="stream", choices=["stream", "qam16", "serving", "batched", "kk", "kk_batch", "kkrx_batch"],
                    help="stream: the 2^24-symbol DP-QPSK stream (default line); qam16: DP-16QAM 5,000 km "
                         "with FP16 and FP32 sample storage against the FP64 oracle; serving: 16 mixed "
                         "channel streams through the serving layer at 80 %% of its capacity; batched: 64 "
                         "streams with uneven blocks, FFT sizes from the heuristic and from the autotuner; "
                         "kk: the paper's Kramers-Kronig receiver on 2^22-sample buffers of 12-bit codes; "
                         "kk_batch: 64 KK front ends with small uneven pushes, one graph replay per round; "
                         "kkrx_batch: 64 whole KK receivers the same way")
    args = ap.parse_args()
    if args.kk_oracle_child:
        kk_oracle_child(args.kk_oracle_child)
        return
    if args.oracle_child:
        name, n_sym, reps, stride = args.oracle_child
        oracle_child(name, int(n_sym), int(reps), int(stride))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        # one stream: replicas, every rank runs its own stream on its own
        # GPU; the 64-stream workload: the streams shard over the ranks
        import torch
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
        args.cpu_baseline = False  # the CPU baseline is taken on one rank at N=1 only
        args.batched = False       # as is the 64-stream sub-record

        def reduce_op(op):
            def f(vals):
                t = torch.tensor(vals, device="cuda", dtype=torch.float64)
                dist.all_reduce(t, op=op)
                return t.tolist()
            return f

        reduce_max = reduce_op(dist.ReduceOp.MAX)
        if args.workload == "batched":
            part = run_batched(args, rank, world, barrier=dist.barrier)
            line = combine_shards(part, world, reduce_max, reduce_op(dist.ReduceOp.SUM))
        else:
            line = combine_replicas(run_ours(args), world, reduce_max)
        if rank == 0:
            print(json.dumps(line), flush=True)
        dist.destroy_process_group()
        return
    if args.workload == "qam16":
        print(json.dumps(run_qam16(args)), flush=True)
        return
    if args.workload == "serving":
        print(json.dumps(run_serving(args)), flush=True)
        return
    if args.workload == "batched":
        print(json.dumps(run_batched(args)), flush=True)
        return
    if args.workload == "kk":
        print(json.dumps(run_kk(args)), flush=True)
        return
    if args.workload == "kk_batch":
        print(json.dumps(run_kk_batch(args)), flush=True)
        return
    if args.workload == "kkrx_batch":
        print(json.dumps(run_kkrx_batch(args)), flush=True)
        return
    print(json.dumps(run_ours(args)), flush=True)


if __name__ == "__main__":
    main()
