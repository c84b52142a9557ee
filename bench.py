#!/usr/bin/env python
"""Throughput benchmark of the reconstruction path (FFT -> window -> IFFT -> HG overlap).

Workload (per GPU and step): 1000 frames of 320x256 uint16 (12-bit, Poisson), two 128x128 polarisation
windows, 64x64 fields and 45 Hermite-Gaussian coefficients per window.  Synthetic, seeded frames.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` is whole-job frames/s with the frames already in HBM; ``e2e`` is the
same metric through the public API from pinned host frames to host results; ``roofline`` is the dominant
kernel's algorithmic work per launch over its event-timed launch duration, against the binding ceiling: the
FP32 peak (derived from SM count, lanes and clock) when algorithmic flops limit the frame rate before the
measured HBM bandwidth does, else the HBM peak; both are reported under ``roofline.alu`` / ``roofline.hbm``;
``cpu_baseline`` is the FP64 oracle on the host cores.  ``--impl reference`` times the oracle itself, as the
reference arm.  Multi-GPU runs (torchrun) are weak-scaled: every rank processes its own batch, with no
collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "frames/s (FFT→window→IFFT→HG overlap) on 1 GB300, % HBM roofline; p99 latency"
WORKLOAD = "batching: 1000 frames 320x256 u16, 2 pol windows 128x128, 64x64 fields, HG groups 0-8 (45 modes)"
FRAMES = 1000
ROTATE = 4                      # distinct input batches cycled between steps (4 x 164 MB > 129 MB L2)
FALLBACK_HBM_GBS = 6800.0
VARIANTS = {"auto": 0, "fused": 1, "fused_pruned": 2, "generic": 3, "fused_groups": 4}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "split_bf16"], default="fp32")
    ap.add_argument("--variant", choices=list(VARIANTS), default="auto",
                    help="kernel variant the handle is held to (dh_set_variant); auto: the library's choice")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-case", action="store_true",
                    help="skip the precision configuration's and the kernel variants' sub-records in the default line")
    ap.add_argument("--sustain-s", type=float, default=2.5,
                    help="seconds of back-to-back steps after the timed region (latency percentiles, clocks)")
    ap.add_argument("--frames", type=int, default=FRAMES, help="frames per step and GPU (default: the workload's 1000)")
    ap.add_argument("--workload", choices=["batching", "serving", "plain", "precision", "large_batch", "extensions"],
                    default="batching")
    ap.add_argument("--requests", type=int, default=2000, help="requests per serving run")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------ helpers


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value_ms, ws, device=None):
    """Largest per-rank value (the job's wall time); a plain float when there is one rank."""
    if ws <= 1:
        return float(value_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, frames_per_rank, steps, max_ms):
    """Frames per second of the whole job: every rank processed frames_per_rank frames per step."""
    return ws * frames_per_rank * steps / (max_ms / 1e3)


def rank_shard(frames_per_rank, rank):
    """The contiguous range of the job's global frame stream that one rank processes (weak scaling: rank r
    takes frames [r F, (r + 1) F) of the one seeded stream, F frames per rank); returns (first, count)."""
    return rank * frames_per_rank, frames_per_rank


def bytes_per_frame(setup, m, modes):
    """Algorithmic bytes per frame: window pixels read plus fields and coefficients written."""
    px_bytes = 2 if setup.dtype == "u16" else 4
    n = setup.window
    return setup.pol_count * (n * n * px_bytes + m * m * 8 + modes * 8)


def window_rows(setup):
    """Frame rows the host-buffer call copies to the device: from the first to the last row of any
    polarisation window (window origin round_half_away(c / px) - N/2)."""
    def rha(v):
        return int(math.floor(abs(v) + 0.5)) * (1 if v >= 0 else -1)
    oy = [rha(setup.beam_centre[p][1] / setup.pixel) - setup.window // 2 for p in range(setup.pol_count)]
    return max(oy) + setup.window - min(oy)


def flops_per_frame(setup, m, modes):
    """Algorithmic FP32 flops per frame by the nominal counts: 2.5 N log2 N per real and 5 N log2 N per
    complex transform of length N, the forward transform pruned to the M box columns (N real rows, M complex
    columns), the M x M inverse, and the separable overlap 4 M^2 G + 4 M modes."""
    n = setup.window
    g = setup.group_count
    lg_n, lg_m = math.log2(n), math.log2(m)
    per_window = (n * 2.5 * n * lg_n + m * 5.0 * n * lg_n + 2 * m * 5.0 * m * lg_m
                  + (4.0 * m * m * g + 4.0 * m * modes if g else 0.0))
    return setup.pol_count * per_window


def fp32_peak_tflops(dev):
    """FP32 peak derived from unit counts and the maximum SM clock: SMs x 128 FP32 lanes x 2 flops (FMA) x
    clock (MEASURED_PEAKS.json sm_max_mhz, else 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, src = 2070.0, "nominal 2070 MHz"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, src = float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except Exception:
        pass
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"derived: {sms} SMs x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz ({src})"


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s"


# source file of each timed kernel; its hash also covers the device headers every kernel includes
KERNEL_SOURCES = {"k_fused128": "k_fused.cu", "k_fused128p": ("k_fused_pr.cu", "fused_pr.hpp"), "k_fused128g": "k_fused_g.cu",
                  "k_fused256": "k_fused256.cu",
                  "k_yinv_tc": "k_overlap_tc.cu", "k_ypass": "k_split.cu", "k_xpass": "k_split.cu", "k_yinv": "k_split.cu"}
DEVICE_HEADERS = ("fft.cuh", "kernels.cuh", "sync.cuh", "umma.cuh", "check.cuh")


def kernel_source_hash(kernel):
    """sha256 (first 16 hex digits) over the kernel's source file and the shared device headers, or None
    for a kernel without a recorded source."""
    if kernel not in KERNEL_SOURCES:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2204_02348_gb300", "csrc")
    src = KERNEL_SOURCES[kernel]
    for name in (src if isinstance(src, tuple) else (src,)) + DEVICE_HEADERS:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, frames_per_launch):
    """DRAM bytes per launch from the committed ncu summary, scaled to this launch size, or None when the
    summary was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash(kernel)
    for line in open(path):
        m = re.match(r"\|\s*(\w+)\s*\|\s*([0-9a-f]+)\s*\|\s*([0-9.eE+]+)\s*\|\s*(\d+)\s*\|", line)
        if m and m.group(1) == kernel and m.group(2) == src:
            return float(m.group(3)) / int(m.group(4)) * frames_per_launch
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.stamps = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.stamps.append(time.perf_counter())

    def samples(self):
        """(host time, SM MHz, power W) of every sample read so far."""
        out = []
        for t, ln in zip(list(self.stamps), list(self.lines)):
            parts = [p.strip() for p in ln.split(",")]
            try:
                out.append((t, float(parts[1]), float(parts[3])))
            except (ValueError, IndexError):
                continue
        return out

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_worker(args):
    frames, setup = args
    from oracle import digholo_oracle as orc
    orc.process_batch(frames, setup)
    return frames.shape[0]


class OraclePool:
    """Spawn-started process pool running the FP64 oracle over frame chunks, one BLAS thread per worker."""

    def __init__(self, workers):
        import concurrent.futures as cf
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.workers = workers
        self.ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))

    def warm(self, setup, frames):
        list(self.ex.map(_oracle_worker, [(frames[:1], setup)] * self.workers))

    def run(self, setup, frames, repeat=1):
        """Process `repeat` passes over `frames`; returns (frames/s, seconds, frames processed)."""
        import numpy as np
        chunks = []
        for _ in range(repeat):
            chunks += [c for c in np.array_split(frames, self.workers * 2) if len(c)]
        t0 = time.perf_counter()
        n = sum(self.ex.map(_oracle_worker, [(c, setup) for c in chunks]))
        dt = time.perf_counter() - t0
        return n / dt, dt, n

    def close(self):
        self.ex.shutdown()


# ------------------------------------------------------------------------------------------ arms


def run_reference(args, ws, rank):
    """Reference arm: the FP64 oracle, as it stands, on the host cores, on the same workload and metric."""
    from synth import holograms as syn
    if rank != 0:
        return
    setup = syn.setup_batching()
    sample = 200                                     # frames per step: a bounded sample of the 1000-frame batch
    data = syn.make_frames(setup, sample)["frames"]
    workers = os.cpu_count() or 1
    pool = OraclePool(workers)
    pool.warm(setup, data)
    for _ in range(args.warmup):
        pool.run(setup, data[: max(1, sample // 10)])
    times = []
    for _ in range(args.steps):
        _, dt, n = pool.run(setup, data)
        times.append(dt)
    pool.close()
    total = sum(times)
    value = args.steps * sample / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": sample,
                   "note": "FP64 oracle (explicit DFTs, direct sums) on host cores; each step a 200-frame sample"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": workers, "kind": "oracle",
                         "sample": f"{sample} frames of the batching workload per step"},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2204_02348_gb300 as dh
    from synth import holograms as syn

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    setup = syn.setup_batching()
    prec = dh.DH_PRECISION_SPLIT_BF16 if args.precision == "split_bf16" else dh.DH_PRECISION_FP32
    frames_n = args.frames
    first, _ = rank_shard(frames_n, rank)
    data = syn.make_frames(setup, frames_n, seed=syn.BASE_SEED, first=first)
    host = torch.from_numpy(data["frames"]).pin_memory()
    inputs = [host.to(dev) for _ in range(ROTATE)]
    h = dh.dh_create()
    dh.configure(h, setup)
    dh.dh_set_precision(h, prec)
    dh.dh_set_variant(h, VARIANTS[args.variant])
    m, modes, _ = dh.dh_get_output_dims(h)
    P = setup.pol_count
    variant = {v: k for k, v in VARIANTS.items()}[dh.dh_get_variant(h)]
    fields = torch.empty((frames_n, P, m, m), dtype=torch.complex64, device=dev)
    coefs = torch.empty((frames_n, P, modes), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(k):
        dh.dh_process_batch(h, inputs[k % ROTATE], dh.DH_DTYPE_U16, frames_n, fields, coefs, stream)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for k in range(max(args.warmup, 3)):
        step(k)
    torch.cuda.synchronize()

    # ---- timed region: K steps between two events.  An event recorded between launches ends the overlap of one
    # persistent launch's tail with the next one's start (on the batching step: +2 us per step for an event per
    # step, +4 us for the library's per-kernel pair, on 98 us), so the timed region carries no other events
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)                 # let the sampler start before the clock runs
    import gc
    gc.collect()
    gc.disable()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(args.steps):
        step(k)
    ev1.record(stream)
    torch.cuda.synchronize()
    gc.enable()
    barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    value = whole_job_rate(ws, frames_n, args.steps, total_ms)
    # ---- the same K steps again with an event per step and the library's per-kernel events: step latencies,
    # each kernel's launches and average launch duration (bracketed by its own events), the launches per step
    dh.dh_set_profiling(h, True)
    barrier()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for k in range(args.steps):
        step(k)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    prof = dh.dh_get_profile(h)
    dh.dh_set_profiling(h, False)
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]

    # ---- sustained: the same step back to back for at least 2.5 s, in segments of 1000 steps (each drained
    # with a synchronize, so its host interval brackets its device work); per-step events give the latency
    # percentiles over every step, clock samples are binned by the segment they fall in
    sustained = None
    if rank == 0 and args.sustain_s > 0:
        sampler2 = ClockSampler(local)
        sampler2.start()
        time.sleep(0.5)
        seg_steps, segs, lat2 = 1000, [], []
        t_start = time.perf_counter()
        k = 0
        while time.perf_counter() - t_start < args.sustain_s:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(seg_steps + 1)]
            torch.cuda.synchronize()
            h0 = time.perf_counter()
            ev[0].record(stream)
            for i in range(seg_steps):
                step(k)
                k += 1
                ev[i + 1].record(stream)
            torch.cuda.synchronize()
            h1 = time.perf_counter()
            ms = ev[0].elapsed_time(ev[-1])
            lat2.extend(ev[i].elapsed_time(ev[i + 1]) for i in range(seg_steps))
            segs.append((h0, h1, ms))
        smp = sampler2.samples()
        sampler2.stop()
        bins = {}
        seg_mhz = []
        for (h0, h1, ms) in segs:
            inside = [mhz for (t, mhz, _) in smp if h0 <= t <= h1]
            mhz = statistics.median(inside) if inside else None
            seg_mhz.append(mhz)
            if mhz is not None:
                b = int(round(mhz / 30.0) * 30)
                n, tot = bins.get(b, (0, 0.0))
                bins[b] = (n + 1, tot + ms)
        lat2.sort()
        tot_ms = sum(ms for (_, _, ms) in segs)
        loaded = [mhz for (t, mhz, _) in smp if segs and segs[0][0] <= t <= segs[-1][1]]
        power = [w for (t, _, w) in smp if segs and segs[0][0] <= t <= segs[-1][1]]
        sustained = {
            "seconds": tot_ms / 1e3, "steps": len(lat2),
            "frames_per_s": frames_n * len(lat2) / (tot_ms / 1e3),
            "sm_mhz_median": statistics.median(loaded) if loaded else None,
            "power_w_max": max(power) if power else None, "clock_samples": len(loaded),
            "latency_ms": {"p50": lat2[len(lat2) // 2], "p99": lat2[min(len(lat2) - 1, int(0.99 * len(lat2)))],
                           "max": lat2[-1], "unit": f"ms per {frames_n}-frame batch"},
            "by_clock": [{"sm_mhz": b, "segments": n, "frames_per_s": frames_n * seg_steps * n / (t / 1e3)}
                         for b, (n, t) in sorted(bins.items())],
        }

    # ---- dominant kernel roofline
    peak, peak_src = measured_peak()
    bpf = bytes_per_frame(setup, m, modes)
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    launches = sum(v[0] for v in prof.values())
    roofline = None
    if dom:
        name, (nl, tms) = dom
        launches_per_step = nl / args.steps
        frames_per_launch = frames_n / launches_per_step
        avg_s = tms / nl / 1e3
        achieved = frames_per_launch * bpf / avg_s / 1e9
        traffic = recorded_traffic(name, frames_per_launch)
        # the binding ceiling is the lower of the HBM and the FP32 ones (frames/s at peak bytes or flops)
        fpf = flops_per_frame(setup, m, modes)
        fpk, fpk_src = fp32_peak_tflops(dev)
        alu_tflops = frames_per_launch * fpf / avg_s / 1e12
        hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
               "peak_source": peak_src, "bytes_per_frame": bpf, "ceiling_frames_per_s": peak * 1e9 / bpf}
        alu = {"achieved": alu_tflops, "peak": fpk, "unit": "TFLOP/s", "frac": alu_tflops / fpk,
               "peak_source": fpk_src, "flops_per_frame": fpf, "ceiling_frames_per_s": fpk * 1e12 / fpf}
        bound, lim = ("alu", alu) if alu["ceiling_frames_per_s"] < hbm["ceiling_frames_per_s"] else ("hbm", hbm)
        roofline = {"bound": bound, "kernel": name, "achieved": lim["achieved"], "peak": lim["peak"],
                    "unit": lim["unit"], "frac": lim["frac"], "traffic": traffic, "peak_source": lim["peak_source"],
                    "frames_per_launch": frames_per_launch,
                    "kernel_share": tms / sum(v[1] for v in prof.values()),
                    "step_frac": (value / ws) / lim["ceiling_frames_per_s"],
                    "hbm": hbm, "alu": alu}

    # ---- end to end through the public host-buffer calls: pinned host frames in, fields and coefficients out,
    # every step's copies inside the wall-clock interval.  The stream of batches goes through
    # dh_process_batch_host_async (the next batch's uploads start behind this one's downloads) and ends with
    # dh_process_batch_host_wait; the blocking dh_process_batch_host, which drains its pipeline on every call, is
    # timed beside it
    host_f = torch.empty((frames_n, P, m, m), dtype=torch.complex64).pin_memory()
    host_c = torch.empty((frames_n, P, modes), dtype=torch.complex64).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))

    def e2e_time(step, finish):
        for _ in range(2):
            step()
        finish()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            step()
        finish()
        return max_over_ranks(1e3 * (time.perf_counter() - t0), ws, dev)

    e_ms = e2e_time(lambda: dh.dh_process_batch_host_async(h, host, dh.DH_DTYPE_U16, frames_n, host_f, host_c, stream),
                    lambda: dh.dh_process_batch_host_wait(h))
    b_ms = e2e_time(lambda: dh.dh_process_batch_host(h, host, dh.DH_DTYPE_U16, frames_n, host_f, host_c, stream),
                    torch.cuda.synchronize)
    e2e = {"value": whole_job_rate(ws, frames_n, e2e_steps, e_ms), "unit": "frames/s",
           "h2d_bytes_per_step": int(frames_n * window_rows(setup) * setup.frame_w * 2),
           "d2h_bytes_per_step": int(host_f.numel() * 8 + host_c.numel() * 8), "steps": e2e_steps,
           "api": "dh_process_batch_host_async + dh_process_batch_host_wait",
           "blocking": {"value": whole_job_rate(ws, frames_n, e2e_steps, b_ms), "api": "dh_process_batch_host"}}

    # ---- CPU baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        workers = os.cpu_count() or 1
        pool = OraclePool(workers)
        pool.warm(setup, data["frames"])
        # one pass to size the sample, then about ten seconds of oracle work
        _, dt0, _ = pool.run(setup, data["frames"])
        rate, dt, n = pool.run(setup, data["frames"], repeat=max(1, min(200, int(round(10.0 / max(dt0, 1e-3))))))
        pool.close()
        cpu = {"value": rate, "unit": "frames/s", "cores": workers, "kind": "oracle",
               "sample": f"{n} frames (repeated passes over the step's batch) in {dt:.1f} s on {workers} processes"}

    # ---- every kernel variant of the 128 x 128 path on the same resident batches (rank 0, N = 1 only): the
    # measured ground for the library's default and the tuner's candidates
    var_case = None
    if rank == 0 and ws == 1 and not args.no_precision_case:
        var_case = {}
        for name in ("fused", "fused_groups", "fused_pruned", "generic"):
            dh.dh_set_variant(h, VARIANTS[name])
            ms = _event_time(lambda: [step(k) for k in range(ROTATE)], 25, 3) / ROTATE
            var_case[name] = {"runs": {v: k for k, v in VARIANTS.items()}[dh.dh_get_variant(h)],
                              "frames_per_s": frames_n / (ms / 1e3), "ms_per_batch": ms}
        dh.dh_set_variant(h, VARIANTS[args.variant])
    dh.dh_destroy(h)
    # ---- the precision configuration beside the headline one (rank 0, N = 1 only)
    prec_case = None
    if rank == 0 and ws == 1 and not args.no_precision_case:
        del inputs, fields, coefs
        torch.cuda.empty_cache()
        prec_case = precision_case(20, dev)
    if rank == 0:
        lat = sorted(per_step)
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if frames_n == FRAMES else WORKLOAD.replace("1000", str(frames_n)),
                       "frames_per_step_per_gpu": frames_n, "frame": [320, 256],
                       "pols": P, "window": setup.window, "field": m, "modes": modes,
                       "overlap": args.precision, "variant": variant, "l2": f"{ROTATE} rotating input batches "
                       f"({ROTATE * host.numel() * 2 / 1e6:.0f} MB) > 129 MB L2",
                       "parallelism": f"replicas x{ws}"},
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "unit": f"ms per {frames_n}-frame batch"},
            "timing": "value: the K steps between two events; latency, kernels, roofline, gpu_launches: the same K "
                      "steps again with an event per step and per-kernel events",
            "roofline": roofline,
            "kernels": {k: {"launches": v[0], "total_ms": v[1]} for k, v in prof.items()},
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "sustained": sustained,
            "precision_case": prec_case,
            "variants_case": var_case,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


SERVING_METRIC = "serving frames/s with p50/p99 request latency (mixed geometries, continuous batching) on 1 GB300"


def run_serving(args, ws, rank, local):
    """Mixed-geometry request stream through the serving loop: requests of U{1..256} frames over three
    geometries (256x256/1 pol, 512x512 with two 256x256 windows, 1024x1024/1 pol), window radius
    U(0.15, 0.32) w_max, G in {6..16}, coefficients returned to host.  A saturation run (all requests at
    once) measures the service rate; Poisson arrivals at 0.5 and 0.9 of it measure latency.  Runs with the
    FP32 and the split-BF16 overlap."""
    import numpy as np
    import torch

    import paper_2204_02348_gb300 as dh
    from synth import holograms as syn

    torch.cuda.set_device(local)
    rng = np.random.default_rng(syn.BASE_SEED + 3)
    kinds = list(syn.SERVING_KINDS)
    pools, geos = {}, {}
    for ki, kind in enumerate(kinds):
        gl = [syn.serving_geometry(kind, rng) for _ in range(8)]          # device-resident plans per kind
        geos[kind] = gl
        base = syn.make_frames(gl[0], 4, seed=syn.BASE_SEED + 50 + ki)["frames"]
        pools[kind] = torch.from_numpy(np.ascontiguousarray(np.resize(base, (256,) + base.shape[1:]))).pin_memory()
    plan_req = []
    for _ in range(args.requests):
        kind = kinds[int(rng.integers(0, 3))]
        plan_req.append((kind, int(rng.integers(0, 8)), int(rng.integers(1, 257))))
    total_frames = sum(n for _, _, n in plan_req)
    out = {}
    for prec_name, prec in (("fp32", dh.DH_PRECISION_FP32), ("split_bf16", dh.DH_PRECISION_SPLIT_BF16)):
        handles = {}
        outs = []
        for kind in kinds:
            for gi, g in enumerate(geos[kind]):
                h = dh.dh_create()
                dh.configure(h, g)
                dh.dh_set_precision(h, prec)
                handles[(kind, gi)] = h
        for kind, gi, n in plan_req:
            m, modes, _ = dh.dh_get_output_dims(handles[(kind, gi)])
            outs.append(torch.empty((n, geos[kind][gi].pol_count, modes), dtype=torch.complex64).pin_memory())

        def run(load, arr_rng, budget=8 << 30, fifo=False):
            srv = dh.dh_server_create(budget, 8)
            if fifo:
                dh.dh_server_set_admission(srv, 0, 0)   # strictly in arrival order
            try:
                # upload every plan and warm the kernels outside the clock
                for (kind, gi), h in handles.items():
                    m, modes, _ = dh.dh_get_output_dims(h)
                    tmp = torch.empty((1, geos[kind][gi].pol_count, modes), dtype=torch.complex64).pin_memory()
                    dh.dh_server_wait(srv, dh.dh_server_submit(srv, h, pools[kind], dh.DH_DTYPE_U16, 1, None, tmp), -1)
                srv2 = srv
                tickets = []
                mean_gap = None if load is None else (total_frames / len(plan_req)) / (load * out[prec_name]["saturated"])
                t0 = time.perf_counter()
                next_t = t0
                for (kind, gi, n), o in zip(plan_req, outs):
                    if mean_gap is not None:
                        next_t += float(arr_rng.exponential(mean_gap))
                        while time.perf_counter() < next_t:
                            pass
                    tickets.append(dh.dh_server_submit(srv2, handles[(kind, gi)], pools[kind], dh.DH_DTYPE_U16, n, None, o))
                for t in tickets:
                    dh.dh_server_wait(srv2, t, -1)
                wall = time.perf_counter() - t0
                st = dh.dh_server_stats(srv2)
            finally:
                dh.dh_server_destroy(srv)
            return {"frames_per_s": total_frames / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                    "max_ms": st["max_ms"], "peak_inflight": st["peak_inflight"], "peak_bytes": st["peak_bytes"],
                    "wait_p50_ms": st["wait_p50_ms"], "wait_p99_ms": st["wait_p99_ms"],
                    "kernel_p50_ms": st["kernel_p50_ms"], "kernel_p99_ms": st["kernel_p99_ms"],
                    "span_p50_ms": st["span_p50_ms"], "span_p99_ms": st["span_p99_ms"],
                    "kernel_ms_total": st["kernel_ms_total"], "bypassed": st["bypassed"],
                    "kernel_frames_per_s": total_frames / (st["kernel_ms_total"] / 1e3) if st["kernel_ms_total"] else None}

        sat = run(None, None)
        out[prec_name] = {"saturated": sat["frames_per_s"], "saturation_run": sat}
        for load in (0.5, 0.9):
            out[prec_name][f"load_{load}"] = run(load, np.random.default_rng(7))
        # the same 0.9 load with strictly arrival-ordered admission (no request passes one that does not fit)
        out[prec_name]["load_0.9_fifo"] = run(0.9, np.random.default_rng(7), fifo=True)
        # stress: the same saturated stream through a 256 MiB budget (requests chunked to fit)
        out[prec_name]["saturated_256MiB"] = run(None, None, budget=256 << 20)
        for h in handles.values():
            dh.dh_destroy(h)
    if rank == 0:
        line = {
            "metric": SERVING_METRIC, "value": out["split_bf16"]["saturated"], "unit": "frames/s", "n_gpus": ws,
            "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 FFT, split-bf16 overlap", "data": "synthetic",
            "config": {"workload": "serving: %d requests of U{1..256} frames over 256x256/1pol, 512x512/2pol, "
                                   "1024x1024/1pol; radius U(0.15,0.32) w_max; G 6..16; 8 GiB budget (and a 256 MiB "
                                   "stress run); 8 streams" %
                                   args.requests, "frames": total_frames,
                       "frame_content": "per-kind pools of seeded synthetic frames, tiled; per-request geometry from "
                                        "8 resident plans per kind", "outputs": "coefficients to pinned host memory"},
            "serving": out,
        }
        print(json.dumps(line), flush=True)


def _tiled_frames(setup, count, distinct, seed):
    """count frames of the seeded stream: `distinct` generated frames repeated (frame content does not change
    the work; the generator is the expensive part for large frames)."""
    import numpy as np
    from synth import holograms as syn
    base = syn.make_frames(setup, distinct, seed=seed)
    idx = np.arange(count) % distinct
    return base, np.ascontiguousarray(base["frames"][idx])


def precision_case(steps, dev):
    """The precision configuration (1024 frames 640x512 u16, two 256x256 windows, 96x96 fields, 120 modes) with
    the FP32 and the split-BF16 overlap: frames/s from CUDA events over `steps` batches (the 671 MB input is
    larger than L2), the step's fraction of the HBM and FP32 ceilings, per-kernel event times, and the
    split-BF16 coefficients' deviation from the FP32 ones."""
    import numpy as np
    import torch

    import paper_2204_02348_gb300 as dh
    from synth import holograms as syn
    s = syn.setup_precision()
    B = 1024
    _, frames = _tiled_frames(s, B, 16, syn.BASE_SEED + 2)
    fr = torch.from_numpy(frames).to(dev)
    peak, _ = measured_peak()
    fpk, _ = fp32_peak_tflops(dev)
    res, c_fp32 = {}, None
    for name, prec in (("fp32", dh.DH_PRECISION_FP32), ("split_bf16", dh.DH_PRECISION_SPLIT_BF16)):
        h = dh.dh_create()
        dh.configure(h, s)
        dh.dh_set_precision(h, prec)
        m, modes, _ = dh.dh_get_output_dims(h)
        f = torch.empty((B, 2, m, m), dtype=torch.complex64, device=dev)
        c = torch.empty((B, 2, modes), dtype=torch.complex64, device=dev)
        ms = _event_time(lambda: dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, B, f, c), steps, 3)
        dh.dh_set_profiling(h, True)
        dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, B, f, c)
        torch.cuda.synchronize()
        prof = dh.dh_get_profile(h)
        dh.dh_set_profiling(h, False)
        cc = c.cpu().numpy().astype(np.complex128)
        # the generic three-kernel path held, for comparison with the default
        variant = dh.dh_get_variant(h)
        dh.dh_set_variant(h, dh.DH_VARIANT_GENERIC)
        ms_g = _event_time(lambda: dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, B, f, c), steps, 3)
        dh.dh_set_variant(h, dh.DH_VARIANT_AUTO)
        # the tuner's choice for this geometry, timed the same way after the default
        dh.dh_autotune(h, fr, dh.DH_DTYPE_U16, B, f, c, reps=3)
        tuning = dh.dh_get_tuning(h)
        ms_t = _event_time(lambda: dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, B, f, c), steps, 3)
        fps = B / (ms / 1e3)
        bpf, fpf = bytes_per_frame(s, m, modes), flops_per_frame(s, m, modes)
        # DRAM traffic of a single-kernel step from the committed capture (null for other kernel sources)
        tr = recorded_traffic(next(iter(prof)), B) if len(prof) == 1 else None
        res[name] = {"frames_per_s": fps, "ms_per_batch": ms, "variant": variant,
                     "traffic_per_frame": None if tr is None else tr / B,
                     "traffic_over_algorithmic": None if tr is None else tr / B / bpf,
                     "generic": {"frames_per_s": B / (ms_g / 1e3), "ms_per_batch": ms_g},
                     "tuned": {"tuning": tuning, "frames_per_s": B / (ms_t / 1e3), "ms_per_batch": ms_t},
                     "hbm_frac": fps * bpf / 1e9 / peak, "alu_frac": fps * fpf / 1e12 / fpk,
                     "bytes_per_frame": bpf, "flops_per_frame": fpf,
                     "kernels_ms": {k: v[1] / max(v[0], 1) for k, v in prof.items()}}
        if c_fp32 is None:
            c_fp32 = cc
        else:
            dev_rel = np.linalg.norm(cc - c_fp32, axis=-1) / np.linalg.norm(c_fp32, axis=-1)
            res[name]["coef_rel_l2_vs_fp32_max"] = float(dev_rel.max())
        dh.dh_destroy(h)
    del fr
    return res


def _event_time(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def run_workload(args, ws, rank, local):
    """Secondary workloads, one JSON line each:
    plain       1 frame 128x128 float32, 15 modes, 32x32 field: latency of single-frame calls (p50/p99), device
                input and end to end from host;
    precision   1024 frames 640x512 u16, two 256x256 windows, 120 modes: FP32 and split-BF16 overlaps, frames/s,
                and the split-BF16 coefficients' deviation from the FP32 ones (accuracy against the FP64 oracle is
                what the parity tests establish);
    large_batch 2000 frames 1280x1024 u16, two 512x512 windows, 210 modes, 64 alignment candidates scored with
                the split-BF16 overlap: frames/s (every frame under all 64 candidates)."""
    import numpy as np
    import torch

    import paper_2204_02348_gb300 as dh
    from synth import holograms as syn

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = {"metric": None, "n_gpus": ws, "data": "synthetic", "vs_baseline": None, "scaling": "weak",
           "higher_is_better": True}
    if args.workload == "plain":
        s = syn.setup_plain()
        d = syn.make_frames(s, 1)
        h = dh.dh_create()
        dh.configure(h, s)
        m, modes, _ = dh.dh_get_output_dims(h)
        fr = torch.from_numpy(d["frames"]).to(dev)
        f = torch.empty((1, 1, m, m), dtype=torch.complex64, device=dev)
        c = torch.empty((1, 1, modes), dtype=torch.complex64, device=dev)
        host = torch.from_numpy(d["frames"]).pin_memory()
        hc = torch.empty((1, 1, modes), dtype=torch.complex64).pin_memory()
        hf = torch.empty((1, 1, m, m), dtype=torch.complex64).pin_memory()
        stream = torch.cuda.current_stream(dev)
        lat, lat_e2e = [], []
        for it in range(args.steps + args.warmup):
            t0 = time.perf_counter()
            dh.dh_process_batch(h, fr, dh.DH_DTYPE_F32, 1, f, c, stream)
            stream.synchronize()
            t1 = time.perf_counter()
            fr.copy_(host, non_blocking=True)
            dh.dh_process_batch(h, fr, dh.DH_DTYPE_F32, 1, f, c, stream)
            hf.copy_(f, non_blocking=True)
            hc.copy_(c, non_blocking=True)
            stream.synchronize()
            t2 = time.perf_counter()
            if it >= args.warmup:
                lat.append(1e3 * (t1 - t0))
                lat_e2e.append(1e3 * (t2 - t1))
        dh.dh_destroy(h)
        lat.sort()
        lat_e2e.sort()
        pct = lambda l, p: l[min(len(l) - 1, int(p * len(l)))]
        out.update({"metric": "single-frame latency (plain 128x128 f32 case), ms", "value": pct(lat, 0.5), "unit": "ms",
                    "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
                    "config": {"workload": "plain: 1 frame 128x128 f32, 15 modes, 32x32 field, one call per frame"},
                    "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99)},
                    "e2e_latency_ms": {"p50": pct(lat_e2e, 0.5), "p99": pct(lat_e2e, 0.99),
                                       "note": "host frame in, host field and coefficients out"}})
    elif args.workload == "precision":
        res = precision_case(max(3, args.steps // 20), dev)
        out.update({"metric": "frames/s, precision case (split-BF16 vs FP32 overlap)", "value": res["split_bf16"]["frames_per_s"],
                    "unit": "frames/s", "steps": max(3, args.steps // 20), "warmup": 3, "dtype": "f32 FFT, split-bf16 overlap",
                    "config": {"workload": "precision: 1024 frames 640x512 u16, 2 windows 256x256, 96x96 fields, 120 modes",
                               "frame_content": "16 seeded frames tiled"},
                    "precision": res,
                    "hbm_frac": {k: v["hbm_frac"] for k, v in res.items()}})
    elif args.workload == "large_batch":
        s = syn.setup_large_batch()
        # 2000 frames unless --frames names another count (smaller counts serve profiler captures)
        B, S = (2000 if args.frames == FRAMES else args.frames), 64
        _, frames = _tiled_frames(s, B, 8, syn.BASE_SEED + 4)
        fr = torch.from_numpy(frames).to(dev)
        cand = syn.candidate_settings(s, S)
        h = dh.dh_create()
        dh.configure(h, s)
        dh.dh_set_precision(h, dh.DH_PRECISION_SPLIT_BF16)
        sets = [dh.make_setting(cand["tilt_deg"][k], cand["defocus"][k], cand["waist"][k]) for k in range(S)]
        pw = torch.empty((B, S), dtype=torch.float32, device=dev)
        dh.dh_set_profiling(h, True)
        ms = _event_time(lambda: dh.dh_score_settings(h, fr, dh.DH_DTYPE_U16, B, sets, pw), 2, 1)
        prof = dh.dh_get_profile(h)
        dh.dh_destroy(h)
        out.update({"metric": "frames/s scored under 64 alignment candidates (large case, split-BF16)", "value": B / (ms / 1e3),
                    "unit": "frames/s", "steps": 2, "warmup": 1, "dtype": "f32 FFT, split-bf16 overlap",
                    "config": {"workload": f"large_batch: {B} frames 1280x1024 u16, 2 windows 512x512, 176x176 fields, 210 "
                                           "modes, 64 candidates (tilt +-0.02 deg, defocus U(0,0.05) waves, waist x U(0.9,1.1))",
                               "frame_content": "8 seeded frames tiled"},
                    "ms_per_batch": ms, "candidate_windows_per_s": B * 2 * S / (ms / 1e3),
                    "kernels": {k: {"launches": v[0], "total_ms": v[1]} for k, v in prof.items()}})
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_extensions(args, ws, rank, local):
    """The optional stages on the batching geometry (320x256 u16 frames, two 128x128 windows, M = 64, 45 modes),
    one JSON line: batch averaging (4000 input frames in sequential groups of 4 -> 1000 outputs), LG
    coefficients, fill-factor correction, reference-wave calibration (1000 frames each), transfer-matrix metrics
    of a 90 x 90 coefficient batch, and the fine-alignment search on 16 frames from a perturbed start.  Device
    buffers; CUDA events on the launching stream; per-kernel times from the library's profiler."""
    import numpy as np
    import torch

    import paper_2204_02348_gb300 as dh
    from synth import holograms as syn

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    steps = max(5, args.steps // 20)
    base = syn.setup_batching()
    res = {}

    def timed(setup, frames, call, n_out, extra=None):
        h = dh.dh_create()
        dh.configure(h, setup)
        m, modes, _ = dh.dh_get_output_dims(h)
        fr = torch.from_numpy(frames).to(dev)
        f = torch.empty((n_out, setup.pol_count, m, m), dtype=torch.complex64, device=dev)
        c = torch.empty((n_out, setup.pol_count, modes), dtype=torch.complex64, device=dev)
        for _ in range(3):
            call(h, fr, f, c)
        torch.cuda.synchronize()
        dh.dh_set_profiling(h, True)
        ms = _event_time(lambda: call(h, fr, f, c), steps, 0)
        prof = dh.dh_get_profile(h)
        dh.dh_destroy(h)
        out = {"ms_per_call": ms, "kernels": {k: {"launches": v[0], "ms_per_call": v[1] / steps} for k, v in prof.items()}}
        out.update(extra or {})
        return out

    # batch averaging: 1000 groups of 4 sequential frames
    A, G = 4, 1000
    d = syn.make_avg_frames(base, 16, A, 0, seed=syn.BASE_SEED + 20)
    frames = np.ascontiguousarray(np.resize(d["frames"], (A * G,) + d["frames"].shape[1:]))
    r = timed(base, frames, lambda h, fr, f, c: dh.dh_process_batch_avg(h, fr, dh.DH_DTYPE_U16, G, A, 0, f, c), G)
    r["input_frames_per_s"] = A * G / (r["ms_per_call"] / 1e3)
    r["output_fields_per_s"] = G / (r["ms_per_call"] / 1e3)
    res["averaging_4_sequential"] = r
    # LG basis, fill factor, reference calibration: 1000 frames each
    _, frames = _tiled_frames(base, 1000, 16, syn.BASE_SEED + 21)
    plain_call = lambda h, fr, f, c: dh.dh_process_batch(h, fr, dh.DH_DTYPE_U16, 1000, f, c)
    for name, setup in (("lg_basis", syn.with_(base, basis="lg")), ("fill_factor", syn.with_(base, fill_factor=True))):
        r = timed(setup, frames, plain_call, 1000)
        r["frames_per_s"] = 1000 / (r["ms_per_call"] / 1e3)
        res[name] = r
    cal, amp = syn.reference_profile(base, sigma_fraction=0.15, floor=200)
    sc = syn.with_(base, ref_amplitude=amp, ref_cal=cal)
    _, frames_c = _tiled_frames(sc, 1000, 16, syn.BASE_SEED + 22)
    r = timed(sc, frames_c, plain_call, 1000)
    r["frames_per_s"] = 1000 / (r["ms_per_call"] / 1e3)
    res["ref_calibration"] = r
    # transfer-matrix metrics of a 90 x 90 batch (45 frames x 2 pols would be rectangular: use 90 rows)
    rng = np.random.default_rng(syn.BASE_SEED + 23)
    coefs = torch.from_numpy((rng.standard_normal((90, 2, 45)) + 1j * rng.standard_normal((90, 2, 45))).astype(np.complex64)).to(dev)
    h = dh.dh_create()
    dh.configure(h, base)
    dh.dh_calc_metrics(h, coefs, 90)
    t0 = time.perf_counter()
    for _ in range(steps):
        vals, _ = dh.dh_calc_metrics(h, coefs, 90)
    res["metrics_90x90"] = {"ms_per_call": 1e3 * (time.perf_counter() - t0) / steps, "IL_dB": vals["IL"], "MDL_dB": vals["MDL"]}
    dh.dh_destroy(h)
    # fine-alignment search on 16 frames from a perturbed start
    s16 = syn.setup_batching()
    d16 = syn.make_frames(s16, 16, seed=syn.BASE_SEED + 24)
    off = syn.with_(s16, tilt_deg=[(t[0] + 0.03, t[1] - 0.02) for t in s16.tilt_deg], waist=[w * 1.05 for w in s16.waist])
    h = dh.dh_create()
    dh.configure(h, off)
    fr = torch.from_numpy(d16["frames"]).to(dev)
    t0 = time.perf_counter()
    power, its = dh.dh_auto_align(h, fr, dh.DH_DTYPE_U16, 16)
    wall = time.perf_counter() - t0
    tilt, _, waist = dh.dh_get_alignment(h)
    dh.dh_destroy(h)
    res["auto_align_16_frames"] = {"ms_per_search": 1e3 * wall, "scorings": its, "candidates_per_scoring": 17,
                                   "tilt_error_deg": max(abs(tilt[p][a] - s16.tilt_deg[p][a]) for p in range(2) for a in range(2)),
                                   "waist_rel_error": max(abs(waist[p] / s16.waist[p] - 1) for p in range(2))}
    if rank == 0:
        print(json.dumps({"metric": "optional stages on the batching geometry (frames/s per stage)",
                          "value": res["averaging_4_sequential"]["input_frames_per_s"], "unit": "input frames/s",
                          "n_gpus": ws, "steps": steps, "warmup": 3, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": "extensions: batching geometry 320x256 u16, 2 windows 128x128, M 64, 45 modes",
                                     "frame_content": "16 seeded frames tiled"},
                          "extensions": res}), flush=True)


def main():
    args = parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "serving":
        run_serving(args, ws, rank, local)
    elif args.workload in ("plain", "precision", "large_batch"):
        run_workload(args, ws, rank, local)
    elif args.workload == "extensions":
        run_extensions(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
