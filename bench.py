#!/usr/bin/env python
"""Benchmark of the sliCQ hot path: forward + inverse of a 60 s stereo clip.

One step = slicq_forward (Algorithm 3: slicing, real FFT_2N, band multiply
and fold, per-band inverse FFT) + slicq_inverse (Algorithm 4: per-band FFT,
dual-window multiply and overlap into the slice spectrum, inverse real
FFT_2N, overlap-add) of 2 x 2,646,000 samples at 44.1 kHz with B = 48,
fmin = 32.7 Hz, fmax = 22050 Hz, 2N = 65536, M = 16384 (Hann windows).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  The L2 cache is flushed (256 MiB write)
between timed steps, outside the per-step CUDA events.  N > 1 runs N
independent replicas (one clip per GPU; the transform has no exchange step).
--impl reference times the FP64 CPU oracle (the only other implementation
of the method) on the host cores instead.

Beside the step the line reports the sliCQ spectrogram epilogue, the
streaming mode's per-call latency, the differentiation workload
(multi-resolution log-magnitude loss and its backward through the adjoint),
the split-precision tensor-core band DFTs against the FP32 form, and the
ragged batch of 256 clips over 16 plans (one CUDA-graph replay per step).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sliCQ fwd+inv audio samples/s on 1 GB300 at rel. err ≤1e-5; % HBM roofline"
UNIT = "samples/s"
WORKLOAD = dict(fs=44100.0, fmin=32.7, fmax=22050.0, bins_per_octave=48, slice_len=65536,
                trans_len=16384, seconds=60, channels=2)
WORKLOAD_NAME = ("60 s stereo 44.1 kHz, pink noise + 20 decaying harmonic tones; Hann CQ windows "
                 "B=48, fmin=32.7 Hz, fmax=22050 Hz; slice 2N=65536, transition 16384")
KERNELS = ("slice_forward", "band_analysis", "band_synthesis", "band_boundary", "slice_inverse",
           "slice_ola", "spectrogram")


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1210_0084_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = _source_sha()
    for line in open(path):
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if kv.get("kernel") == kernel and kv.get("source_sha") == sha:
            try:
                return float(kv["dram_bytes_per_launch"])
            except (KeyError, ValueError):
                return None
    return None


def max_over_ranks(value, world, device=None):
    """The largest of a per-rank value over all ranks (the slowest replica sets
    the step time); the value itself with one rank.  Needs an initialised
    process group when world > 1 (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi clock / throttle samples while the GPU works."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.samples = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu=timestamp,{self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                self.samples.append(dict(sm=float(parts[1]), sm_max=float(parts[2]),
                                         hw=parts[5], hw_th=parts[6], sw_th=parts[7],
                                         sw_pc=parts[8]))
            except ValueError:
                pass

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [s["sm"] for s in self.samples]
        reasons = set()
        for s in self.samples:
            for key, name in (("hw", "hw_slowdown"), ("hw_th", "hw_thermal_slowdown"),
                              ("sw_th", "sw_thermal_slowdown"), ("sw_pc", "sw_power_cap")):
                if s[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(s["sm_max"] for s in self.samples),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------- CPU oracle ---

def _oracle_job(args):
    """FP64 oracle forward + inverse of one segment (runs in a spawned worker)."""
    seg, p = args
    import numpy as np
    import oracle as O
    plan = O.make_plan(O.SliCQParams(*p))
    c = O.slicq_forward(seg.astype(np.float64), plan)
    y = O.slicq_inverse(c, plan, seg.shape[0])
    return seg.shape[0], float(np.linalg.norm(y - seg) / np.linalg.norm(seg))


def _oracle_pool(workers):
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    return mp.get_context("spawn").Pool(workers)


def _oracle_segments(x, count, seg_len):
    n = x.shape[-1]
    segs = []
    for i in range(count):
        ch = i % x.shape[0]
        off = (i * 7919 * seg_len) % max(1, n - seg_len)
        segs.append(x[ch, off:off + seg_len].copy())
    return segs


def _oracle_params():
    w = WORKLOAD
    return (w["fs"], w["fmin"], w["fmax"], w["bins_per_octave"], w["slice_len"], w["trans_len"])


def cpu_baseline(x, seconds_target=15.0):
    """Time the oracle on the host cores over a bounded sample of the workload."""
    cores = os.cpu_count() or 1
    seg_len = 2 * WORKLOAD["slice_len"]      # 4 slices of the workload's plan per job
    pool = _oracle_pool(cores)
    try:
        pool.map(_oracle_job, [(s, _oracle_params()) for s in _oracle_segments(x, cores, WORKLOAD["slice_len"])])
        jobs, done, t0 = 0, 0, time.perf_counter()
        while time.perf_counter() - t0 < seconds_target and jobs < 64 * cores:
            segs = _oracle_segments(x[:, (jobs * 131) % 1000:], cores, seg_len)
            res = pool.map(_oracle_job, [(s, _oracle_params()) for s in segs])
            done += sum(r[0] for r in res)
            jobs += cores
        dt = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{jobs} segments of {seg_len} samples of the workload (FP64 forward + "
                      f"inverse per segment, one process per core, {dt:.1f} s wall)"}


def run_reference(args, x, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    seg_len = WORKLOAD["slice_len"]
    pool = _oracle_pool(cores)
    times, samples = [], 0
    try:
        for i in range(args.warmup + args.steps):
            segs = _oracle_segments(x[:, (i * 97) % 1000:], cores, seg_len)
            t0 = time.perf_counter()
            res = pool.map(_oracle_job, [(s, _oracle_params()) for s in segs])
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                times.append(dt)
                samples = sum(r[0] for r in res)
    finally:
        pool.close()
        pool.join()
    ms = 1e3 * statistics.mean(times)
    value = samples / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: {cores} segments of {seg_len} samples of the "
                                   "workload, FP64 forward + inverse, one process per core"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(world, mk_policy="pow2", precision="fp32", slice_cluster=None):
    name = WORKLOAD_NAME + ("" if mk_policy == "pow2" else "; rectangular representation (one M_k)")
    name += "" if precision == "fp32" else f"; band DFT stages {precision} on the tensor cores"
    return {"workload": name, "fs": WORKLOAD["fs"], "bins_per_octave": WORKLOAD["bins_per_octave"],
            "fmin": WORKLOAD["fmin"], "fmax": WORKLOAD["fmax"], "slice_len": WORKLOAD["slice_len"],
            "trans_len": WORKLOAD["trans_len"], "channels": WORKLOAD["channels"],
            "samples_per_channel": WORKLOAD["seconds"] * int(WORKLOAD["fs"]),
            "mk_policy": mk_policy, "precision": precision, "slice_cluster": slice_cluster,
            "l2": "flushed between timed steps (256 MiB write, outside the events)",
            "parallelism": f"replicas x{world} (independent clips, no exchange)"}


def differentiation(dev, stream, flush, peak, steps=10, warmup=3):
    """Differentiation workload: batch 32 x 6 s mono at 44.1 kHz (noisy/clean
    tone mixtures), multi-resolution log-magnitude L1 loss over B = 12, 24, 48
    (fmin 40 Hz, fmax 22050 Hz, 2N 8192, M 2048, eps 1e-6).  One step =
    three forward transforms of the noisy batch through slicq_transform,
    three of the clean batch, the loss (torch elementwise ops) and its
    backward (three slicq_adjoint calls).  Also timed: the nine transforms
    alone on the same buffers, so the loss arithmetic's share is visible."""
    import torch
    from paper_1210_0084_gb300 import signals
    from paper_1210_0084_gb300.slicq import SliCQParams, SliCQPlan, slicq_transform

    fs, n, batch, eps = 44100.0, 6 * 44100, 32, 1e-6
    noisy, clean = signals.noisy_clean_tone_mixtures(batch, n, fs, seed=signals.seed_for(4))
    plans = [SliCQPlan(SliCQParams(fs, 40.0, fs / 2, B, 8192, 2048), dev.index) for B in (12, 24, 48)]
    xt = torch.from_numpy(noisy).to(dev)
    tt = torch.from_numpy(clean).to(dev)

    def step():
        x = xt.detach().requires_grad_(True)
        loss = 0.0
        for p in plans:
            c = slicq_transform(x, p)
            with torch.no_grad():
                ct = p.forward(tt)
            loss = loss + (torch.log(c.abs() + eps) - torch.log(ct.abs() + eps)).abs().mean()
        loss.backward()
        return loss

    coefs = [torch.empty((batch, p.num_slices(n), p.coefs_per_slice), dtype=torch.complex64, device=dev)
             for p in plans]
    ct_buf = [torch.empty_like(c) for c in coefs]
    g_buf = torch.empty((batch, n), dtype=torch.float32, device=dev)

    def transforms():
        for p, c, ct in zip(plans, coefs, ct_buf):
            p.forward(xt, out=c)
            p.forward(tt, out=ct)
            p.adjoint(c, n, out=g_buf)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for i in range(steps):
            flush.fill_(i & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    step_ms = timed(step)
    tr_ms = timed(transforms)
    # algorithmic bytes of the nine transforms: forward 4 + 8 cps/N per input
    # sample, adjoint 8 cps/N + 4 (per resolution, noisy forward + clean
    # forward + adjoint)
    tr_bytes = 0
    for p in plans:
        S, cps = p.num_slices(n), p.coefs_per_slice
        tr_bytes += 3 * batch * (4 * n + 8 * S * cps)
    return {"workload": "batch 32 x 6 s mono 44.1 kHz, noisy/clean tone mixtures; log-magnitude L1 "
                        "loss over B = 12, 24, 48 (fmin 40 Hz, 2N 8192, M 2048); custom backward",
            "ms_per_step": step_ms, "samples_per_s": batch * n / (step_ms * 1e-3),
            "transforms_ms": tr_ms, "transforms_alg_bytes": tr_bytes,
            "transforms_gbs": tr_bytes / (tr_ms * 1e-3) / 1e9,
            "transforms_frac": tr_bytes / (tr_ms * 1e-3) / 1e9 / peak,
            "loss_share": max(0.0, 1.0 - tr_ms / step_ms)}


def precision_compare(dev, stream, flush, x_stereo, steps=10, warmup=3):
    """The plain FP32 form against the split-precision tensor-core band DFTs
    (FP16 and BF16 hi + lo), forward + inverse at equal inputs: the headline
    60 s stereo workload and the 10 min mono 48 kHz workload (B = 96,
    fmin 27.5 Hz, fmax 24 kHz, 2N 131072, M 32768; noise + exponential
    chirps).  Per precision: ms per step, samples/s, reconstruction error,
    and the traced band-kernel times."""
    import torch
    from paper_1210_0084_gb300 import signals
    from paper_1210_0084_gb300.slicq import SliCQParams, SliCQPlan

    n10 = 600 * 48000
    x10 = signals.noise_plus_chirps(n10, 48000.0, seed=signals.seed_for(3))[None]
    workloads = [
        ("60 s stereo 44.1 kHz, B 48, 2N 65536", x_stereo,
         (WORKLOAD["fs"], WORKLOAD["fmin"], WORKLOAD["fmax"], WORKLOAD["bins_per_octave"],
          WORKLOAD["slice_len"], WORKLOAD["trans_len"])),
        ("10 min mono 48 kHz, B 96, fmin 27.5 Hz, 2N 131072, M 32768", x10,
         (48000.0, 27.5, 24000.0, 96, 131072, 32768)),
    ]
    out = []
    for name, x, prm in workloads:
        xd = torch.from_numpy(x).to(dev)
        batch, n = x.shape
        res = {"workload": name, "samples": batch * n}
        for prec in ("fp32", "split_fp16", "split_bf16"):
            plan = SliCQPlan(SliCQParams(*prm, precision=prec), dev.index)
            S = plan.num_slices(n)
            c = torch.empty((batch, S, plan.coefs_per_slice), dtype=torch.complex64, device=dev)
            y = torch.empty((batch, n), dtype=torch.float32, device=dev)
            for _ in range(warmup):
                plan.forward(xd, out=c)
                plan.inverse(c, n, out=y)
            torch.cuda.synchronize()
            ms = []
            for i in range(steps):
                flush.fill_(i & 255)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.forward(xd, out=c)
                plan.inverse(c, n, out=y)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            plan.trace(True)
            for i in range(steps):
                flush.fill_(i & 255)
                plan.forward(xd, out=c)
                plan.inverse(c, n, out=y)
            torch.cuda.synchronize()
            per = {}
            for k, t in plan.trace_read():
                per.setdefault(k, []).append(t)
            plan.trace(False)
            plan.check()
            med = statistics.median(ms)
            res[prec] = {"ms_per_step": med, "samples_per_s": batch * n / (med * 1e-3),
                         "recon_rel_err": float(torch.linalg.norm(y - xd) / torch.linalg.norm(xd)),
                         "band_analysis_ms": statistics.mean(per.get("band_analysis", [0.0])),
                         "band_synthesis_ms": statistics.mean(per.get("band_synthesis", [0.0]))}
            del plan, c, y
        for prec in ("split_fp16", "split_bf16"):
            res[prec]["speedup_vs_fp32"] = res["fp32"]["ms_per_step"] / res[prec]["ms_per_step"]
        out.append(res)
        del xd
    return out


# ---------------------------------------------------------------- native ---

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-clock-load", action="store_true",
                    help="skip the 1 s load phases around the timed region (for profiler runs)")
    ap.add_argument("--mk-policy", choices=("pow2", "const"), default="pow2",
                    help="band lengths: pow2 (headline) or const (rectangular representation)")
    ap.add_argument("--precision", choices=("fp32", "split_fp16", "split_bf16"), default="fp32",
                    help="band-DFT arithmetic of the timed step (fp32 is the headline)")
    ap.add_argument("--slice-cluster", type=int, default=0,
                    help="CTAs per slice FFT; 0 lets the plan time the valid sizes and keep the "
                         "fastest (pin it under a profiler, whose serialised launches skew that timing)")
    ap.add_argument("--only-step", action="store_true",
                    help="time the step and its kernels only (no e2e, epilogue, streaming, "
                         "differentiation, precision or CPU measurements)")
    ap.add_argument("--workload", choices=("stereo60", "ragged"), default="stereo60",
                    help="stereo60: the headline workload; ragged: 256 clips over 16 plans "
                         "in one CUDA-graph replay per step")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.workload == "ragged":
        run_ragged(args, rank, world, local_rank)
        return

    import numpy as np
    from paper_1210_0084_gb300 import signals

    n = WORKLOAD["seconds"] * int(WORKLOAD["fs"])
    x = signals.pink_noise_harmonic_tones(n, WORKLOAD["fs"], WORKLOAD["channels"],
                                          seed=signals.seed_for(1, rank))
    if args.impl == "reference":
        run_reference(args, x, rank, world)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if local_rank == 0:
        from paper_1210_0084_gb300 import build as B
        B.build()
    if world > 1:
        dist.barrier()
    from paper_1210_0084_gb300.slicq import SliCQParams, SliCQPlan

    p = SliCQParams(WORKLOAD["fs"], WORKLOAD["fmin"], WORKLOAD["fmax"], WORKLOAD["bins_per_octave"],
                    WORKLOAD["slice_len"], WORKLOAD["trans_len"], mk_policy=args.mk_policy,
                    precision=args.precision, slice_cluster=args.slice_cluster)
    plan = SliCQPlan(p, local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    batch = x.shape[0]
    xd = torch.from_numpy(x).to(dev)
    S = plan.num_slices(n)
    c = torch.empty((batch, S, plan.coefs_per_slice), dtype=torch.complex64, device=dev)
    y = torch.empty((batch, n), dtype=torch.float32, device=dev)
    plan.workspace(n, batch)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        plan.forward(xd, out=c)
        plan.inverse(c, n, out=y)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    recon_err = float(torch.linalg.norm(y - xd) / torch.linalg.norm(xd))

    props = torch.cuda.get_device_properties(dev)
    try:
        gpu_id = "%08X:%02X:%02X.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:
        gpu_id = str(local_rank)
    # keep the GPU busy for ~1 s before the timed region so the clock samples
    # below see the loaded state
    sampler = ClockSampler(gpu_id)
    t_end = time.perf_counter() + (0.0 if args.no_clock_load else 1.0)
    while time.perf_counter() < t_end:
        for _ in range(20):
            step()
        torch.cuda.synchronize()

    # the timed steps run without the per-kernel trace: its events between
    # launches would serialise kernels that otherwise overlap their start-up
    # with the previous kernel's tail (programmatic dependent launch)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i & 255)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # per-kernel times: the same number of steps again with the trace on
    plan.trace(True)
    for i in range(args.steps):
        flush.fill_(i & 255)
        step()
    torch.cuda.synchronize()
    traced = plan.trace_read()
    plan.trace(False)
    # a second second of load, so that short timed regions still get samples
    t_end = time.perf_counter() + (0.0 if args.no_clock_load else 0.5)
    while time.perf_counter() < t_end:
        for _ in range(20):
            step()
        torch.cuda.synchronize()
    sampler.stop()

    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ms, world, dev)
    samples_all = batch * n * world
    value = samples_all / (ms_max / 1e3)

    # per-kernel launch times (events around each launch on the call's stream)
    per = {k: [] for k in KERNELS}
    for name, t in traced:
        per[name].append(t)
    cps = plan.coefs_per_slice
    # band_boundary and slice_ola move no algorithmic bytes (they add the two
    # partial sums of the bins two band groups share and of the transition
    # samples two slices share)
    alg_bytes = {"slice_forward": batch * n * 4, "band_analysis": batch * S * cps * 8,
                 "band_synthesis": batch * S * cps * 8, "band_boundary": 0,
                 "slice_inverse": batch * n * 4, "slice_ola": 0,
                 "spectrogram": batch * S * cps * 10}
    peak, peak_kind = _peaks()
    kern = {}
    for k in KERNELS:
        if per[k]:
            avg = statistics.mean(per[k])
            kern[k] = {"launches": len(per[k]), "avg_ms": avg, "share": sum(per[k]),
                       "alg_bytes_per_launch": alg_bytes[k],
                       "gbs": alg_bytes[k] / (avg * 1e-3) / 1e9}
    tot = sum(v["share"] for v in kern.values()) or 1.0
    for v in kern.values():
        v["share"] = v["share"] / tot
    dom = max(kern, key=lambda k: kern[k]["share"])
    traffic = _ncu_traffic(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak,
                "unit": "GB/s", "frac": kern[dom]["gbs"] / peak, "traffic": traffic,
                "peak_kind": f"of {peak_kind}"}
    step_bytes = batch * (8 * n + 16 * S * cps)
    step_roof = {"alg_bytes": step_bytes, "achieved": step_bytes / (ms * 1e-3) / 1e9,
                 "frac": step_bytes / (ms * 1e-3) / 1e9 / peak}

    if args.only_step:
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _config(world, args.mk_policy, args.precision, plan.slice_cluster), "recon_rel_err": recon_err,
                "roofline": roofline, "step_roofline": step_roof, "kernels": kern,
                "gpu_launches": len(traced), "clocks": sampler.summary(),
                "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms)}), flush=True)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # end to end through the public API with pinned host buffers
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty((batch, n), dtype=torch.float32).pin_memory()
    xin = torch.empty_like(xd)
    e_ms = []
    for i in range(args.warmup + args.e2e_steps):
        flush.fill_(i & 255)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        xin.copy_(xh, non_blocking=True)
        plan.forward(xin, out=c)
        plan.inverse(c, n, out=y)
        yh.copy_(y, non_blocking=True)
        s1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e_ms.append(s0.elapsed_time(s1))
    serial_ms = statistics.mean(e_ms)
    serial_err = float(np.linalg.norm(yh.numpy() - x) / np.linalg.norm(x))
    # the same step with the channels on their own streams: channel 1's upload
    # overlaps channel 0's transforms, channel 0's download channel 1's
    yh.zero_()
    chan_streams = [torch.cuda.Stream(dev) for _ in range(batch)]
    e_ms = []
    for i in range(args.warmup + args.e2e_steps):
        flush.fill_(i & 255)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for b, cs_ in enumerate(chan_streams):
            cs_.wait_stream(stream)
            with torch.cuda.stream(cs_):
                xin[b].copy_(xh[b], non_blocking=True)
                plan.forward(xin[b:b + 1], out=c[b:b + 1])
                plan.inverse(c[b:b + 1], n, out=y[b:b + 1])
                yh[b].copy_(y[b], non_blocking=True)
        for cs_ in chan_streams:
            stream.wait_stream(cs_)
        s1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e_ms.append(s0.elapsed_time(s1))
    e2e_err = float(np.linalg.norm(yh.numpy() - x) / np.linalg.norm(x))
    e_ms_max = max_over_ranks(statistics.mean(e_ms), world, dev)
    e2e = {"value": samples_all / (e_ms_max / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(xh.numel() * 4), "d2h_bytes_per_step": int(yh.numel() * 4),
           "ms_per_step": e_ms_max, "recon_rel_err": e2e_err,
           "how": "one stream per channel: upload, forward, inverse, download; the channels' "
                  "copies overlap each other's transforms",
           "serial": {"ms_per_step": serial_ms, "value": samples_all / (serial_ms / 1e3),
                      "recon_rel_err": serial_err}}

    # the sliCQ spectrogram |s0 + s1|^2 of the step's coefficients (Sec. 4.1):
    # not part of the step; timed alone (reads every coefficient once, writes
    # one float per two coefficients)
    spec = torch.empty((batch, S * (cps // 2)), dtype=torch.float32, device=dev)
    for _ in range(3):
        plan.spectrogram(c, n, out=spec)
    sp_ms = []
    for i in range(10):
        flush.fill_(i & 255)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        plan.spectrogram(c, n, out=spec)
        s1.record(stream)
        torch.cuda.synchronize()
        sp_ms.append(s0.elapsed_time(s1))
    sp_bytes = batch * S * cps * 10
    sp_avg = statistics.median(sp_ms)
    epilogues = {"spectrogram": {"ms": sp_avg, "alg_bytes": sp_bytes,
                                 "gbs": sp_bytes / (sp_avg * 1e-3) / 1e9,
                                 "frac": sp_bytes / (sp_avg * 1e-3) / 1e9 / peak,
                                 "bound": "hbm", "peak_kind": f"of {peak_kind}"}}

    # streaming mode: one slice per call (N new samples in, one slice of
    # coefficients out; one slice in, N samples out), per-call latency
    from paper_1210_0084_gb300.slicq import SliCQStream
    sst = SliCQStream(plan)
    hop = sst.hop
    blk = xd[0, :hop].contiguous()
    cs = torch.empty(cps, dtype=torch.complex64, device=dev)
    ys = torch.empty(hop, dtype=torch.float32, device=dev)
    for _ in range(5):
        sst.forward(blk, out=cs)
        sst.inverse(cs, out=ys)
    f_ms, i_ms = [], []
    for _ in range(20):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        sst.forward(blk, out=cs)
        e1.record(stream)
        sst.inverse(cs, out=ys)
        e2.record(stream)
        torch.cuda.synchronize()
        f_ms.append(e0.elapsed_time(e1))
        i_ms.append(e1.elapsed_time(e2))
    fm, im = statistics.median(f_ms), statistics.median(i_ms)
    streaming = {"hop_samples": hop, "forward_ms_per_call": fm, "inverse_ms_per_call": im,
                 "realtime_factor": (hop / WORKLOAD["fs"]) / ((fm + im) * 1e-3),
                 "delay_samples": "one slice: output lags input by N - a0 - 1 after a slice's block"}
    del sst

    diff = differentiation(dev, stream, flush, peak)
    prec_cmp = precision_compare(dev, stream, flush, x)
    ragged = ragged_measure(rank, local_rank, steps=5, warmup=3) if world == 1 else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(x)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(world, args.mk_policy, args.precision, plan.slice_cluster), "recon_rel_err": recon_err,
            "roofline": roofline, "step_roofline": step_roof, "kernels": kern, "epilogues": epilogues,
            "streaming": streaming, "differentiation": diff, "precision": prec_cmp,
            "ragged_batch": ragged,
            "gpu_launches": len(traced), "e2e": e2e, "cpu_baseline": cpu,
            "clocks": sampler.summary(), "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


RAGGED_WORKLOAD = ("ragged batch: 256 mono clips, 1-30 s, fs {16, 22.05, 44.1, 48} kHz, "
                   "B {12, 24, 48, 96}, fmin 50 Hz, fmax min(22 kHz, fs/2), 2N 16384, "
                   "M 4096; one CUDA-graph replay per step")


def ragged_measure(rank, local_rank, steps, warmup, world=1):
    """256 mono clips, lengths U[1, 30] s, fs in {16, 22.05, 44.1, 48} kHz, B in
    {12, 24, 48, 96}; fmin 50 Hz, fmax min(22 kHz, fs/2), 2N = 16384, M = 4096.
    One step = batch forward + batch inverse, captured once in a CUDA graph
    (plans as parallel branches) and replayed.  Returns the measurements
    (time max over ranks when world > 1)."""
    import torch
    from paper_1210_0084_gb300 import signals
    from paper_1210_0084_gb300.slicq import SliCQBatch, SliCQParams, SliCQPlan

    clips = signals.ragged_clips(256, seed=signals.seed_for(3, rank))
    keys = sorted({(c.fs, c.bins_per_octave) for c in clips})
    plans = [SliCQPlan(SliCQParams(fs, 50.0, min(22000.0, fs / 2), B, 16384, 4096), local_rank)
             for fs, B in keys]
    clip_plan = [keys.index((c.fs, c.bins_per_octave)) for c in clips]
    lens = [c.signal.shape[0] for c in clips]
    batch = SliCQBatch(plans, clip_plan, lens)
    sig = batch.pack([c.signal for c in clips])
    coef = torch.empty(batch.coef_total, dtype=torch.complex64, device=sig.device)
    rec = torch.zeros_like(sig)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=sig.device)
    batch.forward(sig, coef)
    batch.inverse(coef, rec)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    with torch.cuda.stream(cs):
        with torch.cuda.graph(g, stream=cs):
            batch.forward(sig, coef)
            batch.inverse(coef, rec)
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    err = max(float(torch.linalg.norm(batch.clip_signal(rec, c) - batch.clip_signal(sig, c)) /
                    torch.linalg.norm(batch.clip_signal(sig, c))) for c in range(len(clips)))
    stream = torch.cuda.current_stream()
    st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(i & 255)
        st[i].record(stream)
        g.replay()
        en[i].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(s.elapsed_time(e) for s, e in zip(st, en))
    ms_max = max_over_ranks(ms, world, sig.device)
    total = int(sum(lens))
    step_bytes = sum(8 * lens[c] + 16 * int(batch.slices[c]) * plans[clip_plan[c]].coefs_per_slice
                     for c in range(len(clips)))
    peak, peak_kind = _peaks()
    return {"workload": RAGGED_WORKLOAD, "clips": len(clips), "plans": len(plans), "samples": total,
            "ms_per_step": ms_max, "samples_per_s": total * world / (ms_max / 1e3),
            "max_clip_recon_rel_err": err,
            "step_roofline": {"alg_bytes": step_bytes, "achieved": step_bytes / (ms * 1e-3) / 1e9,
                              "peak": peak, "frac": step_bytes / (ms * 1e-3) / 1e9 / peak,
                              "peak_kind": f"of {peak_kind}"}}


def run_ragged(args, rank, world, local_rank):
    """The ragged batch as the bench's workload: its own JSON line."""
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if local_rank == 0:
        from paper_1210_0084_gb300 import build as B
        B.build()
    if world > 1:
        dist.barrier()
    r = ragged_measure(rank, local_rank, args.steps, args.warmup, world)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": r["samples_per_s"], "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": RAGGED_WORKLOAD, "clips": r["clips"], "plans": r["plans"],
                       "samples": r["samples"],
                       "l2": "flushed between timed steps (256 MiB write, outside the events)"},
            "max_clip_recon_rel_err": r["max_clip_recon_rel_err"],
            "step_roofline": r["step_roofline"],
        }), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
