#!/usr/bin/env python3
"""Throughput of the FX correlator on the paper's real-time workload.

Workload (Sec. 1 of the paper: 44 elements, 4-bit, 512-point FFT, sampling
rate restricted to ~35 MS/s): N = 44 antennas, K = 512, one step = one 1 s
integration at 35 MS/s = 68359 whole spectra per antenna (35e6 // 512),
pushed through the C ABI in 2^20-sample chunks (33 x 2048 spectra + 775),
then dumped to a device buffer.  Input: seeded synthetic 4-bit data (N(0, 2)
noise + 1% correlated component + a 0.5 LSB tone at channel 97), 770 MB per
step resident in HBM -- larger than the 126 MB L2, so no flush is needed.

value       antenna-samples/s over the timed steps (whole job);
rtf         real-time factor = value / (N * 35e6);
e2e         same metric through the C ABI from pinned host memory, H2D of each
            step's input and D2H of its visibilities inside the timed region;
roofline    dominant kernel: algorithmic work per launch / its CUDA-event time;
cpu_baseline the FP64 oracle on the host cores, on a bounded sample.

``--impl reference`` times the oracle itself (the only reference this method
has) on the same metric, one bounded sample of the workload per step.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "antenna-samples/s & real-time factor (44 el, 35 MS/s); TC vs FP32 at stated error"
UNIT = "antenna-samples/s"
N_ANT, K_FFT, RATE = 44, 512, 35e6
SPEC_PER_STEP = int(RATE // K_FFT)            # 68359 whole spectra in 1 s
CHUNK_FRAMES = (1 << 20) // K_FFT             # 2048 spectra per push
SEED = 11020148 + 2
PROF_EVERY = 10
# The paper's cluster handles the real-time rate of this workload:
# 770e6 B/s of 4-bit samples = 1.54e9 antenna-samples/s (Sec. 1, abstract).
PAPER_RATE = N_ANT * RATE

# DRAM bytes (read + write) of one launch of the dominant kernel over the
# given number of frames, from one ncu capture of the current kernels
# (summaries under profiles/); scaled to the average launch below.  Remove an
# entry when its kernel changes.
NCU_TRAFFIC = {
    ("fengine", "fp32"): (145.93e6, 2048,
                          "ncu --set full, fengine_k512<SPEC_F16X2, corrections off>, one "
                          "2048-frame launch: 23.09 MB read + 122.84 MB written "
                          "(profiles/fengine_k512_n44_2048frames_fp32.txt)"),
}

# Tensor-pipe activity of the X-engine's one pass over a whole 1 s
# integration (the configuration timed here), from one ncu capture
# (sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_elapsed, summary
# under profiles/).  Remove an entry when its kernel changes.
NCU_XENGINE_TENSOR_PCT = {
    "fp32": 36.38,   # profiles/xengine_tc_n44_k512_onepass_fp32.txt
}

WORKLOAD = ("N=44 antennas, K=512-point real FFT -> 256 channels, 990 outputs/channel, "
            "35 MS/s, 1 s integration = 68359 spectra per step in 2^20-sample pushes")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="fp32", choices=["fp32", "fp16", "fp8", "fp32_simt"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision / batching / differentiation measurements")
    ap.add_argument("--chunk", type=int, default=0,
                    help="spectra per internal pass (corr_set_chunk); 0 = library default")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def max_over_ranks(dist, seconds, device):
    """The slowest rank's time (every rank gets it); `dist` None = one rank."""
    if dist is None:
        return seconds
    import torch
    tt = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(world, units_per_rank, seconds):
    """Units all ranks processed (replicas: each rank the same amount) per
    second of the slowest rank."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_id)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()

    def result(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = []
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except (ValueError, IndexError):
                continue
        os.unlink(self.f.name)
        inside = [r for r in rows if self.t0 - 0.15 <= r[0] <= self.t1 + 0.15]
        use = inside if inside else rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[1] for r in use),
                "sm_max_mhz": max(r[2] for r in use), "reasons": reasons,
                "samples": len(use), "in_region": bool(inside)}


def gpu_id_for_smi(local_rank):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local_rank).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[local_rank] if vis else str(local_rank)


# ----------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ----------------------------------------------------------------------------

def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_input(frames, seed=SEED):
    from paper_1102_0148_gb300 import synth
    packed, _ = synth.make_samples(N_ANT, frames * K_FFT, K_FFT, seed=seed, tone_amp=0.5)
    return packed


def time_oracle(packed):
    import oracle
    frames = packed.shape[0]
    t0 = time.perf_counter()
    V, n = oracle.correlate(packed, N_ANT, K_FFT)
    dt = time.perf_counter() - t0
    assert n == frames and V.shape == (990, 256)
    return dt


def oracle_frames_for(seconds):
    """Frames the oracle processes in about `seconds` (probe + proportional)."""
    probe = 1024
    dt = time_oracle(oracle_input(probe))
    frames = int(probe * seconds / max(dt, 1e-3))
    return max(16, min(SPEC_PER_STEP, frames))


def cpu_model():
    """The host CPU's model name (x86 'model name', or lscpu's on Arm)."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


_ORACLE_CHILD = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import oracle
from paper_1102_0148_gb300 import synth
N, K, frames, seed, tone = int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), int(sys.argv[5]), float(sys.argv[6])
packed, _ = synth.make_samples(N, frames * K, K, seed=seed, tone_amp=tone)
t0 = time.perf_counter()
V, n = oracle.correlate(packed, N, K)
dt = time.perf_counter() - t0
assert n == frames
print(json.dumps({"seconds": dt}))
"""


def time_oracle_threads(frames, threads, seed, tone):
    """The oracle on `frames` spectra of the 44-antenna workload in a fresh
    process whose BLAS runs `threads` threads (0 = the library's default,
    all cores); returns its wall time (input generation excluded)."""
    env = dict(os.environ)
    if threads:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS",
                  "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS"):
            env[k] = str(threads)
    r = subprocess.run([sys.executable, "-c", _ORACLE_CHILD, ROOT, str(N_ANT), str(K_FFT),
                        str(frames), str(seed), str(tone)],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle child failed: {r.stderr[-500:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])["seconds"]


def cpu_baseline(seconds):
    """The FP64 oracle on the host cores, at one thread and at all cores, on
    the plain-FX workload (N = 44, 2^17 samples = 256 spectra) and on a
    prefix of the real-time one (1 s at 35 MS/s; the prefix sized to about
    `seconds` of CPU work at all cores, a quarter of that at one thread)."""
    cores = os.cpu_count() or 1
    frames = oracle_frames_for(seconds)
    frames1 = max(16, frames // max(1, min(cores, 16)) * 2)
    runs = []
    for name, fr, seed, tone in (("plain FX: N=44, K=512, 2^17 samples (256 spectra)", 256,
                                  11020148 + 1, 0.0),
                                 (None, None, SEED, 0.5)):
        for threads in (1, 0):
            f = fr if fr else (frames1 if threads == 1 else frames)
            dt = time_oracle_threads(f, threads, seed, tone)
            runs.append({"workload": name or f"real time: first {f} of the 68359 spectra of a "
                                              f"1 s integration at 35 MS/s (+ 0.5 LSB tone)",
                         "threads": threads or cores, "spectra": f, "seconds": dt,
                         "value": N_ANT * f * K_FFT / dt, "rtf": N_ANT * f * K_FFT / dt / PAPER_RATE})
    head = runs[-1]
    return {"value": head["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"first {head['spectra']} of the 68359 spectra of one 1 s integration "
                      f"({head['spectra'] * K_FFT} samples x 44 antennas), numpy FP64 oracle, "
                      f"all {cores} cores, {head['seconds']:.1f} s",
            "runs": runs}


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    budget = 90.0 / max(1, args.steps + args.warmup)
    frames = oracle_frames_for(budget)
    packed = oracle_input(frames)
    for _ in range(args.warmup):
        time_oracle(packed)
    times = [time_oracle(packed) for _ in range(args.steps)]
    total = sum(times)
    value = N_ANT * frames * K_FFT * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_RATE, "dtype": "f64",
        "data": "synthetic", "rtf": value / PAPER_RATE,
        "config": {"workload": WORKLOAD, "sample_spectra_per_step": frames},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                         "sample": f"{frames} spectra x 44 antennas per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1102_0148_gb300 import corr, synth, workload
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    bf16_sus = peaks.get("bf16_tflops_sustained", 1700.0)
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    peak_src = "measured" if peaks else "fallback"

    dtype = corr.DTYPES[args.dtype]
    frames = SPEC_PER_STEP
    rec = N_ANT * K_FFT // 2
    dev_in, info = synth.make_samples_torch(N_ANT, frames * K_FFT, K_FFT, seed=SEED + rank,
                                            device="cuda", tone_amp=0.5)
    dev_in = dev_in.reshape(-1)
    stream = torch.cuda.current_stream()
    h = corr.corr_create(N_ANT, K_FFT, dtype)
    if args.chunk:
        corr.corr_set_chunk(h, args.chunk)
    corr.corr_set_stream(h, stream.cuda_stream)
    info_h = corr.corr_info(h)
    P, C = info_h["P"], info_h["C"]
    vis = torch.empty((P, C), dtype=torch.complex64, device="cuda")
    base = dev_in.data_ptr()
    pushes = [(f0, min(CHUNK_FRAMES, frames - f0)) for f0 in range(0, frames, CHUNK_FRAMES)]

    def step(src_base):
        for f0, nf in pushes:
            corr.corr_push(h, src_base + f0 * rec, nf * K_FFT)
        return corr.corr_dump(h, vis)

    for _ in range(args.warmup):
        assert step(base) == frames
    torch.cuda.synchronize()
    corr.corr_profile_enable(h, True)
    corr.corr_profile_read(h)

    sampler = ClockSampler(gpu_id_for_smi(local_rank))
    time.sleep(1.0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler.start()
    ev0.record(stream)
    # kernel timing: CUDA events around every launch of every PROF_EVERY-th
    # step (events on every launch slow the whole step by ~5%)
    profiled = 0
    for it in range(args.steps):
        on = it % PROF_EVERY == 0
        corr.corr_profile_enable(h, on)
        profiled += on
        step(base)
    ev1.record(stream)
    torch.cuda.synchronize()
    sampler.stop()
    if dist:
        dist.barrier()
    t = max_over_ranks(dist, ev0.elapsed_time(ev1) / 1e3, "cuda")
    clocks = sampler.result()
    prof = corr.corr_profile_read(h)
    corr.corr_profile_enable(h, False)
    # every step launches the same kernels
    launches = sum(v[0] for v in prof.values()) * args.steps // max(1, profiled)

    value = whole_job_rate(world, N_ANT * frames * K_FFT * args.steps, t)

    # roofline of the dominant kernel (largest summed event time)
    spec_total = frames * profiled
    dom = max(("fengine", "xengine", "fused"), key=lambda c: prof[c][1])
    n_launch, ms = prof[dom]
    if dom == "fused":
        # One fused F/X launch per integration, its spectra kept in an
        # L2-resident ring: only the 4-bit input touches HBM, and the kernel is
        # bound by instruction issue in its F-engine warps.  Reported here: the
        # F-engine warps' transform work (the paper's 2.5 K log2 K flops per
        # spectrum) against the FP32 pipe; the X-engine warps' tensor work is in
        # the xengine block.
        work = workload.fengine_flops(N_ANT, K_FFT, spec_total) / n_launch
        bound, unit = "alu", "TFLOP/s"
        peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        psrc = f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz"
        achieved = work / (ms / n_launch / 1e3) / 1e12
    elif dom == "xengine":
        work = workload.xengine_flops(N_ANT, K_FFT, spec_total) / n_launch
        if args.dtype == "fp32_simt":
            bound, unit = "alu", "TFLOP/s"
            peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
            psrc = f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz"
        else:
            # FP32 mode issues kind::f16 (two FP16 planes), FP8 kind::f8f6f4
            bound, unit = "tensor", "TFLOP/s"
            ratio = 2.0 if args.dtype == "fp8" else 1.0
            peak = bf16_sus * ratio
            psrc = (f"{peak_src} bf16 sustained {bf16_sus} TF/s x nominal "
                    f"{'fp8/bf16 = 2' if ratio == 2.0 else 'fp16/bf16 = 1'}")
        achieved = work / (ms / n_launch / 1e3) / 1e12
    else:
        ob = {"fp32": 4, "fp32_simt": 4, "fp16": 2, "fp8": 1}[args.dtype]
        work = workload.fengine_bytes(N_ANT, K_FFT, spec_total, ob) / n_launch
        bound, unit = "hbm", "GB/s"
        peak = hbm_peak
        psrc = f"{peak_src} hbm_gbs"
        achieved = work / (ms / n_launch / 1e3) / 1e9
    traffic = None
    tr = NCU_TRAFFIC.get((dom, args.dtype))
    if tr and not args.chunk:
        traffic = tr[0] * (spec_total / n_launch) / tr[1]
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic,
                "traffic_source": tr[2] if traffic else None, "peak_source": psrc,
                "work_per_launch": work,
                "kernel_ms": {c: prof[c][1] for c in prof},
                "kernel_launches": {c: prof[c][0] for c in prof},
                "profiled_steps": profiled}

    # the X-engine at its tensor-pipe fraction: useful flops (8 per complex
    # MAC, all pairs) and the flops its MMAs issue (tile padding, and the
    # three FP16 products of FP32 mode), against the peak of the MMA kind
    # it issues, per CUDA-event time of its launches
    xengine = None
    xkey = "fused" if prof["fused"][0] > 0 else "xengine"
    if args.dtype != "fp32_simt" and prof[xkey][0] > 0:
        # (in the fused kernel the X-engine warps run beside the F-engine
        # warps, so the rates are over the whole fused kernel's time)
        n_x, ms_x = prof[xkey]
        s_pad = -(-frames // 128) * 128          # every step's passes, padded frames
        sec = ms_x / 1e3
        useful = workload.xengine_flops(N_ANT, K_FFT, frames) * profiled / sec / 1e12
        issued = workload.xengine_issued_flops(N_ANT, K_FFT, s_pad, args.dtype) * profiled / sec / 1e12
        ratio = 2.0 if args.dtype == "fp8" else 1.0
        xengine = {
            "kernel": "fx_fused_kernel (X-engine warps)" if xkey == "fused" else "xengine_tc_kernel",
            "instruction": "tcgen05.mma kind::f8f6f4" if args.dtype == "fp8" else "tcgen05.mma kind::f16",
            "ms_per_step": ms_x / profiled, "launches_per_step": n_x / profiled,
            "useful_tflops": useful, "issued_tflops": issued,
            "peak_tflops": bf16_sus * ratio, "peak_burst_tflops": bf16_peak * ratio,
            "peak_source": f"{peak_src} bf16 (sustained and burst) x nominal "
                           f"{'fp8/bf16 = 2' if ratio == 2.0 else 'fp16/bf16 = 1'}",
            "useful_frac": useful / (bf16_sus * ratio), "issued_frac": issued / (bf16_sus * ratio),
            "ncu_tensor_pipe_pct": NCU_XENGINE_TENSOR_PCT.get(args.dtype) if not args.chunk else None,
        }

    # end to end from pinned host memory through the C ABI
    e2e = None
    if args.e2e_steps > 0:
        host_in = torch.empty(dev_in.numel(), dtype=torch.uint8, pin_memory=True)
        host_in.copy_(dev_in)
        host_vis = torch.empty((P, C), dtype=torch.complex64, pin_memory=True)
        hb = host_in.data_ptr()

        def step_host():
            # pushes from pinned host memory, then the integration's
            # visibilities queued into pinned host memory: the next step's
            # copies start while this one is reduced and read back
            for f0, nf in pushes:
                corr.corr_push(h, hb + f0 * rec, nf * K_FFT)
            return corr.corr_dump_async(h, host_vis)

        step_host()
        corr.corr_sync(h)
        # the host link's rate in this run: one step's input, pinned host ->
        # device, as a single copy (CUDA events, best of 3)
        scratch = torch.empty_like(dev_in)
        copy_ms = []
        for _ in range(3):
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            scratch.copy_(host_in, non_blocking=True)
            c1.record(stream)
            c1.synchronize()
            copy_ms.append(c0.elapsed_time(c1))
        del scratch
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            step_host()
        corr.corr_sync(h)                   # the last step's visibilities are in host memory
        te = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
        e2e = {"value": whole_job_rate(world, N_ANT * frames * K_FFT * args.e2e_steps, te),
               "unit": UNIT,
               "h2d_bytes_per_step": frames * rec,
               "d2h_bytes_per_step": host_vis.numel() * host_vis.element_size(),
               "steps": args.e2e_steps, "dump": "corr_dump_async into pinned host memory",
               "ms_per_step": 1e3 * te / args.e2e_steps,
               "h2d_gbs": frames * rec / (min(copy_ms) * 1e-3) / 1e9,
               "h2d_ms_per_step": min(copy_ms)}
        del host_in

    # TC vs FP32: the other X-engine precisions on the same integration
    variants = None
    if not args.no_variants and rank == 0:
        variants = measure_variants(corr, torch, np, dev_in, pushes, rec, args.dtype, args.chunk)

    corr.corr_destroy(h)
    del dev_in
    torch.cuda.empty_cache()

    forms = None
    if rank == 0 and not args.no_forms:
        forms = {"precision": measure_precision_form(corr, torch, np),
                 "batching": measure_batch_form(corr, torch, np),
                 "differentiation": measure_grad_form(corr, torch, np),
                 "streaming": measure_streaming_form(corr, torch, np)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_RATE,
            "dtype": "f32" if args.dtype.startswith("fp32") else args.dtype,
            "data": "synthetic",
            "rtf": value / (world * N_ANT * RATE),
            "config": {"workload": WORKLOAD, "x_engine": args.dtype,
                       "spectra_per_step": frames, "chunk_samples": CHUNK_FRAMES * K_FFT,
                       "pass_spectra": args.chunk or "default",
                       "input_bytes_per_step": frames * rec,
                       "l2": "inputs (770 MB/step) larger than L2; no flush",
                       "parallelism": f"replicas x{world}"},
            "clocks": clocks, "gpu_launches": launches, "roofline": roofline,
            "xengine": xengine,
            "e2e": e2e, "cpu_baseline": cpu, "variants": variants, "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def measure_variants(corr, torch, np, dev_in, pushes, rec, main_dtype, chunk, steps=20):
    """Throughput of each X-engine precision and its normalised visibility
    error against the FP32 tensor-core path on the same 1 s integration;
    fp32_fused is FP32 mode on the fused F/X-engine (corr_set_fused)."""
    out = {}
    ref = None
    order = ["fp32", "fp32_fused", "fp32_simt", "fp16", "fp8"]
    res = {}
    for name in order:
        try:
            h = corr.corr_create(N_ANT, K_FFT, corr.DTYPES[name.replace("_fused", "")])
            if chunk:
                corr.corr_set_chunk(h, chunk)
            if name == "fp32_fused":         # the fused F/X-engine (one launch per integration)
                corr.corr_set_fused(h, True)
        except corr.CorrError as e:
            out[name] = {"unavailable": str(e)}
            continue
        stream = torch.cuda.current_stream()
        corr.corr_set_stream(h, stream.cuda_stream)
        vis = torch.empty((990, 256), dtype=torch.complex128, device="cuda")
        base = dev_in.data_ptr()

        def step():
            for f0, nf in pushes:
                corr.corr_push(h, base + f0 * rec, nf * K_FFT)
            return corr.corr_dump(h, vis, fp64=True)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1e3
        V = vis.cpu().numpy()
        corr.corr_destroy(h)
        res[name] = V
        val = N_ANT * SPEC_PER_STEP * K_FFT * steps / t
        out[name] = {"value": val, "rtf": val / (N_ANT * RATE), "ms_per_step": 1e3 * t / steps}
    ref = res.get("fp32")
    if ref is not None:
        autos = [i * N_ANT - i * (i - 1) // 2 for i in range(N_ANT)]
        A = np.abs(ref[autos])
        ii = [i for i in range(N_ANT) for j in range(i, N_ANT)]
        jj = [j for i in range(N_ANT) for j in range(i, N_ANT)]
        nrm = np.sqrt(A[ii] * A[jj])
        for name, V in res.items():
            out[name]["err_vs_fp32"] = float(np.max(np.abs(V - ref) / nrm))
    return out


def _norm_err(np, V, R, N):
    autos = [i * N - i * (i - 1) // 2 for i in range(N)]
    A = np.abs(R[autos])
    ii = [i for i in range(N) for j in range(i, N)]
    jj = [j for i in range(N) for j in range(i, N)]
    nrm = np.sqrt(A[ii] * A[jj])
    return float(np.max(np.abs(np.asarray(V, np.complex128) - R) / np.maximum(nrm, 1e-300)))


def _events_ms(torch, fn, steps, stream):
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_precision_form(corr, torch, np, steps=3):
    """Full 40 MHz band: N = 44 at 80 MS/s, K = 512, 1 s integrations
    (156250 spectra) pushed in 2^20-sample chunks; error of each X-engine
    precision against the FP64 oracle on the 2^20-sample prefix."""
    import oracle
    from paper_1102_0148_gb300 import synth
    rate = 80e6
    frames = int(rate // K_FFT)
    rec = N_ANT * K_FFT // 2
    dev, _ = synth.make_samples_torch(N_ANT, frames * K_FFT, K_FFT, seed=SEED + 1, device="cuda",
                                      tone_amp=0.5)
    dev = dev.reshape(-1)
    R, _ = oracle.correlate(dev[: CHUNK_FRAMES * rec].cpu().numpy(), N_ANT, K_FFT)
    stream = torch.cuda.current_stream()
    pushes = [(f0, min(CHUNK_FRAMES, frames - f0)) for f0 in range(0, frames, CHUNK_FRAMES)]
    out = {"workload": "N=44, K=512, 80 MS/s, 1 s = 156250 spectra; error on the 2^20-sample prefix"}
    for name in ("fp32", "fp16", "fp8"):
        with corr.Correlator(N_ANT, K_FFT, name, stream=stream.cuda_stream) as c:
            c.push(dev[: CHUNK_FRAMES * rec], CHUNK_FRAMES * K_FFT)
            V, _ = c.dump(fp64=True)
            err = _norm_err(np, V, R, N_ANT)
            vis = torch.empty((990, 256), dtype=torch.complex64, device="cuda")

            def step():
                for f0, nf in pushes:
                    corr.corr_push(c.h, dev.data_ptr() + f0 * rec, nf * K_FFT)
                corr.corr_dump(c.h, vis)

            ms = _events_ms(torch, step, steps, stream)
        val = N_ANT * frames * K_FFT / (ms * 1e-3)
        out[name] = {"value": val, "unit": UNIT, "rtf": val / (N_ANT * rate), "err_vs_oracle": err}
    del dev
    torch.cuda.empty_cache()
    return out


def measure_batch_form(corr, torch, np, steps=5):
    """Modes (44, 512), (22, 2048), (11, 4096) and the (256, 1024) scale-up,
    2^22 samples per antenna each, in one graph-captured step whose X-engine
    work is one persistent launch; tiles from a short autotuner sweep.  Error
    against the FP64 oracle on a 2^16-sample prefix of every mode."""
    import oracle
    from paper_1102_0148_gb300 import synth, tune
    modes = [(44, 512), (22, 2048), (11, 4096), (256, 1024)]
    T = 1 << 22
    data = []
    for m, (N, K) in enumerate(modes):
        d, _ = synth.make_samples_torch(N, T, K, seed=SEED + 10 + m, device="cuda")
        data.append(d.reshape(-1))
    Tp = 1 << 16
    refs = [oracle.correlate(x[: Tp * N // 2].cpu().numpy(), N, K)[0] for x, (N, K) in zip(data, modes)]
    out = {"workload": "modes (44,512), (22,2048), (11,4096), (256,1024); 2^22 samples/antenna/mode",
           "samples_per_step": sum(N * T for N, _ in modes)}
    tiles = {}
    # *_one_launch: the modes' F-engines as one multi-mode launch
    # (corr_batch_set_one_launch), with the tiles tuned for the default form
    for name, dt, one in (("fp16", "fp16", False), ("fp32", "fp32", False),
                          ("fp16_one_launch", "fp16", True)):
        if dt not in tiles:
            tiles[dt] = tune.tune_batch(modes, dt, T=T, repeats=2, save=False,
                                        windows=(128, 256) if dt == "fp32" else (512, 1024, 2048),
                                        stages=(3, 4, 6), splits=(0, 1))
        t = tiles[dt]
        with corr.CorrelatorBatch(modes, dt, window=t["window"], stages=t["stages"],
                                  split=t["split"], one_launch=one) as b:
            for h, (N, K) in zip(b.handles, modes):
                corr.corr_set_chunk(h, T // K)           # one pass per mode and push
                corr.corr_profile_enable(h, True)
                corr.corr_profile_read(h)
            b.push([x[: Tp * N // 2] for x, (N, _) in zip(data, modes)],
                   [Tp] * len(modes))
            vis_p, _ = b.dump(fp64=True)
            # launches of one step, by kernel class, over the modes' handles
            # (the captured graph replays the same sequence)
            launches = {}
            for h in b.handles:
                for c, (n_l, _) in corr.corr_profile_read(h).items():
                    launches[c] = launches.get(c, 0) + n_l
                corr.corr_profile_enable(h, False)
            errs = [_norm_err(np, V, R, N) for V, R, (N, _) in zip(vis_p, refs, modes)]
            vis = [torch.empty((N * (N + 1) // 2, K // 2), dtype=torch.complex64, device="cuda")
                   for N, K in modes]
            b.capture(data, vis)
            s = torch.cuda.ExternalStream(b.stream)
            ms = _events_ms(torch, b.replay, steps, s)
        val = out["samples_per_step"] / (ms * 1e-3)
        out[name] = {"value": val, "unit": UNIT, "ms_per_step": ms, "tiles": t,
                     "err_vs_oracle_per_mode": errs, "launches_per_step": launches}
    del data
    torch.cuda.empty_cache()
    return out


def measure_streaming_form(corr, torch, np, steps=5):
    """The headline integration with coarse integer delays on the stream
    (the synthetic model's own delays d_i compensated, D_i = max d - d_i):
    throughput with the delay pass, and the error against the FP64 oracle of
    the delayed stream on the 2^20-sample prefix."""
    import oracle
    from paper_1102_0148_gb300 import synth
    frames = int(RATE // K_FFT)
    rec = N_ANT * K_FFT // 2
    dev, info = synth.make_samples_torch(N_ANT, frames * K_FFT, K_FFT, seed=SEED + 3,
                                         device="cuda", tone_amp=0.5)
    dev = dev.reshape(-1)
    D = (info["delays"].max() - info["delays"]).astype(np.int32)
    R, _ = oracle.correlate(dev[: CHUNK_FRAMES * rec].cpu().numpy(), N_ANT, K_FFT, sample_delays=D)
    stream = torch.cuda.current_stream()
    pushes = [(f0, min(CHUNK_FRAMES, frames - f0)) for f0 in range(0, frames, CHUNK_FRAMES)]
    with corr.Correlator(N_ANT, K_FFT, "fp32", stream=stream.cuda_stream) as c:
        corr.corr_set_sample_delays(c.h, D)
        c.push(dev[: CHUNK_FRAMES * rec], CHUNK_FRAMES * K_FFT)
        V, _ = c.dump(fp64=True)
        err = _norm_err(np, V, R, N_ANT)
        vis = torch.empty((990, 256), dtype=torch.complex64, device="cuda")

        def step():
            for f0, nf in pushes:
                corr.corr_push(c.h, dev.data_ptr() + f0 * rec, nf * K_FFT)
            corr.corr_dump(c.h, vis)

        ms = _events_ms(torch, step, steps, stream)
    val = N_ANT * frames * K_FFT / (ms * 1e-3)
    del dev
    torch.cuda.empty_cache()
    return {"workload": "N=44, K=512, 35 MS/s, 1 s, integer sample delays 0..15 compensated; "
                        "error on the 2^20-sample prefix",
            "sample_delays": {"value": val, "unit": UNIT, "rtf": val / (N_ANT * RATE),
                              "ms_per_step": ms, "err_vs_oracle": err}}


def measure_grad_form(corr, torch, np, steps=5):
    """N = 44, K = 512, 2^20 samples: L = sum |V(g, tau) - M|^2 with gains
    g ~ CN(1, 0.1^2) and delays tau ~ U(-0.5, 0.5) applied in the F-engine;
    forward and backward times and the gradient's error against the
    oracle's closed form."""
    import oracle
    from paper_1102_0148_gb300 import synth
    from paper_1102_0148_gb300.autograd import visibilities
    T = 1 << 20
    packed, _ = synth.make_samples(N_ANT, T, K_FFT, seed=SEED + 5)
    R, _ = oracle.correlate(packed, N_ANT, K_FFT)
    g, tau = synth.gains_delays(N_ANT, seed=SEED + 5)
    g = np.asarray(g, np.complex64).astype(np.complex128)
    tau = np.asarray(tau, np.float32).astype(np.float64)
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    M = torch.from_numpy(R).cuda()
    stream = torch.cuda.current_stream()
    with corr.Correlator(N_ANT, K_FFT, "fp32") as c:
        gt = torch.tensor(g, dtype=torch.complex64, device="cuda", requires_grad=True)
        tt = torch.tensor(tau, dtype=torch.float32, device="cuda", requires_grad=True)

        def fwd():
            return (visibilities(gt, tt, dev, c) - M).abs().pow(2).sum()

        f_ms = _events_ms(torch, fwd, steps, stream)

        def fwd_bwd():
            gt.grad = None
            tt.grad = None
            fwd().backward()

        fb_ms = _events_ms(torch, fwd_bwd, steps, stream)
        gg = gt.grad.cpu().numpy().astype(np.complex128)
        gtau = tt.grad.cpu().numpy().astype(np.float64)
    _, og, ot = oracle.loss_and_grad(R, g, tau, K_FFT)
    return {"workload": "N=44, K=512, 2^20 samples; loss sum |V(g,tau) - V(1,0)|^2",
            "forward_ms": f_ms, "backward_ms": fb_ms - f_ms,
            "grad_g_rel_err": float(np.abs(gg - og).max() / np.abs(og).max()),
            "grad_tau_rel_err": float(np.abs(gtau - ot).max() / np.abs(ot).max())}


if __name__ == "__main__":
    sys.exit(main())
