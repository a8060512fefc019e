"""Time whole workspace passes of one geometry, kernel class by kernel class.

    python -m paper_1102_0148_gb300.passes --N 256 --K 1024 --dtype fp16 --frames 4096
    python -m paper_1102_0148_gb300.passes --batch 44:512,22:2048,11:4096,256:1024 --dtype fp16

Each step pushes ``frames`` spectra per antenna of synthetic device-resident
input (drawn on the GPU) as one pass and dumps the integration.  After
``--warmup`` steps, ``--steps`` steps run with the handle's profiler on and
the CUDA-event time of every kernel class is printed per step, with the
tensor-core X-engine's issued TFLOP/s.  ``--window/--stages/--split/--atoms``
set the X-engine tiles (0: the planner's choice).  This is the command the
profiler summaries of single passes are taken with (one small geometry, a
few launches).
"""

import argparse
import json

from . import corr, synth, workload


def run(N, K, dtype="fp32", frames=4096, steps=5, warmup=3, window=0, stages=0, split=0,
        atoms=0, seed=5):
    import torch
    dev, _ = synth.make_samples_torch(N, frames * K, K, seed=seed, device="cuda")
    dev = dev.reshape(-1)
    h = corr.corr_create(N, K, corr.DTYPES[dtype])
    try:
        corr.corr_set_chunk(h, frames)
        if window or stages or split or atoms:
            corr.corr_set_tiles(h, window, stages, split, atoms)
        corr.corr_set_stream(h, torch.cuda.current_stream().cuda_stream)
        vis = torch.empty((N * (N + 1) // 2, K // 2), dtype=torch.complex64, device="cuda")

        def step():
            corr.corr_push(h, dev.data_ptr(), frames * K)
            corr.corr_dump(h, vis)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        corr.corr_profile_enable(h, True)
        corr.corr_profile_read(h)
        for _ in range(steps):
            step()
        prof = corr.corr_profile_read(h)
    finally:
        corr.corr_destroy(h)
    out = {"N": N, "K": K, "dtype": dtype, "frames": frames, "steps": steps,
           "ms_per_step": {c: ms / steps for c, (n, ms) in prof.items() if n},
           "launches_per_step": {c: n / steps for c, (n, ms) in prof.items() if n}}
    xms = out["ms_per_step"].get("xengine")
    if xms and dtype != "fp32_simt":
        s_pad = (frames + 127) // 128 * 128
        out["xengine_issued_tflops"] = workload.xengine_issued_flops(N, K, s_pad, dtype) / (xms * 1e-3) / 1e12
    return out


def run_batch(modes, dtype="fp16", samples=1 << 22, steps=20, warmup=3, window=0, stages=0,
              split=0, seed=5, one_launch=False):
    """Replays of the captured step of a batch (push of ``samples`` per antenna
    and mode, one pass per mode, and the dump), timed with CUDA events on the
    batch's stream; eager per-class launch counts of one step."""
    import torch
    data = []
    for m, (N, K) in enumerate(modes):
        d, _ = synth.make_samples_torch(N, samples, K, seed=seed + m, device="cuda")
        data.append(d.reshape(-1))
    with corr.CorrelatorBatch(modes, dtype, window=window, stages=stages, split=split,
                              one_launch=one_launch) as b:
        for h, (N, K) in zip(b.handles, modes):
            corr.corr_set_chunk(h, samples // K)
            corr.corr_profile_enable(h, True)
            corr.corr_profile_read(h)
        b.push(data)
        b.dump()
        for h in b.handles:
            corr.corr_profile_read(h)
        b.push(data)                     # the second eager step is the one profiled
        b.dump()
        launches, eager_ms = {}, {}
        for h in b.handles:
            for c, (n, t) in corr.corr_profile_read(h).items():
                if n:
                    launches[c] = launches.get(c, 0) + n
                    eager_ms[c] = eager_ms.get(c, 0.0) + t
            corr.corr_profile_enable(h, False)
        vis = [torch.empty((N * (N + 1) // 2, K // 2), dtype=torch.complex64, device="cuda")
               for N, K in modes]
        b.capture(data, vis)
        s = torch.cuda.ExternalStream(b.stream)
        for _ in range(warmup):
            b.replay()
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            b.replay()
        e1.record(s)
        b.sync()
        ms = e0.elapsed_time(e1) / steps
    return {"modes": [list(m) for m in modes], "dtype": dtype, "samples": samples,
            "one_launch": one_launch, "ms_per_step": ms, "launches_per_step": launches, "eager_ms_per_class": eager_ms}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--N", type=int)
    ap.add_argument("--K", type=int)
    ap.add_argument("--batch", default=None,
                    help="modes N:K,N:K,... (a captured batch step instead of one handle)")
    ap.add_argument("--samples", type=int, default=1 << 22, help="per antenna and mode (--batch)")
    ap.add_argument("--one-launch", action="store_true",
                    help="(--batch) the modes' F-engines as one launch")
    ap.add_argument("--dtype", default="fp32", choices=sorted(corr.DTYPES))
    ap.add_argument("--frames", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--window", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--split", type=int, default=0)
    ap.add_argument("--atoms", type=int, default=0)
    a = ap.parse_args()
    if a.batch:
        modes = [tuple(int(v) for v in m.split(":")) for m in a.batch.split(",")]
        print(json.dumps(run_batch(modes, a.dtype, a.samples, a.steps, a.warmup, a.window,
                                   a.stages, a.split, one_launch=a.one_launch)))
        return
    if a.N is None or a.K is None:
        ap.error("--N and --K (or --batch) are required")
    print(json.dumps(run(a.N, a.K, a.dtype, a.frames, a.steps, a.warmup, a.window, a.stages,
                         a.split, a.atoms)))


if __name__ == "__main__":
    main()
