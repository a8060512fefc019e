"""Time whole workspace passes of one geometry, kernel class by kernel class.

    python -m paper_1102_0148_gb300.passes --N 256 --K 1024 --dtype fp16 --frames 4096

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


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--N", type=int, required=True)
    ap.add_argument("--K", type=int, required=True)
    ap.add_argument("--dtype", default="fp32", choices=sorted(corr.DTYPES))
    ap.add_argument("--frames", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--window", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--split", type=int, default=0)
    ap.add_argument("--atoms", type=int, default=0)
    a = ap.parse_args()
    print(json.dumps(run(a.N, a.K, a.dtype, a.frames, a.steps, a.warmup, a.window, a.stages,
                         a.split, a.atoms)))


if __name__ == "__main__":
    main()
