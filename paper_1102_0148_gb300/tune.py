"""Autotuner for the correlator's tile choices.

    python -m paper_1102_0148_gb300.tune --N 44 --K 512 --dtype fp32
    python -m paper_1102_0148_gb300.tune --batch 44x512,22x2048,11x4096 --dtype fp32

For one correlator it sweeps the pass size (spectra per workspace pass), the
TMEM accumulation window of the tensor-core X-engine and its shared-memory
stage count, timing push + dump of seeded synthetic data with CUDA events on
the device, and keeps the fastest.  For a batch it sweeps window and stages
of the shared persistent launch, timing replays of the captured graph.
Windows are limited per precision so that the tensor core's biased FP32
accumulation stays far below the parity bound (<= 256 spectra in FP32
mode, ~1e-6 normalised).

Results are cached as JSON (``$GBCORR_TUNE_CACHE`` or
``~/.cache/gbcorr/tune.json``) keyed by geometry, precision and GPU name;
``apply`` / ``apply_batch`` set a handle's tiles from the cache.
"""

import argparse
import itertools
import json
import os

WINDOWS = {"fp32": (64, 128, 256), "fp16": (128, 256, 512, 1024, 2048),
           "fp8": (256, 512, 1024, 2048, 4096)}
STAGES = (2, 3, 4, 6, 8)
CHUNKS = (1024, 2048, 4096)
SPLITS = (0, 1, 2, 4)


def cache_path():
    return os.environ.get("GBCORR_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "gbcorr", "tune.json")


def _load():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(key, value):
    d = _load()
    d[key] = value
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _gpu():
    import torch
    return torch.cuda.get_device_name(0)


def key(N, K, dtype):
    return f"{_gpu()}|{N}x{K}|{dtype}"


def key_batch(modes, dtype):
    return f"{_gpu()}|batch:" + ",".join(f"{N}x{K}" for N, K in modes) + f"|{dtype}"


def lookup(N, K, dtype):
    return _load().get(key(N, K, dtype))


def apply(c, N, K, dtype):
    """Set chunk and tiles of Correlator `c` from the cache; True if found."""
    from . import corr
    t = lookup(N, K, dtype)
    if not t:
        return False
    corr.corr_set_chunk(c.h, t["chunk"])
    corr.corr_set_tiles(c.h, t["window"], t["stages"], t.get("split", 0))
    return True


def apply_batch(b, modes, dtype):
    from . import corr
    t = _load().get(key_batch(modes, dtype))
    if not t:
        return False
    corr.corr_batch_set_tiles(b.b, t["window"], t["stages"], t.get("split", 0))
    return True


def _time(fn, repeats, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(repeats):
        fn()
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / repeats


def tune(N, K, dtype="fp32", frames=8192, repeats=3, save=True, windows=None, stages=None,
         chunks=None, splits=None):
    """Sweep (chunk, window, stages, split) for one correlator; returns the best."""
    import torch
    from . import corr, synth
    dev, _ = synth.make_samples_torch(N, frames * K, K, seed=7, device="cuda")
    dev = dev.reshape(-1)
    stream = torch.cuda.current_stream()
    P, C = N * (N + 1) // 2, K // 2
    vis = torch.empty((P, C), dtype=torch.complex64, device="cuda")
    best, results = None, []
    for ch, w, st, sp in itertools.product(chunks or CHUNKS, windows or WINDOWS[dtype],
                                           stages or STAGES, splits or SPLITS):
        try:
            with corr.Correlator(N, K, dtype, chunk=ch, stream=stream.cuda_stream) as c:
                corr.corr_set_tiles(c.h, w, st, sp)

                def step():
                    corr.corr_push(c.h, dev, frames * K)
                    corr.corr_dump(c.h, vis)

                ms = _time(step, repeats, stream)
        except corr.CorrError:
            continue
        results.append((ms, ch, w, st, sp))
        if best is None or ms < best[0]:
            best = (ms, ch, w, st, sp)
    out = {"chunk": best[1], "window": best[2], "stages": best[3], "split": best[4], "ms": best[0],
           "spectra_per_s": frames / (best[0] * 1e-3), "frames": frames,
           "candidates": len(results)}
    if save:
        _save(key(N, K, dtype), out)
    return out


def tune_batch(modes, dtype="fp32", T=1 << 22, repeats=3, save=True, windows=None, stages=None,
               splits=None):
    """Sweep (window, stages, split) for a batch, timing replays of its graph."""
    import torch
    from . import corr, synth
    data = []
    for m, (N, K) in enumerate(modes):
        d, _ = synth.make_samples_torch(N, T, K, seed=11 + m, device="cuda")
        data.append(d.reshape(-1))
    vis = [torch.empty((N * (N + 1) // 2, K // 2), dtype=torch.complex64, device="cuda")
           for N, K in modes]
    best, results = None, []
    for w, st, sp in itertools.product(windows or WINDOWS[dtype], stages or STAGES,
                                       splits or SPLITS):
        try:
            with corr.CorrelatorBatch(modes, dtype) as b:
                for h, (N, K) in zip(b.handles, modes):
                    corr.corr_set_chunk(h, T // K)       # one pass per mode and push
                corr.corr_batch_set_tiles(b.b, w, st, sp)
                b.capture(data, vis)
                s = torch.cuda.ExternalStream(b.stream)
                ms = _time(b.replay, repeats, s)
        except corr.CorrError:
            continue
        results.append((ms, w, st, sp))
        if best is None or ms < best[0]:
            best = (ms, w, st, sp)
    out = {"window": best[1], "stages": best[2], "split": best[3], "ms": best[0],
           "samples_per_antenna": T,
           "candidates": len(results)}
    if save:
        _save(key_batch(modes, dtype), out)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=44)
    ap.add_argument("--K", type=int, default=512)
    ap.add_argument("--dtype", default="fp32", choices=sorted(WINDOWS))
    ap.add_argument("--batch", default=None, help="modes as NxK,NxK,...")
    a = ap.parse_args()
    if a.batch:
        modes = [tuple(int(v) for v in m.split("x")) for m in a.batch.split(",")]
        print(json.dumps(tune_batch(modes, a.dtype)))
    else:
        print(json.dumps(tune(a.N, a.K, a.dtype)))


if __name__ == "__main__":
    main()
