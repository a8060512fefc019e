"""Batching form (GPU): several modes of uneven N and K whose X-engine work
shares one persistent tensor-core launch per pass, eagerly and replayed as a
captured CUDA graph.  Every mode's visibilities are checked against the FP64
oracle with the parity bound of its precision.

The modes are the batching workload's: (44, 512), (22, 2048), (11, 4096) and
the 256-antenna, K = 1024 scale-up, here at short lengths so the oracle
finishes in seconds.
"""

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth

pytestmark = pytest.mark.gpu

MODES3 = [(44, 512), (22, 2048), (11, 4096)]
MODES4 = MODES3 + [(256, 1024)]


def norm_err(V, R, N):
    autos = np.array([oracle.baseline_index(i, i, N) for i in range(N)])
    A = np.abs(R[autos])
    pairs = oracle.baseline_pairs(N)
    nrm = np.sqrt(A[[p[0] for p in pairs]] * A[[p[1] for p in pairs]])
    return float(np.max(np.abs(np.asarray(V, np.complex128) - R) / np.maximum(nrm, 1e-300)))


def make_inputs(modes, T, seed):
    import torch
    packed, refs = [], []
    for m, (N, K) in enumerate(modes):
        p, _ = synth.make_samples(N, T, K, seed=seed + 100 * m)
        packed.append(torch.from_numpy(p.reshape(-1)).cuda())
        refs.append(oracle.correlate(p, N, K)[0])
    return packed, refs


# one: the modes' F-engines as one multi-mode launch (corr_batch_set_one_launch)
@pytest.mark.parametrize("one", [False, True])
@pytest.mark.parametrize("modes,T", [(MODES3, 1 << 17), (MODES4, 1 << 16)])
def test_batch_matches_oracle(lib, modes, T, one):
    dev, refs = make_inputs(modes, T, seed=11020148 + 40)
    with lib.CorrelatorBatch(modes, "fp32", one_launch=one) as b:
        b.push(dev)
        vis, n = b.dump(fp64=True)
    for (N, K), V, R, nm in zip(modes, vis, refs, n):
        assert nm == T // K
        assert norm_err(V, R, N) <= 1e-5, (N, K)


def test_batch_multiple_passes(lib):
    """Chunks smaller than the pushes: the modes have different numbers of
    passes, so later launches cover only some of them."""
    modes = MODES3
    T = 1 << 17                                   # 256, 64 and 32 frames
    dev, refs = make_inputs(modes, T, seed=11020148 + 41)
    with lib.CorrelatorBatch(modes, "fp32", chunk=128) as b:
        b.push(dev)
        b.push(dev)                               # accumulate twice
        vis, n = b.dump(fp64=True)
    for (N, K), V, R, nm in zip(modes, vis, refs, n):
        assert nm == 2 * T // K
        assert norm_err(V, 2 * R, N) <= 1e-5


@pytest.mark.parametrize("one", [False, True])
def test_batch_graph_replay(lib, one):
    import torch
    modes = MODES3
    T = 1 << 16
    dev_a, refs_a = make_inputs(modes, T, seed=11020148 + 42)
    dev_b, refs_b = make_inputs(modes, T, seed=11020148 + 43)
    bufs = [x.clone() for x in dev_a]
    with lib.CorrelatorBatch(modes, "fp32", one_launch=one) as b:
        vis = [torch.empty((N * (N + 1) // 2, K // 2), dtype=torch.complex128, device="cuda")
               for N, K in modes]
        b.capture(bufs, vis, fp64=True)
        for dev, refs in ((dev_a, refs_a), (dev_b, refs_b), (dev_a, refs_a)):
            for buf, x in zip(bufs, dev):
                buf.copy_(x)
            torch.cuda.synchronize()
            n = b.replay()
            b.sync()
            for (N, K), V, R, nm in zip(modes, vis, refs, n):
                assert nm == T // K
                assert norm_err(V.cpu().numpy(), R, N) <= 1e-5


@pytest.mark.parametrize("one", [False, True])
def test_batch_fp16(lib, one):
    modes = MODES3
    T = 1 << 17
    dev, refs = make_inputs(modes, T, seed=11020148 + 44)
    with lib.CorrelatorBatch(modes, "fp16", one_launch=one) as b:
        b.push(dev)
        vis, n = b.dump(fp64=True)
    for (N, K), V, R in zip(modes, vis, refs):
        from conftest import report_err
        # about twice the measured 1.3e-4, 2.6e-4, 3.7e-4
        bound = {512: 2.6e-4, 2048: 5.2e-4, 4096: 7.4e-4}[K]
        assert report_err(f"batch-fp16-N{N}-K{K}", norm_err(V, R, N)) <= bound


def test_batch_rejects_mixed_or_bad_arguments(lib):
    with pytest.raises(lib.CorrError):
        lib.CorrelatorBatch([(44, 512)] * 5, "fp32")
    with pytest.raises(lib.CorrError):
        lib.CorrelatorBatch(MODES3, "fp32_simt")


@pytest.mark.parametrize("one", [False, True])
def test_batch_multiblock_passes_and_replays(lib, one):
    """A multi-block mode (N = 130: three antenna blocks) whose pass results
    go through the FP32 slot and the reduction: several passes per push (the
    first into a zero accumulator is stored, later ones added), pushes
    accumulated across calls, and graph replays of fresh data; every result
    against the oracle.  A replay after an eager push is refused."""
    import torch
    modes = [(130, 256), (44, 512)]
    T = 1 << 16                                   # 256 and 128 frames
    dev_a, refs_a = make_inputs(modes, T, seed=11020148 + 45)
    dev_b, refs_b = make_inputs(modes, T, seed=11020148 + 46)
    with lib.CorrelatorBatch(modes, "fp32", chunk=128, one_launch=one) as b:   # 2 passes and 1
        b.push(dev_a)
        b.push(dev_b)
        vis, n = b.dump(fp64=True)
        for (N, K), V, Ra, Rb, nm in zip(modes, vis, refs_a, refs_b, n):
            assert nm == 2 * T // K
            assert norm_err(V, Ra + Rb, N) <= 1e-5, (N, K)
        bufs = [x.clone() for x in dev_a]
        out = [torch.empty((N * (N + 1) // 2, K // 2), dtype=torch.complex128, device="cuda")
               for N, K in modes]
        b.capture(bufs, out, fp64=True)
        for dev, refs in ((dev_b, refs_b), (dev_a, refs_a)):
            for buf, x in zip(bufs, dev):
                buf.copy_(x)
            torch.cuda.synchronize()
            b.replay()
            b.sync()
            for (N, K), V, R in zip(modes, out, refs):
                assert norm_err(V.cpu().numpy(), R, N) <= 1e-5, (N, K)
        b.push(dev_a)
        with pytest.raises(lib.CorrError) as ei:
            b.replay()
        assert ei.value.code == lib.CORR_ESTATE
        vis, n = b.dump(fp64=True)                # the eager push is still whole
        for (N, K), V, R in zip(modes, vis, refs_a):
            assert norm_err(V, R, N) <= 1e-5, (N, K)


@pytest.mark.parametrize("one", [False, True])
def test_batch_every_fengine_kind_with_corrections(lib, one):
    """Every F-engine body -- K = 512, 1024, 2048 and a generic K (256) --
    each mode with its own gains and fractional delays, as separate launches
    and as one multi-mode launch, against the oracle with the same
    corrections."""
    modes = [(44, 512), (20, 1024), (22, 2048), (5, 256)]
    T = 1 << 16
    dev, _ = make_inputs(modes, T, seed=11020148 + 47)
    refs = []
    with lib.CorrelatorBatch(modes, "fp32", one_launch=one) as b:
        for m, ((N, K), h) in enumerate(zip(modes, b.handles)):
            g, tau = synth.gains_delays(N, seed=500 + m)
            g32 = np.asarray(g, np.complex64)
            t32 = np.asarray(tau * 2.5, np.float32)
            lib.corr_set_corrections(h, g32, t32)
            packed = dev[m].cpu().numpy().reshape(T // K, N, K // 2)
            refs.append(oracle.correlate(packed, N, K, gains=g32.astype(np.complex128),
                                         delays=t32.astype(np.float64))[0])
        b.push(dev)
        vis, n = b.dump(fp64=True)
    for (N, K), V, R, nm in zip(modes, vis, refs, n):
        assert nm == T // K
        assert norm_err(V, R, N) <= 1e-5, (N, K)


# FP16 / FP8 with the four modes (N = 256 as work groups beside the
# single-block modes in one launch; 128, 32, 16 and 64 frames): about twice
# the errors measured on a GB300 (FP16 1.9e-4, 3.8e-4, 5.1e-4, 3.0e-4; FP8
# 2.5e-2, 4.3e-2, 6.3e-2, 3.6e-2 -- FP8's error falls as 1/sqrt(frames))
MIXED_BOUND = {("fp16", 512): 3.9e-4, ("fp16", 2048): 7.6e-4, ("fp16", 4096): 1.03e-3,
               ("fp16", 1024): 6.0e-4, ("fp8", 512): 5.0e-2, ("fp8", 2048): 8.6e-2,
               ("fp8", 4096): 1.27e-1, ("fp8", 1024): 7.2e-2}


@pytest.mark.parametrize("one", [False, True])
@pytest.mark.parametrize("dtype", ["fp16", "fp8"])
def test_batch_reduced_precision_with_a_multiblock_mode(lib, dtype, one):
    from conftest import report_err
    modes = MODES4
    T = 1 << 16
    dev, refs = make_inputs(modes, T, seed=11020148 + 48)
    with lib.CorrelatorBatch(modes, dtype, one_launch=one) as b:
        b.push(dev)
        vis, n = b.dump(fp64=True)
    for (N, K), V, R, nm in zip(modes, vis, refs, n):
        assert nm == T // K
        e = report_err(f"batch4-{dtype}-N{N}-K{K}-one{int(one)}", norm_err(V, R, N))
        assert e <= MIXED_BOUND[(dtype, K)], (N, K, e)


# Full size, as bench.py times the batching workload: 2^22 samples per antenna
# and mode, one pass per mode, the captured step replayed, with the tiles the
# autotuner picks for it on a GB300.  The oracle computes four channels of
# every mode (DC, the tone channel 97, a middle and the last channel) for all
# pairs.  FP16 bounds: about twice the errors measured on a GB300 (2.6e-5,
# 3.3e-5, 4.9e-5, 3.4e-5; FP32 1.3e-6 .. 1.9e-6 against its 1e-5 bar).
FULL_T = 1 << 22
FULL_TILES = {"fp16": (2048, 4, 0), "fp32": (256, 6, 1)}
FULL_FP16_BOUND = {(44, 512): 5e-5, (22, 2048): 6.6e-5, (11, 4096): 1e-4, (256, 1024): 6.8e-5}


@pytest.fixture(scope="module")
def full_batch():
    import torch
    data, refs, chans = [], [], []
    for m, (N, K) in enumerate(MODES4):
        d, _ = synth.make_samples_torch(N, FULL_T, K, seed=11020148 + 60 + m, device="cuda",
                                        tone_amp=0.5)
        d = d.reshape(-1)
        C = K // 2
        ch = [0, 97, C // 2 + 3, C - 1]
        R, S = oracle.visibilities_channels(d.cpu().numpy(), N, K, ch, frames_per_block=256)
        assert S == FULL_T // K
        data.append(d)
        refs.append(R)
        chans.append(ch)
    return data, refs, chans


@pytest.mark.parametrize("dtype", ["fp32", "fp16"])
def test_batch_full_size_sampled_channels(lib, full_batch, dtype):
    import torch
    data, refs, chans = full_batch
    w, st, sp = FULL_TILES[dtype]
    with lib.CorrelatorBatch(MODES4, dtype, window=w, stages=st, split=sp) as b:
        for h, (N, K) in zip(b.handles, MODES4):
            lib.corr_set_chunk(h, FULL_T // K)          # one pass per mode and push
        vis = [torch.empty((N * (N + 1) // 2, K // 2), dtype=torch.complex64, device="cuda")
               for N, K in MODES4]
        b.capture(data, vis)
        n = b.replay()
        b.sync()
    for (N, K), V, R, ch, nm in zip(MODES4, vis, refs, chans, n):
        assert nm == FULL_T // K
        e = norm_err(V.cpu().numpy()[:, ch], R, N)
        print(f"MEASURED_ERR batchfull-{dtype}-N{N}-K{K} {e:.3e}")
        assert e <= (1e-5 if dtype == "fp32" else FULL_FP16_BOUND[(N, K)]), (N, K, e)
