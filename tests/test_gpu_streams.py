"""F-engine side streams (GPU): consecutive pushes' F-engine launches run on
two internal streams, each after the work queued on the handle's stream
before its push; the handle's stream waits for them before the X-engine and
before any call that changes what they read.  These tests check the
orderings that makes visible, against the FP64 oracle.
"""

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
SEED = 11020148 + 70


def vis_error(V, R, N):
    autos = np.array([oracle.baseline_index(i, i, N) for i in range(N)])
    A = np.abs(R[autos])
    pairs = oracle.baseline_pairs(N)
    nrm = np.sqrt(A[[p[0] for p in pairs]] * A[[p[1] for p in pairs]])
    return float(np.max(np.abs(np.asarray(V, np.complex128) - R) / nrm))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("K", [512, 1024])
def test_corrections_change_between_pushes(lib, torch_cuda, K):
    """Frames pushed before corr_set_corrections keep the old (identity)
    corrections even though their F-engine launches may still be queued on a
    side stream when the table changes."""
    torch = torch_cuda
    N, S1, S2 = 6, 96, 160
    packed, _ = synth.make_samples(N, (S1 + S2) * K, K, seed=SEED + K)
    rec = N * K // 2
    g, tau = synth.gains_delays(N, seed=K)
    g = np.asarray(g, np.complex64)
    tau = np.asarray(tau, np.float32)
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    with lib.Correlator(N, K, "fp32") as c:
        for f0 in range(0, S1, 32):                 # several queued launches
            c.push(dev[f0 * rec:(f0 + 32) * rec], 32 * K)
        c.set_corrections(g, tau)
        for f0 in range(S1, S1 + S2, 32):
            c.push(dev[f0 * rec:(f0 + 32) * rec], 32 * K)
        V, n = c.dump(fp64=True)
    assert n == S1 + S2
    R1, _ = oracle.correlate(packed[:S1], N, K)
    R2, _ = oracle.correlate(packed[S1:], N, K, gains=g.astype(np.complex128),
                             delays=tau.astype(np.float64))
    assert vis_error(V, R1 + R2, N) <= TOL


def test_pushes_follow_user_stream_work(lib, torch_cuda):
    """Each push's input is written by a kernel queued on the caller's stream
    just before the push; the F-engine on its side stream must see it."""
    torch = torch_cuda
    N, K, S = 8, 512, 384
    packed, _ = synth.make_samples(N, S * K, K, seed=SEED + 1)
    rec = N * K // 2
    src = torch.from_numpy(packed.reshape(-1)).cuda()
    R, _ = oracle.correlate(packed, N, K)
    s = torch.cuda.Stream()
    keep = []
    with lib.Correlator(N, K, "fp32", stream=s.cuda_stream) as c:
        with torch.cuda.stream(s):
            torch.cuda._sleep(1 << 20)               # the copies below start late
            for f0 in range(0, S, 64):
                b = torch.empty(64 * rec, dtype=torch.uint8, device="cuda")
                b.copy_(src[f0 * rec:(f0 + 64) * rec])
                keep.append(b)
                c.push(b, 64 * K)
        V, n = c.dump(fp64=True)
    assert n == S
    assert vis_error(V, R, N) <= TOL


def test_set_stream_joins_side_launches(lib, torch_cuda):
    """Switching the handle's stream between pushes keeps every frame."""
    torch = torch_cuda
    N, K, S = 5, 512, 256
    packed, _ = synth.make_samples(N, S * K, K, seed=SEED + 2)
    rec = N * K // 2
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    R, _ = oracle.correlate(packed, N, K)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with lib.Correlator(N, K, "fp32", stream=s1.cuda_stream) as c:
        c.push(dev[:128 * rec], 128 * K)
        lib.corr_set_stream(c.h, s2.cuda_stream)
        c.push(dev[128 * rec:], 128 * K)
        V, n = c.dump(fp64=True)
    assert n == S
    assert vis_error(V, R, N) <= TOL
