"""Fused F/X-engine (GPU, through the C ABI): K = 512, CORR_FP32, N <= 44.

With corr_set_fused(h, 1), device-memory pushes of such a handle run as
one persistent kernel per flush, F-engine and X-engine warps side by side
on every SM, the spectra handed over through a three-slot ring of
256-frame chunks.  Every case is
held to the FP32 bar (1e-5, normalised by sqrt|V_ii V_jj|) against the FP64
oracle, and the same pushes through the separate F- and X-engine launches
(corr_set_fused(h, 0)) to the same bar.
"""

import numpy as np
import pytest

import oracle
from conftest import report_err
from paper_1102_0148_gb300 import synth
from test_gpu_parity import TOL, vis_error

pytestmark = pytest.mark.gpu

SEED = 11020148 + 700


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def correlate(lib, torch, packed, N, pushes, fused, gains=None, delays=None, host=False):
    K = 512
    rec = N * K // 2
    buf = torch.from_numpy(np.ascontiguousarray(packed).reshape(-1))
    buf = buf.pin_memory() if host else buf.cuda()
    with lib.Correlator(N, K, "fp32", fused=fused) as c:
        if gains is not None or delays is not None:
            c.set_corrections(gains, delays)
        f0 = 0
        for nf in pushes:
            c.push(buf[f0 * rec:(f0 + nf) * rec], nf * K)
            f0 += nf
        V, n = c.dump(fp64=True)
    assert n == sum(pushes)
    return V


def test_served_and_switchable(lib, torch_cuda):
    with lib.Correlator(44, 512, "fp32") as c:
        assert not lib.corr_get_fused(c.h)          # off by default
        lib.corr_set_fused(c.h, True)
        assert lib.corr_get_fused(c.h)
        lib.corr_set_fused(c.h, False)
        assert not lib.corr_get_fused(c.h)
    for N, K, dtype in [(44, 512, "fp16"), (44, 1024, "fp32"), (45, 512, "fp32"), (8, 512, "fp32_simt")]:
        with lib.Correlator(N, K, dtype) as c:
            assert not lib.corr_get_fused(c.h)
            with pytest.raises(lib.CorrError) as ei:
                lib.corr_set_fused(c.h, True)
            assert ei.value.code == lib.CORR_EUNSUPPORTED


@pytest.mark.parametrize("N,pushes", [
    (44, [256]),                           # the plain-FX workload: one chunk
    (44, [100, 1, 200, 37, 512, 1000]),    # ragged pushes: partial 32-frame blocks
    (44, [2048, 2048, 1000, 775]),         # 11 chunks: the ring turns over 3 times
    (1, [300]), (2, [70, 33]), (5, [600]), (17, [129, 640]), (40, [1100]),
])
def test_fused_matches_oracle_and_separate_path(lib, torch_cuda, N, pushes):
    S = sum(pushes)
    packed, _ = synth.make_samples(N, S * 512, 512, seed=SEED + N * 10 + len(pushes))
    R, _ = oracle.correlate(packed, N, 512)
    Vf = correlate(lib, torch_cuda, packed, N, pushes, fused=True)
    Vs = correlate(lib, torch_cuda, packed, N, pushes, fused=False)
    e = report_err(f"fused-N{N}-S{S}", vis_error(Vf, R, N))
    assert e <= TOL, e
    assert vis_error(Vs, R, N) <= TOL
    assert vis_error(Vf, Vs, N) <= TOL


def test_fused_with_corrections_and_extreme_gains(lib, torch_cuda):
    N, pushes = 5, [700, 333]
    S = sum(pushes)
    packed, _ = synth.make_samples(N, S * 512, 512, seed=SEED + 99, tone_amp=6.0)
    rng = np.random.Generator(np.random.PCG64(SEED + 99))
    g = (np.array([1e-4, 1e-2, 1.0, 50.0, 300.0]) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))).astype(np.complex64)
    tau = rng.uniform(-3.0, 3.0, N).astype(np.float32)
    R, _ = oracle.correlate(packed, N, 512, gains=g.astype(np.complex128), delays=tau.astype(np.float64))
    V = correlate(lib, torch_cuda, packed, N, pushes, fused=True, gains=g, delays=tau)
    assert report_err("fused-gains", vis_error(V, R, N)) <= TOL


def test_fused_mixed_with_host_pushes_and_correction_changes(lib, torch_cuda):
    """Device pushes (fused), a host push (separate launches) and a change of
    gains in one integration: each frame keeps the corrections in force when
    it was pushed."""
    torch = torch_cuda
    N, K = 6, 512
    packed, _ = synth.make_samples(N, 900 * K, K, seed=SEED + 5)
    g1 = np.array([1.0, 2.0, 0.5j, 1.0, -1.0, 3.0], np.complex64)
    g2 = np.array([40.0, 1.0, 1.0, 1e-2j, 1.0, 1.0], np.complex64)
    parts = [(0, 300, g1, False), (300, 500, g1, True), (500, 900, g2, False)]
    R = sum(oracle.correlate(packed[a:b], N, K, gains=g.astype(np.complex128))[0]
            for a, b, g, _ in parts)
    rec = N * K // 2
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    host = torch.from_numpy(packed.reshape(-1)).pin_memory()
    with lib.Correlator(N, K, "fp32", fused=True) as c:
        for a, b, g, on_host in parts:
            c.set_corrections(g, None)
            src = host if on_host else dev
            c.push(src[a * rec:b * rec], (b - a) * K)
        V, n = c.dump(fp64=True)
    assert n == 900 and vis_error(V, R, N) <= TOL


def test_fused_checkpoint_resume(lib, torch_cuda):
    torch = torch_cuda
    N, K = 44, 512
    packed, _ = synth.make_samples(N, 1200 * K, K, seed=SEED + 7)
    rec = N * K // 2
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    with lib.Correlator(N, K, "fp32", fused=True) as a:
        a.push(dev[: 700 * rec], 700 * K)
        state = lib.corr_save_state(a.h)          # runs the waiting fused launch first
        a.push(dev[700 * rec:], 500 * K)
        Va, _ = a.dump(fp64=True)
    with lib.Correlator(N, K, "fp32", fused=True) as b:
        lib.corr_load_state(b.h, state)
        b.push(dev[700 * rec:], 500 * K)
        Vb, n = b.dump(fp64=True)
    assert n == 1200 and np.array_equal(Va, Vb)


def test_fused_bounded_wait_gives_up_and_handle_recovers(lib, torch_cuda):
    """corr_test_fault kind 2: the first chunk of the next fused launch never
    counts as complete, so the producer waits give up after the limit; the
    dump reports CORR_ETIMEOUT, and the next integration is exact."""
    torch = torch_cuda
    N, K, S = 44, 512, 600
    packed, _ = synth.make_samples(N, S * K, K, seed=SEED + 8)
    R, _ = oracle.correlate(packed, N, K)
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    with lib.Correlator(N, K, "fp32", fused=True) as c:
        lib.corr_test_fault(c.h, 2, 0.05)
        c.push(dev, S * K)
        with pytest.raises(lib.CorrError) as ei:
            c.dump(fp64=True)
        assert ei.value.code == lib.CORR_ETIMEOUT
        c.push(dev, S * K)
        V, n = c.dump(fp64=True)
    assert n == S and vis_error(V, R, N) <= TOL
