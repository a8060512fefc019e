"""FP32 paths under extreme per-antenna gains (GPU, through the C ABI).

The correction of Sec. 2.1 multiplies antenna i's spectra by a_i[k] =
g_i exp(-2 pi i k tau_i / K).  In CORR_FP32 mode the corrected spectra enter
the tensor cores as two FP16 planes, so their magnitude must stay inside the
FP16 range whatever |g_i| is: the handle pre-scales antenna i by the power of
two sigma_i = 2^floor(log2(2^15 / (8 K |g_i|))) (|X| <= 8K for 4-bit input)
and divides sigma_i sigma_j out of every visibility.  These tests put gains
of modulus 1e-4 .. 300 on one array, at K = 512 and 4096, with a 6 LSB tone
(and, separately, the worst-case input: every sample -8, |X[0]| = 8K), and
hold both FP32 paths to the 1e-5 bar against the FP64 oracle.  The
normalised error is invariant under gains (both V_ij and sqrt|V_ii V_jj|
scale by |g_i g_j|), so the bar is the same as at unit gain.
"""

import numpy as np
import pytest

import oracle
from conftest import report_err
from paper_1102_0148_gb300 import synth
from test_gpu_parity import TOL, run_gpu, vis_error

pytestmark = pytest.mark.gpu

SEED = 11020148 + 600
MODULI = np.array([1e-4, 1e-2, 1.0, 50.0, 300.0])
# FP16 (scales from the autocorrelations, so also gain-invariant): about twice
# the measured 1.1e-4 (K = 512) and 3.2e-4 (K = 4096)
FP16_BOUND = {512: 2.2e-4, 4096: 6.5e-4}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def extreme_gains(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    phase = rng.uniform(-np.pi, np.pi, MODULI.size)
    g = (MODULI * np.exp(1j * phase)).astype(np.complex64)
    tau = rng.uniform(-3.0, 3.0, MODULI.size).astype(np.float32)
    return g, tau


@pytest.mark.parametrize("dtype", ["fp32", "fp32_fused", "fp32_simt", "fp16"])
@pytest.mark.parametrize("K,S", [(512, 300), (4096, 40)])
def test_extreme_gains_with_tone(lib, torch_cuda, dtype, K, S):
    N = MODULI.size
    packed, _ = synth.make_samples(N, S * K, K, seed=SEED + K, tone_amp=6.0)
    g, tau = extreme_gains(SEED + K)
    R, n_ref = oracle.correlate(packed, N, K, gains=g.astype(np.complex128),
                                delays=tau.astype(np.float64))
    V, n = run_gpu(lib, torch_cuda, packed, N, K, dtype, gains=g, delays=tau)
    assert n == n_ref == S
    e = report_err(f"gains-{dtype}-K{K}", vis_error(V, R, N))
    assert e <= (FP16_BOUND[K] if dtype == "fp16" else TOL), e


@pytest.mark.parametrize("dtype", ["fp32", "fp32_fused", "fp32_simt"])
@pytest.mark.parametrize("K", [512, 4096])
def test_worst_case_input_largest_gain(lib, torch_cuda, dtype, K):
    """Every sample -8 (byte 0x88): |X[0]| = 8K, the bound the pre-scale is
    derived from, times |g| = 300 (9.8e6 at K = 4096, far beyond 65504)."""
    N, S = 3, 4
    packed = np.full((S, N, K // 2), 0x88, np.uint8)
    g = np.array([300.0, -300.0j, 1e-4], np.complex64)
    R, _ = oracle.correlate(packed, N, K, gains=g.astype(np.complex128))
    V, n = run_gpu(lib, torch_cuda, packed, N, K, dtype, gains=g)
    assert n == S
    dc = oracle.baseline_index(0, 0, N)
    assert np.isfinite(V).all()
    assert abs(V[dc, 0] - R[dc, 0]) <= 1e-6 * abs(R[dc, 0])
    # a constant input has power at DC only: channel 0 against the oracle at
    # the FP32 bar, the other channels (zero in exact arithmetic, rounding
    # noise in the oracle's direct DFT) against the DC power
    assert vis_error(V[:, :1], R[:, :1], N) <= TOL
    assert np.abs(V[:, 1:]).max() <= 1e-6 * abs(R[dc, 0])


def test_gains_outside_the_range_are_rejected(lib, torch_cuda):
    N, K = 3, 64
    with lib.Correlator(N, K, "fp32") as c:
        for bad in ([1.0, 2e12, 1.0], [1.0, np.nan, 1.0], [1e-13, 1.0, 1.0]):
            with pytest.raises(lib.CorrError) as ei:
                c.set_corrections(np.asarray(bad, np.complex64), None)
            assert ei.value.code == lib.CORR_EINVAL
        with pytest.raises(lib.CorrError) as ei:
            c.set_corrections(None, np.asarray([0.0, np.inf, 0.0], np.float32))
        assert ei.value.code == lib.CORR_EINVAL
        # zero and the range limits are accepted
        c.set_corrections(np.asarray([0.0, 2.0 ** 40, 2.0 ** -40], np.complex64), None)


def test_corrections_changed_mid_integration(lib, torch_cuda):
    """Frames pushed before a change of gains keep the old corrections even
    when the new gains change the pre-scale (the handle cross-multiplies the
    waiting frames first)."""
    torch = torch_cuda
    N, K, S = 4, 256, 256
    packed, _ = synth.make_samples(N, 2 * S * K, K, seed=SEED + 7)
    g1 = np.array([1.0, 0.5j, 2.0, 1.0], np.complex64)
    g2 = np.array([300.0, 1e-3, -1.0, 40.0j], np.complex64)
    R1, _ = oracle.correlate(packed[:S], N, K, gains=g1.astype(np.complex128))
    R2, _ = oracle.correlate(packed[S:], N, K, gains=g2.astype(np.complex128))
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    rec = N * K // 2
    for dtype in ("fp32", "fp32_simt"):
        with lib.Correlator(N, K, dtype) as c:
            c.set_corrections(g1, None)
            c.push(dev[: S * rec], S * K)
            c.set_corrections(g2, None)
            c.push(dev[S * rec:], S * K)
            V, n = c.dump(fp64=True)
        assert n == 2 * S
        assert vis_error(V, R1 + R2, N) <= TOL, dtype
