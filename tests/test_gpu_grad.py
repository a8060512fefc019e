"""Differentiation form (GPU): dL/dg and dL/dtau through the autograd Function.

Workload: N = 44, K = 512, 2^20 samples per antenna (2048 spectra), FP32.
Gains g ~ CN(1, 0.1^2) and fractional delays tau ~ U(-0.5, 0.5) samples are
applied in the F-engine; L = sum |V_ij - M_ij|^2 with M the visibilities of
the uncorrected instrument (g = 1, tau = 0), from the oracle.  The gradient
from the library's backward kernel is checked against the oracle's closed
form (relative 1e-4 of the largest component) and against central finite
differences (h = 1e-3) of the oracle's FP64 forward; a finite difference of
the GPU forward itself checks the autograd wiring end to end.
"""

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth

pytestmark = pytest.mark.gpu

N, K = 44, 512
S = (1 << 20) // K


@pytest.fixture(scope="module")
def setup():
    import torch
    packed, _ = synth.make_samples(N, S * K, K, seed=11020148 + 5)
    R, _ = oracle.correlate(packed, N, K)
    g, tau = synth.gains_delays(N, seed=11020148 + 5)
    g = np.asarray(g, np.complex64).astype(np.complex128)      # the values the GPU sees
    tau = np.asarray(tau, np.float32).astype(np.float64)
    return torch.from_numpy(packed.reshape(-1)).cuda(), R, g, tau


def gpu_loss_and_grad(lib, dev, R, g, tau, dtype="fp32"):
    import torch
    from paper_1102_0148_gb300.autograd import visibilities
    M = torch.from_numpy(R).cuda()
    gt = torch.tensor(g, dtype=torch.complex64, device="cuda", requires_grad=True)
    tt = torch.tensor(tau, dtype=torch.float32, device="cuda", requires_grad=True)
    with lib.Correlator(N, K, dtype) as c:
        V = visibilities(gt, tt, dev, c)
        L = (V - M).abs().pow(2).sum()
        L.backward()
    return float(L.item()), gt.grad.cpu().numpy().astype(np.complex128), tt.grad.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", ["fp32", "fp32_simt"])
def test_grad_matches_oracle_closed_form(lib, setup, dtype):
    dev, R, g, tau = setup
    L, gg, gt = gpu_loss_and_grad(lib, dev, R, g, tau, dtype)
    L0, og, ot = oracle.loss_and_grad(R, g, tau, K)
    assert abs(L - L0) <= 1e-4 * L0
    scale_g = np.abs(og).max()
    scale_t = np.abs(ot).max()
    assert np.abs(gg - og).max() <= 1e-4 * scale_g, np.abs(gg - og).max() / scale_g
    assert np.abs(gt - ot).max() <= 1e-4 * scale_t, np.abs(gt - ot).max() / scale_t


def test_grad_matches_oracle_finite_differences(lib, setup):
    dev, R, g, tau = setup
    _, gg, gt = gpu_loss_and_grad(lib, dev, R, g, tau)
    h = 1e-3
    scale = max(np.abs(gg).max(), np.abs(gt).max())
    for m in (0, 17, 43):
        e = np.zeros(N)
        e[m] = h
        d_re = (oracle.loss(R, g + e, tau, K) - oracle.loss(R, g - e, tau, K)) / (2 * h)
        d_im = (oracle.loss(R, g + 1j * e, tau, K) - oracle.loss(R, g - 1j * e, tau, K)) / (2 * h)
        d_t = (oracle.loss(R, g, tau + e, K) - oracle.loss(R, g, tau - e, K)) / (2 * h)
        assert abs(gg[m] - (d_re + 1j * d_im)) <= 1e-4 * scale
        assert abs(gt[m] - d_t) <= 1e-4 * scale


def test_grad_matches_gpu_forward_differences(lib, setup):
    """Central differences of the GPU's own FP32 forward (looser: the FP32
    rounding of L enters divided by 2h)."""
    dev, R, g, tau = setup
    _, gg, gt = gpu_loss_and_grad(lib, dev, R, g, tau)
    h = 1e-3
    scale = max(np.abs(gg).max(), np.abs(gt).max())
    for m in (3, 30):
        e = np.zeros(N)
        e[m] = h
        Lp, _, _ = gpu_loss_and_grad(lib, dev, R, g + e, tau)
        Lm, _, _ = gpu_loss_and_grad(lib, dev, R, g - e, tau)
        assert abs(gg[m].real - (Lp - Lm) / (2 * h)) <= 1e-2 * scale
        Lp, _, _ = gpu_loss_and_grad(lib, dev, R, g, tau + e)
        Lm, _, _ = gpu_loss_and_grad(lib, dev, R, g, tau - e)
        assert abs(gt[m] - (Lp - Lm) / (2 * h)) <= 1e-2 * scale


def test_grad_leaves_running_integration_untouched(lib, setup):
    import torch
    dev, R, g, tau = setup
    with lib.Correlator(N, K, "fp32") as c:
        c.push(dev[: 64 * N * K // 2], 64 * K)
        gV = np.ones((c.P, c.C), np.complex128)
        gg = np.empty(N, np.complex64)
        gt = np.empty(N, np.float32)
        lib.corr_grad(c.h, dev, S * K, g.astype(np.complex64), tau.astype(np.float32), gV, True,
                      gg, gt)
        V, n = c.dump(fp64=True)
    assert n == 64
    R64, _ = oracle.correlate(dev[: 64 * N * K // 2].cpu().numpy(), N, K)
    autos = [oracle.baseline_index(i, i, N) for i in range(N)]
    A = np.abs(R64[autos])
    pairs = oracle.baseline_pairs(N)
    nrm = np.sqrt(A[[p[0] for p in pairs]] * A[[p[1] for p in pairs]])
    assert np.max(np.abs(V - R64) / nrm) <= 1e-5
    del torch
