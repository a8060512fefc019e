"""Pins of the oracle's closed-form gradient (CPU): central finite
differences of the oracle's own float64 forward (an independent route to the
same derivative), and the zero-loss, zero-gradient point a = 1."""

import numpy as np

import oracle
from paper_1102_0148_gb300 import synth


def _setup(N=5, K=32, S=24, seed=4):
    packed, _ = synth.make_samples(N, S * K, K, seed=seed)
    R, _ = oracle.correlate(packed, N, K)
    g, tau = synth.gains_delays(N, seed=seed + 1)
    return R, g, tau, K


def test_zero_at_model_point():
    R, g, tau, K = _setup()
    N = len(g)
    L, gg, gt = oracle.loss_and_grad(R, np.ones(N, complex), np.zeros(N), K)
    assert L == 0.0
    assert np.abs(gg).max() == 0.0 and np.abs(gt).max() == 0.0


def test_forward_matches_corrected_correlation():
    N, K, S = 4, 32, 16
    packed, _ = synth.make_samples(N, S * K, K, seed=8)
    R, _ = oracle.correlate(packed, N, K)
    g, tau = synth.gains_delays(N, seed=9)
    V, _ = oracle.correlate(packed, N, K, gains=g, delays=tau)
    L = oracle.loss(R, g, tau, K)
    assert abs(L - np.sum(np.abs(V - R) ** 2)) <= 1e-10 * L


def test_gradient_matches_central_differences():
    R, g, tau, K = _setup()
    N = len(g)
    L, gg, gt = oracle.loss_and_grad(R, g, tau, K)
    h = 1e-6
    for m in range(N):
        e = np.zeros(N)
        e[m] = h
        d_re = (oracle.loss(R, g + e, tau, K) - oracle.loss(R, g - e, tau, K)) / (2 * h)
        d_im = (oracle.loss(R, g + 1j * e, tau, K) - oracle.loss(R, g - 1j * e, tau, K)) / (2 * h)
        d_tau = (oracle.loss(R, g, tau + e, K) - oracle.loss(R, g, tau - e, K)) / (2 * h)
        scale = max(abs(gg).max(), abs(gt).max())
        assert abs(gg[m] - (d_re + 1j * d_im)) < 1e-6 * scale
        assert abs(gt[m] - d_tau) < 1e-6 * scale
