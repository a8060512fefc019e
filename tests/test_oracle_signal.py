"""Physical pins of the oracle (CPU): an injected tone and an injected
correlated fraction come out where the signal model puts them.

* A noise-free tone of 6 LSB at bin 97 of a 512-point transform, delayed by
  d_i samples on antenna i, is periodic in the frame, so every antenna's
  spectrum is the undelayed one times exp(-2 pi i 97 d_i / 512): the
  visibility at channel 97 has modulus S |Q[97]|^2 (Q from numpy's FFT of the
  quantised tone) and phase -2 pi 97 (d_i - d_j) / 512, exactly; applying
  delays tau_i = -d_i removes the slope.
* A 0.5 LSB tone dithered by sigma = 2 noise stands out ~8x in the autos and
  carries the same phase slope within its statistical error.
* A common Gaussian component of 1% of the noise power, after delay
  compensation, gives a channel-summed coherence of rho_q (1 - |d_i - d_j|/K),
  rho_q being the correlation after the 4-bit quantiser (first-order Hermite
  term, computed here from normal-distribution integrals) and (1 - |D|/K) the
  fraction of a frame the two delayed streams share.
"""

import math

import numpy as np
import pytest
from scipy.stats import norm

import oracle
from paper_1102_0148_gb300 import synth

K = 512
CH = 97


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def test_noise_free_tone_phase_and_modulus():
    N = 6
    d = np.array([0, 3, 15, 7, 1, 12])
    packed, _ = synth.make_samples(N, 8 * K, K, seed=1, noise=False, corr_sigma=0.0,
                                   tone_amp=6.0, tone_bin=CH, tone_K=K, delays=d)
    x = oracle.unpack(packed, N, K)
    Q = np.fft.rfft(x[0, :K].astype(np.float64))[CH]          # antenna 0 has d = 0
    V, S = oracle.correlate(packed, N, K)
    assert S == 8
    for p, (i, j) in enumerate(oracle.baseline_pairs(N)):
        want = S * abs(Q) ** 2 * np.exp(-2j * np.pi * CH * (d[i] - d[j]) / K)
        assert abs(V[p, CH] - want) <= 1e-9 * abs(want)
    # Compensating delays flatten the phase slope.
    Vc, _ = oracle.correlate(packed, N, K, delays=-d.astype(float))
    ph = np.angle(Vc[:, CH])
    assert np.abs(ph).max() < 1e-9
    # The tone channel dominates every auto.
    autos = [oracle.baseline_index(i, i, N) for i in range(N)]
    assert (Vc[autos, CH].real > 100 * np.delete(Vc[autos].real, CH, axis=1).max(1)).all()


def test_dithered_tone_stands_out_with_phase_slope():
    N, T = 44, 1 << 17
    packed, info = synth.make_samples(N, T, K, seed=11020148 + 2, tone_amp=0.5,
                                      tone_bin=CH, tone_K=K)
    d = info["delays"]
    V, S = oracle.correlate(packed, N, K)
    autos = [oracle.baseline_index(i, i, N) for i in range(N)]
    A = V[autos].real
    ratio = A[:, CH] / np.median(A, axis=1)
    # Tone power per spectrum (0.5*K/2)^2 = 16384 over noise ~ K*E[q^2] ~ 2110.
    assert (ratio > 6).all() and (ratio < 12).all()
    err = []
    for p, (i, j) in enumerate(oracle.baseline_pairs(N)):
        if i == j:
            continue
        want = -2 * np.pi * CH * (d[i] - d[j]) / K
        err.append(_wrap(np.angle(V[p, CH]) - want))
    err = np.abs(np.array(err))
    # statistical phase error ~ 1/(8 sqrt(S)) ~ 0.008 rad at S = 256
    assert err.max() < 0.06


def _quantiser_moments(sigma):
    """E[x q(x)] and E[q(x)^2] for x ~ N(0, sigma^2) and the 4-bit quantiser
    q = clip(round half away from zero, -8, 7)."""
    exq = 0.0
    eq2 = 0.0
    for v in range(-8, 8):
        lo = -np.inf if v == -8 else v - 0.5
        hi = np.inf if v == 7 else v + 0.5
        p = norm.cdf(hi / sigma) - norm.cdf(lo / sigma)
        ex = sigma * (norm.pdf(lo / sigma) - norm.pdf(hi / sigma))   # E[x; lo<x<hi]
        exq += v * ex
        eq2 += v * v * p
    return exq, eq2


def test_correlated_fraction_recovered():
    N, T = 44, 1 << 17
    sig_n, sig_c = 2.0, 0.2
    packed, info = synth.make_samples(N, T, K, seed=11020148 + 1, sigma=sig_n,
                                      corr_sigma=sig_c)
    d = info["delays"].astype(np.int64)
    var = sig_n ** 2 + sig_c ** 2
    rho = sig_c ** 2 / var
    exq, eq2 = _quantiser_moments(math.sqrt(var))
    rho_q = rho * exq ** 2 / (var * eq2)
    assert 0.0095 < rho_q < 0.0099

    Vc, S = oracle.correlate(packed, N, K, delays=-d.astype(float))
    V0, _ = oracle.correlate(packed, N, K)
    C = K // 2
    k = np.arange(C)
    autos = np.array([oracle.baseline_index(i, i, N) for i in range(N)])
    pw = Vc[autos].real.sum(1)
    got_c, got_0, want_c, want_0 = [], [], [], []
    for p, (i, j) in enumerate(oracle.baseline_pairs(N)):
        if i == j:
            continue
        D = d[i] - d[j]
        nrm = math.sqrt(pw[i] * pw[j])
        got_c.append(Vc[p].real.sum() / nrm)
        got_0.append(V0[p].real.sum() / nrm)
        overlap = 1 - abs(D) / K
        want_c.append(rho_q * overlap)
        want_0.append(rho_q * overlap * np.cos(2 * np.pi * k * D / K).mean())
    got_c, got_0 = np.array(got_c), np.array(got_0)
    want_c, want_0 = np.array(want_c), np.array(want_0)
    sig = 1 / math.sqrt(2 * S * C)                    # per-baseline std
    assert np.abs(got_c - want_c).max() < 5.5 * sig
    assert np.abs(got_0 - want_0).max() < 5.5 * sig
    sig_mean = sig / math.sqrt(len(got_c))
    assert abs(got_c.mean() - want_c.mean()) < 5 * sig_mean
    assert abs(got_0.mean() - want_0.mean()) < 5 * sig_mean
    # A wrong correction sign would double the slope instead of removing it.
    Vw, _ = oracle.correlate(packed, N, K, delays=d.astype(float))
    wrong = np.mean([Vw[p].real.sum() / math.sqrt(pw[i] * pw[j])
                     for p, (i, j) in enumerate(oracle.baseline_pairs(N)) if i != j
                     and d[i] != d[j]])
    assert wrong < 0.5 * want_c.mean()
