"""Pins of the oracle's cross-multiply-accumulate and correction steps (CPU).

* brute force: plain loops over (i, j, s) on a tiny input;
* the lag identity: the inverse transform of one spectrum's cross power
  equals the circular cross-correlation computed in the time domain, which
  fixes the transform's sign, the conjugated operand and the pair order;
* Hermitian symmetry and real, non-negative autos;
* the correction: an applied integer delay equals a circular shift of the
  samples, and a gain scales V_ij by g_i conj(g_j).
"""

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth


def test_pair_order_and_index():
    for N in (1, 2, 5, 44):
        pairs = oracle.baseline_pairs(N)
        assert len(pairs) == N * (N + 1) // 2
        for p, (i, j) in enumerate(pairs):
            assert oracle.baseline_index(i, j, N) == p
    # 44 antennas: 946 cross baselines + 44 autos = 990 outputs per channel.
    assert len(oracle.baseline_pairs(44)) == 990


def test_visibilities_brute_force_loops():
    rng = np.random.default_rng(7)
    N, S, C = 4, 5, 3
    Y = rng.normal(size=(N, S, C)) + 1j * rng.normal(size=(N, S, C))
    V = oracle.visibilities(Y)
    p = 0
    for i in range(N):
        for j in range(i, N):
            for k in range(C):
                acc = 0j
                for s in range(S):
                    acc += Y[i, s, k] * complex(Y[j, s, k].real, -Y[j, s, k].imag)
                assert abs(V[p, k] - acc) < 1e-12
            p += 1


def test_lag_identity_single_spectrum():
    K = 32
    rng = np.random.default_rng(11)
    x = rng.integers(-8, 8, (3, K))
    X = oracle.spectra(x, K, with_nyquist=True)          # [3][1][K/2+1]
    G = oracle.full_visibility_matrix(X)                 # [K/2+1][3][3]
    k = np.arange(1, K // 2)
    for i in range(3):
        for j in range(3):
            for lag in (0, 1, 3, 17, K - 1):
                V = G[:, i, j]
                r = (V[0].real + V[K // 2].real * (-1) ** lag
                     + 2 * np.real(np.sum(V[1:K // 2] * np.exp(2j * np.pi * k * lag / K)))) / K
                brute = sum(int(x[i, (m + lag) % K]) * int(x[j, m]) for m in range(K))
                assert abs(r - brute) < 1e-9, (i, j, lag)


def test_hermitian_and_autos():
    packed, _ = synth.make_samples(6, 64 * 16, 64, seed=3)
    x = oracle.unpack(packed, 6, 64)
    G = oracle.full_visibility_matrix(oracle.spectra(x, 64))
    np.testing.assert_allclose(G, np.conj(G.transpose(0, 2, 1)),
                               atol=1e-12 * np.abs(G).max())
    d = np.diagonal(G, axis1=1, axis2=2)
    assert np.abs(d.imag).max() <= 1e-12 * np.abs(d).max()
    assert (d.real >= 0).all()


def test_integer_delay_equals_circular_shift():
    # a_i[k] = exp(-2 pi i k tau / K) with integer tau applied to one frame is
    # the transform of the frame shifted later by tau samples (circularly).
    K = 64
    rng = np.random.default_rng(4)
    x = rng.integers(-8, 8, (1, K))
    for tau in (1, 3, -2):
        a = oracle.correction_factors(K, delays=[tau])
        Y = oracle.spectra(x, K) * a[:, None, :]
        Xs = oracle.spectra(np.roll(x, tau, axis=1), K)
        np.testing.assert_allclose(Y, Xs, atol=1e-9)


def test_gain_scales_visibility():
    rng = np.random.default_rng(9)
    N, K = 3, 32
    x = rng.integers(-8, 8, (N, 4 * K))
    X = oracle.spectra(x, K)
    g = np.array([1.5 - 0.2j, 0.7 + 0.1j, -1.0 + 0.5j])
    V0 = oracle.visibilities(X)
    V1 = oracle.visibilities(X * oracle.correction_factors(K, gains=g)[:, None, :])
    for p, (i, j) in enumerate(oracle.baseline_pairs(N)):
        np.testing.assert_allclose(V1[p], g[i] * np.conj(g[j]) * V0[p], rtol=1e-12,
                                   atol=1e-9)


@pytest.mark.parametrize("channels", [[0, 97, 255], [13]])
def test_streamed_channel_subset_matches_full(channels):
    N, K = 5, 512
    packed, info = synth.make_samples(N, 40 * K, K, seed=21)
    g = np.linspace(0.9, 1.1, N) * np.exp(1j * np.linspace(0, 1, N))
    tau = np.linspace(-0.5, 0.5, N)
    V, S = oracle.correlate(packed, N, K, gains=g, delays=tau)
    Vs, S2 = oracle.visibilities_channels(packed, N, K, channels, gains=g,
                                          delays=tau, frames_per_block=7)
    assert S == S2 == 40
    np.testing.assert_allclose(Vs, V[:, channels], rtol=1e-10,
                               atol=1e-9 * np.abs(V).max())
