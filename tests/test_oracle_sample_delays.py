"""Pins of the oracle's integer sample delays (streaming form).

* A delay of exactly one frame (D = K) moves every frame to the next frame
  slot, so the spectra of the delayed stream are the original spectra one
  frame later, with an all-zero first frame: an identity between DFTs of
  different frames that no retyping of the shift can fake.
* Physical pin of the sign: the synthetic common signal reaches antenna i
  d_i samples late, so its tone (channel 97 of K = 512) shows in V_ij with
  phase -2 pi 97 (d_i - d_j) / 512.  Delaying antenna i by D_i = max(d) - d_i
  lines the common signal up on every antenna and removes that phase slope;
  the opposite sign would double it.
* Energy: the delayed stream holds the original samples minus the last D_i
  of each antenna.
"""

import numpy as np

import oracle
from paper_1102_0148_gb300 import synth


def test_whole_frame_delay_moves_spectra_by_one_frame():
    N, K, F = 3, 64, 9
    packed, _ = synth.make_samples(N, F * K, K, seed=5)
    x = oracle.unpack(packed, N, K)
    X = oracle.spectra(x, K)
    Y = oracle.spectra(oracle.delay_samples(x, [K, 0, K]), K)
    assert np.array_equal(Y[1], X[1])
    for i in (0, 2):
        assert not np.any(Y[i, 0])
        np.testing.assert_allclose(Y[i, 1:], X[i, :-1], rtol=0, atol=1e-9)


def test_compensating_delays_remove_the_tone_phase_slope():
    N, K, F = 6, 512, 400
    d = np.array([0, 3, 7, 12, 5, 15])
    packed, info = synth.make_samples(N, F * K, K, seed=9, delays=d, tone_amp=2.0)
    assert np.array_equal(info["delays"], d)
    ch = 97
    R, _ = oracle.correlate(packed, N, K)
    D = d.max() - d
    Rc, _ = oracle.correlate(packed, N, K, sample_delays=D)
    for i in range(N):
        for j in range(i + 1, N):
            p = oracle.baseline_index(i, j, N)
            want = -2 * np.pi * ch * (d[i] - d[j]) / K
            before = np.angle(R[p, ch] * np.exp(-1j * want))
            after = np.angle(Rc[p, ch])
            assert abs(before) < 0.05, (i, j, before)      # the uncompensated slope is there
            assert abs(after) < 0.05, (i, j, after)        # and compensation removes it


def test_delay_keeps_all_but_the_last_samples():
    N, K, F = 4, 32, 5
    packed, _ = synth.make_samples(N, F * K, K, seed=3)
    x = oracle.unpack(packed, N, K).astype(np.int64)
    D = [0, 1, 17, 32]
    y = oracle.delay_samples(x, D)
    for i in range(N):
        T = x.shape[1]
        assert np.sum(y[i] ** 2) == np.sum(x[i, :T - D[i]] ** 2)
        assert np.array_equal(np.sort(y[i, D[i]:]), np.sort(x[i, :T - D[i]]))
