"""Pins of the oracle's unpack and DFT steps (CPU only).

Each check compares the oracle with something it does not compute itself:
the two's-complement definition written forwards, hand-derived K = 8
transforms (tests/golden/dft_k8.txt), numpy's FFT, the shift theorem and
Parseval's identity.
"""

import os

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_unpack_exhaustive_256_bytes():
    # Forward construction: a value v in [-8, 7] is stored as v mod 16.
    vals = np.arange(-8, 8)
    lo, hi = np.meshgrid(vals, vals, indexing="ij")
    lo = lo.ravel()
    hi = hi.ravel()
    byte = ((lo % 16) | ((hi % 16) << 4)).astype(np.uint8)
    assert len(set(byte.tolist())) == 256
    x = oracle.unpack(byte, N=1, K=512)          # 256 bytes = one frame
    assert x.dtype == np.int8
    assert np.array_equal(x[0, 0::2], lo)
    assert np.array_equal(x[0, 1::2], hi)


def test_unpack_frame_antenna_layout():
    # Distinct sample values per (antenna, time) survive pack -> unpack.
    rng = np.random.default_rng(5)
    N, K, F = 3, 16, 4
    q = rng.integers(-8, 8, (N, F * K))
    packed = synth.pack_nibbles(q, K)
    assert packed.shape == (F, N, K // 2)
    # byte m of (frame f, antenna i) = samples f*K + 2m (low), f*K + 2m + 1 (high)
    f, i, m = 2, 1, 5
    b = int(packed[f, i, m])
    assert (b & 15) == (q[i, f * K + 2 * m] % 16)
    assert (b >> 4) == (q[i, f * K + 2 * m + 1] % 16)
    assert np.array_equal(oracle.unpack(packed, N, K), q)


def _golden_k8():
    cases = []
    with open(os.path.join(GOLDEN, "dft_k8.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            xs, ys = line.split("|")
            x = np.array([int(v) for v in xs.split()])
            y = np.array([float(v) for v in ys.split()])
            cases.append((x, y[0::2] + 1j * y[1::2]))
    return cases


@pytest.mark.parametrize("case", range(7))
def test_dft_hand_derived_k8(case):
    x, want = _golden_k8()[case]
    X = oracle.spectra(x[None, :], 8, with_nyquist=True)[0, 0]
    np.testing.assert_allclose(X, want, atol=1e-13)


@pytest.mark.parametrize("K", [8, 16, 64, 512, 4096])
def test_dft_matches_numpy_rfft(K):
    rng = np.random.default_rng(K)
    x = rng.integers(-8, 8, (3, 4 * K))
    X = oracle.spectra(x, K)
    ref = np.fft.rfft(x.reshape(3, 4, K).astype(np.float64), axis=-1)[..., :K // 2]
    scale = np.abs(ref).max()
    assert np.abs(X - ref).max() <= 1e-12 * scale * np.log2(K)


def test_dft_impulse_and_constant():
    K = 64
    for n0 in (0, 1, 7, 33):
        x = np.zeros((1, K), np.int64)
        x[0, n0] = 1
        X = oracle.spectra(x, K)[0, 0]
        k = np.arange(K // 2)
        np.testing.assert_allclose(X, np.exp(-2j * np.pi * k * n0 / K), atol=1e-13)
    X = oracle.spectra(np.full((1, K), 3), K)[0, 0]
    assert abs(X[0] - 3 * K) < 1e-12
    assert np.abs(X[1:]).max() < 1e-12


def test_dft_shift_theorem():
    K = 256
    rng = np.random.default_rng(1)
    x = rng.integers(-8, 8, K)
    for m in (1, 5, 100):
        X0 = oracle.spectra(x[None], K)[0, 0]
        X1 = oracle.spectra(np.roll(x, m)[None], K)[0, 0]
        k = np.arange(K // 2)
        np.testing.assert_allclose(X1, X0 * np.exp(-2j * np.pi * k * m / K),
                                   atol=1e-9)


@pytest.mark.parametrize("K", [16, 512])
def test_parseval_with_nyquist_weight(K):
    rng = np.random.default_rng(2)
    x = rng.integers(-8, 8, (2, 8 * K))
    X = oracle.spectra(x, K, with_nyquist=True)
    P = np.abs(X) ** 2
    spec_power = (P[..., 0] + 2 * P[..., 1:K // 2].sum(-1) + P[..., K // 2]) / K
    time_power = (x.reshape(2, 8, K).astype(np.float64) ** 2).sum(-1)
    np.testing.assert_allclose(spec_power, time_power, rtol=1e-12)


def test_channel_subset_matches_full():
    K = 128
    rng = np.random.default_rng(3)
    x = rng.integers(-8, 8, (2, 3 * K))
    full = oracle.spectra(x, K)
    ch = [0, 5, 63]
    part = oracle.spectra(x, K, channels=ch)
    np.testing.assert_allclose(part, full[..., ch], atol=1e-10)
