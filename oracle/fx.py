"""FX correlator oracle, float64: unpack -> direct DFT -> correction -> XMAC.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What the paper computes (Sec. 1): each antenna's sample stream is split into
spectral channels with an FFT, every pair of antennas is cross-multiplied per
channel to form the cross power spectra, and these are accumulated to the
required cadence.  Each function below is the plain definition of one of
those steps.

Readings of the paper used here (the paper prints no formulas for them):

* Input (Sec. 1: 4-bit quantisation; Sec. 2.2: a frame holds K contiguous
  samples from *all* elements): packed bytes laid out ``[frame][antenna][K/2]``;
  byte ``b`` carries two samples, the earlier one in the low nibble, each a
  4-bit two's-complement integer in [-8, 7].
* Transform (Sec. 4: forward, unnormalised, single precision in the paper):
  X_i[s, k] = sum_n x_i[s*K + n] * exp(-2*pi*i*k*n/K), no scaling.
* Channels (Sec. 1, computation-rate paragraph: K channels per 2K-point
  transform): C = K/2 channels k = 0 .. K/2-1; DC kept, Nyquist (k = K/2)
  dropped from the output.
* Correction (Sec. 2.1 mentions a phase applied before accumulation):
  Y_i[s, k] = a_i[k] X_i[s, k] with a_i[k] = g_i * exp(-2*pi*i*k*tau_i/K), i.e.
  a complex gain g_i and a delay of tau_i samples applied to antenna i.
* Cross-multiply (Sec. 1, Sec. 4 "complex cross multiply"):
  V_ij[k] = sum_s Y_i[s, k] * conj(Y_j[s, k]); only i <= j is emitted
  (V_ji = conj(V_ij)), autos included, upper triangle in row-major order.
"""

import numpy as np


# ---------------------------------------------------------------------------
# Baseline bookkeeping
# ---------------------------------------------------------------------------

def baseline_pairs(N):
    """All (i, j) with 0 <= i <= j < N in row-major upper-triangle order.

    There are N(N+1)/2 of them: the N(N-1)/2 cross baselines of Sec. 1 plus
    the N autocorrelations.
    """
    return [(i, j) for i in range(N) for j in range(i, N)]


def baseline_index(i, j, N):
    """Position of pair (i, j), i <= j, in ``baseline_pairs(N)``."""
    if not (0 <= i <= j < N):
        raise ValueError("need 0 <= i <= j < N")
    return i * N - i * (i - 1) // 2 + (j - i)


# ---------------------------------------------------------------------------
# Step 1: 4-bit unpack (Sec. 1, Sec. 2.2)
# ---------------------------------------------------------------------------

def unpack(packed, N, K):
    """Packed bytes ``[F][N][K/2]`` (any shape with that many bytes) -> int8
    samples ``x[N][F*K]``.

    Byte m of a (frame, antenna) record holds sample 2m in its low nibble and
    sample 2m+1 in its high nibble; a nibble v in 0..15 is the two's-complement
    value v - 16 when v >= 8.
    """
    b = np.asarray(packed, dtype=np.uint8).reshape(-1)
    if K % 2 or b.size % (N * (K // 2)):
        raise ValueError("byte count is not a whole number of frames")
    F = b.size // (N * (K // 2))
    b = b.reshape(F, N, K // 2).astype(np.int16)
    lo = b & 0x0F
    hi = (b >> 4) & 0x0F
    lo = np.where(lo >= 8, lo - 16, lo)
    hi = np.where(hi >= 8, hi - 16, hi)
    x = np.empty((F, N, K), dtype=np.int8)
    x[:, :, 0::2] = lo
    x[:, :, 1::2] = hi
    return np.ascontiguousarray(x.transpose(1, 0, 2)).reshape(N, F * K)


# ---------------------------------------------------------------------------
# Step 2: direct DFT (Sec. 1, Sec. 4)
# ---------------------------------------------------------------------------

def dft_matrix(K, channels=None, with_nyquist=False):
    """W[n, c] = exp(-2*pi*i * k_c * n / K) in float64.

    ``channels`` selects which k to return (default 0 .. K/2-1, plus K/2 when
    ``with_nyquist``).  The product k*n is reduced modulo K in integer
    arithmetic before it becomes an angle, so every angle is 2*pi*m/K with an
    exact integer m < K.
    """
    if channels is None:
        channels = np.arange(K // 2 + (1 if with_nyquist else 0))
    k = np.asarray(channels, dtype=np.int64)[None, :]
    n = np.arange(K, dtype=np.int64)[:, None]
    m = (n * k) % K
    theta = 2.0 * np.pi * m / K
    return np.cos(theta) - 1j * np.sin(theta)


def spectra(x, K, with_nyquist=False, channels=None):
    """Samples ``x[N][T]`` (T a multiple of K) -> ``X[N][S][C]`` complex128.

    One unnormalised forward DFT per antenna per frame of K samples; the
    transform is the matrix product of the frames with ``dft_matrix``.
    """
    x = np.asarray(x)
    N, T = x.shape
    if T % K:
        raise ValueError("T must be a multiple of K")
    S = T // K
    frames = x.reshape(N * S, K).astype(np.float64)
    W = dft_matrix(K, channels=channels, with_nyquist=with_nyquist)
    return (frames @ W).reshape(N, S, W.shape[1])


# ---------------------------------------------------------------------------
# Step 3: per-antenna gain and delay (Sec. 2.1)
# ---------------------------------------------------------------------------

def correction_factors(K, gains=None, delays=None, N=None, channels=None):
    """a[i, c] = g_i * exp(-2*pi*i * k_c * tau_i / K), float64/complex128.

    ``gains`` complex, ``delays`` real (samples, any real value).  Missing
    gains are 1 and missing delays 0.
    """
    if N is None:
        N = len(gains) if gains is not None else len(delays)
    g = np.ones(N, np.complex128) if gains is None else np.asarray(gains, np.complex128)
    tau = np.zeros(N) if delays is None else np.asarray(delays, np.float64)
    if channels is None:
        channels = np.arange(K // 2)
    k = np.asarray(channels, dtype=np.float64)
    phase = -2.0 * np.pi * np.outer(tau, k) / K
    return g[:, None] * (np.cos(phase) + 1j * np.sin(phase))


# ---------------------------------------------------------------------------
# Step 4: cross-multiply and accumulate (Sec. 1, Sec. 4)
# ---------------------------------------------------------------------------

def full_visibility_matrix(Y):
    """``Y[N][S][C]`` -> ``V[C][N][N]`` with V[k, i, j] = sum_s Y_i conj(Y_j)."""
    Yk = np.ascontiguousarray(np.asarray(Y, np.complex128).transpose(2, 0, 1))
    return Yk @ Yk.conj().transpose(0, 2, 1)


def visibilities(Y):
    """``Y[N][S][C]`` -> ``V[P][C]``, P = N(N+1)/2, pairs in ``baseline_pairs``
    order."""
    G = full_visibility_matrix(Y)
    N = G.shape[1]
    iu, ju = np.triu_indices(N)
    return np.ascontiguousarray(G[:, iu, ju].T)


def visibilities_channels(packed, N, K, channels, gains=None, delays=None,
                          frames_per_block=4096):
    """V[P][len(channels)] for selected channels only, streaming over frames.

    Same definition as ``visibilities(spectra(...))`` restricted to a few
    channels, so long integrations can be checked at a sampled set of
    outputs without holding every channel's spectra.
    """
    b = np.asarray(packed, dtype=np.uint8).reshape(-1)
    rec = N * (K // 2)
    F = b.size // rec
    ch = np.asarray(channels, dtype=np.int64)
    W = dft_matrix(K, channels=ch)
    a = correction_factors(K, gains, delays, N=N, channels=ch)
    G = np.zeros((len(ch), N, N), np.complex128)
    for f0 in range(0, F, frames_per_block):
        f1 = min(F, f0 + frames_per_block)
        x = unpack(b[f0 * rec:f1 * rec], N, K)
        S = f1 - f0
        X = (x.reshape(N * S, K).astype(np.float64) @ W).reshape(N, S, len(ch))
        Y = X * a[:, None, :]
        Yk = np.ascontiguousarray(Y.transpose(2, 0, 1))
        G += Yk @ Yk.conj().transpose(0, 2, 1)
    iu, ju = np.triu_indices(N)
    return np.ascontiguousarray(G[:, iu, ju].T), F


# ---------------------------------------------------------------------------
# Streaming form: coarse integer delays on the sample stream
# ---------------------------------------------------------------------------

def delay_samples(x, sample_delays):
    """y_i[t] = x_i[t - D_i] for t >= D_i, 0 before (the stream starts at t = 0).

    Reading (the paper mentions only a phase applied before accumulation,
    Sec. 2.1; the integer shift is the coarse delay tracking of an FX
    correlator's streaming input): antenna i's samples are delayed by D_i
    whole samples, so a common signal that reaches antenna i d_i samples late
    lines up on every antenna when D_i = max(d) - d_i.
    """
    x = np.asarray(x)
    N, T = x.shape
    y = np.zeros_like(x)
    for i in range(N):
        D = int(sample_delays[i])
        if D < T:
            y[i, D:] = x[i, :T - D]          # y[i, t] = x[i, t - D] for t >= D
    return y


def correlate(packed, N, K, gains=None, delays=None, sample_delays=None):
    """End to end: bytes -> V[P][K/2] and the number of spectra accumulated
    (with optional integer sample delays on the stream, then the DFT, then the
    optional gain/phase correction)."""
    x = unpack(packed, N, K)
    if sample_delays is not None:
        x = delay_samples(x, sample_delays)
    X = spectra(x, K)
    if gains is not None or delays is not None:
        X = X * correction_factors(K, gains, delays, N=N)[:, None, :]
    return visibilities(X), X.shape[1]
