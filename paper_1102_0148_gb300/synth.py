"""Seeded synthetic antenna data, packed as the correlator's input bytes.

This module only *makes inputs*; it holds none of the correlator's arithmetic
(no transform, no correction, no cross-multiply).  Both the CUDA path's tests
and the CPU oracle consume the bytes it writes, so the bytes are the contract.

Signal model (a synthetic stand-in for the 44 phased-array beams of the paper,
Sec. 1: real samples, Nyquist-sampled, 4-bit quantised):

    x_i[t] = clip(round(n_i[t] + c[t - d_i] + A cos(2 pi f (t - d_i) / K0)), -8, 7)

* n_i ~ N(0, sigma^2) independent per antenna (sigma = 2 LSB by default);
* c   ~ N(0, corr_sigma^2), one common stream; corr_sigma = 0.2 makes the
  correlated component 1% of the noise power;
* d_i integer delays drawn uniformly from [0, max_delay);
* an optional common tone of amplitude A at bin f of a K0-point transform;
* round = half away from zero.

Layout of the result: ``[frame][antenna][K/2]`` bytes, frame = K consecutive
samples of every antenna; within an antenna's K/2 bytes, byte m holds sample
2m in its low nibble and sample 2m+1 in its high nibble, each as a 4-bit
two's-complement code.
"""

import numpy as np

# Fixed block length of the numpy generator, so the bytes for a given seed do
# not depend on how long a stream is requested.
_BLOCK = 1 << 16


def _round_half_away(x):
    return np.where(x >= 0, np.floor(x + 0.5), np.ceil(x - 0.5))


def pack_nibbles(q, K):
    """int samples ``q[N][T]`` in [-8, 7] -> bytes ``[T/K][N][K/2]``."""
    q = np.asarray(q)
    N, T = q.shape
    nib = (q.astype(np.int16) & 0x0F).astype(np.uint8)
    pairs = nib[:, 0::2] | (nib[:, 1::2] << 4)            # [N][T/2]
    F = T // K
    return np.ascontiguousarray(pairs.reshape(N, F, K // 2).transpose(1, 0, 2))


def make_samples(N, T, K, seed, sigma=2.0, corr_sigma=0.2, max_delay=16,
                 tone_amp=0.0, tone_bin=97, tone_K=512, noise=True,
                 delays=None):
    """numpy generator (PCG64).  Returns ``(packed uint8 [T/K][N][K/2], info)``.

    ``info`` holds the integer delays d_i and the model parameters.  Suited to
    inputs of up to a few times 2^22 samples per antenna.
    """
    if T % K or K % 2:
        raise ValueError("T must be a multiple of the even frame length K")
    rng = np.random.Generator(np.random.PCG64(seed))
    if delays is None:
        d = rng.integers(0, max_delay, N) if max_delay > 0 else np.zeros(N, np.int64)
    else:
        d = np.asarray(delays, np.int64)
    hist = max(int(max_delay), int(d.max()) + 1 if N else 1)
    out = np.empty((T // K, N, K // 2), np.uint8)
    c_prev = np.zeros(hist)
    blk = max(K, (_BLOCK // K) * K)
    for t0 in range(0, T, blk):
        tb = min(blk, T - t0)
        c_new = rng.normal(0.0, corr_sigma, tb) if corr_sigma > 0 else np.zeros(tb)
        c_ext = np.concatenate([c_prev, c_new])
        x = rng.normal(0.0, sigma, (N, tb)) if noise else np.zeros((N, tb))
        t = np.arange(t0, t0 + tb, dtype=np.float64)
        for i in range(N):
            x[i] += c_ext[hist - d[i]: hist - d[i] + tb]
            if tone_amp:
                x[i] += tone_amp * np.cos(2.0 * np.pi * tone_bin * (t - d[i]) / tone_K)
        q = np.clip(_round_half_away(x), -8, 7).astype(np.int8)
        out[t0 // K:(t0 + tb) // K] = pack_nibbles(q, K)
        c_prev = c_ext[-hist:]
    info = dict(delays=d, sigma=sigma, corr_sigma=corr_sigma, tone_amp=tone_amp,
                tone_bin=tone_bin, tone_K=tone_K, seed=seed)
    return out, info


def make_samples_torch(N, T, K, seed, device, sigma=2.0, corr_sigma=0.2,
                       max_delay=16, tone_amp=0.0, tone_bin=97, tone_K=512,
                       frames_per_block=2048, out=None):
    """Same model drawn with torch's generator on ``device`` (for inputs too
    large to draw on the host quickly).  Returns ``(packed uint8 tensor
    [T/K][N][K/2], info)``.  Its bytes differ from ``make_samples`` for the
    same seed; both are valid draws of the model.
    """
    import torch

    if T % K or K % 2:
        raise ValueError("T must be a multiple of the even frame length K")
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    d = torch.randint(0, max(1, max_delay), (N,), generator=g, device=device)
    if max_delay <= 0:
        d.zero_()
    hist = max(1, int(max_delay))
    F = T // K
    if out is None:
        out = torch.empty((F, N, K // 2), dtype=torch.uint8, device=device)
    c_prev = torch.zeros(hist, dtype=torch.float32, device=device)
    ar = torch.arange(0, 0, device=device)
    for f0 in range(0, F, frames_per_block):
        f1 = min(F, f0 + frames_per_block)
        tb = (f1 - f0) * K
        c_new = torch.randn(tb, generator=g, device=device) * corr_sigma
        c_ext = torch.cat([c_prev, c_new])
        x = torch.randn((N, tb), generator=g, device=device) * sigma
        if ar.numel() != tb:
            ar = torch.arange(tb, device=device)
        idx = (hist - d)[:, None] + ar[None, :]
        x += c_ext[idx]
        if tone_amp:
            t = (ar[None, :] + f0 * K - d[:, None]).double()
            x += (tone_amp * torch.cos(2.0 * np.pi * tone_bin * t / tone_K)).float()
        q = torch.where(x >= 0, torch.floor(x + 0.5), torch.ceil(x - 0.5))
        q = q.clamp_(-8, 7).to(torch.int16)
        nib = (q & 0x0F).to(torch.uint8)
        pairs = nib[:, 0::2] | (nib[:, 1::2] << 4)
        out[f0:f1] = pairs.reshape(N, f1 - f0, K // 2).transpose(0, 1)
        c_prev = c_ext[-hist:]
    info = dict(delays=d.cpu().numpy(), sigma=sigma, corr_sigma=corr_sigma,
                tone_amp=tone_amp, tone_bin=tone_bin, tone_K=tone_K, seed=seed)
    return out, info


def gains_delays(N, seed, gain_sigma=0.1, delay_range=0.5):
    """Per-antenna complex gains g ~ CN(1, gain_sigma^2) and fractional delays
    tau ~ U(-delay_range, delay_range) samples (the gradient workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = 1.0 + (rng.normal(0, gain_sigma / np.sqrt(2), N)
               + 1j * rng.normal(0, gain_sigma / np.sqrt(2), N))
    tau = rng.uniform(-delay_range, delay_range, N)
    return g.astype(np.complex128), tau
