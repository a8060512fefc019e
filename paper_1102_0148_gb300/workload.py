"""Work and traffic accounting for the FX correlator (no device code).

Two flop counts are kept apart:

* the paper's load model (Sec. 1): an FFT costs 2.5 log2(K) real flops per
  input sample (K log2 K complex operations per 2K-point transform), and the
  cross multiply-accumulate costs N^2 flops per sample-time (about N^2/2
  complex MACs per channel sample, one op per multiply-add);
* the algorithmic count used for rooflines: 8 real flops per complex
  multiply-accumulate, N(N+1)/2 pairs (autos included) per channel per
  spectrum, K/2 channels.
"""

import math


def n_pairs(N):
    return N * (N + 1) // 2


def paper_fft_gflops_per_msps(N, K):
    """FFT load per MS/s of sampling rate, in Gflops (Sec. 1)."""
    return 2.5 * math.log2(K) * N * 1e6 / 1e9


def paper_xmac_gflops_per_msps(N):
    """Cross multiply-accumulate load per MS/s, in Gflops (Sec. 1)."""
    return N * N * 1e6 / 1e9


def input_bytes_per_second(N, R_sps, bits=4):
    return N * R_sps * bits / 8.0


def xengine_flops(N, K, n_spec):
    """Useful X-engine flops: 8 per complex MAC, every pair incl. autos."""
    return 8.0 * n_pairs(N) * (K // 2) * n_spec


def fengine_flops(N, K, n_spec):
    """Algorithmic F-engine flops, the paper's 2.5 log2(K) per sample."""
    return 2.5 * math.log2(K) * N * K * n_spec


def fengine_bytes(N, K, n_spec, out_bytes_per_real):
    """Algorithmic HBM bytes of the F-engine: 0.5 B/sample in, and the
    corner-turned spectra out (2 reals per channel, K/2 channels)."""
    return N * n_spec * (K / 2.0 + K * out_bytes_per_real)


def xengine_issued_flops(N, K, s_pad, dtype):
    """Flops the tensor-core X-engine issues for one pass of ``s_pad`` padded
    spectra: 2 M N K per tcgen05.mma, with the tile shapes the kernel uses.

    Antennas come in blocks of 64 (rows [Re; Im], 2 nb of them), M = 128
    rows.  Per spectrum and channel:
    * one block (N <= 64): FP32 mode (two FP16 planes) one MMA whose B is
      [hi; lo], N = 2 r (r = 2N rounded up to 8); FP16 / FP8 one MMA with
      N = 2N rounded up to 16;
    * several blocks: work groups of block b1 against blocks b2 .. b2 +
      nbB - 1 (b2 = b1, b1 + 2, ...; nbB = 2, or 1 for a row's last), one
      MMA with N = 128 nbB (three in FP32 mode: hi hi, hi lo, lo hi).
    """
    nblk = (N + 63) // 64
    if nblk == 1:
        if dtype == "fp32":
            per = 2 * 128 * (2 * ((2 * N + 7) // 8 * 8))
        else:
            per = 2 * 128 * ((2 * N + 15) // 16 * 16)
    else:
        per = 0
        for b1 in range(nblk):
            for b2 in range(b1, nblk, 2):
                nn = 128 * min(2, nblk - b2)
                per += (3 if dtype == "fp32" else 1) * 2 * 128 * nn
    return float(per) * (K // 2) * s_pad
