"""Precision form (GPU): FP16 and FP8-E4M3 tensor-core inputs with
per-antenna, per-channel scaling from the autocorrelations, FP32
accumulation (Sec. 4: float output converted to a narrower type with
prescaling before the cross-multiply).

Stated errors, normalised by sqrt(|V_ii V_jj|) against the FP64 oracle on a
2^20-sample prefix (2048 spectra), about twice the error measured on a GB300
for this seeded input:
  FP16 (11 significant bits): <= 1e-4 (4.9e-5 measured);
  FP8-E4M3 (4 significant bits): <= 1.4e-2 (7.0e-3 measured).
A 6 LSB tone with automatic scales: FP8 <= 5e-2 (2.5e-2 measured).
The workload is the full-band one: N = 44, 80 MS/s, K = 512, 4-bit, with the
oracle run on the first 2^20 samples per antenna.
"""

import numpy as np
import pytest

import oracle
from conftest import report_err
from paper_1102_0148_gb300 import synth

pytestmark = pytest.mark.gpu

N, K = 44, 512
BOUND = {"fp16": 1e-4, "fp8": 1.4e-2}
TONE_BOUND_FP8 = 5e-2


def norm_err(V, R, N):
    autos = np.array([oracle.baseline_index(i, i, N) for i in range(N)])
    A = np.abs(R[autos])
    pairs = oracle.baseline_pairs(N)
    nrm = np.sqrt(A[[p[0] for p in pairs]] * A[[p[1] for p in pairs]])
    return float(np.max(np.abs(np.asarray(V, np.complex128) - R) / np.maximum(nrm, 1e-300)))


def correlate(lib, dev, S, dtype, scales=None):
    with lib.Correlator(N, K, dtype) as c:
        if scales is not None:
            lib.corr_set_scales(c.h, scales)
        c.push(dev, S * K)
        V, n = c.dump(fp64=True)
        assert n == S
        return V


@pytest.fixture(scope="module")
def prefix_packed():
    S = (1 << 20) // K
    packed, _ = synth.make_samples(N, S * K, K, seed=11020148 + 3, tone_amp=0.5)
    return packed, S


@pytest.fixture(scope="module")
def prefix(prefix_packed):
    import torch
    packed, S = prefix_packed
    R, _ = oracle.correlate(packed, N, K)
    return torch.from_numpy(packed.reshape(-1)).cuda(), R, S


@pytest.mark.parametrize("dtype", ["fp16", "fp8"])
def test_full_band_prefix_error(lib, prefix, dtype):
    dev, R, S = prefix
    V = correlate(lib, dev, S, dtype)
    e = report_err(f"prefix80-{dtype}", norm_err(V, R, N))
    assert e <= BOUND[dtype]


def test_scaling_prevents_fp8_saturation(lib):
    """A 6 LSB tone puts ~1500 into channel 97, beyond FP8-E4M3's 448: with
    unit scales the tone channel saturates, with scales from the
    autocorrelations it does not."""
    import torch
    S = 256
    packed, _ = synth.make_samples(N, S * K, K, seed=5, tone_amp=6.0)
    R, _ = oracle.correlate(packed, N, K)
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    e_auto = norm_err(correlate(lib, dev, S, "fp8"), R, N)
    ones = np.ones((N, K // 2), np.float32)
    e_unit = norm_err(correlate(lib, dev, S, "fp8", scales=ones), R, N)
    report_err("fp8-tone6-auto", e_auto)
    report_err("fp8-tone6-unit", e_unit)
    assert e_auto <= TONE_BOUND_FP8
    assert e_unit > 10 * e_auto


@pytest.mark.parametrize("dtype,target", [("fp16", 64.0), ("fp8", 16.0)])
def test_scales_follow_autocorrelations(lib, prefix, dtype, target):
    dev, R, S = prefix
    with lib.Correlator(N, K, dtype) as c:
        c.push(dev, S * K)
        first = lib.corr_get_scales(c.h)          # from the estimation pass
        V, n = c.dump(fp64=True)
        after = lib.corr_get_scales(c.h)          # from this integration's autos
    autos = np.array([oracle.baseline_index(i, i, N) for i in range(N)])
    P = V[autos].real / n
    want = target / np.sqrt(P / 2)
    # powers of two, the nearest in log2 to the target scale
    assert np.all(np.exp2(np.round(np.log2(after))) == after)
    assert np.max(np.abs(np.log2(after / want))) <= 0.5 + 1e-9
    # the 256-frame estimate picks the same power of two almost everywhere
    assert np.mean(first == after) > 0.8


def test_user_scales_do_not_bias(lib, prefix):
    dev, R, S = prefix
    rng = np.random.default_rng(0)
    sc = (2.0 ** rng.integers(-3, 4, (N, K // 2))).astype(np.float32) * 16
    V = correlate(lib, dev, S, "fp16", scales=sc)
    assert report_err("prefix80-fp16-user-scales", norm_err(V, R, N)) <= BOUND["fp16"]


def test_scales_rejected_on_fp32_handles(lib):
    with lib.Correlator(N, K, "fp32") as c:
        with pytest.raises(lib.CorrError) as ei:
            lib.corr_get_scales(c.h)
        assert ei.value.code == lib.CORR_EINVAL


def round_to_bits(v, m):
    """v rounded to the nearest value with m fraction bits (ties to even),
    exponent unbounded: FP16 (m = 10) and E4M3 (m = 3) rounding away from
    their subnormal and overflow ranges."""
    f, e = np.frexp(v)
    return np.ldexp(np.round(f * 2.0 ** (m + 1)), e - (m + 1))


# |mean GPU bias - mean model bias| bounds: the model leaves out the tensor
# core's FP32 accumulation (-2.0e-6 measured for FP16 on a GB300) and the few
# roundings that the F-engine's FP32 spectra take the other way (E4M3:
# -7.1095e-4 measured against -7.1024e-4 modelled)
AUTO_BIAS_TOL = {"fp16": 5e-6, "fp8": 5e-6}


@pytest.mark.parametrize("dtype,m", [("fp16", 10), ("fp8", 3)])
def test_quantisation_bias_on_autos(lib, prefix, prefix_packed, dtype, m):
    """Rounding the scaled spectra to the X-engine's input type changes each
    autocorrelation by sum_s |q(Y)|^2 - |Y|^2.  The scales are powers of two,
    so q(s Y) / s = q(Y) and that change follows from the oracle's FP64
    spectra alone; the GPU's mean relative bias on V_ii must match it.  On a
    floating-point grid the bias is negative, not the +Delta^2/12 of a
    uniform grid: the spacing doubles at each power of two, so values just
    above one round down onto it from the wider cell, and for spectra whose
    magnitudes spread over several octaves that outweighs the mean-square
    rounding error (about -7e-4 of V_ii for E4M3, below 1e-6 for FP16).  A
    conversion that truncated instead of rounding would move the E4M3 bias
    to about -8e-2."""
    dev, R, S = prefix
    packed, _ = prefix_packed
    V = correlate(lib, dev, S, dtype)
    autos = np.array([oracle.baseline_index(i, i, N) for i in range(N)])
    Ra = R[autos].real
    Y = oracle.spectra(oracle.unpack(packed, N, K), K)                # [N][S][C]
    Q = round_to_bits(Y.real, m) ** 2 + round_to_bits(Y.imag, m) ** 2
    b_model = float(np.mean(Q.sum(axis=1) / Ra - 1.0))
    b_gpu = float(np.mean(np.asarray(V[autos].real, np.float64) / Ra - 1.0))
    print(f"MEASURED_BIAS autos-{dtype} gpu {b_gpu:.4e} model {b_model:.4e}")
    if dtype == "fp8":
        assert -1.2e-3 < b_model < -3e-4
    assert abs(b_gpu - b_model) <= AUTO_BIAS_TOL[dtype], (b_gpu, b_model)
