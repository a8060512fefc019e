"""Coarse integer delays on the pushed stream (GPU), against the oracle.

The oracle delays the whole stream from t = 0 and correlates it; the GPU
delays each pushed chunk on the device, taking the samples before it from
the end of the previous chunk.  Delays cover 0, odd, even and a whole frame,
chunks are ragged and cross several workspace passes, inputs come from
device and host memory.
"""

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
SEED = 61


def vis_error(V, R, N):
    autos = np.array([oracle.baseline_index(i, i, N) for i in range(N)])
    A = np.abs(R[autos])
    pairs = oracle.baseline_pairs(N)
    nrm = np.sqrt(A[[p[0] for p in pairs]] * A[[p[1] for p in pairs]])
    return float(np.max(np.abs(np.asarray(V, np.complex128) - R) / nrm))


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.mark.parametrize("dtype", ["fp32", "fp32_simt", "fp16"])
@pytest.mark.parametrize("K,host", [(512, False), (64, True), (2048, False)])
def test_delayed_stream_matches_oracle(lib, torch, dtype, K, host):
    N = 5
    D = np.array([0, 1, 6, K - 3, K], np.int32)
    pushes = [70, 1, 200, 33, 129]
    F = sum(pushes)
    packed, _ = synth.make_samples(N, F * K, K, seed=SEED + K)
    R, _ = oracle.correlate(packed, N, K, sample_delays=D)
    buf = torch.from_numpy(packed.reshape(-1))
    buf = buf.pin_memory() if host else buf.cuda()
    rec = N * K // 2
    with lib.Correlator(N, K, dtype, chunk=256) as c:
        lib.corr_set_sample_delays(c.h, D)
        f0 = 0
        for nf in pushes:
            c.push(buf[f0 * rec:(f0 + nf) * rec], nf * K)
            f0 += nf
        V, n = c.dump(fp64=True)
    assert n == F
    from conftest import report_err
    e = report_err(f"sdelay-{dtype}-K{K}-host{int(host)}", vis_error(V, R, N))
    assert e <= (TOL if dtype != "fp16" else 2e-4)      # FP16: 0.8e-4 .. 0.9e-4 measured


def test_delays_change_mid_stream_and_persist_across_dumps(lib, torch):
    N, K = 4, 128
    A, B = 150, 170
    packed, _ = synth.make_samples(N, (A + B) * K, K, seed=SEED + 1)
    x = oracle.unpack(packed, N, K)
    D1 = np.array([3, 0, 128, 77], np.int32)
    D2 = np.array([0, 5, 1, 64], np.int32)
    y1 = oracle.delay_samples(x, D1)[:, :A * K]
    y2 = oracle.delay_samples(x, D2)[:, A * K:]
    R1 = oracle.visibilities(oracle.spectra(y1, K))
    R2 = oracle.visibilities(oracle.spectra(y2, K))
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    rec = N * K // 2
    with lib.Correlator(N, K, "fp32") as c:
        lib.corr_set_sample_delays(c.h, D1)
        c.push(dev[:A * rec], A * K)
        V1, n1 = c.dump(fp64=True)             # the stream goes on across the dump
        lib.corr_set_sample_delays(c.h, D2)
        c.push(dev[A * rec:], B * K)
        V2, n2 = c.dump(fp64=True)
    assert (n1, n2) == (A, B)
    assert vis_error(V1, R1, N) <= TOL and vis_error(V2, R2, N) <= TOL


def test_checkpoint_carries_the_stream_history(lib, torch):
    N, K = 6, 512
    packed, _ = synth.make_samples(N, 400 * K, K, seed=SEED + 2)
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    rec = N * K // 2
    D = np.array([9, 0, 511, 2, 300, 512], np.int32)
    with lib.Correlator(N, K, "fp32") as c:
        lib.corr_set_sample_delays(c.h, D)
        c.push(dev[: 250 * rec], 250 * K)
        c.push(dev[250 * rec:], 150 * K)
        V_one, _ = c.dump(fp64=True)
    with lib.Correlator(N, K, "fp32") as c:
        lib.corr_set_sample_delays(c.h, D)
        c.push(dev[: 250 * rec], 250 * K)
        state = lib.corr_save_state(c.h)
    with lib.Correlator(N, K, "fp32") as c2:
        lib.corr_load_state(c2.h, state)
        c2.push(dev[250 * rec:], 150 * K)
        V_two, _ = c2.dump(fp64=True)
    assert np.array_equal(V_one, V_two)


def test_delay_arguments_are_checked(lib, torch):
    N, K = 3, 64
    with lib.Correlator(N, K, "fp32") as c:
        for bad in ([0, -1, 0], [0, K + 1, 0]):
            with pytest.raises(lib.CorrError) as ei:
                lib.corr_set_sample_delays(c.h, bad)
            assert ei.value.code == lib.CORR_EINVAL
        lib.corr_set_sample_delays(c.h, [1, 2, 3])
        lib.corr_set_sample_delays(c.h, None)        # off again
    modes = [(8, 512), (4, 1024)]
    with lib.CorrelatorBatch(modes, "fp16") as b:
        lib.corr_set_sample_delays(b.handles[0], [1] * 8)
        data = [torch.zeros(N_ * 256 * K_ // 2, dtype=torch.uint8, device="cuda") for N_, K_ in modes]
        with pytest.raises(lib.CorrError) as ei:
            b.push(data)
        assert ei.value.code == lib.CORR_EINVAL
