"""Allocation failures on the host side (GPU; no device fault involved).

The library routes every device allocation of a handle through one helper
with a test hook: while CORR_TEST_FAIL_ALLOC holds a positive integer k, the
k-th allocation counted since the variable last changed value fails as if
cudaMalloc had run out of memory.  Each failing call must return
CORR_ENOMEM, leave nothing half-made behind, and leave the handle usable:
the same work then succeeds and matches the FP64 oracle.
"""

import os

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth
from test_gpu_parity import TOL, vis_error

pytestmark = pytest.mark.gpu

VAR = "CORR_TEST_FAIL_ALLOC"


@pytest.fixture()
def fail_alloc():
    def arm(k):
        os.environ[VAR] = str(k)

    yield arm
    os.environ.pop(VAR, None)


def _input(N, K, S, seed):
    packed, _ = synth.make_samples(N, S * K, K, seed=seed)
    R, _ = oracle.correlate(packed, N, K)
    return packed, R


@pytest.mark.parametrize("k", [1, 2, 5])
def test_create_fails_cleanly(lib, fail_alloc, k):
    fail_alloc(k)
    with pytest.raises(lib.CorrError) as ei:
        lib.corr_create(8, 256, lib.CORR_FP32)
    assert ei.value.code == lib.CORR_ENOMEM
    os.environ.pop(VAR)
    h = lib.corr_create(8, 256, lib.CORR_FP32)
    lib.corr_destroy(h)


@pytest.mark.parametrize("k", [1, 7, 16])
def test_host_staging_ring_all_or_nothing(lib, fail_alloc, k):
    """The first push from host memory makes 16 staging buffers; failing the
    k-th must release the others, and the next push makes all 16 again."""
    import torch
    N, K, S = 6, 256, 300
    packed, R = _input(N, K, S, seed=11020148 + 70 + k)
    host = torch.from_numpy(packed.reshape(-1)).pin_memory()
    with lib.Correlator(N, K, "fp32") as c:
        fail_alloc(k)
        with pytest.raises(lib.CorrError) as ei:
            c.push(host, S * K)
        assert ei.value.code == lib.CORR_ENOMEM
        os.environ.pop(VAR)
        c.push(host, S * K)
        V, n = c.dump(fp64=True)
    assert n == S                      # the failed push added nothing
    assert vis_error(V, R, N) <= TOL


def test_workspace_resize_failure_keeps_the_old_one(lib, fail_alloc):
    import torch
    N, K, S = 5, 128, 400
    packed, R = _input(N, K, S, seed=11020148 + 80)
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    with lib.Correlator(N, K, "fp32", chunk=256) as c:
        fail_alloc(1)
        with pytest.raises(lib.CorrError) as ei:
            lib.corr_set_chunk(c.h, 1024)
        assert ei.value.code == lib.CORR_ENOMEM
        os.environ.pop(VAR)
        c.push(dev, S * K)
        V, n = c.dump(fp64=True)
    assert n == S and vis_error(V, R, N) <= TOL


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sample_delay_buffers_all_or_nothing(lib, fail_alloc, k):
    import torch
    N, K, S = 4, 128, 200
    packed, _ = synth.make_samples(N, S * K, K, seed=11020148 + 90)
    D = np.array([0, 3, 17, 128], np.int32)
    R, _ = oracle.correlate(packed, N, K, sample_delays=D)
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    with lib.Correlator(N, K, "fp32") as c:
        fail_alloc(k)
        with pytest.raises(lib.CorrError) as ei:
            lib.corr_set_sample_delays(c.h, D)
        assert ei.value.code == lib.CORR_ENOMEM
        os.environ.pop(VAR)
        lib.corr_set_sample_delays(c.h, D)
        c.push(dev, S * K)
        V, n = c.dump(fp64=True)
    assert n == S and vis_error(V, R, N) <= TOL


def test_gradient_buffers_fail_then_work(lib, fail_alloc):
    import torch
    N, K, S = 4, 64, 64
    packed, R = _input(N, K, S, seed=11020148 + 95)
    dev = torch.from_numpy(packed.reshape(-1)).cuda()
    G = np.ones((N * (N + 1) // 2, K // 2), np.complex64)
    gg = np.zeros(N, np.complex64)
    gt = np.zeros(N, np.float32)
    with lib.Correlator(N, K, "fp32") as c:
        fail_alloc(1)
        with pytest.raises(lib.CorrError) as ei:
            lib.corr_grad(c.h, dev, S * K, None, None, G, False, gg, gt)
        assert ei.value.code == lib.CORR_ENOMEM
        os.environ.pop(VAR)
        lib.corr_grad(c.h, dev, S * K, None, None, G, False, gg, gt)
        c.push(dev, S * K)
        V, n = c.dump(fp64=True)
    assert np.all(np.isfinite(gg)) and np.all(np.isfinite(gt))
    assert n == S and vis_error(V, R, N) <= TOL
