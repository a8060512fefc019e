"""corr_correlate_noalloc, the entry point for callers that must not allocate
device memory (a real-time acquisition loop in which cudaMalloc/cudaFree
could stall the device, or a process whose device memory is all owned by
another allocator).

It is checked through the C ABI against the handle path (corr_create ->
corr_push -> corr_dump, FP32 CUDA-core X-engine) and against the FP64
oracle on the same bytes, within the tolerance every parity test uses, on
two calls in a row with different inputs: the second call must not see
anything the first left in the shared scratch array.  Two geometries: the
paper's (N = 44, K = 512, the register-FFT F-engine) and a small one
(N = 5, K = 64, the generic F-engine with the twiddles this entry point
computes itself).  This file is collected last so that a failure here stops a
`-x` run only after every other test has run; it also passes on its own in a
fresh process.
"""

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _norm_err(V, R, N):
    autos = np.array([oracle.baseline_index(i, i, N) for i in range(N)])
    A = np.abs(R[autos]).astype(np.float64)
    pairs = oracle.baseline_pairs(N)
    nrm = np.sqrt(A[[p[0] for p in pairs]] * A[[p[1] for p in pairs]])
    return float(np.max(np.abs(V.astype(np.complex128) - R) / np.maximum(nrm, 1e-300)))


def _handle_path(lib, dev, N, K, S):
    with lib.Correlator(N, K, lib.CORR_FP32_SIMT) as c:
        c.push(dev, S * K)
        V, n = c.dump(fp64=True)
    assert n == S
    return V


@pytest.mark.parametrize("N,K,calls", [
    # 300 frames: more than one internal pass, with a ragged last pass
    (44, 512, [(300, 11020148 + 31), (130, 11020148 + 32)]),
    (5, 64, [(150, 11020148 + 33), (37, 11020148 + 34)]),
])
def test_noalloc_matches_handle_path_twice(lib, N, K, calls):
    import torch
    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream()
    P, C = N * (N + 1) // 2, K // 2
    out = torch.empty((P, C), dtype=torch.complex64, device="cuda")
    for call, (S, seed) in enumerate(calls):
        packed, _ = synth.make_samples(N, S * K, K, seed=seed)
        dev = torch.from_numpy(packed.reshape(-1)).cuda()
        ref = _handle_path(lib, dev, N, K, S)
        R, n_ref = oracle.correlate(packed, N, K)
        assert n_ref == S
        out.fill_(complex(3e30, -3e30))          # stale garbage must be overwritten
        lib.corr_correlate_noalloc(dev, S * K, N, K, out, stream)
        torch.cuda.synchronize()
        V = out.cpu().numpy()
        e = _norm_err(V, ref, N)
        assert e <= TOL, f"call {call}: normalised error {e:.3g} against the handle path"
        e = _norm_err(V, R, N)
        assert e <= TOL, f"call {call}: normalised error {e:.3g} against the oracle"


def test_noalloc_rejects_oversize_and_bad_sizes(lib):
    import torch
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.CorrError) as ei:
        lib.corr_correlate_noalloc(dummy, 0, 512, 4096, out)
    assert ei.value.code == lib.CORR_EINVAL
    assert "bytes of scratch" in str(ei.value)
    with pytest.raises(lib.CorrError) as ei:
        lib.corr_correlate_noalloc(dummy, 7, 4, 16, out)
    assert ei.value.code == lib.CORR_EINVAL
