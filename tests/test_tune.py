"""Autotuner: cache bookkeeping (CPU) and a small sweep whose choice keeps
parity (GPU)."""

import json

import numpy as np
import pytest

import oracle
from paper_1102_0148_gb300 import synth, tune


def test_cache_roundtrip(tmp_path, monkeypatch):
    monkeypatch.setenv("GBCORR_TUNE_CACHE", str(tmp_path / "t.json"))
    monkeypatch.setattr(tune, "_gpu", lambda: "FakeGPU")
    assert tune.lookup(44, 512, "fp32") is None
    tune._save(tune.key(44, 512, "fp32"), {"chunk": 1024, "window": 64, "stages": 3})
    tune._save(tune.key_batch([(44, 512), (22, 2048)], "fp16"), {"window": 128, "stages": 4})
    assert tune.lookup(44, 512, "fp32")["window"] == 64
    d = json.loads((tmp_path / "t.json").read_text())
    assert "FakeGPU|44x512|fp32" in d and "FakeGPU|batch:44x512,22x2048|fp16" in d
    assert tune.lookup(44, 512, "fp16") is None


def test_window_limits_respect_accuracy():
    # FP32 mode accumulates at most 256 spectra per TMEM window
    assert max(tune.WINDOWS["fp32"]) <= 256
    assert all(w % 128 == 0 for w in tune.WINDOWS["fp8"])


@pytest.mark.gpu
def test_tune_and_apply_keep_parity(lib, tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("GBCORR_TUNE_CACHE", str(tmp_path / "t.json"))
    N, K = 12, 512
    best = tune.tune(N, K, "fp32", frames=512, repeats=1, windows=(64, 128), stages=(2, 4),
                     chunks=(256, 512), splits=(0, 2))
    assert best["candidates"] == 16 and best["ms"] > 0
    S = 300
    packed, _ = synth.make_samples(N, S * K, K, seed=99)
    R, _ = oracle.correlate(packed, N, K)
    with lib.Correlator(N, K, "fp32") as c:
        assert tune.apply(c, N, K, "fp32")
        c.push(torch.from_numpy(packed.reshape(-1)).cuda(), S * K)
        V, n = c.dump(fp64=True)
    autos = [oracle.baseline_index(i, i, N) for i in range(N)]
    A = np.abs(R[autos])
    pairs = oracle.baseline_pairs(N)
    nrm = np.sqrt(A[[p[0] for p in pairs]] * A[[p[1] for p in pairs]])
    assert np.max(np.abs(V - R) / nrm) <= 1e-5


@pytest.mark.gpu
def test_tune_batch(lib, tmp_path, monkeypatch):
    monkeypatch.setenv("GBCORR_TUNE_CACHE", str(tmp_path / "t.json"))
    modes = [(44, 512), (11, 4096)]
    best = tune.tune_batch(modes, "fp16", T=1 << 16, repeats=1, windows=(64, 128), stages=(3,),
                           splits=(1,))
    assert best["candidates"] == 2
    with lib.CorrelatorBatch(modes, "fp16") as b:
        assert tune.apply_batch(b, modes, "fp16")
