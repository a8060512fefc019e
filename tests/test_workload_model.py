"""The load model the benchmark reports against reproduces the paper's printed
numbers (tests/golden/paper_load.txt, Sec. 1 and the abstract)."""

import os

from paper_1102_0148_gb300 import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_load.txt")


def _golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                out[line[0]] = float(line[1])
    return out


def test_paper_load_numbers():
    g = _golden()
    N, K, R = int(g["N"]), int(g["K"]), g["R_msps"]
    fft = workload.paper_fft_gflops_per_msps(N, K)
    xmac = workload.paper_xmac_gflops_per_msps(N)
    assert round(fft, 2) == g["fft_gflops_per_msps"]
    assert round(xmac, 2) == g["xmac_gflops_per_msps"]
    assert (fft + xmac) * R > g["total_gflops_min"]
    bps = workload.input_bytes_per_second(N, R * 1e6)
    assert abs(bps / 1e6 - g["input_MBps"]) < 1e-9
    assert round(bps / 2 ** 20 / 5) * 5 == g["input_MiBps_abstract"]


def test_pair_count():
    assert workload.n_pairs(44) == 990
    # one second at 35 MS/s holds 68359 whole 512-point frames
    assert int(35e6 // 512) == 68359
    assert workload.xengine_flops(44, 512, 68359) == 8 * 990 * 256 * 68359
