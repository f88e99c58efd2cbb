"""The allocation-free entry point, cwt_execute_noalloc.

It exists for callers that must not allocate GPU memory once running (a
real-time EEG / BCI loop whose deadline a blocking cudaMalloc could break, or a
plug-in whose host owns the GPU memory).  This file checks, through the C ABI,
that two calls in a row (different sizes, so the second reuses scratch the
first one filled) give the plan path's results (cwt_plan_create +
cwt_execute) within the FP32 tolerance, and the FP64 oracle's on sampled rows,
and that oversized requests are refused.
It is named to be collected last; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
from eeg_synth import eeg
from tests.metrics import FP32_TOL, complex_err, phase_err, power_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_07793_gb300 as p
    return p


def plan_path(lib, x, fs, freqs, cycles):
    t = lib.CWT(x.shape[0], x.shape[1], fs, freqs, cycles, outputs=("complex", "power", "phase"))
    out = t(x)
    import torch
    torch.cuda.synchronize()
    t.close()
    return {k: v.cpu().numpy() for k, v in out.items()}


CASES = [
    (64, 10000, 1000.0, np.geomspace(1, 100, 100), np.linspace(3, 10, 100)),
    (5, 777, 250.0, [2.0, 9.0, 31.0, 120.0], [3.0, 7.0, 7.0, 10.0]),
]


def test_two_calls_in_a_row_match_plan_path(lib):
    import torch
    for i, (C, n, fs, freqs, cycles) in enumerate(CASES):
        x = torch.from_numpy(eeg(900 + i, C, n, fs, np.float32)).cuda()
        S = len(freqs)
        c = torch.empty((C, S, n), dtype=torch.complex64, device="cuda")
        p = torch.empty((C, S, n), dtype=torch.float32, device="cuda")
        ph = torch.empty((C, S, n), dtype=torch.float32, device="cuda")
        lib.cwt_execute_noalloc(x, C, n, fs, freqs, cycles, c, p, ph)
        torch.cuda.synchronize()
        ref = plan_path(lib, x, fs, freqs, cycles)
        rc = ref["complex"].astype(np.complex128)
        assert complex_err(c.cpu().numpy(), rc).max() <= FP32_TOL
        assert power_err(p.cpu().numpy(), rc).max() <= FP32_TOL
        assert phase_err(ph.cpu().numpy(), rc).max() <= FP32_TOL
        assert np.abs(p.cpu().numpy() - ref["power"]).max() <= FP32_TOL * ref["power"].max()
        # and directly against the FP64 oracle on a few rows (every row of the small case)
        rows = [(0, 0), (C - 1, S - 1), (C // 2, S // 2)] if C > 8 else [(a, b) for a in range(C) for b in range(S)]
        xo = x.cpu().numpy().astype(np.float64)
        orc = oracle.cwt_rows(xo, lib.cwt_fft_length(n), fs, freqs, cycles, rows)
        got = c.cpu().numpy()
        assert complex_err(np.stack([got[a, b] for a, b in rows]), orc).max() <= FP32_TOL


def test_oversized_request_is_refused(lib):
    import torch
    x = torch.zeros((512, 16384), device="cuda")
    out = torch.zeros(16, device="cuda")
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_execute_noalloc(x, 512, 16384, 1000.0, [10.0] * 100, [7.0] * 100, None, out, None)
    assert e.value.status == lib.CWT_EINVAL
