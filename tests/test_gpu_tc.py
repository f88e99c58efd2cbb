"""GPU parity of the tensor-core inverse FFTs (CWT_PREC_TC_FP16 / _BF16).

The radix-16 stages of every inverse FFT run as DFT matrix products on the
tensor cores (mma.sync.m16n8k16) with hi/lo split FP16 or BF16 operands and
FP32 accumulation; pass 0, the twiddles, the cross-CTA stage and the epilogue
stay FP32.  Each case compares the library, through the C ABI, with the FP64
oracle on the same seeded inputs, row by row, at the reduced-precision bar
(2e-3 of the row's peak power; tests/metrics.py), and reports the error per
frequency (the precision workload's metric):
  * every row at N = 16384 (single CTAs), 32768 and 65536 (clusters of 2 and
    4 CTAs), narrow bands (sparse pass 0) and wide bands (dense pass 0),
    complex, power and phase, decimation, f64 I/O;
  * the precision workload at full size (256 ch x 122880 @2048 Hz, N =
    131072 on clusters of 8 CTAs, 128 scales, power + phase) on sampled rows,
    in the launch configuration the benchmark times, for FP16 and BF16.
"""
import os

import numpy as np
import pytest

import oracle
from eeg_synth import eeg, workload
from tests.metrics import TC_TOL, complex_err, phase_err, power_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_07793_gb300 as p
    return p


def run_tc(lib, x, fs, freqs, cycles, outputs, precision, **kw):
    import torch
    C, n = x.shape
    t = lib.CWT(C, n, fs, freqs, cycles, outputs=outputs, precision=precision, **kw)
    try:
        assert t.info.precision == {"tc_fp16": 1, "tc_bf16": 2}[precision]
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        out = t(xt)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}, t.info.fft_length
    finally:
        t.close()


def errors(res, ref):
    e = {}
    if "complex" in res:
        e["complex"] = complex_err(res["complex"], ref)
    if "power" in res:
        e["power"] = power_err(res["power"], ref)
    if "phase" in res:
        e["phase"] = phase_err(res["phase"], ref)
    return e


CASES = [
    # (C, n, fs, freqs, n_cycles): N = 16384 / 32768 / 65536
    (3, 12000, 1000.0, [0.7, 4.0, 13.0, 60.0, 240.0, 480.0], [3.0, 7.0, 7.0, 5.0, 12.0, 3.0]),
    (2, 20000, 1000.0, [0.8, 13.0, 240.0], [3.0, 7.0, 12.0]),
    (1, 40000, 2000.0, [3.0, 600.0, 950.0], [7.0, 5.0, 3.0]),
]


@pytest.mark.parametrize("precision", ["tc_fp16", "tc_bf16"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_tc_every_row(lib, case, precision):
    """Every row against the oracle; 480 and 950 Hz with 3 cycles have bands
    wider than 4096 bins per residue class (the dense pass 0)."""
    C, n, fs, freqs, cycles = CASES[case]
    x = eeg(900 + case, C, n, fs, np.float32)
    res, N = run_tc(lib, x, fs, freqs, cycles, ("complex", "power", "phase"), precision)
    assert N >= 16384
    ref = oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles)
    e = errors(res, ref)
    worst = {k: float(v.max()) for k, v in e.items()}
    print(precision, N, worst)
    for k, v in worst.items():
        assert v <= TC_TOL, (k, v)
    # the compensated products keep far more than the bar (FP16 hi/lo ~2^-22,
    # BF16 hi/lo ~2^-16 per product; measured 3e-6 .. 1.4e-5 on these rows)
    assert worst["power"] <= (5e-5 if precision == "tc_fp16" else 2e-4), worst


@pytest.mark.parametrize("precision", ["tc_fp16", "tc_bf16"])
def test_tc_decimation_and_f64_io(lib, precision):
    C, n, fs = 2, 16384, 1000.0
    freqs, cycles = [2.0, 30.0, 200.0], [7.0, 7.0, 9.0]
    x = eeg(950, C, n, fs, np.float64)
    res, N = run_tc(lib, x, fs, freqs, cycles, ("complex", "power"), precision, decimation=3,
                    dtype="f64")
    assert res["power"].dtype == np.float64 and res["power"].shape == (C, 3, -(-n // 3))
    ref = oracle.cwt(x, N, fs, freqs, cycles, decimation=3)
    for k, v in errors(res, ref).items():
        assert v.max() <= TC_TOL, (k, v.max())


def test_tc_unsupported_lengths(lib):
    """The tensor-core path covers power-of-two N of 16384 .. 131072."""
    o = lib.cwt_options_init()
    o.precision = lib.CWT_PREC_TC_FP16
    for n, pad in ((8000, lib.CWT_PAD_POW2), (12000, lib.CWT_PAD_SMOOTH)):  # N = 8192, 12000
        o.pad_policy = pad
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_plan_create(1, n, 1000.0, [10.0], [7.0], 0, lib.CWT_OUT_POWER, o)
        assert e.value.status == lib.CWT_EUNSUPPORTED


@pytest.mark.parametrize("precision", ["tc_fp16", "tc_bf16"])
def test_tc_precision_workload_full_size_sampled_rows(lib, precision):
    """256 ch x 122880 @2048 Hz (N = 131072, clusters of 8 CTAs), 128 log
    freqs 0.5-200 Hz, power + phase: error against the oracle per frequency
    on sampled rows, at the 2e-3 bar."""
    import torch
    w = workload("precision")
    t = lib.CWT(w.channels, w.samples, w.fs, w.freqs, w.n_cycles, outputs=("power", "phase"),
                precision=precision)
    try:
        assert t.info.fft_length == 131072
        x = w.signal()
        out = t(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        rows = [(0, 0), (255, 127), (17, 64), (200, 100), (99, 115), (3, 33), (128, 120), (64, 8)]
        ref = oracle.cwt_rows(x.astype(np.float64), 131072, w.fs, w.freqs, w.n_cycles, rows,
                              threads=os.cpu_count())
        pw = np.stack([out["power"][c, s].cpu().numpy() for c, s in rows])
        ph = np.stack([out["phase"][c, s].cpu().numpy() for c, s in rows])
        e_p, e_ph = power_err(pw, ref), phase_err(ph, ref)
        for (c, s), a, b in zip(rows, e_p, e_ph):
            print(f"{precision} F={w.freqs[s]:8.3f} Hz  power err {a:.2e}  phase err {b:.2e}")
        assert e_p.max() <= TC_TOL and e_ph.max() <= TC_TOL
        assert bool(torch.isfinite(out["power"]).all()) and bool(torch.isfinite(out["phase"]).all())
    finally:
        t.close()
