"""Plan-time specialization (cwt_options.specialize): a smooth length with no
fixed-length kernel compiled in gets one compiled at plan creation (NVRTC) for
its scheduler schedule.  Same schedule, same arithmetic: the outputs must be
bitwise those of the runtime-schedule kernels, and within the FP32 bar of the
FP64 oracle (Section "Fast Fourier transform" for the padding)."""
import numpy as np
import pytest

import oracle
from eeg_synth import eeg
from tests.metrics import FP32_TOL, complex_err, power_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_07793_gb300 as p
    return p

# (n = N, C, fs, freqs, cycles, dtype, decimation): runtime-schedule lengths of
# several shapes -- many rows per CTA (42, 105), a generic and a pair schedule,
# four passes, one row per CTA up to 512 threads.
CASES = [
    (42, 5, 100.0, [8.0, 30.0], [3.0, 5.0], "f32", 1),
    (105, 4, 100.0, [6.0, 35.0], [4.0, 7.0], "f32", 1),
    (250, 3, 500.0, [5.0, 60.0, 200.0], [5.0, 7.0, 9.0], "f32", 2),
    (1323, 3, 500.0, [3.0, 40.0, 220.0], [5.0, 7.0, 10.0], "f64", 1),
    (6300, 2, 1000.0, [1.0, 30.0, 400.0], [3.0, 7.0, 12.0], "f32", 1),
    (11025, 2, 1000.0, [0.8, 50.0, 450.0], [4.0, 7.0, 11.0], "f32", 3),
]


def _run(lib, x, n, fs, freqs, cycles, dtype, d, specialize):
    import torch
    t = lib.CWT(x.shape[0], n, fs, freqs, cycles, outputs=("complex", "power", "phase"), dtype=dtype,
                decimation=d, pad="smooth", specialize=specialize)
    info = t.info
    out = t(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    t.close()
    return res, info


@pytest.mark.parametrize("case", range(len(CASES)))
def test_specialized_kernels_match_runtime_schedule_and_oracle(lib, case):
    n, C, fs, freqs, cycles, dtype, d = CASES[case]
    x = eeg(1500 + case, C, n, fs, np.float64 if dtype == "f64" else np.float32)
    plain, info0 = _run(lib, x, n, fs, freqs, cycles, dtype, d, False)
    spec, info1 = _run(lib, x, n, fs, freqs, cycles, dtype, d, True)
    assert info0.fft_length == info1.fft_length == n
    assert info0.specialized == 0 and info0.fixed_kernel == 0
    assert info1.specialized == 1 and info1.fixed_kernel == 1
    for k in plain:
        assert np.array_equal(plain[k], spec[k]), k
    ref = oracle.cwt(x.astype(np.float64), n, fs, freqs, cycles, decimation=d)
    assert complex_err(spec["complex"], ref).max() <= FP32_TOL
    assert power_err(spec["power"], ref).max() <= FP32_TOL


# cluster rows whose local length has no kernel compiled in, split the same
# way with and without specialization: (n = N, C, fs, freqs, cycles,
# decimation, CL)
CLUSTER_CASES = [
    (19683, 1, 2000.0, [1.5, 100.0, 800.0], [20.0, 7.0, 4.0], 4, 3),
    (14175, 2, 1000.0, [2.0, 40.0, 300.0], [5.0, 7.0, 10.0], 1, 3),
]


@pytest.mark.parametrize("case", range(len(CLUSTER_CASES)))
def test_specialized_cluster_kernels_match_runtime_schedule_and_oracle(lib, case):
    """The cluster kernels compiled for the local length of the split: bitwise
    the runtime-schedule cluster kernels, and within the bar of the oracle."""
    n, C, fs, freqs, cycles, d, CL = CLUSTER_CASES[case]
    x = eeg(1600 + case, C, n, fs, np.float32)
    plain, info0 = _run(lib, x, n, fs, freqs, cycles, "f32", d, False)
    spec, info1 = _run(lib, x, n, fs, freqs, cycles, "f32", d, True)
    assert info0.cluster == info1.cluster == CL
    assert info0.specialized == 0 and info1.specialized == 1 and info1.fixed_kernel == 1
    for k in plain:
        assert np.array_equal(plain[k], spec[k]), k
    ref = oracle.cwt(x.astype(np.float64), n, fs, freqs, cycles, decimation=d)
    assert power_err(spec["power"], ref).max() <= FP32_TOL


# splits that only plan-time compilation opens (local rows two CTAs per SM
# hold, clusters above 8 CTAs): (n = N, fs, freqs, cycles, decimation, CL
# with specialize, CL without)
WIDE_CASES = [
    (105000, 1000.0, [0.8, 60.0, 450.0], [7.0, 7.0, 12.0], 8, 10, 7),
    (115200, 1920.0, [0.5, 40.0, 900.0], [7.0, 7.0, 10.0], 8, 9, 8),
    (14406, 500.0, [1.0, 30.0, 200.0], [3.0, 7.0, 12.0], 1, 7, 2),
]


@pytest.mark.parametrize("case", range(len(WIDE_CASES)))
def test_specialized_wide_splits_match_oracle(lib, case):
    """With specialize the cluster split may take local rows that only a
    kernel compiled at plan creation runs two CTAs per SM, on up to 16 CTAs
    (non-portable cluster sizes): parity with the oracle, and with the
    portable split of the same length."""
    n, fs, freqs, cycles, d, CL1, CL0 = WIDE_CASES[case]
    x = eeg(1650 + case, 1, n, fs, np.float32)
    plain, info0 = _run(lib, x, n, fs, freqs, cycles, "f32", d, False)
    spec, info1 = _run(lib, x, n, fs, freqs, cycles, "f32", d, True)
    assert info0.cluster == CL0 and info1.cluster == CL1
    assert info1.specialized == 1 and info1.fixed_kernel == 1
    assert int(np.prod([r for r in info1.radices if r])) == n // CL1
    ref = oracle.cwt(x.astype(np.float64), n, fs, freqs, cycles, decimation=d)
    assert complex_err(spec["complex"], ref).max() <= FP32_TOL
    assert power_err(spec["power"], ref).max() <= FP32_TOL
    peak = plain["power"].max(axis=-1, keepdims=True)
    assert (np.abs(spec["power"] - plain["power"]) / peak).max() <= 2 * FP32_TOL


@pytest.mark.parametrize("n,pad", [(10000, "smooth"), (1000, "pow2"), (20000, "smooth")])
def test_specialize_leaves_compiled_in_paths(lib, n, pad):
    """A length with a kernel compiled in (10000), a power of two and a cluster
    row on a compiled-in local length (20000 = 2 x 10000) run their usual
    kernels: nothing is compiled at plan creation."""
    t = lib.CWT(1, n, 1000.0, [10.0, 50.0], [7.0, 7.0], outputs=("power",), pad=pad, specialize=True)
    assert t.info.specialized == 0
    t.close()


@pytest.mark.parametrize("case", [1, 3, 4])
def test_tuned_specialization_parity(lib, case):
    """specialize = 2: candidate schedules compiled and timed at plan creation,
    the fastest kept (its radices reported); parity with the oracle."""
    n, C, fs, freqs, cycles, dtype, d = CASES[case]
    x = eeg(1700 + case, C, n, fs, np.float64 if dtype == "f64" else np.float32)
    res, info = _run(lib, x, n, fs, freqs, cycles, dtype, d, 2)
    assert info.specialized == 2 and info.fixed_kernel == 1
    assert int(np.prod([r for r in info.radices if r])) == n
    ref = oracle.cwt(x.astype(np.float64), n, fs, freqs, cycles, decimation=d)
    assert complex_err(res["complex"], ref).max() <= FP32_TOL
    assert power_err(res["power"], ref).max() <= FP32_TOL


@pytest.mark.parametrize("n", [1000, 10000])
def test_tuning_competes_with_compiled_in_kernels(lib, n):
    """specialize = 2 on a length with a compiled-in kernel: the compiled-in
    kernel competes with the candidates; whichever runs, parity holds."""
    fs, freqs, cycles = 1000.0, [3.0, 40.0, 300.0], [5.0, 7.0, 10.0]
    x = eeg(1800 + n, 2, n, fs, np.float32)
    res, info = _run(lib, x, n, fs, freqs, cycles, "f32", 1, 2)
    assert info.specialized in (0, 2) and info.fixed_kernel == 1
    ref = oracle.cwt(x.astype(np.float64), n, fs, freqs, cycles)
    assert power_err(res["power"], ref).max() <= FP32_TOL


@pytest.mark.parametrize("case,n", [(0, None), (1, None), (1, 30720), (1, 60000)])
def test_tuned_cluster_rows_parity(lib, case, n):
    """specialize = 2 on cluster rows: the candidates are schedules of the local
    length NL = N / CL (30720 = 3 x 10240; the compiled-in cluster kernel of NL
    competing where there is one, 60000 = 5 x 12000); parity holds."""
    n0, C, fs, freqs, cycles, d, CL = CLUSTER_CASES[case]
    if n is not None:
        n0, CL = n, {30720: 3, 60000: 5}[n]
    x = eeg(1900 + case, C, n0, fs, np.float32)
    res, info = _run(lib, x, n0, fs, freqs, cycles, "f32", d, 2)
    assert info.cluster == CL and info.fixed_kernel == 1
    assert info.specialized in ((0, 2) if n == 60000 else (2,))
    assert int(np.prod([r for r in info.radices if r])) == n0 // CL
    ref = oracle.cwt(x.astype(np.float64), n0, fs, freqs, cycles, decimation=d)
    assert complex_err(res["complex"], ref).max() <= FP32_TOL
    assert power_err(res["power"], ref).max() <= FP32_TOL
