"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every case draws seeded synthetic inputs from eeg_synth, runs the library on
cuda:0 and compares element by element with oracle/ on the same inputs:
  * the plain workload (8 ch x 500 @500 Hz, f64 I/O, power): every row;
  * the fused workload at full size (64 ch x 10000 @1000 Hz, complex + power),
    in the launch configuration the benchmark times: a spread of sampled rows;
  * edge cases: n = 1, n at and just past a power of two, the largest
    single-pass length, one channel / one scale, frequencies near Nyquist,
    small and large n_cycles, Gabor, decimation, phase, f64 I/O.
Bar: FP32 paths within 1e-5 per row (tests/metrics.py).
"""
import numpy as np
import pytest

import oracle
from eeg_synth import eeg, workload
from tests.metrics import FP32_TOL, complex_err, paper_style_error, phase_err, power_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_07793_gb300 as p
    return p


def run_gpu(lib, x, fs, freqs, cycles, outputs, dtype="f32", decimation=1, wavelet="morlet",
            fft_length=0, pad="pow2", gmw_gamma=3.0, edge="cyclic", normalization="unit"):
    import torch
    C, n = x.shape
    t = lib.CWT(C, n, fs, freqs, cycles, outputs=outputs, dtype=dtype, decimation=decimation,
                wavelet=wavelet, fft_length=fft_length, pad=pad, gmw_gamma=gmw_gamma, edge=edge,
                normalization=normalization)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = t(xt)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    N = t.info.fft_length
    t.close()
    return res, N


def check(res, ref, tol=FP32_TOL):
    worst = {}
    if "complex" in res:
        worst["complex"] = complex_err(res["complex"], ref).max()
    if "power" in res:
        worst["power"] = power_err(res["power"], ref).max()
    if "phase" in res:
        worst["phase"] = phase_err(res["phase"], ref).max()
    for k, v in worst.items():
        assert v <= tol, f"{k} row error {v:.3e} > {tol:.0e}"
    return worst


def test_fft_matches_library_fft_and_parseval(lib):
    import torch
    rng = np.random.default_rng(1)
    for log2n in range(5, 18):  # 2^15..2^17 run on thread-block clusters
        n = 1 << log2n
        z = (rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))).astype(np.complex64)
        d_in = torch.from_numpy(z).cuda()
        for direction in (-1, 1):
            d_out = torch.empty_like(d_in)
            lib.cwt_fft(d_in, d_out, n, 3, direction)
            torch.cuda.synchronize()
            got = d_out.cpu().numpy().astype(np.complex128)
            zz = z.astype(np.complex128)
            ref = np.fft.fft(zz, axis=1) if direction < 0 else np.fft.ifft(zz, axis=1) * n
            rel = np.abs(got - ref).max() / np.abs(ref).max()
            assert rel < 2e-6 * log2n, (n, direction, rel)
            # Parseval: sum |x|^2 = (1/n) sum |X|^2
            assert np.allclose((np.abs(got) ** 2).sum(1) / n, (np.abs(zz) ** 2).sum(1), rtol=1e-5)
    # in place
    z = (rng.standard_normal((2, 1024)) + 1j * rng.standard_normal((2, 1024))).astype(np.complex64)
    d = torch.from_numpy(z).cuda()
    lib.cwt_fft(d, d, 1024, 2, -1)
    torch.cuda.synchronize()
    assert np.abs(d.cpu().numpy() - np.fft.fft(z.astype(np.complex128), axis=1)).max() < 1e-3


@pytest.mark.parametrize("F,sigma,fs,n", [(10.0, 7.0, 500.0, 500), (1.0, 3.0, 1000.0, 10000),
                                          (240.0, 3.0, 500.0, 300), (40.0, 10.0, 250.0, 2048),
                                          (0.5, 7.0, 2048.0, 4096)])
def test_bank_matches_oracle_wavelet_spectrum(lib, F, sigma, fs, n):
    """The FP64-generated, FP32-stored bank equals the DFT of the oracle's
    unit-energy periodised wavelet (times 1/N), and its band holds every bin
    above 1e-10 of the peak."""
    plan = lib.cwt_plan_create(1, n, fs, [F], [sigma], 0, lib.CWT_OUT_POWER)
    try:
        bank, start, length = lib.cwt_plan_bank(plan)
        N = lib.cwt_plan_info(plan).fft_length
    finally:
        lib.cwt_plan_destroy(plan)
    W = np.fft.fft(oracle.wavelet(F, sigma, fs, N)).real / N
    assert np.abs(bank[0] - W).max() <= 1e-6 * np.abs(W).max()
    k = np.arange(N)
    inside = ((k - start[0]) % N) < length[0]
    assert np.all(np.abs(W[~inside]) <= 2e-10 * np.abs(W).max())


def test_plain_workload_every_row(lib):
    w = workload("plain")
    x = w.signal()
    res, N = run_gpu(lib, x, w.fs, w.freqs, w.n_cycles, w.outputs, dtype=w.dtype)
    assert res["power"].dtype == np.float64 and res["power"].shape == (8, 40, 500)
    ref = oracle.cwt(x, N, w.fs, w.freqs, w.n_cycles)
    check(res, ref)


def test_fused_workload_full_size_sampled_rows(lib):
    """64 x 10000, complex64 + power, exactly as the benchmark launches it;
    the oracle recomputes a spread of rows (lowest/highest scale, smallest and
    largest n_cycles, first/last channel)."""
    w = workload("fused")
    x = w.signal()
    res, N = run_gpu(lib, x, w.fs, w.freqs, w.n_cycles, w.outputs)
    assert res["complex"].shape == (64, 100, 10000) and res["complex"].dtype == np.complex64
    rows = [(c, s) for c in (0, 31, 63) for s in (0, 1, 37, 64, 98, 99)]
    ref = oracle.cwt_rows(x, N, w.fs, w.freqs, w.n_cycles, rows)
    got = {k: np.stack([v[c, s] for c, s in rows]) for k, v in res.items()}
    check(got, ref)
    # power is |complex|^2 of the same kernel output
    assert np.allclose(res["power"][0], np.abs(res["complex"][0]) ** 2, rtol=1e-5, atol=0)


EDGE = [
    # (C, n, fs, freqs, cycles, kwargs)
    (1, 1, 100.0, [10.0], [7.0], {}),
    (2, 31, 100.0, [5.0, 30.0], [3.0, 7.0], {}),
    (2, 32, 100.0, [5.0, 30.0], [3.0, 7.0], {}),
    (3, 33, 100.0, [5.0, 30.0, 49.0], [3.0, 7.0, 10.0], {}),
    (5, 3001, 1000.0, np.geomspace(1, 400, 7), np.linspace(2, 12, 7), {}),
    (2, 16384, 1000.0, [0.7, 499.0], [7.0, 3.0], {}),
    (1, 700, 500.0, [2.0], [1.0], {}),
    (2, 1000, 250.0, [124.0, 100.0], [2.0, 7.0], {}),
    (3, 900, 300.0, [9.0, 41.0], [7.0, 5.0], dict(wavelet="gabor")),
    (2, 777, 500.0, [6.0, 60.0], [7.0, 7.0], dict(fft_length=4096)),
]


@pytest.mark.parametrize("case", range(len(EDGE)))
def test_edge_cases_all_outputs(lib, case):
    C, n, fs, freqs, cycles, kw = EDGE[case]
    x = eeg(100 + case, C, n, fs, np.float32)
    res, N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power", "phase"), **kw)
    ref = oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles, wavelet=kw.get("wavelet", "morlet"))
    check(res, ref)


@pytest.mark.parametrize("d", [2, 3, 4, 6, 8, 16])
def test_decimation(lib, d):
    C, n, fs = 3, 2500, 1000.0
    freqs, cycles = np.geomspace(2, 80, 9), np.clip(np.geomspace(2, 80, 9) / 2, 3, 12)
    x = eeg(200 + d, C, n, fs, np.float32)
    res, N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power"), decimation=d)
    assert res["power"].shape == (C, 9, -(-n // d))
    ref = oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles, decimation=d)
    check(res, ref)


def test_f64_io_complex_and_phase(lib):
    x = eeg(300, 2, 1200, 512.0, np.float64)
    res, N = run_gpu(lib, x, 512.0, [3.0, 12.0, 100.0], [7.0, 7.0, 7.0],
                     ("complex", "power", "phase"), dtype="f64")
    assert res["complex"].dtype == np.complex128
    check(res, oracle.cwt(x, N, 512.0, [3.0, 12.0, 100.0], [7.0, 7.0, 7.0]))


def test_host_buffers_match_device_path_and_repeat_bitwise(lib):
    import torch
    w = workload("plain")
    x = np.ascontiguousarray(w.signal()[:, :])
    plan = lib.cwt_plan_create(8, 500, w.fs, w.freqs, w.n_cycles, 0, lib.CWT_OUT_COMPLEX | lib.CWT_OUT_POWER,
                               _opts(lib, io=lib.CWT_DTYPE_F64))
    try:
        hc = np.empty((8, 40, 500), np.complex128)
        hp = np.empty((8, 40, 500), np.float64)
        lib.cwt_execute_host(plan, x, hc, hp, None)
        xt = torch.from_numpy(x).cuda()
        dc = torch.empty((8, 40, 500), dtype=torch.complex128, device="cuda")
        dp = torch.empty((8, 40, 500), dtype=torch.float64, device="cuda")
        lib.cwt_execute(plan, xt, dc, dp, None)
        lib.cwt_execute(plan, xt, dc, dp, None)
        torch.cuda.synchronize()
        assert np.array_equal(dc.cpu().numpy(), hc) and np.array_equal(dp.cpu().numpy(), hp)
    finally:
        lib.cwt_plan_destroy(plan)


@pytest.mark.parametrize("pad", ["pow2", "smooth"])
def test_pinned_host_outputs_written_directly_equal_device_path(lib, pad):
    """cwt_execute_host with page-locked, device-mapped outputs (written by the
    kernels over the host link) and with a mix of pinned and pageable outputs:
    bitwise equal to the device path (power-of-two and smooth kernels)."""
    import torch
    w = workload("fused")
    C, n = 4, w.samples
    x = np.ascontiguousarray(w.signal()[:C])
    o = lib.cwt_options_init()
    o.pad_policy = lib.CWT_PAD_SMOOTH if pad == "smooth" else lib.CWT_PAD_POW2
    plan = lib.cwt_plan_create(C, n, w.fs, w.freqs, w.n_cycles, 0, lib.CWT_OUT_COMPLEX | lib.CWT_OUT_POWER, o)
    try:
        shape = (C, w.scales, n)
        xt = torch.from_numpy(x).cuda()
        dc = torch.empty(shape, dtype=torch.complex64, device="cuda")
        dp = torch.empty(shape, dtype=torch.float32, device="cuda")
        lib.cwt_execute(plan, xt, dc, dp, None)
        torch.cuda.synchronize()
        ref_c, ref_p = dc.cpu().numpy(), dp.cpu().numpy()
        hc = torch.empty(shape, dtype=torch.complex64).pin_memory()
        hp = torch.empty(shape, dtype=torch.float32).pin_memory()
        lib.cwt_execute_host(plan, torch.from_numpy(x).pin_memory(), hc, hp, None)
        assert np.array_equal(hc.numpy(), ref_c) and np.array_equal(hp.numpy(), ref_p)
        hp2 = np.empty(shape, np.float32)  # pageable: staged
        hc.zero_()
        lib.cwt_execute_host(plan, x, hc, hp2, None)
        assert np.array_equal(hc.numpy(), ref_c) and np.array_equal(hp2, ref_p)
    finally:
        lib.cwt_plan_destroy(plan)


def test_bad_pointers_rejected_on_host(lib):
    import torch
    plan = lib.cwt_plan_create(1, 100, 500.0, [10.0], [7.0], 0, lib.CWT_OUT_POWER)
    try:
        x = torch.zeros(100, device="cuda")
        out = torch.zeros(100, device="cuda")
        host = np.zeros(100, np.float32)
        for sig, o in ((host, out), (x, host), (x[1:], out), (x, None)):
            with pytest.raises(lib.CWTError) as e:
                lib.cwt_execute(plan, sig, None, o, None)
            assert e.value.status == lib.CWT_EINVAL
        with pytest.raises(lib.CWTError):  # complex not requested at creation
            lib.cwt_execute(plan, x, torch.zeros(200, device="cuda"), out, None)
    finally:
        lib.cwt_plan_destroy(plan)


def test_profiling_counts_launches(lib):
    import torch
    plan = lib.cwt_plan_create(4, 1000, 500.0, [10.0, 20.0], [7.0, 7.0], 0, lib.CWT_OUT_POWER)
    try:
        lib.cwt_plan_set_profiling(plan, True)
        x = torch.zeros((4, 1000), device="cuda")
        out = torch.empty((4, 2, 1000), device="cuda")
        for _ in range(3):
            lib.cwt_execute(plan, x, None, out, None)
        n_f, ms_f = lib.cwt_plan_profile_read(plan, lib.CWT_KERNEL_FORWARD_FFT)
        n_s, ms_s = lib.cwt_plan_profile_read(plan, lib.CWT_KERNEL_SCALE_BLOCK)
        assert (n_f, n_s) == (3, 3) and ms_f > 0 and ms_s > 0
        assert lib.cwt_plan_profile_read(plan, lib.CWT_KERNEL_SCALE_BLOCK) == (0, 0.0)
        nb, bank_ms = lib.cwt_plan_profile_read(plan, lib.CWT_KERNEL_BANK)
        assert nb == 1 and bank_ms > 0
    finally:
        lib.cwt_plan_destroy(plan)


def test_paper_style_error_report(lib):
    """Table 1's metric (|diff| / SD over the 20-80 % interior, threshold
    1e-5 SD) for 1 s at 1000 Hz, sigma 7, 30-90 Hz by 1 Hz, against the oracle."""
    fs, n = 1000.0, 1000
    freqs = np.arange(30.0, 91.0)
    x = eeg(400, 1, n, fs, np.float32)
    res, N = run_gpu(lib, x, fs, freqs, np.full(len(freqs), 7.0), ("complex",))
    ref = oracle.cwt(x.astype(np.float64), N, fs, freqs, np.full(len(freqs), 7.0))
    rep = paper_style_error(res["complex"].astype(np.complex128), ref)
    assert rep["real"][2] == 0 and rep["imag"][2] == 0, rep


def _opts(lib, **kw):
    o = lib.cwt_options_init()
    if "io" in kw:
        o.io_dtype = kw["io"]
    return o


def test_cluster_lengths_every_row(lib):
    """N = 32768 and 65536 (rows on clusters of 2 and 4 CTAs), every row."""
    for C, n, fs, freqs, cycles in [(2, 20000, 1000.0, [0.8, 13.0, 240.0], [3.0, 7.0, 12.0]),
                                    (1, 40000, 2000.0, [3.0, 600.0], [7.0, 5.0])]:
        x = eeg(600 + n, C, n, fs, np.float32)
        res, N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power", "phase"))
        assert N > 16384
        check(res, oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles))


def test_precision_workload_full_size_sampled_rows(lib):
    """256 ch x 122880 @2048 Hz (N = 131072: clusters of 8 CTAs), 128 log
    freqs 0.5-200 Hz, power + phase, FP32; error per frequency on sampled rows."""
    import os
    import torch
    w = workload("precision")
    C, S = w.channels, w.scales
    t = lib.CWT(C, w.samples, w.fs, w.freqs, w.n_cycles, outputs=("power", "phase"))
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
            print(f"F={w.freqs[s]:8.3f} Hz  power err {a:.2e}  phase err {b:.2e}")
        assert e_p.max() <= FP32_TOL and e_ph.max() <= FP32_TOL
    finally:
        t.close()


def test_channel_shards_equal_the_whole(lib):
    """Rows are independent: transforming channel blocks separately (as ranks
    of a multi-GPU run do) gives bitwise the whole-recording result."""
    import torch
    from paper_2506_07793_gb300.partition import shard_channels
    C, n, fs = 10, 3000, 500.0
    freqs, cycles = np.geomspace(2, 120, 11), np.full(11, 7.0)
    x = torch.from_numpy(eeg(77, C, n, fs, np.float32)).cuda()
    whole = lib.CWT(C, n, fs, freqs, cycles, outputs=("complex", "power"))
    ref = whole(x)
    for world in (2, 3):
        for r in range(world):
            c0, c1 = shard_channels(C, world, r)
            part = lib.CWT(c1 - c0, n, fs, freqs, cycles, outputs=("complex", "power"))
            out = part(x[c0:c1].contiguous())
            torch.cuda.synchronize()
            assert torch.equal(out["complex"], ref["complex"][c0:c1])
            assert torch.equal(out["power"], ref["power"][c0:c1])
            part.close()
    whole.close()


SMOOTH = [
    # (C, n, fs, freqs, cycles, kwargs) -- smooth padded lengths: 98, 125, 500, 3024, 10000, 14000
    (2, 97, 100.0, [9.0, 30.0], [3.0, 7.0], {}),
    (3, 122, 125.0, [11.0, 50.0], [5.0, 7.0], {}),
    (2, 500, 500.0, [4.0, 40.0, 200.0], [3.0, 7.0, 10.0], dict(dtype="f64")),
    (3, 3001, 1000.0, np.geomspace(1, 400, 6), np.linspace(3, 10, 6), dict(decimation=3)),
    (2, 10000, 1000.0, [0.8, 10.0, 99.0], [3.0, 6.0, 10.0], {}),
    (1, 14000, 2000.0, [5.0, 300.0], [7.0, 7.0], {}),
    (2, 33, 100.0, [5.0, 30.0], [3.0, 7.0], {}),            # N = 35 = 5 x 7, the shortest
    (1, 1, 100.0, [10.0], [7.0], {}),                         # one sample: N = 32
]


@pytest.mark.parametrize("case", range(len(SMOOTH)))
def test_smooth_padding_every_row(lib, case):
    """The paper's padding (Section "Fast Fourier transform"): 2,3,5,7-smooth N,
    mixed-radix kernels; parity with the oracle at the same N."""
    C, n, fs, freqs, cycles, kw = SMOOTH[case]
    kw = dict(kw)
    dtype = kw.pop("dtype", "f32")
    x = eeg(950 + case, C, n, fs, np.float64 if dtype == "f64" else np.float32)
    res, N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power", "phase"), dtype=dtype,
                     pad="smooth", **kw)
    assert N == lib.cwt_fft_length(n, lib.CWT_PAD_SMOOTH) and N <= 16384
    ref = oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles, decimation=kw.get("decimation", 1))
    check(res, ref)


def test_fused_workload_smooth_padding_sampled_rows(lib):
    """The fused workload under the paper's own padding: N = 10000 (no padding)."""
    w = workload("fused")
    x = w.signal()
    res, N = run_gpu(lib, x, w.fs, w.freqs, w.n_cycles, w.outputs, pad="smooth")
    assert N == 10000
    rows = [(c, s) for c in (0, 63) for s in (0, 1, 50, 99)]
    ref = oracle.cwt_rows(x, N, w.fs, w.freqs, w.n_cycles, rows)
    check({k: np.stack([v[c, s] for c, s in rows]) for k, v in res.items()}, ref)


SMOOTH_CLUSTER = [
    # (C, n, fs, freqs, cycles, kwargs, N, CL): smooth N above 16384, one
    # thread-block cluster of CL CTAs per row, NL = N / CL points each.
    # Narrow bands (a low carrier with many cycles) take the sparse first
    # pass, wide ones the dense pass.
    (1, 16400, 1000.0, [2.0, 40.0, 300.0], [5.0, 7.0, 10.0], {}, 16464, 2),
    (2, 20000, 2000.0, [0.5, 50.0, 900.0], [3.0, 7.0, 12.0], dict(dtype="f64"), 20000, 2),
    # local rows two CTAs per SM hold, compiled in: 10000, 12000, 12288, on
    # clusters of up to 10 CTAs (above 8: a non-portable cluster size)
    (1, 50000, 1000.0, [1.0, 100.0, 450.0], [20.0, 7.0, 4.0], dict(decimation=4), 50000, 5),
    (1, 100000, 4000.0, [0.3, 60.0, 1900.0], [7.0, 7.0, 10.0], dict(decimation=8), 100000, 10),
    (1, 122880, 2048.0, [0.5, 13.0, 200.0], [7.0, 7.0, 7.0], dict(decimation=8), 122880, 10),
    (1, 30000, 500.0, [1.0, 40.0, 240.0], [7.0, 7.0, 12.0], dict(decimation=4), 30000, 3),
    (1, 60000, 1000.0, [0.6, 80.0, 480.0], [5.0, 7.0, 12.0], dict(decimation=8, dtype="f64"), 60000, 5),
    (1, 48000, 800.0, [0.8, 50.0, 380.0], [7.0, 7.0, 10.0], dict(decimation=4), 48000, 4),
    # the runtime schedule of 14400 on 8 CTAs
    (1, 115200, 1920.0, [0.5, 40.0, 900.0], [7.0, 7.0, 10.0], dict(decimation=8), 115200, 8),
    # smooth lengths of at most 16384 that no one-CTA schedule covers, odd
    # cluster sizes, and the compiled-in local length 15360 on 6 and 7 CTAs
    (1, 14175, 1000.0, [2.0, 40.0, 300.0], [5.0, 7.0, 10.0], {}, 14175, 3),
    (2, 14406, 500.0, [1.0, 30.0, 200.0], [3.0, 7.0, 12.0], dict(dtype="f64"), 14406, 2),
    (1, 15625, 1000.0, [0.7, 80.0, 450.0], [7.0, 7.0, 7.0], dict(decimation=2), 15625, 5),
    (1, 19683, 2000.0, [1.5, 100.0, 800.0], [7.0, 7.0, 7.0], {}, 19683, 3),
    (1, 92160, 4096.0, [0.5, 50.0, 1800.0], [7.0, 7.0, 7.0], dict(decimation=16), 92160, 6),
    (1, 107520, 4096.0, [0.4, 120.0, 2000.0], [7.0, 7.0, 12.0], dict(decimation=16), 107520, 7),
    # the compiled-in local row 15000 (a minute and a half at 500 Hz)
    (1, 45000, 500.0, [1.0, 30.0, 230.0], [5.0, 7.0, 12.0], dict(decimation=4), 45000, 3),
]

# local lengths whose schedule is compiled into the cluster kernels (for
# every cluster size these cases use)
CLUSTER_FIXED_NL = (15360, 15000, 10000, 12000, 12288)


@pytest.mark.parametrize("case", range(len(SMOOTH_CLUSTER)))
def test_smooth_cluster_every_row(lib, case):
    """Smooth lengths one CTA does not run (Section "Fast Fourier transform"):
    the row of N = CL NL points runs on a cluster, each CTA a residue class
    through the NL-point mixed-radix passes, then one radix-CL stage across
    the cluster; parity with the oracle at the same N for every output kind."""
    import torch
    C, n, fs, freqs, cycles, kw, N_want, CL = SMOOTH_CLUSTER[case]
    kw = dict(kw)
    dtype = kw.pop("dtype", "f32")
    d = kw.get("decimation", 1)
    x = eeg(1100 + case, C, n, fs, np.float64 if dtype == "f64" else np.float32)
    t = lib.CWT(C, n, fs, freqs, cycles, outputs=("complex", "power", "phase"), dtype=dtype,
                pad="smooth", **kw)
    info = t.info
    assert info.fft_length == N_want and info.cluster == CL
    assert info.fixed_kernel == (N_want // CL in CLUSTER_FIXED_NL)
    rad = [r for r in info.radices if r]
    assert int(np.prod(rad)) == N_want // CL
    out = t(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    t.close()
    ref = oracle.cwt(x.astype(np.float64), N_want, fs, freqs, cycles, decimation=d)
    check(res, ref)


GMW = [
    # (C, n, fs, freqs, betas, gamma, kwargs)
    (2, 500, 500.0, [4.0, 40.0, 200.0], [20.0, 20.0, 20.0], 3.0, {}),
    (3, 1000, 1000.0, np.geomspace(2, 300, 5), [3.0, 8.0, 20.0, 60.0, 120.0], 3.0, dict(decimation=2)),
    (2, 777, 256.0, [5.0, 100.0], [3.0, 6.5], 1.0, {}),  # Cauchy; 100 Hz aliases past fs
    (1, 3001, 1000.0, [10.0, 90.0], [8.0, 4.0], 2.0, dict(pad="smooth")),
    (2, 300, 200.0, [1.0, 50.0], [1.5, 30.0], 0.7, dict(dtype="f64")),
    (1, 20000, 2000.0, [3.0, 700.0], [20.0, 20.0], 3.0, {}),  # cluster path (N = 32768)
]


@pytest.mark.parametrize("case", range(len(GMW)))
def test_gmw_every_row(lib, case):
    """Generalized Morse wavelet (Eq. 5 with U(omega)): the bank generator's
    alias-summed spectrum against the oracle's inverse-DFT definition."""
    C, n, fs, freqs, betas, gam, kw = GMW[case]
    kw = dict(kw)
    dtype = kw.pop("dtype", "f32")
    x = eeg(970 + case, C, n, fs, np.float64 if dtype == "f64" else np.float32)
    res, N = run_gpu(lib, x, fs, freqs, betas, ("complex", "power", "phase"), dtype=dtype,
                     wavelet="gmw", gmw_gamma=gam, **kw)
    ref = oracle.cwt(x.astype(np.float64), N, fs, freqs, betas, decimation=kw.get("decimation", 1),
                     wavelet="gmw", gamma=gam)
    check(res, ref)


LINEAR = [
    # (C, n, fs, freqs, cycles, kwargs)
    (2, 500, 500.0, [4.0, 40.0, 200.0], [3.0, 7.0, 10.0], {}),
    (2, 1000, 1000.0, np.geomspace(2, 300, 5), np.linspace(3, 10, 5), dict(decimation=3)),
    (1, 3000, 1000.0, [5.0, 90.0], [7.0, 7.0], dict(pad="smooth")),
    (2, 300, 200.0, [9.0, 50.0], [5.0, 7.0], dict(wavelet="gabor", dtype="f64")),
    (1, 20000, 1000.0, [2.0, 60.0], [5.0, 7.0], dict(pad="smooth")),  # N = 22680 on a cluster of 2
    # GMW (Eq. 5; the cycles column holds beta): support radius measured by the library
    (2, 800, 500.0, [6.0, 60.0], [20.0, 40.0], dict(wavelet="gmw")),
    (1, 600, 250.0, [3.0, 40.0], [8.0, 60.0], dict(wavelet="gmw", gmw_gamma=2.0, pad="smooth")),
]


def _support_radius(fs, freqs, cycles):
    a = max(c / (2 * np.pi * f) for f, c in zip(freqs, cycles))
    return int(np.ceil(6.5 * a * fs))


@pytest.mark.parametrize("case", range(len(LINEAR)))
def test_linear_edges_equal_linear_convolution(lib, case):
    """Linear ("same"-mode) edges: N >= n + R + 1 with R the largest scale's
    support radius, parity with the oracle at that N, and agreement with a
    direct linear convolution of the signal with the sampled wavelet
    (normalised like the oracle's) at every output, edges included.  Morlet
    and Gabor take their Gaussian closed form; the GMW, which has none, the
    oracle's periodised wavelet over a period much longer than its support."""
    C, n, fs, freqs, cycles, kw = LINEAR[case]
    kw = dict(kw)
    dtype = kw.pop("dtype", "f32")
    wavelet = kw.pop("wavelet", "morlet")
    gamma = kw.get("gmw_gamma", 3.0)
    x = eeg(990 + case, C, n, fs, np.float64 if dtype == "f64" else np.float32)
    res, N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power"), dtype=dtype, wavelet=wavelet,
                     edge="linear", **kw)
    kind = {"morlet": lib.CWT_WAVELET_MORLET, "gabor": lib.CWT_WAVELET_GABOR, "gmw": lib.CWT_WAVELET_GMW}[wavelet]
    radii = [lib.cwt_support_radius(kind, F, sg, fs, gamma) for F, sg in zip(freqs, cycles)]
    if wavelet != "gmw":
        assert max(radii) == _support_radius(fs, freqs, cycles)
    assert N >= n + max(radii) + 1
    d = kw.get("decimation", 1)
    ref = oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles, decimation=d, wavelet=wavelet, gamma=gamma)
    check(res, ref)
    # direct linear convolution with the unperiodised sampled wavelet
    lin = np.empty_like(ref)
    for s, (F, sg) in enumerate(zip(freqs, cycles)):
        if wavelet == "gmw":
            Rs = int(1.5 * radii[s]) + 1
            Nbig = 1 << int(np.ceil(np.log2(8 * Rs)))
            big = oracle.periodised_wavelet(F, sg, fs, Nbig, wavelet="gmw", gamma=gamma)
            psi = big[np.arange(-Rs, Rs + 1) % Nbig]
        else:
            a = sg / (2 * np.pi * F)
            Rs = int(np.ceil(40 * a * fs))
            tau = np.arange(-Rs, Rs + 1) / fs
            kappa = 0.0 if wavelet == "gabor" else np.exp(-0.5 * sg * sg)
            psi = np.exp(-tau ** 2 / (2 * a * a)) * (np.exp(2j * np.pi * F * tau) - kappa)
        psi = psi / np.sqrt(np.sum(np.abs(oracle.periodised_wavelet(F, sg, fs, N, wavelet=wavelet,
                                                                     gamma=gamma)) ** 2))
        for c in range(C):
            lin[c, s] = np.convolve(x[c].astype(np.float64), psi)[Rs:Rs + n][::d]
    check({"complex": res["complex"]}, lin)


@pytest.mark.parametrize("n", [200, 250, 320, 400, 500, 1000, 1600, 2000, 2500, 3200, 5000, 6400, 8000])
def test_smooth_padding_common_eeg_lengths(lib, n):
    """2^a 5^b lengths (whole seconds of EEG at 250 / 500 / 1000 Hz among
    them): the scale block runs on a fixed-length kernel (500 ... 8000) or on
    an inlined radix pair (every pair that some smooth length schedules at
    least once over this list: 200, 250, 320, 400, 1600, 3200, 6400), the
    forward FFT on the pair -- parity with the oracle at that N."""
    fs = 1000.0
    freqs, cycles = [3.0, 20.0, 90.0], [5.0, 7.0, 9.0]
    x = eeg(1010 + n, 2, n, fs, np.float32)
    res, N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power"), pad="smooth")
    assert N == n
    check(res, oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles))


FIXED = [
    # (n = N, C, freqs, cycles, dtype, decimation) at fs = 1 kHz: the
    # fixed-length scale-block kernels; bands from narrow (sparse first pass)
    # to the widest (dense), FP64 I/O, and decimations with and without a
    # linear epilogue stride (T d a multiple of 16)
    (10000, 3, np.geomspace(0.5, 450.0, 8), np.linspace(3.0, 12.0, 8), "f32", 1),
    (10000, 2, [0.7, 8.0, 120.0, 480.0], [3.0, 5.0, 9.0, 14.0], "f64", 3),
    (10000, 2, [2.0, 40.0, 300.0], [4.0, 7.0, 10.0], "f32", 7),
    (8000, 3, np.geomspace(0.5, 450.0, 6), np.linspace(3.0, 12.0, 6), "f32", 1),
    (8000, 2, [1.0, 60.0, 400.0], [4.0, 7.0, 12.0], "f64", 5),
    (5000, 3, np.geomspace(1.0, 450.0, 6), np.linspace(3.0, 12.0, 6), "f32", 1),
    (5000, 2, [0.9, 30.0, 250.0], [3.0, 7.0, 10.0], "f32", 3),
    (4000, 3, np.geomspace(1.0, 450.0, 6), np.linspace(3.0, 12.0, 6), "f64", 1),
    (4000, 2, [2.0, 45.0, 350.0], [5.0, 7.0, 11.0], "f32", 9),
    (2500, 3, np.geomspace(2.0, 450.0, 5), np.linspace(3.0, 12.0, 5), "f32", 1),   # 2 rows per CTA
    (2000, 5, [3.0, 40.0, 300.0], [4.0, 7.0, 10.0], "f64", 2),                     # odd row count
    (1000, 7, np.geomspace(4.0, 450.0, 3), [5.0, 7.0, 12.0], "f32", 1),            # 5 rows per CTA
    (500, 3, [10.0, 100.0, 400.0, 480.0], [6.0, 7.0, 9.0, 12.0], "f32", 4),         # 10 rows per CTA
    (15000, 2, np.geomspace(0.5, 450.0, 5), np.linspace(3.0, 12.0, 5), "f32", 1),  # four passes
    (12000, 2, [0.6, 50.0, 420.0], [3.0, 7.0, 12.0], "f64", 1),
    (9000, 2, np.geomspace(1.0, 450.0, 4), np.linspace(3.0, 12.0, 4), "f32", 3),
    (7500, 3, [0.8, 25.0, 330.0], [3.0, 7.0, 10.0], "f32", 1),
    (6000, 2, [1.5, 70.0, 440.0], [4.0, 7.0, 12.0], "f32", 2),
    (3000, 5, np.geomspace(2.0, 450.0, 3), [5.0, 7.0, 12.0], "f32", 1),             # 2 rows per CTA
    (1500, 6, [4.0, 90.0, 470.0], [5.0, 7.0, 9.0], "f64", 1),                      # 4 rows per CTA
    (14000, 2, [0.5, 30.0, 400.0], [3.0, 7.0, 12.0], "f32", 1),
    (13500, 1, [0.9, 60.0, 450.0], [4.0, 7.0, 10.0], "f32", 2),
    (12500, 2, [0.7, 20.0, 300.0], [3.0, 7.0, 12.0], "f64", 1),
    (10500, 2, [1.2, 45.0, 380.0], [5.0, 7.0, 9.0], "f32", 3),
    (7000, 3, [0.8, 35.0, 460.0], [3.0, 7.0, 12.0], "f32", 1),
    (4500, 3, [1.5, 25.0, 330.0], [4.0, 7.0, 10.0], "f32", 1),
    (3750, 3, [2.0, 50.0, 410.0], [5.0, 7.0, 12.0], "f64", 2),
    (3500, 3, [1.8, 70.0, 260.0], [4.0, 7.0, 9.0], "f32", 1),
    (2250, 5, [3.0, 40.0, 350.0], [5.0, 7.0, 10.0], "f32", 1),                     # 2 rows per CTA
    (1750, 5, [3.5, 80.0, 420.0], [5.0, 7.0, 11.0], "f32", 1),                     # 2 rows per CTA
    (1250, 7, [4.0, 60.0, 440.0], [5.0, 7.0, 9.0], "f32", 1),                      # 4 rows per CTA
    (750, 9, [8.0, 100.0, 470.0], [6.0, 7.0, 12.0], "f32", 1),                     # 8 rows per CTA
]


@pytest.mark.parametrize("case", range(len(FIXED)))
def test_fixed_length_kernel_every_row(lib, case):
    """The 27 whole-second lengths 750 ... 15000 run on the kernels compiled
    for that length and schedule (several rows per CTA below 3500, row counts
    that leave a CTA partly idle); parity with the oracle for every output
    kind."""
    n, C, freqs, cycles, dtype, d = FIXED[case]
    fs = 1000.0
    x = eeg(1200 + case, C, n, fs, np.float64 if dtype == "f64" else np.float32)
    t = lib.CWT(C, n, fs, freqs, cycles, outputs=("complex", "power", "phase"), dtype=dtype,
                decimation=d, pad="smooth")
    assert t.info.fixed_kernel == 1 and t.info.fft_length == n
    t.close()
    res, N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power", "phase"), dtype=dtype,
                     decimation=d, pad="smooth")
    check(res, oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles, decimation=d))


def test_smooth_plan_reports_schedule(lib):
    """The fused workload's smooth length N = 10000 runs 16 x 25 x 25 (on 416
    threads) on the kernel compiled for that length and schedule, and so do
    8000, 5000, 4000 and 2000 on the pass orders measured fastest; 1600 and 250 run on inlined
    pairs, and a length outside the pairs runs the generic one."""
    o = lib.cwt_options_init()
    o.pad_policy = lib.CWT_PAD_SMOOTH
    for n, pair, rad, fixed in ((10000, (0, 0), [16, 25, 25], 1), (3001, (0, 0), None, 0),
                                (5000, (0, 0), [20, 10, 25], 1), (8000, (0, 0), [16, 25, 20], 1),
                                (4000, (0, 0), [16, 10, 25], 1), (2000, (0, 0), [20, 10, 10], 1),
                                (1600, (10, 16), None, 0), (250, (10, 25), None, 0)):
        plan = lib.cwt_plan_create(1, n, 1000.0, [10.0], [7.0], 0, lib.CWT_OUT_POWER, o)
        try:
            info = lib.cwt_plan_info(plan)
            if pair is not None:
                assert tuple(info.inlined_pair) == pair
            assert info.fixed_kernel == fixed
            got = [r for r in info.radices if r]
            assert int(np.prod(got)) == info.fft_length
            if rad is not None:
                assert got == rad
        finally:
            lib.cwt_plan_destroy(plan)


@pytest.mark.parametrize("N", [4000, 4096, 1215, 2401])
def test_explicit_smooth_fft_length(lib, N):
    """An explicit 2,3,5,7-smooth N (on an inlined pair, a power of two, a pure
    3-smooth and a pure 7-smooth length): parity with the oracle at that N."""
    fs, freqs, cycles = 500.0, [6.0, 60.0], [7.0, 7.0]
    x = eeg(1100 + N, 2, 777, fs, np.float32)
    res, got_N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power", "phase"), fft_length=N)
    assert got_N == N
    check(res, oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles))


# For every radix the scheduler uses, the shortest smooth length whose
# schedule takes it as the first pass and as a later pass (the host schedule
# is pinned in test_abi.py; here the kernels run it).
RADIX_LENGTHS = [40, 35, 13125, 36, 49, 80, 48, 81, 45, 100, 144, 72, 196, 70, 225, 75, 320, 112,
                 324, 108, 400, 180, 441, 147, 576, 192, 625, 125, 729, 189, 784, 280, 900, 300, 640]


@pytest.mark.parametrize("N", RADIX_LENGTHS)
def test_every_radix_in_every_position(lib, N):
    """Each mixed-radix DFT (prime, prime-power and coprime composite radices
    4 ... 32, Section "Fast Fourier transform") in the first and in a later
    pass, forward and inverse: parity with the oracle at an explicit N."""
    fs, freqs, cycles = 100.0, [8.0, 30.0], [3.0, 5.0]
    n = N - 3
    x = eeg(1400 + N, 1, n, fs, np.float32)
    res, got_N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power"), fft_length=N)
    assert got_N == N
    check(res, oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles))


@pytest.mark.parametrize("pad,edge", [("pow2", "cyclic"), ("smooth", "cyclic"), ("pow2", "linear")])
def test_mne_normalisation(lib, pad, edge):
    """MNE-python's wavelet normalisation (sum |w|^2 = 2) on every row, against
    the oracle under the same convention, including linear edges (MNE's own
    "same"-mode convolution)."""
    fs, n = 1000.0, 3000
    freqs, cycles = np.array([4.0, 12.0, 40.0, 90.0]), np.array([5.0, 7.0, 7.0, 9.0])
    x = eeg(1300, 2, n, fs, np.float32)
    res, N = run_gpu(lib, x, fs, freqs, cycles, ("complex", "power"), pad=pad, edge=edge,
                     normalization="mne")
    check(res, oracle.cwt(x.astype(np.float64), N, fs, freqs, cycles, normalization="mne"))
