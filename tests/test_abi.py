"""CPU-only checks of the C ABI: the library loads, exports every function that
include/*.h declares, and its host-side logic (argument validation, padding
policy, status strings) behaves as documented.  No CUDA compute is issued: each
call here returns before the library's first CUDA call."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_07793_gb300 as p
    return p


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"\b(cwt_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_status_strings(lib):
    for s in (0, 1, 2, 3, 4, 5, 6, 8):
        assert lib.cwt_status_str(s).startswith("CWT_") and "UNKNOWN" not in lib.cwt_status_str(s)
    assert "UNKNOWN" in lib.cwt_status_str(7)  # no status 7: nothing waits on the device
    assert "UNKNOWN" in lib.cwt_status_str(99)


def test_bounds_check_build_compiles_and_exports(lib):
    """The bounds-checked variant (-DCWT_BOUNDS_CHECK) builds and exports the
    same symbols (its kernels run in tests/test_gpu_bounds_check.py)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_cwt_build", os.path.join(ROOT, "paper_2506_07793_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    so = ctypes.CDLL(b.build(check=True))
    for name in declared_functions():
        assert hasattr(so, name), name


def test_options_defaults(lib):
    o = lib.cwt_options_init()
    assert (o.precision, o.decimation, o.pad_policy, o.fft_length, o.io_dtype) == (0, 1, 0, 0, 0)


@pytest.mark.parametrize("n,N", [(1, 32), (31, 32), (32, 32), (33, 64), (500, 512), (10000, 16384),
                                 (16384, 16384), (16385, 32768), (122880, 131072), (131072, 131072)])
def test_pow2_padding(lib, n, N):
    assert lib.cwt_fft_length(n) == N


@pytest.mark.parametrize("n,N", [(1, 32), (97, 98), (122, 125), (500, 500), (3001, 3024),
                                 (10000, 10000), (14000, 14000), (14401, 14406), (15000, 15000),
                                 (15100, 15120), (16001, 16128), (16383, 16384), (16385, 16464),
                                 (19683, 19683), (20000, 20000), (50000, 50000), (59000, 59535),
                                 (59049, 59535), (78125, 78400), (122880, 122880), (128000, 131072),
                                 (131072, 131072)])
def test_smooth_padding(lib, n, N):
    """Section "Fast Fourier transform": the smallest 2,3,5,7-smooth length >= n
    that the kernels run.  14406 = 2 3 7^4 and 15120 = 2^4 3^3 5 7 have no
    one-CTA schedule (at most 32 values per thread, 512 threads) but split as
    2 x 7203 and 2 x 7560 over a cluster; 16128 = 2^8 3^2 7 likewise; 16464
    = 2 x 8232 is the first smooth length past 16384; 19683 = 3 x 6561 runs
    on a cluster of 3.  3^10 = 59049 has no split with NL <= 16384 (3 is its
    only factor), so 59000 and 59049 pad to 59535 = 5 x 11907; 5^7 = 78125
    splits only as 5 x 15625, unscheduled, and pads to 78400 = 2^6 5^2 7^2;
    122880 = 8 x 15360 (run as 10 x 12288) needs no padding; 128000 = 8 x 16000 and
    129024 = 8 x 16128 split only into unscheduled NL, so 128000 pads to 2^17."""
    assert lib.cwt_fft_length(n, lib.CWT_PAD_SMOOTH) == N


def _smooth(m):
    for f in (2, 3, 5, 7):
        while m % f == 0:
            m //= f
    return m == 1


def _one_cta(lib, m):
    try:
        lib.cwt_smooth_schedule(m)
        return True
    except lib.CWTError as e:
        assert e.status == lib.CWT_EUNSUPPORTED
        return False


def test_smooth_cluster_split_rule(lib):
    """Every smooth length in [32, 2^17] that is not a power of two is kept by
    the SMOOTH policy exactly when the one-CTA scheduler covers it (N <= 16384)
    or some CL in 2 ... 8 divides it with N / CL <= 16384 a length that
    scheduler covers."""
    passed_over = []
    for m in range(32, 131073):
        if not _smooth(m) or (m & (m - 1)) == 0:
            continue
        ok = m <= 16384 and _one_cta(lib, m)
        for cl in range(2, 9):
            if ok:
                break
            ok = m % cl == 0 and m // cl <= 16384 and _one_cta(lib, m // cl)
        assert (lib.cwt_fft_length(m, lib.CWT_PAD_SMOOTH) == m) == ok, m
        if not ok:
            passed_over.append(m)
    assert len(passed_over) == 43 and passed_over[:3] == [59049, 78125, 84375]


# (N, specialize, CTAs per row, local length, compiled in)
CLUSTER_LAYOUTS = [
    (10000, 0, 1, 10000, 1),     # one CTA per row
    (20000, 0, 2, 10000, 1),     # 2 x 10000: two CTAs per SM already
    (30000, 0, 3, 10000, 1),     # not 2 x 15000 (one CTA per SM)
    (45000, 0, 3, 15000, 1),     # no local row two CTAs per SM hold is compiled in
    (60000, 0, 5, 12000, 1),     # not 4 x 15000
    (92160, 0, 6, 15360, 1),
    (100000, 0, 10, 10000, 1),   # a non-portable cluster, compiled in; not 8 x 12500
    (122880, 0, 10, 12288, 1),   # not 8 x 15360
    (115200, 0, 8, 14400, 0),    # 10 x 11520 is not compiled in
    (14406, 0, 2, 7203, 0),
    (45000, 1, 4, 11250, 0),     # plan-time kernels: any local row two CTAs per SM hold
    (105000, 1, 10, 10500, 0),
    (115200, 1, 9, 12800, 0),
    (14406, 1, 7, 2058, 0),
    (30720, 1, 3, 10240, 0),
    (100000, 1, 10, 10000, 1),   # fewest passes first: 3 (10 x 10000) before 4 (8 x 12500)
    (120000, 2, 10, 12000, 1),
]


@pytest.mark.parametrize("N,spec,CL,NL,fixed", CLUSTER_LAYOUTS)
def test_smooth_cluster_layout(lib, N, spec, CL, NL, fixed):
    """The cluster split of a smooth length (host-only): local rows that two
    CTAs per SM hold are preferred where a kernel is built for them -- fewest
    passes, then the smallest cluster; sizes above 8 CTAs only on compiled-in
    local rows or with plan-time compilation -- else the smallest cluster."""
    cl, rad, fx = lib.cwt_smooth_cluster(N, spec)
    assert (cl, int(np.prod(rad)), fx) == (CL, NL, fixed)


def test_smooth_cluster_layout_invariants(lib):
    """Every smooth length the SMOOTH policy keeps has a layout: CL local rows
    whose radices multiply to N / CL; above 8 CTAs only on a compiled-in row
    unless specialized; the same padding either way."""
    for m in list(range(16385, 131073, 97)) + [122880, 61440, 98304]:
        if not _smooth(m) or (m & (m - 1)) == 0 or lib.cwt_fft_length(m, lib.CWT_PAD_SMOOTH) != m:
            continue
        for spec in (0, 1):
            cl, rad, fx = lib.cwt_smooth_cluster(m, spec)
            assert 2 <= cl <= 16 and cl * int(np.prod(rad)) == m, (m, spec)
            assert spec or cl <= 8 or fx, m


def test_smooth_cluster_layout_refusals(lib):
    for N in (4096, 78125, 31, 131073):
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_smooth_cluster(N)
        assert e.value.status == lib.CWT_EUNSUPPORTED
    for spec in (-1, 3):
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_smooth_cluster(30000, spec)
        assert e.value.status == lib.CWT_EINVAL


def test_padding_limits(lib):
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_fft_length(0)
    assert e.value.status == lib.CWT_EINVAL
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_fft_length(131073)
    assert e.value.status == lib.CWT_EUNSUPPORTED
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_fft_length(131073, lib.CWT_PAD_SMOOTH)
    assert e.value.status == lib.CWT_EUNSUPPORTED


BAD = [
    dict(channels=0), dict(samples=0), dict(fs=0.0), dict(fs=float("nan")),
    dict(freqs=[10.0, 0.0]), dict(freqs=[10.0, 250.0]), dict(freqs=[-1.0]),
    dict(n_cycles=[7.0, 0.0]), dict(n_cycles=[7.0, float("inf")]),
    dict(wavelet=7), dict(kinds=0), dict(kinds=8), dict(decimation=0), dict(io=5),
    dict(precision=9), dict(fft_length=101), dict(fft_length=64, samples=100),
    dict(wavelet=2, gamma=0.0), dict(wavelet=2, gamma=-3.0), dict(wavelet=2, gamma=float("nan")),
    dict(wavelet=2, gamma=65.0), dict(wavelet=2, n_cycles=[20.0, 1001.0]), dict(edge=2), dict(edge=-1),
    dict(edge=1, fft_length=128),  # linear edges need N >= n + R + 1 (here 100 + 363 + 1)
    dict(norm=2), dict(norm=-1), dict(specialize=3), dict(specialize=-1),
    # a carrier far below the first DFT bin: 1.5 Hz with sigma 7 in a 32-point
    # window at 500 Hz (first bin 15.6 Hz) has a spectrum below 1e-150 on every
    # bin, so its unit-energy normalisation would underflow
    dict(samples=32, freqs=[1.5, 20.0]),
    # Gabor keeps a DC term exp(-sigma^2 / 2): below 1e-150 only for sigma > 26
    dict(samples=32, freqs=[1.5, 20.0], wavelet=1, n_cycles=[30.0, 7.0]),
    dict(samples=32, freqs=[1.5, 20.0], wavelet=2, n_cycles=[20.0, 20.0]),  # GMW
]


@pytest.mark.parametrize("bad", BAD)
def test_invalid_arguments_rejected_before_cuda(lib, bad):
    a = dict(channels=2, samples=100, fs=500.0, freqs=[10.0, 20.0], n_cycles=[7.0, 7.0],
             wavelet=0, kinds=2, decimation=1, io=0, precision=0, fft_length=0, gamma=3.0, edge=0,
             norm=0, specialize=0)
    a.update(bad)
    o = lib.cwt_options_init()
    o.decimation, o.io_dtype, o.precision, o.fft_length = a["decimation"], a["io"], a["precision"], a["fft_length"]
    o.gmw_gamma = a["gamma"]
    o.edge_mode = a["edge"]
    o.normalization = a["norm"]
    o.specialize = a["specialize"]
    f = np.asarray(a["freqs"], dtype=np.float64)
    c = np.asarray(a["n_cycles"], dtype=np.float64)
    if len(c) != len(f):
        c = np.resize(c, len(f))
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_plan_create(a["channels"], a["samples"], a["fs"], f, c, a["wavelet"], a["kinds"], o)
    assert e.value.status == lib.CWT_EINVAL


def test_option_struct_layout(lib):
    """The ctypes mirrors of the option structs match the C layout (checked
    there by static_assert) and the defaults of the *_init functions."""
    o = lib.cwt_options_init()
    assert ctypes.sizeof(o) == 64 and type(o).gmw_gamma.offset == 24
    assert o.gmw_gamma == 3.0 and o.decimation == 1
    assert type(o).edge_mode.offset == 20 and o.edge_mode == lib.CWT_EDGE_CYCLIC
    assert type(o).normalization.offset == 32 and o.normalization == lib.CWT_NORM_UNIT_ENERGY
    assert type(o).specialize.offset == 36 and o.specialize == 0
    assert ctypes.sizeof(lib.cwt_plan_info_t) == 120 and lib.cwt_plan_info_t.radices.offset == 64
    assert lib.cwt_plan_info_t.fixed_kernel.offset == 104 and lib.cwt_plan_info_t.cluster.offset == 112
    assert lib.cwt_plan_info_t.specialized.offset == 116
    so = lib.cwt_server_options_init()
    assert ctypes.sizeof(so) == 56 and type(so).gmw_gamma.offset == 32
    assert so.gmw_gamma == 3.0 and so.max_streams == 32


def test_linear_edges_too_long(lib):
    """Linear edges pad by the support radius: refused when n + R + 1 exceeds
    2^17 (0.01 Hz with 7 cycles at 4 kHz; a GMW with beta = 0.3, whose
    envelope decays only as |t|^-1.3)."""
    o = lib.cwt_options_init()
    o.edge_mode = lib.CWT_EDGE_LINEAR
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_plan_create(1, 100, 4000.0, [0.01], [7.0], 0, lib.CWT_OUT_POWER, o)
    assert e.value.status == lib.CWT_EUNSUPPORTED
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_plan_create(1, 100, 500.0, [10.0], [0.3], lib.CWT_WAVELET_GMW, lib.CWT_OUT_POWER, o)
    assert e.value.status == lib.CWT_EUNSUPPORTED


@pytest.mark.parametrize("kind,F,sig,fs", [(0, 10.0, 7.0, 1000.0), (1, 3.0, 5.0, 250.0), (0, 0.5, 3.0, 2048.0)])
def test_support_radius_gaussian(lib, kind, F, sig, fs):
    """Morlet and Gabor: the Gaussian envelope exp(-t^2 / (2 a^2)) is 1e-9 of
    its peak at a sqrt(2 ln 1e9) = 6.44 a; the radius is ceil(6.5 a fs)."""
    a = sig / (2 * np.pi * F)
    assert lib.cwt_support_radius(kind, F, sig, fs) == int(np.ceil(6.5 * a * fs))
    assert np.exp(-(6.5 * a) ** 2 / (2 * a * a)) < 1e-9 < np.exp(-(6.4 * a) ** 2 / (2 * a * a))


@pytest.mark.parametrize("F,beta,gamma,fs", [(10.0, 20.0, 3.0, 1000.0), (40.0, 3.0, 3.0, 500.0),
                                             (10.0, 20.0, 1.0, 1000.0), (5.0, 17.5, 3.0, 2048.0)])
def test_support_radius_gmw_against_fourier_quadrature(lib, F, beta, gamma, fs):
    """GMW (Eq. 5 with U(nu)): the library measures the radius from the
    spectrum with an FP64 inverse FFT; here |psi(t)| = |int G(nu) e^(2 pi i nu t)
    dnu| comes from scipy's Fourier-integral quadrature (QAWF).  At the radius
    the envelope is below 1e-9 of its peak psi(0) = int G, and at 0.9 of it
    above."""
    integrate = pytest.importorskip("scipy.integrate")
    wp = (beta / gamma) ** (1 / gamma)

    def G(nu):
        return np.exp(beta * np.log(wp * nu / F) - (wp * nu / F) ** gamma) if nu > 0 else 0.0

    def env(t):
        w = 2 * np.pi * t
        c = integrate.quad(G, 0, np.inf, weight="cos", wvar=w, limlst=200)[0]
        s = integrate.quad(G, 0, np.inf, weight="sin", wvar=w, limlst=200)[0]
        return np.hypot(c, s)

    R = lib.cwt_support_radius(lib.CWT_WAVELET_GMW, F, beta, fs, gamma)
    peak = integrate.quad(G, 0, np.inf, limit=500)[0]
    assert env(R / fs) <= 1.05e-9 * peak
    assert env(0.9 * R / fs) > 1e-9 * peak


def test_support_radius_refusals(lib):
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_support_radius(lib.CWT_WAVELET_GMW, 10.0, 0.3, 500.0)
    assert e.value.status == lib.CWT_EUNSUPPORTED
    for bad in [(5, 10.0, 7.0, 500.0), (0, 0.0, 7.0, 500.0), (0, 300.0, 7.0, 500.0), (0, 10.0, -1.0, 500.0)]:
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_support_radius(*bad)
        assert e.value.status == lib.CWT_EINVAL


@pytest.mark.parametrize("what", ["tc_fp16", "tc_bf16", "too_long", "odd_smooth", "unsplit_smooth",
                                  "tc_smooth"])
def test_unsupported_requests(lib, what):
    """The tensor-core inverse FFTs cover power-of-two N of 16384 .. 131072
    only (here N = 128, then the smooth 20000); 140000 samples exceed the
    longest padding; an explicit smooth fft_length with no cluster split
    (5^7 = 78125 splits only as 5 x 15625; 128000 = 8 x 16000, both NL
    unscheduled) is refused."""
    o = lib.cwt_options_init()
    wavelet, samples = 0, 100
    if what == "tc_fp16":
        o.precision = lib.CWT_PREC_TC_FP16
    elif what == "tc_bf16":
        o.precision = lib.CWT_PREC_TC_BF16
    elif what == "odd_smooth":
        o.fft_length = 78125
    elif what == "unsplit_smooth":
        o.fft_length = 128000
    elif what == "tc_smooth":
        o.precision, o.fft_length = lib.CWT_PREC_TC_FP16, 20000
    else:
        samples = 140000
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_plan_create(1, samples, 500.0, [10.0], [7.0], wavelet, lib.CWT_OUT_POWER, o)
    assert e.value.status == lib.CWT_EUNSUPPORTED


def test_null_plan_calls(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    so.cwt_plan_workspace_bytes.restype = ctypes.c_size_t
    assert so.cwt_plan_workspace_bytes(None) == 0
    assert so.cwt_plan_destroy(None) == 0
    assert so.cwt_execute(None, None, None, None, None, None) == lib.CWT_EINVAL
    assert so.cwt_plan_info(None, None) == lib.CWT_EINVAL
    so.cwt_plan_last_error.restype = ctypes.c_char_p
    assert so.cwt_plan_last_error(None) == b""
    rad, pair = (ctypes.c_int * 8)(), (ctypes.c_int * 2)()
    t, fixed = ctypes.c_int(), ctypes.c_int()
    assert so.cwt_smooth_schedule(10000, None, ctypes.byref(t), pair, ctypes.byref(fixed)) == lib.CWT_EINVAL
    assert so.cwt_smooth_schedule(10000, rad, None, pair, ctypes.byref(fixed)) == lib.CWT_EINVAL
    assert so.cwt_smooth_schedule(10000, rad, ctypes.byref(t), None, ctypes.byref(fixed)) == lib.CWT_EINVAL
    assert so.cwt_smooth_schedule(10000, rad, ctypes.byref(t), pair, None) == lib.CWT_EINVAL
    assert so.cwt_smooth_schedule(-5, rad, ctypes.byref(t), pair, ctypes.byref(fixed)) == lib.CWT_EUNSUPPORTED


# The fixed-length kernels run only when the host scheduler picks exactly the
# schedule they were compiled for: pin that choice (and the inlined pair of
# the forward FFT) for each of them, on the host.
FIXED_SCHEDULES = {
    10000: ([16, 25, 25], 416, (0, 0)),
    8000: ([16, 25, 20], 416, (0, 0)),
    5000: ([20, 10, 25], 256, (0, 0)),
    4000: ([16, 10, 25], 256, (0, 0)),
    2500: ([25, 10, 10], 100, (0, 0)),
    2000: ([20, 10, 10], 100, (0, 0)),
    1000: ([10, 10, 10], 50, (10, 16)),
    500: ([20, 25], 25, (20, 25)),
    15000: ([10, 10, 10, 15], 512, (0, 0)),
    12000: ([16, 25, 30], 512, (0, 0)),
    9000: ([24, 15, 25], 384, (0, 0)),
    7500: ([25, 10, 30], 384, (0, 0)),
    6000: ([24, 10, 25], 256, (0, 0)),
    3000: ([24, 5, 25], 125, (0, 0)),
    1500: ([10, 10, 15], 50, (0, 0)),
    14000: ([14, 10, 10, 10], 512, (0, 0)),
    13500: ([6, 10, 15, 15], 512, (0, 0)),
    12500: ([10, 10, 5, 25], 512, (0, 0)),
    10500: ([28, 15, 25], 448, (0, 0)),
    7000: ([28, 10, 25], 288, (0, 0)),
    4500: ([10, 15, 30], 160, (0, 0)),
    3750: ([25, 6, 25], 256, (0, 0)),
    3500: ([28, 5, 25], 192, (0, 0)),
    2250: ([10, 15, 15], 75, (0, 0)),
    1750: ([14, 5, 25], 70, (0, 0)),
    1250: ([25, 10, 5], 50, (0, 0)),
    750: ([25, 30], 30, (0, 0)),
}


@pytest.mark.parametrize("N", sorted(FIXED_SCHEDULES))
def test_fixed_length_kernels_are_scheduled(lib, N):
    rad, threads, pair, fixed = lib.cwt_smooth_schedule(N)
    assert (rad, threads, pair, fixed) == FIXED_SCHEDULES[N] + (1,)


def test_smooth_schedules_on_the_host(lib):
    """Every schedulable smooth length below 16384: passes multiply to N, at
    most 32 values per thread and pass, T <= 512, and the pair kernels only
    where the pair's radices suffice; the lengths no schedule covers are
    refused."""
    seen_fixed = set()
    for N in range(32, 16385):
        x = N
        for f in (2, 3, 5, 7):
            while x % f == 0:
                x //= f
        if x != 1 or (N & (N - 1)) == 0:
            continue
        try:
            rad, T, pair, fixed = lib.cwt_smooth_schedule(N)
        except lib.CWTError as e:
            assert e.status == lib.CWT_EUNSUPPORTED and 14175 <= N <= 16200, N
            continue
        assert int(np.prod(rad)) == N and 1 <= T <= 512 and len(rad) >= 2
        for R in rad:
            assert 4 <= R <= 32 and (-(-(N // R) // T)) * R <= max(32, R), (N, rad, T)
        if pair != (0, 0):
            assert set(rad) <= set(pair), (N, rad, pair)
        if fixed:
            seen_fixed.add(N)
    assert seen_fixed == set(FIXED_SCHEDULES)
    for N in (1024, 3001 * 7 + 1, 20000, 16):
        with pytest.raises(lib.CWTError):
            lib.cwt_smooth_schedule(N)


def test_grid_check_boundary(lib):
    """The refusal is the 1e-150 floor on the sampled spectrum, not a rule on
    the carrier's bin: 6 Hz with sigma 5 in a 32-point window at 500 Hz (0.38
    of the first bin, peak ~1e-14 on the grid) passes the host-side checks and
    fails only for lack of a GPU here, while 2 Hz with sigma 12 is refused."""
    import torch
    o = lib.cwt_options_init()
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_plan_create(1, 32, 500.0, [2.0], [12.0], 0, lib.CWT_OUT_POWER, o)
    assert e.value.status == lib.CWT_EINVAL
    if torch.cuda.is_available():
        plan = lib.cwt_plan_create(1, 32, 500.0, [6.0], [5.0], 0, lib.CWT_OUT_POWER, o)
        lib.cwt_plan_destroy(plan)
    else:
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_plan_create(1, 32, 500.0, [6.0], [5.0], 0, lib.CWT_OUT_POWER, o)
        assert e.value.status != lib.CWT_EINVAL


@pytest.mark.parametrize("N", [6300, 42, 105000, 14175])
def test_specialize_check_compiles_on_the_host(lib, N):
    """The plan-time compiler builds the fixed-length kernels of a smooth
    length's one-CTA schedule (6300, 42), or the cluster kernels on its local
    length (105000 = 10 x 10500 on a non-portable cluster of 10 CTAs,
    14175 = 3 x 4725), from the embedded source, without a device."""
    assert lib.cwt_specialize_check(N) == ""  # no warnings either


@pytest.mark.parametrize("N", [4096, 78125, 31, 131072 * 2])
def test_specialize_check_refuses_other_lengths(lib, N):
    """Powers of two, smooth lengths with neither a schedule nor a split, and
    lengths outside [32, 131072] have nothing to specialize."""
    with pytest.raises(lib.CWTError) as e:
        lib.cwt_specialize_check(N)
    assert e.value.status == lib.CWT_EUNSUPPORTED


def _specialize_check_in_child(cache_dir, N):
    """cwt_specialize_check(N) in a fresh process with CWT_JIT_CACHE_DIR set;
    returns its wall time in seconds."""
    import subprocess
    import sys
    code = ("import time, paper_2506_07793_gb300 as p; t = time.perf_counter(); "
            f"assert p.cwt_specialize_check({N}) == ''; print(time.perf_counter() - t)")
    env = dict(os.environ, CWT_JIT_CACHE_DIR=str(cache_dir))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    return float(r.stdout.strip().splitlines()[-1])


def test_plan_time_module_cache_on_disk(lib, tmp_path):
    """CWT_JIT_CACHE_DIR keeps each plan-time compiled module on disk: a second
    process loads it instead of compiling (one file per schedule, no
    temporaries left), and a damaged file reads as a miss and is rewritten."""
    N = 6300
    t_compile = _specialize_check_in_child(tmp_path, N)
    files = sorted(tmp_path.iterdir())
    assert len(files) == 1 and files[0].name.startswith("cwt_jit_") and files[0].suffix == ".bin"
    good = files[0].read_bytes()
    assert good.startswith(b"cwt-jit-module 1\n") and b":6300/" in good.split(b"\n")[1]
    t_load = _specialize_check_in_child(tmp_path, N)
    assert t_load < 0.5 * t_compile, (t_load, t_compile)
    assert sorted(tmp_path.iterdir()) == files
    # a truncated file: a miss, compiled again and rewritten whole (the same
    # header; the compiler's output need not be byte-identical run to run)
    files[0].write_bytes(good[: len(good) // 2])
    _specialize_check_in_child(tmp_path, N)
    again = files[0].read_bytes()
    head = again.split(b"\n", 5)
    assert head[:4] == good.split(b"\n", 5)[:4] and int(head[4]) == len(head[5]) > 0
    # another schedule: a second file
    _specialize_check_in_child(tmp_path, 14175)
    assert len(list(tmp_path.iterdir())) == 2
