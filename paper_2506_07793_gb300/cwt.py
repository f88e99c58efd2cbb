"""Thin ctypes binding of libcwt_gb300.so (include/cwt.h), same names as the C ABI.

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels.  torch is used for device memory and streams (a tensor's
data_ptr() and torch.cuda.current_stream().cuda_stream are passed as plain
pointers).  If the library has not been built, importing this module raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CWT_GB300_LIB selects another build of the library (the bounds-checked
# variant, _lib/libcwt_gb300_check.so); default the ordinary one.
LIB_PATH = os.environ.get("CWT_GB300_LIB") or os.path.join(_HERE, "_lib", "libcwt_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()'). There is no CPU fallback.")

_lib = ctypes.CDLL(LIB_PATH)

# ---- constants (mirror include/cwt.h) ----
CWT_OK, CWT_EINVAL, CWT_ENOMEM, CWT_EUNSUPPORTED, CWT_ECUDA = 0, 1, 2, 3, 4
CWT_EAGAIN, CWT_EBUSY, CWT_EDEVICE = 5, 6, 8
CWT_WAVELET_MORLET, CWT_WAVELET_GABOR, CWT_WAVELET_GMW = 0, 1, 2
CWT_EDGE_CYCLIC, CWT_EDGE_LINEAR = 0, 1
CWT_OUT_COMPLEX, CWT_OUT_POWER, CWT_OUT_PHASE = 1, 2, 4
CWT_PREC_FP32, CWT_PREC_TC_FP16, CWT_PREC_TC_BF16 = 0, 1, 2
CWT_DTYPE_F32, CWT_DTYPE_F64 = 0, 1
CWT_PAD_POW2, CWT_PAD_SMOOTH = 0, 1
CWT_NORM_UNIT_ENERGY, CWT_NORM_MNE = 0, 1
CWT_KERNEL_BANK, CWT_KERNEL_FORWARD_FFT, CWT_KERNEL_SCALE_BLOCK, CWT_KERNEL_BATCH = 0, 1, 2, 3


class cwt_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("decimation", ctypes.c_int),
                ("pad_policy", ctypes.c_int), ("fft_length", ctypes.c_int),
                ("io_dtype", ctypes.c_int), ("edge_mode", ctypes.c_int),
                ("gmw_gamma", ctypes.c_double), ("normalization", ctypes.c_int),
                ("specialize", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class cwt_plan_info_t(ctypes.Structure):
    _fields_ = [("channels", ctypes.c_int), ("samples", ctypes.c_int), ("scales", ctypes.c_int),
                ("fft_length", ctypes.c_int), ("n_out", ctypes.c_int), ("decimation", ctypes.c_int),
                ("fold", ctypes.c_int), ("inverse_length", ctypes.c_int), ("device", ctypes.c_int),
                ("io_dtype", ctypes.c_int), ("output_kinds", ctypes.c_uint),
                ("workspace_bytes", ctypes.c_size_t), ("bank_ms", ctypes.c_double),
                ("radices", ctypes.c_int * 8), ("inlined_pair", ctypes.c_int * 2),
                ("fixed_kernel", ctypes.c_int), ("precision", ctypes.c_int),
                ("cluster", ctypes.c_int), ("specialized", ctypes.c_int)]


class cwt_epoch(ctypes.Structure):
    _fields_ = [("in_offset", ctypes.c_longlong), ("out_offset", ctypes.c_longlong),
                ("samples", ctypes.c_int), ("reserved", ctypes.c_int)]


class cwt_batch_stats(ctypes.Structure):
    _fields_ = [("items", ctypes.c_int), ("grid", ctypes.c_int), ("inverse_radix", ctypes.c_int),
                ("order", ctypes.c_int), ("tuned", ctypes.c_int), ("reserved", ctypes.c_int),
                ("tune_ms", ctypes.c_double * 4), ("graph_launches", ctypes.c_longlong),
                ("bank_bytes", ctypes.c_size_t)]


class cwt_server_options(ctypes.Structure):
    _fields_ = [("max_streams", ctypes.c_int), ("window", ctypes.c_int),
                ("hop_seconds", ctypes.c_double), ("mem_budget_bytes", ctypes.c_size_t),
                ("output_kinds", ctypes.c_uint), ("reserved0", ctypes.c_int),
                ("gmw_gamma", ctypes.c_double), ("reserved", ctypes.c_int * 4)]


class cwt_server_stats_t(ctypes.Structure):
    _fields_ = [("open_streams", ctypes.c_int), ("reserved", ctypes.c_int),
                ("admitted", ctypes.c_longlong), ("refused", ctypes.c_longlong),
                ("hops", ctypes.c_longlong), ("launches", ctypes.c_longlong),
                ("coefficients", ctypes.c_longlong), ("device_bytes", ctypes.c_size_t),
                ("latency_p50_s", ctypes.c_double), ("latency_p99_s", ctypes.c_double),
                ("latency_max_s", ctypes.c_double), ("latency_mean_s", ctypes.c_double),
                ("span_s", ctypes.c_double)]


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("cwt_status_str", ctypes.c_char_p, [ctypes.c_int])
_sig("cwt_options_init", ctypes.c_int, [ctypes.POINTER(cwt_options)])
_sig("cwt_fft_length", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _ip])
_sig("cwt_smooth_schedule", ctypes.c_int, [ctypes.c_int, _ip, _ip, _ip, _ip])
_sig("cwt_smooth_cluster", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _ip, _ip, _ip])
_sig("cwt_specialize_check", ctypes.c_int, [ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t])
_sig("cwt_support_radius", ctypes.c_int,
     [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _ip])
_sig("cwt_plan_create", ctypes.c_int,
     [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, ctypes.c_int, _dp,
      ctypes.c_int, ctypes.c_uint, ctypes.POINTER(cwt_options)])
_sig("cwt_plan_destroy", ctypes.c_int, [_vp])
_sig("cwt_plan_info", ctypes.c_int, [_vp, ctypes.POINTER(cwt_plan_info_t)])
_sig("cwt_plan_workspace_bytes", ctypes.c_size_t, [_vp])
_sig("cwt_plan_last_error", ctypes.c_char_p, [_vp])
_sig("cwt_execute", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp])
_sig("cwt_execute_host", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp])
_sig("cwt_plan_bank", ctypes.c_int, [_vp, _fp, _ip, _ip])
_sig("cwt_fft", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp])
_sig("cwt_measure_peak", ctypes.c_int, [ctypes.c_int, _dp])
_sig("cwt_execute_noalloc", ctypes.c_int,
     [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_int, _vp, _vp, _vp, _vp])
_sig("cwt_execute_batch", ctypes.c_int,
     [_vp, ctypes.POINTER(cwt_epoch), ctypes.c_int, _vp, _vp, _vp, _vp, _vp])
_sig("cwt_plan_batch_stats", ctypes.c_int, [_vp, ctypes.POINTER(cwt_batch_stats)])
_sig("cwt_server_options_init", ctypes.c_int, [ctypes.POINTER(cwt_server_options)])
_sig("cwt_server_create", ctypes.c_int, [ctypes.POINTER(_vp), _dp, _dp, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(cwt_server_options)])
_sig("cwt_server_destroy", ctypes.c_int, [_vp])
_sig("cwt_stream_open", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, _ip])
_sig("cwt_stream_push", ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int])
_sig("cwt_server_step", ctypes.c_int, [_vp, _ip])
_sig("cwt_server_sync", ctypes.c_int, [_vp])
_sig("cwt_stream_pull", ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _ip,
                                       ctypes.POINTER(ctypes.c_longlong)])
_sig("cwt_stream_close", ctypes.c_int, [_vp, ctypes.c_int])
_sig("cwt_server_stats", ctypes.c_int, [_vp, ctypes.POINTER(cwt_server_stats_t)])
_sig("cwt_server_reset_stats", ctypes.c_int, [_vp])
_sig("cwt_plan_set_profiling", ctypes.c_int, [_vp, ctypes.c_int])
_sig("cwt_plan_profile_read", ctypes.c_int,
     [_vp, ctypes.c_int, _ip, _dp, ctypes.c_int])


class CWTError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {cwt_status_str(status)}")


def _check(status, what):
    if status != CWT_OK:
        raise CWTError(status, what)


def _ptr(x):
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- the C ABI, same names ----

def cwt_status_str(status):
    return _lib.cwt_status_str(int(status)).decode()


def cwt_options_init():
    o = cwt_options()
    _check(_lib.cwt_options_init(ctypes.byref(o)), "cwt_options_init")
    return o


def cwt_fft_length(samples, pad_policy=CWT_PAD_POW2):
    n = ctypes.c_int(0)
    _check(_lib.cwt_fft_length(int(samples), int(pad_policy), ctypes.byref(n)), "cwt_fft_length")
    return n.value


def cwt_smooth_schedule(n_fft):
    """(radices, threads per row, inlined pair, fixed_kernel) of a smooth length."""
    rad = (ctypes.c_int * 8)()
    pair = (ctypes.c_int * 2)()
    t, fixed = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib.cwt_smooth_schedule(int(n_fft), rad, ctypes.byref(t), pair, ctypes.byref(fixed)),
           "cwt_smooth_schedule")
    return [r for r in rad if r], t.value, (pair[0], pair[1]), fixed.value


def cwt_smooth_cluster(n_fft, specialize=0):
    """(cluster, radices, fixed_kernel) of a smooth length's row layout."""
    rad = (ctypes.c_int * 8)()
    cl, fixed = ctypes.c_int(0), ctypes.c_int(0)
    _check(_lib.cwt_smooth_cluster(int(n_fft), int(specialize), ctypes.byref(cl), rad, ctypes.byref(fixed)),
           "cwt_smooth_cluster")
    return cl.value, [r for r in rad if r], fixed.value


def cwt_support_radius(wavelet, freq_hz, n_cycles, fs, gmw_gamma=3.0):
    """Support radius in samples (envelope below 1e-9 of its peak beyond it)."""
    r = ctypes.c_int(0)
    _check(_lib.cwt_support_radius(int(wavelet), float(freq_hz), float(n_cycles), float(gmw_gamma),
                                   float(fs), ctypes.byref(r)), "cwt_support_radius")
    return r.value


def cwt_specialize_check(n_fft):
    """Compile (host only, for sm_103a) the fixed-length kernels of the one-CTA
    schedule of n_fft that cwt_options.specialize would build; returns the
    compiler's log.  Raises CWTError (CWT_EUNSUPPORTED: no such schedule;
    CWT_ECUDA: the compile failed, log in the message)."""
    buf = ctypes.create_string_buffer(1 << 16)
    st = _lib.cwt_specialize_check(int(n_fft), buf, ctypes.sizeof(buf))
    if st != CWT_OK:
        raise CWTError(st, f"cwt_specialize_check({n_fft}): {buf.value.decode(errors='replace')[:2000]}")
    return buf.value.decode(errors="replace")


def cwt_plan_create(channels, samples, fs, freqs_hz, n_cycles, wavelet=CWT_WAVELET_MORLET,
                    output_kinds=CWT_OUT_POWER, options=None):
    """Returns an opaque plan handle (int).  Raises CWTError on failure."""
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64).reshape(-1))
    c = np.ascontiguousarray(np.broadcast_to(np.asarray(n_cycles, dtype=np.float64), f.shape))
    h = _vp()
    st = _lib.cwt_plan_create(ctypes.byref(h), int(channels), int(samples), float(fs),
                              f.ctypes.data_as(_dp), len(f), c.ctypes.data_as(_dp), int(wavelet),
                              int(output_kinds), ctypes.byref(options) if options is not None else None)
    _check(st, "cwt_plan_create")
    return h.value


def cwt_plan_destroy(plan):
    _check(_lib.cwt_plan_destroy(plan), "cwt_plan_destroy")


def cwt_plan_info(plan):
    info = cwt_plan_info_t()
    _check(_lib.cwt_plan_info(plan, ctypes.byref(info)), "cwt_plan_info")
    return info


def cwt_plan_workspace_bytes(plan):
    return int(_lib.cwt_plan_workspace_bytes(plan))


def cwt_plan_last_error(plan):
    return _lib.cwt_plan_last_error(plan).decode()


def cwt_execute(plan, signal, complex_out=None, power_out=None, phase_out=None, stream=None):
    st = _lib.cwt_execute(plan, _ptr(signal), _ptr(complex_out), _ptr(power_out), _ptr(phase_out),
                          _stream(stream))
    _check(st, "cwt_execute")


def cwt_execute_host(plan, signal, complex_out=None, power_out=None, phase_out=None, stream=None):
    st = _lib.cwt_execute_host(plan, _ptr(signal), _ptr(complex_out), _ptr(power_out),
                               _ptr(phase_out), _stream(stream))
    _check(st, "cwt_execute_host")


def cwt_plan_bank(plan):
    """(bank [S][N] float32, band_start [S], band_len [S]) copied to host."""
    info = cwt_plan_info(plan)
    bank = np.empty((info.scales, info.fft_length), dtype=np.float32)
    start = np.empty(info.scales, dtype=np.int32)
    length = np.empty(info.scales, dtype=np.int32)
    _check(_lib.cwt_plan_bank(plan, bank.ctypes.data_as(_fp), start.ctypes.data_as(_ip),
                              length.ctypes.data_as(_ip)), "cwt_plan_bank")
    return bank, start, length


def cwt_fft(d_in, d_out, n, batch, direction, stream=None):
    _check(_lib.cwt_fft(_ptr(d_in), _ptr(d_out), int(n), int(batch), int(direction),
                        _stream(stream)), "cwt_fft")


def cwt_measure_peak(what):
    """Measured TFLOP/s of the current GPU: 0 FP32 FMA, 1 mma.sync FP16, 2 mma.sync BF16."""
    v = ctypes.c_double()
    _check(_lib.cwt_measure_peak(int(what), ctypes.byref(v)), "cwt_measure_peak")
    return v.value


def cwt_execute_noalloc(signal, channels, samples, fs, freqs_hz, n_cycles, complex_out=None,
                        power_out=None, phase_out=None, stream=None):
    """The transform without any GPU allocation (for callers that may not
    allocate while running, e.g. real-time loops); see include/cwt.h."""
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64).reshape(-1))
    c = np.ascontiguousarray(np.broadcast_to(np.asarray(n_cycles, dtype=np.float64), f.shape))
    st = _lib.cwt_execute_noalloc(_ptr(signal), int(channels), int(samples), float(fs),
                                  f.ctypes.data_as(_dp), c.ctypes.data_as(_dp), len(f),
                                  _ptr(complex_out), _ptr(power_out), _ptr(phase_out),
                                  _stream(stream))
    _check(st, "cwt_execute_noalloc")


def pack_epochs(lengths, channels, scales, decimation=1):
    """Packed layout for cwt_execute_batch: epochs back to back, each epoch's
    signal [C][n_e] and outputs [C][S][ceil(n_e/d)].  Returns (epochs array,
    total input elements, total output elements per output array)."""
    arr = (cwt_epoch * len(lengths))()
    i_off = o_off = 0
    for k, n in enumerate(lengths):
        n = int(n)
        arr[k].in_offset, arr[k].out_offset, arr[k].samples = i_off, o_off, n
        i_off += channels * n
        o_off += channels * scales * (-(-n // decimation))
    return arr, i_off, o_off


def cwt_execute_batch(plan, epochs, d_in, complex_out=None, power_out=None, phase_out=None,
                      stream=None):
    st = _lib.cwt_execute_batch(plan, epochs, len(epochs), _ptr(d_in), _ptr(complex_out),
                                _ptr(power_out), _ptr(phase_out), _stream(stream))
    _check(st, "cwt_execute_batch")


def cwt_plan_batch_stats(plan):
    s = cwt_batch_stats()
    _check(_lib.cwt_plan_batch_stats(plan, ctypes.byref(s)), "cwt_plan_batch_stats")
    return s


def cwt_plan_set_profiling(plan, enable):
    _check(_lib.cwt_plan_set_profiling(plan, int(bool(enable))), "cwt_plan_set_profiling")


def cwt_plan_profile_read(plan, kernel, reset=True):
    """(launches, total_ms) of one kernel since the last reset."""
    n = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(_lib.cwt_plan_profile_read(plan, int(kernel), ctypes.byref(n), ctypes.byref(ms),
                                      int(bool(reset))), "cwt_plan_profile_read")
    return n.value, ms.value


# ---- convenience wrapper over torch tensors ----

_KIND_BITS = {"complex": CWT_OUT_COMPLEX, "power": CWT_OUT_POWER, "phase": CWT_OUT_PHASE}


class CWT:
    """A plan plus torch output allocation.

    >>> t = CWT(channels=64, samples=10000, fs=1000.0, freqs=f, n_cycles=c,
    ...         outputs=("complex", "power"))
    >>> out = t(x_cuda)          # dict of torch tensors [C][S][n_out]
    """

    def __init__(self, channels, samples, fs, freqs, n_cycles, outputs=("power",),
                 wavelet="morlet", dtype="f32", decimation=1, fft_length=0, pad="pow2",
                 gmw_gamma=3.0, edge="cyclic", precision="fp32", normalization="unit",
                 specialize=False):
        opt = cwt_options_init()
        opt.normalization = {"unit": CWT_NORM_UNIT_ENERGY, "mne": CWT_NORM_MNE}[normalization]
        opt.specialize = int(specialize)  # False / True / 2 (tune)
        opt.precision = {"fp32": CWT_PREC_FP32, "tc_fp16": CWT_PREC_TC_FP16,
                         "tc_bf16": CWT_PREC_TC_BF16}[precision]
        opt.decimation = int(decimation)
        opt.pad_policy = {"pow2": CWT_PAD_POW2, "smooth": CWT_PAD_SMOOTH}[pad]
        opt.gmw_gamma = float(gmw_gamma)
        opt.edge_mode = {"cyclic": CWT_EDGE_CYCLIC, "linear": CWT_EDGE_LINEAR}[edge]
        opt.io_dtype = CWT_DTYPE_F64 if dtype in ("f64", "float64") else CWT_DTYPE_F32
        opt.fft_length = int(fft_length)
        kinds = 0
        for o in outputs:
            kinds |= _KIND_BITS[o]
        wv = {"morlet": CWT_WAVELET_MORLET, "gabor": CWT_WAVELET_GABOR, "gmw": CWT_WAVELET_GMW}[wavelet]
        self.outputs = tuple(outputs)
        self.dtype = "f64" if opt.io_dtype == CWT_DTYPE_F64 else "f32"
        self.plan = cwt_plan_create(channels, samples, fs, freqs, n_cycles, wv, kinds, opt)
        self.info = cwt_plan_info(self.plan)

    def close(self):
        if self.plan:
            cwt_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_outputs(self, device=None):
        import torch
        i = self.info
        shape = (i.channels, i.scales, i.n_out)
        rt = torch.float64 if self.dtype == "f64" else torch.float32
        ct = torch.complex128 if self.dtype == "f64" else torch.complex64
        dev = device if device is not None else torch.device("cuda", i.device)
        out = {}
        for o in self.outputs:
            out[o] = torch.empty(shape, dtype=ct if o == "complex" else rt, device=dev)
        return out

    def __call__(self, signal, out=None, stream=None):
        if out is None:
            out = self.alloc_outputs(signal.device)
        cwt_execute(self.plan, signal, out.get("complex"), out.get("power"), out.get("phase"),
                    stream)
        return out


# ---- streaming server ----

def cwt_server_options_init():
    o = cwt_server_options()
    _check(_lib.cwt_server_options_init(ctypes.byref(o)), "cwt_server_options_init")
    return o


def cwt_server_create(freqs_hz, n_cycles, wavelet=CWT_WAVELET_MORLET, options=None):
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64).reshape(-1))
    c = np.ascontiguousarray(np.broadcast_to(np.asarray(n_cycles, dtype=np.float64), f.shape))
    h = _vp()
    _check(_lib.cwt_server_create(ctypes.byref(h), f.ctypes.data_as(_dp), c.ctypes.data_as(_dp),
                                  len(f), int(wavelet),
                                  ctypes.byref(options) if options is not None else None),
           "cwt_server_create")
    return h.value


def cwt_server_destroy(srv):
    _check(_lib.cwt_server_destroy(srv), "cwt_server_destroy")


def cwt_stream_open(srv, channels, fs):
    i = ctypes.c_int(-1)
    _check(_lib.cwt_stream_open(srv, int(channels), float(fs), ctypes.byref(i)), "cwt_stream_open")
    return i.value


def cwt_stream_push(srv, stream_id, samples):
    """samples: [C][k] float32 (numpy, C-contiguous, or a torch tensor)."""
    if isinstance(samples, np.ndarray):
        samples = np.ascontiguousarray(samples, dtype=np.float32)
        k = samples.shape[-1]
    else:
        k = samples.shape[-1]
    _check(_lib.cwt_stream_push(srv, int(stream_id), _ptr(samples), int(k)), "cwt_stream_push")


def cwt_server_step(srv):
    n = ctypes.c_int(0)
    _check(_lib.cwt_server_step(srv, ctypes.byref(n)), "cwt_server_step")
    return n.value


def cwt_server_sync(srv):
    _check(_lib.cwt_server_sync(srv), "cwt_server_sync")


def cwt_stream_pull(srv, stream_id, out):
    """Fill `out` ([max_hops][C][S][H] float32, C-contiguous) with completed
    hops; returns (n_hops, first_sample) -- (0, None) when none is ready."""
    n = ctypes.c_int(0)
    first = ctypes.c_longlong(0)
    st = _lib.cwt_stream_pull(srv, int(stream_id), _ptr(out), int(out.shape[0]), ctypes.byref(n),
                              ctypes.byref(first))
    if st == CWT_EAGAIN:
        return 0, None
    _check(st, "cwt_stream_pull")
    return n.value, first.value


def cwt_stream_close(srv, stream_id):
    _check(_lib.cwt_stream_close(srv, int(stream_id)), "cwt_stream_close")


def cwt_server_stats(srv):
    s = cwt_server_stats_t()
    _check(_lib.cwt_server_stats(srv, ctypes.byref(s)), "cwt_server_stats")
    return s


def cwt_server_reset_stats(srv):
    _check(_lib.cwt_server_reset_stats(srv), "cwt_server_reset_stats")
