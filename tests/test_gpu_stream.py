"""GPU tests of the streaming server (overlap-save CWT on live windows).

* Each emitted hop equals the oracle's cyclic CWT power of its window
  x[e - W, e) (zeros before the first sample, N = W = 2048) at the H centred
  positions [W - D - H, W - D), D = floor((W - H) / 2), within 1e-5 of each
  row's peak power over that window.
* A stream's results are bitwise the same alone and batched together with
  other streams of different channel counts and sampling rates (continuous
  batching does not change a stream's arithmetic).
* Admission by slots and by device-memory budget, back-pressure and error codes.
"""
import numpy as np
import pytest

import oracle
from eeg_synth import eeg
from tests.metrics import FP32_TOL

pytestmark = pytest.mark.gpu

W = 2048
FREQS = np.geomspace(1.0, 100.0, 64)
CYCLES = np.full(64, 7.0)


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_07793_gb300 as p
    return p


def server(lib, max_streams=32, budget=0, wavelet=None, cycles=CYCLES, gamma=3.0):
    o = lib.cwt_server_options_init()
    o.max_streams = max_streams
    o.mem_budget_bytes = budget
    o.gmw_gamma = gamma
    wv = lib.CWT_WAVELET_MORLET if wavelet is None else wavelet
    return lib.cwt_server_create(FREQS, cycles, wv, o)


def feed(lib, srv, sid, x, chunks, H, C, S):
    """Push x in the given chunk sizes, stepping and pulling as we go.
    Returns {hop_first_sample: [C][S][H] power}."""
    out = {}
    buf = np.empty((16, C, S, H), np.float32)
    pos = 0
    for k in chunks:
        lib.cwt_stream_push(srv, sid, x[:, pos:pos + k])
        pos += k
        lib.cwt_server_step(srv)
        lib.cwt_server_sync(srv)
        while True:
            n, first = lib.cwt_stream_pull(srv, sid, buf)
            if n == 0:
                break
            for h in range(n):
                out[first + h * H] = buf[h].copy()
    return out


def hop_reference(x, e, H, fs, wavelet="morlet", cycles=CYCLES, gamma=3.0):
    """Oracle coefficients of the hop, and each row's peak power over the
    whole window.  Errors are normalised by the window peak: the FFT's
    rounding scales with the window, while inside one hop the true values can
    be ~0 (e.g. a short wavelet centred before the first sample)."""
    D = (W - H) // 2
    win = np.zeros((x.shape[0], W))
    lo = e - W
    seg = x[:, max(lo, 0):e]
    win[:, W - seg.shape[1]:] = seg
    c = oracle.cwt(win, W, fs, FREQS, cycles, wavelet=wavelet, gamma=gamma)
    return c[..., W - D - H:W - D], oracle.power(c).max(axis=-1)


def test_gmw_hops_match_oracle(lib):
    """The server with the generalized Morse wavelet (Eq. 5; beta 20, gamma 3)."""
    fs, C = 1000.0, 2
    H = 50
    betas = np.full(len(FREQS), 20.0)
    x = eeg(702, C, 10 * H, fs, np.float32)
    srv = server(lib, wavelet=lib.CWT_WAVELET_GMW, cycles=betas, gamma=3.0)
    try:
        sid = lib.cwt_stream_open(srv, C, fs)
        out = feed(lib, srv, sid, x, [3 * H, 3 * H, 4 * H], H, C, len(FREQS))
        assert len(out) == 10
        D = (W - H) // 2
        for first in sorted(out)[::4]:
            ref, peak = hop_reference(x.astype(np.float64), first + D + H, H, fs, "gmw", betas, 3.0)
            err = np.abs(out[first] - oracle.power(ref)).max(axis=-1) / peak
            assert err.max() <= FP32_TOL, (first, err.max())
    finally:
        lib.cwt_server_destroy(srv)


def test_hops_match_oracle(lib):
    fs, C = 500.0, 3
    H = int(np.ceil(fs * 0.05))
    x = eeg(700, C, 12 * H + 7, fs, np.float32)
    srv = server(lib)
    try:
        sid = lib.cwt_stream_open(srv, C, fs)
        rng = np.random.default_rng(1)
        chunks, tot = [], 0
        while tot < x.shape[1]:
            k = int(min(rng.integers(1, 2 * H), x.shape[1] - tot))
            chunks.append(k)
            tot += k
        out = feed(lib, srv, sid, x, chunks, H, C, len(FREQS))
        assert len(out) == x.shape[1] // H
        D = (W - H) // 2
        for first in sorted(out)[::3]:
            e = first + D + H
            ref, peak = hop_reference(x.astype(np.float64), e, H, fs)
            err = np.abs(out[first] - oracle.power(ref)).max(axis=-1) / peak
            assert err.max() <= FP32_TOL, (first, err.max())
        st = lib.cwt_server_stats(srv)
        assert st.hops == len(out) and st.latency_p99_s > 0
    finally:
        lib.cwt_server_destroy(srv)


def test_alone_equals_in_the_mix(lib):
    fs, C = 1000.0, 8
    H = 50
    x = eeg(701, C, 30 * H, fs, np.float32)
    chunks = [37, 120, 5, 300, 88, 399, 400]  # each push carries at most 8 hops (8 * H)
    srv = server(lib)
    try:
        sid = lib.cwt_stream_open(srv, C, fs)
        alone = feed(lib, srv, sid, x, chunks, H, C, len(FREQS))
    finally:
        lib.cwt_server_destroy(srv)
    srv = server(lib)
    try:
        others = []
        for i, (c2, f2) in enumerate([(32, 250.0), (64, 2000.0), (16, 4000.0), (3, 500.0)]):
            oid = lib.cwt_stream_open(srv, c2, f2)
            others.append((oid, eeg(800 + i, c2, 4000, f2, np.float32), int(np.ceil(f2 * 0.05)), c2))
        sid = lib.cwt_stream_open(srv, C, fs)
        mixed = {}
        buf = np.empty((16, C, len(FREQS), H), np.float32)
        obuf = {o[0]: np.empty((16, o[3], len(FREQS), o[2]), np.float32) for o in others}
        pos = 0
        opos = 0
        for k in chunks:
            for oid, ox, oh, oc in others:  # interleave the other streams' pushes
                kk = min(oh, ox.shape[1] - opos)
                if kk > 0:
                    lib.cwt_stream_push(srv, oid, ox[:, opos:opos + kk])
            opos += 50
            lib.cwt_stream_push(srv, sid, x[:, pos:pos + k])
            pos += k
            lib.cwt_server_step(srv)
            lib.cwt_server_sync(srv)
            for oid, _, _, _ in others:
                while lib.cwt_stream_pull(srv, oid, obuf[oid])[0]:
                    pass
            while True:
                n, first = lib.cwt_stream_pull(srv, sid, buf)
                if n == 0:
                    break
                for h in range(n):
                    mixed[first + h * H] = buf[h].copy()
        assert sorted(mixed) == sorted(alone)
        for key in alone:
            assert np.array_equal(mixed[key], alone[key])
    finally:
        lib.cwt_server_destroy(srv)


def test_admission_by_slots_and_budget(lib):
    srv = server(lib, max_streams=2)
    try:
        a = lib.cwt_stream_open(srv, 8, 500.0)
        b = lib.cwt_stream_open(srv, 8, 500.0)
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_stream_open(srv, 8, 500.0)
        assert e.value.status == lib.CWT_EBUSY
        lib.cwt_stream_close(srv, a)
        c = lib.cwt_stream_open(srv, 8, 500.0)  # the freed slot is reused
        assert c == a and b != a
        st = lib.cwt_server_stats(srv)
        assert (st.admitted, st.refused, st.open_streams) == (3, 1, 2)
    finally:
        lib.cwt_server_destroy(srv)
    srv = server(lib, budget=64 << 20)
    try:
        lib.cwt_stream_open(srv, 8, 250.0)
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_stream_open(srv, 256, 4000.0)  # its batch buffers alone exceed 64 MB
        assert e.value.status == lib.CWT_EBUSY
    finally:
        lib.cwt_server_destroy(srv)


def test_backpressure_and_errors(lib):
    srv = server(lib)
    try:
        sid = lib.cwt_stream_open(srv, 2, 1000.0)
        buf = np.empty((4, 2, 64, 50), np.float32)
        assert lib.cwt_stream_pull(srv, sid, buf) == (0, None)       # nothing yet
        for _ in range(8):
            lib.cwt_stream_push(srv, sid, np.zeros((2, 50), np.float32))
        with pytest.raises(lib.CWTError) as e:                          # 8 hops unpulled
            lib.cwt_stream_push(srv, sid, np.zeros((2, 50), np.float32))
        assert e.value.status == lib.CWT_EBUSY
        assert lib.cwt_server_step(srv) == 8
        lib.cwt_server_sync(srv)
        n, first = lib.cwt_stream_pull(srv, sid, buf)
        assert n == 4 and first == 50 - (W - 50) // 2 - 50
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_stream_open(srv, 2, 150.0)  # 100 Hz scale above Nyquist
        assert e.value.status == lib.CWT_EINVAL
        with pytest.raises(lib.CWTError):
            lib.cwt_stream_push(srv, 31, np.zeros((2, 5), np.float32))  # not open
    finally:
        lib.cwt_server_destroy(srv)


def test_stream_refused_when_the_window_cannot_hold_a_scale(lib):
    """A 0.1 Hz scale with 7 cycles has a spectrum below 1e-150 on every bin
    of the 2048-point window at 4 kHz (first bin 1.95 Hz): such a stream is
    refused (CWT_EINVAL, not counted as an admission refusal), while the same
    scales at 250 Hz (first bin 0.12 Hz) are admitted."""
    o = lib.cwt_server_options_init()
    srv = lib.cwt_server_create(np.array([0.1, 10.0]), np.array([7.0, 7.0]), lib.CWT_WAVELET_MORLET, o)
    try:
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_stream_open(srv, 2, 4000.0)
        assert e.value.status == lib.CWT_EINVAL
        sid = lib.cwt_stream_open(srv, 2, 250.0)
        lib.cwt_stream_close(srv, sid)
    finally:
        lib.cwt_server_destroy(srv)
