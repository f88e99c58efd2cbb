"""GPU parity of the batch path (cwt_execute_batch) against the FP64 oracle.

Each epoch is the plain transform of its own samples with padded length
N_e = next power of two >= max(n_e, 32); the oracle computes every epoch
separately with its own N_e.  Cases: a small batch of ragged lengths (1 up to
the 8192 maximum, powers of two and one past them) checked on every row for
several decimations, and the full batching workload (2048 epochs of
U{256..8192} samples x 64 channels, 64 scales, power decimated x4) in the
launch configuration the benchmark times, checked on sampled rows.
"""
import numpy as np
import pytest

import oracle
from eeg_synth import batch_signal, eeg, workload
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


def make_plan(lib, C, n_max, fs, freqs, cycles, kinds, d, edge=0):
    o = lib.cwt_options_init()
    o.decimation = d
    o.edge_mode = edge
    return lib.cwt_plan_create(C, n_max, fs, freqs, cycles, 0, kinds, o)


def test_linear_edges_batch(lib):
    """Linear edges in a batch: each epoch padded to a power of two >= n + R + 1."""
    import torch
    C, fs, d = 2, 500.0, 2
    freqs = np.array([6.0, 20.0, 70.0])
    cycles = np.array([5.0, 7.0, 9.0])
    R = int(np.ceil(6.5 * max(cycles / (2 * np.pi * freqs)) * fs))
    lengths = [40, 300, 1000, 3000]
    plan = make_plan(lib, C, 3000, fs, freqs, cycles, lib.CWT_OUT_POWER, d, edge=lib.CWT_EDGE_LINEAR)
    try:
        ep, n_in, n_o = lib.pack_epochs(lengths, C, len(freqs), d)
        xs = [eeg(600 + k, C, n, fs, np.float32) for k, n in enumerate(lengths)]
        x = torch.from_numpy(np.concatenate([a.reshape(-1) for a in xs])).cuda()
        pw = torch.full((n_o,), np.nan, dtype=torch.float32, device="cuda")
        lib.cwt_execute_batch(plan, ep, x, None, pw, None)
        torch.cuda.synchronize()
        pw = pw.cpu().numpy()
        for k, n in enumerate(lengths):
            N = lib.cwt_fft_length(n + R + 1)
            ref = oracle.cwt(xs[k].astype(np.float64), N, fs, freqs, cycles, decimation=d)
            no = -(-n // d)
            sl = slice(ep[k].out_offset, ep[k].out_offset + C * len(freqs) * no)
            assert power_err(pw[sl].reshape(C, len(freqs), no), ref).max() <= FP32_TOL
    finally:
        lib.cwt_plan_destroy(plan)


@pytest.mark.parametrize("d", [1, 3, 4])
def test_small_ragged_batch_every_row(lib, d):
    import torch
    C, fs = 3, 500.0
    # 3 Hz sits at 0.19 of the first bin of the 32-point epochs: an unresolved
    # row, checked like the others (the oracle takes the spectral side of
    # Poisson summation there)
    freqs = np.array([3.0, 6.0, 20.0, 70.0, 240.0])
    cycles = np.array([3.0, 5.0, 7.0, 9.0, 12.0])
    lengths = [1, 31, 32, 33, 100, 257, 1000, 2048, 4097, 8192, 640]
    kinds = lib.CWT_OUT_POWER | (lib.CWT_OUT_COMPLEX if d == 1 else 0)
    plan = make_plan(lib, C, 8192, fs, freqs, cycles, kinds, d)
    try:
        ep, n_in, n_o = lib.pack_epochs(lengths, C, len(freqs), d)
        xs = [eeg(500 + k, C, n, fs, np.float32) for k, n in enumerate(lengths)]
        x = torch.from_numpy(np.concatenate([a.reshape(-1) for a in xs])).cuda()
        pw = torch.full((n_o,), np.nan, dtype=torch.float32, device="cuda")
        cx = torch.empty((n_o,), dtype=torch.complex64, device="cuda") if d == 1 else None
        lib.cwt_execute_batch(plan, ep, x, cx, pw, None)
        torch.cuda.synchronize()
        pw = pw.cpu().numpy()
        cx = cx.cpu().numpy() if cx is not None else None
        for k, n in enumerate(lengths):
            N = lib.cwt_fft_length(n)
            ref = oracle.cwt(xs[k].astype(np.float64), N, fs, freqs, cycles, decimation=d)
            no = -(-n // d)
            sl = slice(ep[k].out_offset, ep[k].out_offset + C * len(freqs) * no)
            got = pw[sl].reshape(C, len(freqs), no)
            assert power_err(got, ref).max() <= FP32_TOL, (n, power_err(got, ref).max())
            if cx is not None:
                assert complex_err(cx[sl].reshape(C, len(freqs), no), ref).max() <= FP32_TOL
        st = lib.cwt_plan_batch_stats(plan)
        assert st.tuned == 1 and st.items > 0 and st.inverse_radix in (16, 32)
        if d % 2:  # an 8192-point inverse row: only the 32-point staging holds it
            assert st.inverse_radix == 32 and st.tune_ms[0] == -1.0 and st.tune_ms[2] == -1.0
    finally:
        lib.cwt_plan_destroy(plan)


def test_batching_workload_full_size_sampled_rows(lib):
    import torch
    w = workload("batch")
    lengths = w.extra["epoch_lengths"]
    C, S, d = w.channels, w.scales, w.decimation
    plan = make_plan(lib, C, 8192, w.fs, w.freqs, w.n_cycles, lib.CWT_OUT_POWER, d)
    try:
        ep, n_in, n_o = lib.pack_epochs(lengths, C, S, d)
        xn, offs, _ = batch_signal(w)
        assert len(xn) == n_in and all(int(offs[k]) == ep[k].in_offset for k in range(len(lengths)))
        xd = torch.from_numpy(xn).cuda()
        pw = torch.empty(n_o, dtype=torch.float32, device="cuda")
        for _ in range(2):  # first call tunes, second replays the graph
            lib.cwt_execute_batch(plan, ep, xd, None, pw, None)
        torch.cuda.synchronize()
        rng = np.random.default_rng(33)
        picks = [(int(np.argmax(lengths)), 0, 0), (int(np.argmin(lengths)), C - 1, S - 1)]
        picks += [(int(rng.integers(len(lengths))), int(rng.integers(C)), int(rng.integers(S)))
                  for _ in range(22)]
        for e_, c, s in picks:
            n = int(lengths[e_])
            N = lib.cwt_fft_length(n)
            xe = xn[ep[e_].in_offset:ep[e_].in_offset + C * n].reshape(C, n)
            ref = oracle.cwt_rows(xe.astype(np.float64), N, w.fs, w.freqs, w.n_cycles, [(c, s)],
                                  decimation=d)[0]
            no = -(-n // d)
            start = ep[e_].out_offset + (c * S + s) * no
            got = pw[start:start + no].cpu().numpy()
            assert power_err(got[None], ref[None]).max() <= FP32_TOL, (e_, c, s)
        st = lib.cwt_plan_batch_stats(plan)
        assert st.graph_launches >= 2 and st.tuned == 1
    finally:
        lib.cwt_plan_destroy(plan)


def test_batch_argument_checks(lib):
    import torch
    plan = make_plan(lib, 2, 1000, 500.0, [10.0], [7.0], lib.CWT_OUT_POWER, 1)
    try:
        x = torch.zeros(4000, device="cuda")
        out = torch.zeros(4000, device="cuda")
        ep, _, _ = lib.pack_epochs([1001], 2, 1, 1)
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_execute_batch(plan, ep, x, None, out, None)
        assert e.value.status == lib.CWT_EINVAL
        ep, _, _ = lib.pack_epochs([10], 2, 1, 1)
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_execute_batch(plan, ep, x, out, out, None)  # complex not requested
        assert e.value.status == lib.CWT_EINVAL
    finally:
        lib.cwt_plan_destroy(plan)
    plan = make_plan(lib, 1, 9000, 500.0, [10.0], [7.0], lib.CWT_OUT_POWER, 1)
    try:
        ep, _, _ = lib.pack_epochs([9000], 1, 1, 1)
        with pytest.raises(lib.CWTError) as e:
            lib.cwt_execute_batch(plan, ep, torch.zeros(9000, device="cuda"), None,
                                  torch.zeros(9000, device="cuda"), None)
        assert e.value.status == lib.CWT_EUNSUPPORTED
    finally:
        lib.cwt_plan_destroy(plan)


def test_batch_refuses_an_epoch_too_short_for_a_scale(lib):
    """1.5 Hz with 7 cycles is fine at the plan's 8192 points (500 Hz) but
    has a spectrum below 1e-150 on every bin of a 32-point epoch: the batch
    is refused before any device work, and a batch of long epochs still runs."""
    import torch
    C, fs, freqs, cycles = 1, 500.0, np.array([1.5, 20.0]), np.array([7.0, 7.0])
    plan = make_plan(lib, C, 8192, fs, freqs, cycles, lib.CWT_OUT_POWER, 1)
    try:
        for lengths, ok in (([4000, 20], False), ([4000, 3000], True)):
            ep, n_in, n_o = lib.pack_epochs(lengths, C, len(freqs), 1)
            x = torch.zeros((n_in,), dtype=torch.float32, device="cuda")
            pw = torch.zeros((n_o,), dtype=torch.float32, device="cuda")
            if ok:
                lib.cwt_execute_batch(plan, ep, x, None, pw, None)
                torch.cuda.synchronize()
            else:
                with pytest.raises(lib.CWTError) as e:
                    lib.cwt_execute_batch(plan, ep, x, None, pw, None)
                assert e.value.status == lib.CWT_EINVAL
    finally:
        lib.cwt_plan_destroy(plan)
