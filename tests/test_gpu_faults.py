"""Out-of-memory paths, by host-side failure injection (no GPU fault).

CWT_FAULT_ALLOC_AT=k makes the k-th allocation the library makes (after the
variable last changed) fail as out of memory before any CUDA call (csrc/alloc.cu).
Each case walks k over every allocation of an entry point: the call must
return CWT_ENOMEM, leave nothing allocated (device free memory back where it
was) and leave the library usable -- the same call then succeeds and its
result matches the oracle."""
import os

import numpy as np
import pytest

import oracle
from eeg_synth import eeg
from tests.metrics import FP32_TOL, power_err

pytestmark = pytest.mark.gpu

SLACK = 2 << 20  # allocation granularity of the driver


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_07793_gb300 as p
    return p


@pytest.fixture
def inject():
    def set_(k, tag):
        os.environ["CWT_FAULT_ALLOC_AT"] = f"{k}:{tag}"
    yield set_
    os.environ.pop("CWT_FAULT_ALLOC_AT", None)


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def walk(lib, inject, tag, call, max_k=40):
    """Fail allocation k = 1, 2, ... of call() until it succeeds; returns its result."""
    for k in range(1, max_k):
        before = free_bytes()
        inject(k, tag)
        try:
            out = call()
        except lib.CWTError as e:
            assert e.status == lib.CWT_ENOMEM, (tag, k, e.status)
            assert free_bytes() >= before - SLACK, (tag, k, "leak")
            continue
        finally:
            os.environ.pop("CWT_FAULT_ALLOC_AT", None)
        assert k > 1, f"{tag}: no allocation was made"
        return out
    raise AssertionError(f"{tag}: still failing after {max_k} allocations")


@pytest.mark.parametrize("precision", ["fp32", "tc_fp16"])
def test_plan_create_and_host_execute_enomem(lib, inject, precision):
    import torch
    C, n, fs = 2, 20000 if precision != "fp32" else 700, 1000.0
    freqs, cycles = np.array([6.0, 40.0]), np.array([7.0, 7.0])
    x = eeg(1500, C, n, fs, np.float32)

    def create():
        return lib.CWT(C, n, fs, freqs, cycles, outputs=("power",), precision=precision)
    t = walk(lib, inject, "create-" + precision, create)
    try:
        h_in = torch.from_numpy(x)
        h_out = torch.empty((C, 2, n), dtype=torch.float32)   # pageable: staged through the device

        def host_call():
            lib.cwt_execute_host(t.plan, h_in, None, h_out, None, None)
            return True
        walk(lib, inject, "host-" + precision, host_call)
        ref = oracle.cwt(x.astype(np.float64), t.info.fft_length, fs, freqs, cycles)
        tol = FP32_TOL if precision == "fp32" else 2e-3
        assert power_err(h_out.numpy(), ref).max() <= tol
    finally:
        t.close()


def test_batch_new_shape_enomem(lib, inject):
    import torch
    C, fs = 2, 500.0
    freqs, cycles = np.array([6.0, 20.0]), np.array([5.0, 7.0])
    o = lib.cwt_options_init()
    plan = lib.cwt_plan_create(C, 3000, fs, freqs, cycles, 0, lib.CWT_OUT_POWER, o)
    try:
        lengths = [300, 3000, 1000]
        ep, n_in, n_o = lib.pack_epochs(lengths, C, len(freqs), 1)
        xs = [eeg(1600 + k, C, n, fs, np.float32) for k, n in enumerate(lengths)]
        x = torch.from_numpy(np.concatenate([a.reshape(-1) for a in xs])).cuda()
        pw = torch.zeros((n_o,), dtype=torch.float32, device="cuda")

        def run():
            lib.cwt_execute_batch(plan, ep, x, None, pw, None)
            torch.cuda.synchronize()
            return True
        walk(lib, inject, "batch", run)
        p = pw.cpu().numpy()
        for k, n in enumerate(lengths):
            ref = oracle.cwt(xs[k].astype(np.float64), lib.cwt_fft_length(n), fs, freqs, cycles)
            got = p[ep[k].out_offset:ep[k].out_offset + C * 2 * n].reshape(C, 2, n)
            assert power_err(got, ref).max() <= FP32_TOL
    finally:
        lib.cwt_plan_destroy(plan)


def test_stream_open_enomem_keeps_the_server_usable(lib, inject):
    o = lib.cwt_server_options_init()
    srv = lib.cwt_server_create(np.array([5.0, 20.0]), np.array([7.0, 7.0]), lib.CWT_WAVELET_MORLET, o)
    try:
        sid = walk(lib, inject, "stream", lambda: lib.cwt_stream_open(srv, 4, 500.0))
        st = lib.cwt_server_stats(srv)
        assert st.open_streams == 1 and st.admitted == 1
        lib.cwt_stream_push(srv, sid, np.zeros((4, 100), np.float32))
        lib.cwt_server_step(srv)
        lib.cwt_server_sync(srv)
        lib.cwt_stream_close(srv, sid)
    finally:
        lib.cwt_server_destroy(srv)
