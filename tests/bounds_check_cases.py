"""Small cases of every kernel family, run in a process that loaded the
library named by CWT_GB300_LIB (the bounds-checked build): each case must
finish without CWT_EDEVICE (no out-of-range shared-memory access or index was
recorded) and match the FP64 oracle.  Prints one line per case; exits non-zero
on the first failure.  Run by tests/test_gpu_bounds_check.py."""
import os
import sys
import zlib

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_2506_07793_gb300 as lib  # noqa: E402
from eeg_synth import eeg  # noqa: E402
from tests.metrics import FP32_TOL, TC_TOL, complex_err, power_err  # noqa: E402

assert lib.LIB_PATH == os.environ["CWT_GB300_LIB"], lib.LIB_PATH


def plan_case(name, C, n, fs, freqs, cycles, tol=FP32_TOL, **kw):
    x = eeg(zlib.crc32(name.encode()) % 1000, C, n, fs, np.float64 if kw.get("dtype") == "f64" else np.float32)
    t = lib.CWT(C, n, fs, freqs, cycles, outputs=("complex", "power"), **kw)
    try:
        out = t(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        ref = oracle.cwt(x.astype(np.float64), t.info.fft_length, fs, freqs, cycles,
                         decimation=kw.get("decimation", 1))
        e = max(complex_err(out["complex"].cpu().numpy(), ref).max(),
                power_err(out["power"].cpu().numpy(), ref).max())
        assert e <= tol, (name, e)
        print(f"{name}: N = {t.info.fft_length}, max row error {e:.2e}")
    finally:
        t.close()


F5 = np.array([3.0, 11.0, 40.0, 120.0, 230.0])
S5 = np.array([5.0, 7.0, 7.0, 9.0, 12.0])
plan_case("pow2 one CTA", 2, 700, 500.0, F5, S5)
plan_case("pow2 16384 (32 points per thread)", 1, 12000, 500.0, F5, S5)
plan_case("pow2 cluster of 2", 1, 20000, 1000.0, F5, S5)
plan_case("pow2 decimation 4 (spectral fold)", 2, 3000, 500.0, F5, S5, decimation=4)
plan_case("f64 I/O", 2, 500, 500.0, F5, S5, dtype="f64")
plan_case("smooth fixed 10000", 2, 10000, 1000.0, F5, S5, pad="smooth")
plan_case("smooth fixed 1000 (several rows per CTA)", 3, 1000, 500.0, F5, S5, pad="smooth")
plan_case("smooth pair / generic 6000", 2, 6000, 1000.0, F5, S5, pad="smooth")
plan_case("smooth generic 1323", 2, 1323, 500.0, F5, S5, pad="smooth", fft_length=1323)
plan_case("smooth cluster of 2 (16464 = 2 x 8232)", 1, 16400, 1000.0, F5, S5, pad="smooth")
plan_case("smooth cluster of 3 (14175 = 3 x 4725)", 1, 14175, 1000.0, F5, S5, pad="smooth")
plan_case("smooth cluster of 8 (115200 = 8 x 14400)", 1, 115200, 1920.0, F5, S5, pad="smooth",
          decimation=16)
plan_case("smooth cluster of 10 (122880 = 10 x 12288, compiled in)", 1, 122880, 2048.0, F5, S5,
          pad="smooth", decimation=16)
# plan-time compilation is off in this build: a split that only compiled
# kernels run (105000 = 10 x 10500) falls back to the portable one (7 x 15000)
t = lib.CWT(1, 105000, 1000.0, F5, S5, outputs=("power",), pad="smooth", specialize=True)
try:
    assert (t.info.cluster, t.info.specialized) == (7, 0), (t.info.cluster, t.info.specialized)
    print("specialize without plan-time compilation: cluster", t.info.cluster)
finally:
    t.close()
plan_case("portable split after the fallback (105000 = 7 x 15000)", 1, 105000, 1000.0, F5, S5,
          pad="smooth", decimation=16, specialize=True)
plan_case("tensor cores FP16, 16384", 2, 12000, 500.0, F5, S5, tol=TC_TOL, precision="tc_fp16")
plan_case("tensor cores BF16, cluster of 2", 1, 20000, 1000.0, F5, S5, tol=TC_TOL,
          precision="tc_bf16")

# batch: ragged epochs, both inverse staging widths over two decimations
for d in (1, 3):
    C, fs = 2, 500.0
    lengths = [31, 257, 2048, 4097, 8192, 640]
    o = lib.cwt_options_init()
    o.decimation = d
    plan = lib.cwt_plan_create(C, 8192, fs, F5, S5, 0, lib.CWT_OUT_POWER, o)
    try:
        ep, n_in, n_o = lib.pack_epochs(lengths, C, len(F5), d)
        xs = [eeg(700 + k, C, n, fs, np.float32) for k, n in enumerate(lengths)]
        x = torch.from_numpy(np.concatenate([a.reshape(-1) for a in xs])).cuda()
        pw = torch.zeros((n_o,), dtype=torch.float32, device="cuda")
        lib.cwt_execute_batch(plan, ep, x, None, pw, None)
        torch.cuda.synchronize()
        p = pw.cpu().numpy()
        worst = 0.0
        for k, n in enumerate(lengths):
            ref = oracle.cwt(xs[k].astype(np.float64), lib.cwt_fft_length(n), fs, F5, S5, decimation=d)
            no = -(-n // d)
            got = p[ep[k].out_offset:ep[k].out_offset + C * len(F5) * no].reshape(C, len(F5), no)
            worst = max(worst, power_err(got, ref).max())
        assert worst <= FP32_TOL, ("batch", d, worst)
        print(f"batch d = {d}: max row error {worst:.2e}")
    finally:
        lib.cwt_plan_destroy(plan)

# streaming server: two streams, several hops, then a sync (collects violations)
so = lib.cwt_server_options_init()
srv = lib.cwt_server_create(np.array([5.0, 20.0, 60.0]), np.array([7.0, 7.0, 7.0]),
                            lib.CWT_WAVELET_MORLET, so)
try:
    ids = [lib.cwt_stream_open(srv, 3, 500.0), lib.cwt_stream_open(srv, 2, 1000.0)]
    for step in range(6):
        for sid, (C, fs) in zip(ids, [(3, 500.0), (2, 1000.0)]):
            lib.cwt_stream_push(srv, sid, eeg(800 + step, C, int(0.05 * fs), fs, np.float32))
        lib.cwt_server_step(srv)
        lib.cwt_server_sync(srv)
    print("stream: hops", lib.cwt_server_stats(srv).hops)
finally:
    lib.cwt_server_destroy(srv)

# batched FFT building block, one CTA and cluster lengths
for n in (64, 4096, 16384, 65536):
    z = (torch.randn(2, n, dtype=torch.float32) + 1j * torch.randn(2, n, dtype=torch.float32)).to(torch.complex64)
    d_in = z.cuda()
    d_out = torch.empty_like(d_in)
    lib.cwt_fft(d_in, d_out, n, 2, -1)
    torch.cuda.synchronize()
    ref = np.fft.fft(z.numpy().astype(np.complex128), axis=-1)
    e = np.abs(d_out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert e < 1e-5, ("fft", n, e)
    print(f"fft {n}: {e:.2e}")

# the entry point without allocation
C, n, fs = 2, 3000, 500.0
x = eeg(900, C, n, fs, np.float32)
pw = torch.empty((C, len(F5), n), dtype=torch.float32, device="cuda")
lib.cwt_execute_noalloc(torch.from_numpy(x).cuda(), C, n, fs, F5, S5, power_out=pw)
torch.cuda.synchronize()
ref = oracle.cwt(x.astype(np.float64), lib.cwt_fft_length(n), fs, F5, S5)
e = power_err(pw.cpu().numpy(), ref).max()
assert e <= FP32_TOL, ("noalloc", e)
print(f"noalloc: {e:.2e}")
print("ALL CASES PASSED UNDER BOUNDS CHECKS")
