"""Benchmark: CWT coefficients per second on the fused FP32 workload.

Workload (one step): 64 channels x 10,000 samples (10 s at 1000 Hz) of seeded
synthetic EEG, float32, Morlet with n_cycles rising linearly 3 -> 10 over 100
log-spaced frequencies 1-100 Hz, outputs complex64 coefficients and float32
power: one cwt_execute (forward FFT of every channel + the fused scale-block
kernel) over inputs already resident in HBM.  The wavelet bank is generated
once at plan creation and reported separately (bank_ms).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream; between steps a 256 MB buffer (> the 129 MB L2) is
overwritten outside the events.  N > 1 (torchrun) runs one independent
workload per rank (weak scaling, no collective on the data path); the time is
the max over ranks.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CWT coeffs/sec (ch x scales x samples)"
UNIT = "coeffs/s"
WORKLOAD = "fused"
L2_FLUSH_BYTES = 256 << 20
# committed ncu summaries of the fused workload's scale-block kernel, per
# padding, and the sources each was captured from
PROFILES = {
    "pow2": ("scale_block_fp32_fused_64x100x10000.txt", ["fft_core.cuh", "scale_block.cu"]),
    "smooth": ("mr_fixed_scale_block_fp32_fused_smooth_64x100x10000.txt",
               ["fft_core.cuh", "mixed_radix.cuh", "smooth_device.cuh", "smooth_kernel.cuh", "smooth.cu",
                "smooth_fixed.cuh", "smooth_fixed.cu"]),
}


def kernel_source_hash(pad="pow2"):
    h = hashlib.sha256()
    for f in PROFILES[pad][1]:
        with open(os.path.join(ROOT, "paper_2506_07793_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(pad="pow2"):
    """DRAM bytes per launch of the scale-block kernel from the committed ncu
    summary, or None when the kernel source changed since it was captured."""
    try:
        text = open(os.path.join(ROOT, "profiles", PROFILES[pad][0])).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash(pad):
        return None
    return float(m_bytes.group(1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.dev = device_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def padded_length(n, pad):
    """The workload's padded length, written out here so that the oracle legs
    need nothing from the product library: the next power of two >= max(n, 32),
    or the smallest 2,3,5,7-smooth length >= max(n, 32) (Section "Fast Fourier
    transform").  For the workloads timed here (n = 10000, 122880, 500) this is
    the length the library's plan reports."""
    m = max(int(n), 32)
    if pad == "pow2":
        return 1 << (m - 1).bit_length()
    while True:
        x = m
        for f in (2, 3, 5, 7):
            while x % f == 0:
                x //= f
        if x == 1:
            return m
        m += 1


def host_cores():
    """Host threads this process may use (the oracle runs one per core)."""
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def host_cpu_model():
    """The host CPU's model name: lscpu's "Model name", else /proc/cpuinfo's
    "model name", else its Arm implementer and part codes."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip().lower(), v.strip())
    if "model name" in fields:
        return fields["model name"]
    if "cpu implementer" in fields:
        return f"Arm implementer {fields['cpu implementer']} part {fields.get('cpu part', '?')}"
    return "unknown"


def cpu_baseline(w, x_rows, n_channels, N, n_scales=None, min_seconds=10.0):
    """The FP64 oracle, as it stands, on the host cores: the first n_scales
    (default all) scales of the first channels of the same workload, at the
    padded length N of the timed plan -- n_channels channels, then one more at a
    time until at least min_seconds of work (at most every channel given)."""
    import oracle
    cores = host_cores()
    ns = w.scales if n_scales is None else n_scales
    scales = list(range(0, w.scales, max(1, w.scales // ns)))[:ns]
    x64 = x_rows.astype(np.float64)
    done, dt = 0, 0.0
    while done < len(x64) and (done < n_channels or dt < min_seconds):
        take = n_channels if done == 0 else 1
        rows = [(c, s) for c in range(take) for s in scales]
        t0 = time.perf_counter()
        oracle.cwt_rows(x64[done:done + take], N, w.fs, w.freqs, w.n_cycles, rows, threads=cores)
        dt += time.perf_counter() - t0
        done += take
    coeffs = done * len(scales) * w.n_out
    return {"value": coeffs / dt, "unit": UNIT, "cores": cores, "cpu_model": host_cpu_model(),
            "kind": "oracle",
            "sample": f"{done} of {w.channels} channels x {len(scales)} of {w.scales} scales x "
                      f"{w.n_out} samples ({coeffs} coefficients), {dt:.2f} s wall"}


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, each step a bounded
    sample (1 channel x all scales) of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from eeg_synth import workload
    import oracle
    w = workload(WORKLOAD)
    cores = host_cores()
    N = padded_length(w.samples, args.pad)
    x = w.signal(channels=1).astype(np.float64)
    rows = [(0, s) for s in range(w.scales)]
    for _ in range(args.warmup):
        oracle.cwt_rows(x, N, w.fs, w.freqs, w.n_cycles, rows[:4], threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.cwt_rows(x, N, w.fs, w.freqs, w.n_cycles, rows, threads=cores)
    dt = (time.perf_counter() - t0) / args.steps
    value = len(rows) * w.n_out / dt
    sample = f"1 of {w.channels} channels x all {w.scales} scales x {w.n_out} samples per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.notes, "channels": w.channels, "samples": w.samples,
                   "scales": w.scales, "fft_length": N, "padding": args.pad, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu_model": host_cpu_model(),
                         "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def plain_fp32_pipeline(cw, plan, x, fused_power, w, args, flush, stream):
    """The paper's own GPU design (Section "Optimizing performance": wavelets
    generated in GPU memory, library FFT, elementwise product, library inverse
    FFT), run with torch.fft (cuFFT) as a comparator only: FFT of the
    zero-padded signal, broadcast product with the same FP32 bank, inverse FFT,
    crop, |c|^2.  Same outputs (complex64 + power) as the fused kernel; its step
    time and its largest per-row power difference from the fused result are
    reported."""
    import torch
    info = cw.cwt_plan_info(plan)
    N = info.fft_length
    bank, _, _ = cw.cwt_plan_bank(plan)
    Wt = torch.from_numpy(bank * N).cuda()  # the bank carries 1/N; ifft applies it again
    xp = torch.zeros((w.channels, N), dtype=torch.float32, device="cuda")
    out = {}

    def step():
        xp[:, :w.samples] = x
        X = torch.fft.fft(xp)                           # [C][N] complex64
        c = torch.fft.ifft(X[:, None, :] * Wt[None])    # [C][S][N]
        c = c[..., :w.samples]
        out["c"], out["p"] = c, c.real * c.real + c.imag * c.imag
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms = timed_steps(step, args.steps, flush, stream) / args.steps
    p = out["p"]
    row_err = ((p - fused_power).abs().amax(dim=-1) / fused_power.amax(dim=-1)).max().item()
    del out, xp, Wt
    torch.cuda.empty_cache()
    return {"value": w.coefficients / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "impl": "torch.fft (cuFFT): fft -> broadcast product -> ifft -> crop -> |c|^2",
            "max_row_power_diff_vs_fused": row_err, "speedup_of_fused": None}


def plain_fp32_chunked(cw, plan, x, fused_power, fused_phase, w, args, flush, stream, chunk=8):
    """The plain FP32 pipeline (cuFFT through torch.fft, as in
    plain_fp32_pipeline) for the precision workload, whose [C][S][N] complex
    intermediate (34 GB) is formed `chunk` channels at a time: one FFT of all
    channels, then per chunk the broadcast product with the same FP32 bank, the
    inverse FFT, the crop, |c|^2 and atan2 into the power and phase outputs.
    The fused result is compared on the last step's outputs (per-row power
    difference over the row's peak)."""
    import torch
    info = cw.cwt_plan_info(plan)
    N = info.fft_length
    bank, _, _ = cw.cwt_plan_bank(plan)
    Wt = torch.from_numpy(bank * N).cuda()
    xp = torch.zeros((w.channels, N), dtype=torch.float32, device="cuda")
    ref_p = fused_power[:chunk].clone()
    pw = torch.empty_like(fused_power)
    ph = torch.empty_like(fused_phase)

    def step():
        xp[:, :w.samples] = x
        X = torch.fft.fft(xp)
        for c0 in range(0, w.channels, chunk):
            c = torch.fft.ifft(X[c0:c0 + chunk, None, :] * Wt[None])[..., :w.samples]
            pw[c0:c0 + chunk] = c.real * c.real + c.imag * c.imag
            ph[c0:c0 + chunk] = torch.angle(c)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    steps = max(2, min(args.steps, 5))
    ms = timed_steps(step, steps, flush, stream) / steps
    row_err = ((pw[:chunk] - ref_p).abs().amax(dim=-1) / ref_p.amax(dim=-1)).max().item()
    del pw, ph, xp, Wt
    torch.cuda.empty_cache()
    return {"value": w.coefficients / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "impl": f"torch.fft (cuFFT): fft -> per {chunk}-channel chunk: broadcast product -> ifft "
                    "-> crop -> |c|^2, angle",
            "max_row_power_diff_vs_fused": row_err, "speedup_of_fused": None}


def other_padding(cw, w, kinds, pad, x, outs, flush, stream, args):
    """The same workload under the other padding policy (same outputs, same
    timing method), reported beside the main line for comparison."""
    o = cw.cwt_options_init()
    o.pad_policy = cw.CWT_PAD_SMOOTH if pad == "smooth" else cw.CWT_PAD_POW2
    plan = cw.cwt_plan_create(w.channels, w.samples, w.fs, w.freqs, w.n_cycles,
                              cw.CWT_WAVELET_MORLET, kinds, o)
    N = cw.cwt_plan_info(plan).fft_length
    step = lambda: cw.cwt_execute(plan, x, *outs, stream)  # noqa: E731
    for _ in range(args.warmup):
        step()
    cw.cwt_plan_set_profiling(plan, True)
    cw.cwt_plan_profile_read(plan, cw.CWT_KERNEL_SCALE_BLOCK, reset=True)
    ms = timed_steps(step, args.steps, flush, stream) / args.steps
    n_sb, ms_sb = cw.cwt_plan_profile_read(plan, cw.CWT_KERNEL_SCALE_BLOCK, reset=True)
    cw.cwt_plan_destroy(plan)
    return {"padding": pad, "fft_length": N, "value": w.coefficients / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "kernel_ms": ms_sb / max(n_sb, 1)}


def timed_steps(step, steps, flush, stream):
    """Run `steps` steps, each between CUDA events on `stream`, overwriting
    `flush` (> L2) between them outside the events; returns total ms."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends))


def run_batch(args):
    """Batching workload: 2048 epochs (U{256..8192} samples) x 64 channels,
    64 scales, power decimated x4, one cwt_execute_batch per step."""
    import torch
    import paper_2506_07793_gb300 as cw
    from eeg_synth import batch_signal, workload
    import oracle

    world, rank, local, dist = rank_setup()
    w = workload("batch")
    if args.epochs:
        w.extra["epoch_lengths"] = w.extra["epoch_lengths"][:args.epochs]
        w.extra["epoch_starts"] = w.extra["epoch_starts"][:args.epochs]
    lengths = w.extra["epoch_lengths"]
    C, S, d = w.channels, w.scales, w.decimation
    opt = cw.cwt_options_init()
    opt.decimation = d
    plan = cw.cwt_plan_create(C, 8192, w.fs, w.freqs, w.n_cycles, cw.CWT_WAVELET_MORLET,
                              cw.CWT_OUT_POWER, opt)
    ep, n_in, n_o = cw.pack_epochs(lengths, C, S, d)
    x_host, _, _ = batch_signal(w)
    x = torch.from_numpy(x_host).cuda()
    out = torch.empty(n_o, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    step = lambda: cw.cwt_execute_batch(plan, ep, x, None, out, None, stream)  # noqa: E731
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    cw.cwt_plan_set_profiling(plan, True)
    clocks = ClockSampler(torch.cuda.current_device())
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    total_ms = timed_steps(step, args.steps, flush, stream)
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    n_b, ms_b = cw.cwt_plan_profile_read(plan, cw.CWT_KERNEL_BATCH, reset=True)
    cw.cwt_plan_set_profiling(plan, False)
    stats = cw.cwt_plan_batch_stats(plan)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    coeffs = int(n_o)
    value = coeffs * world / (ms_step * 1e-3)
    peaks, peak_kind = measured_peaks()
    alg_bytes = int(x_host.nbytes) + coeffs * 4 + int(stats.bank_bytes)
    k_s = ms_b / max(n_b, 1) * 1e-3
    achieved = alg_bytes / k_s / 1e9
    roofline = {"kernel": "batch_kernel (persistent, CUDA graph)", "bound": "hbm",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_kind, "traffic": None,
                "alg_bytes_per_launch": alg_bytes, "kernel_ms": k_s * 1e3}
    # end to end: pinned host input -> device, batch, device -> pinned host output
    h_in = torch.from_numpy(x_host).pin_memory()
    h_out = torch.empty(n_o, dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.e2e_steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        x.copy_(h_in, non_blocking=True)
        step()
        h_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": coeffs * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(x_host.nbytes),
           "d2h_bytes_per_step": int(coeffs * 4), "ms_per_step": e2e_s * 1e3}
    cw.cwt_plan_destroy(plan)
    loop = per_epoch_loop(cw, w, x_host, ep, lengths, stream) if world == 1 else None
    if loop is not None:
        loop["speedup_of_batch"] = value / loop["value"]
    plain = (plain_fp32_batch(cw, w, x, out, ep, lengths, flush, stream)
             if world == 1 and not getattr(args, "no_plain", False) else None)
    if plain is not None:
        plain["speedup_of_batch"] = plain["ms_per_step"] / ms_step
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.notes, "epochs": len(lengths), "channels": C, "scales": S,
                       "decimation": d, "coefficients_per_step": coeffs,
                       "l2": "inputs (2.2 GB) and outputs (35 GB) exceed L2; 256 MB buffer also "
                             "overwritten between timed steps",
                       "autotuned": {"inverse_radix": stats.inverse_radix, "order": stats.order,
                                     "candidate_ms": list(stats.tune_ms)},
                       "items": stats.items, "grid": stats.grid, "wall_s_timed_region": wall,
                       "parallelism": f"weak x{world}, no collective"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": args.steps, "clocks": clk,
        }
        if loop is not None:
            line["per_epoch_loop"] = loop
        if plain is not None:
            line["plain_fp32_gpu"] = plain
        if world == 1:
            # the oracle over the first epochs, one at a time until at least 10 s of work
            cores = host_cores()
            t0 = time.perf_counter()
            done = n_ep = 0
            while n_ep < len(lengths) and (n_ep < 2 or time.perf_counter() - t0 < getattr(args, "cpu_seconds", 10.0)):
                n = int(lengths[n_ep])
                xe = x_host[ep[n_ep].in_offset:ep[n_ep].in_offset + C * n].reshape(C, n)
                oracle.cwt(xe.astype(np.float64), padded_length(n, "pow2"), w.fs, w.freqs, w.n_cycles,
                           decimation=d, threads=cores)
                done += C * S * (-(-n // d))
                n_ep += 1
            dt = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": done / dt, "unit": UNIT, "cores": cores,
                                    "cpu_model": host_cpu_model(), "kind": "oracle",
                                    "sample": f"first {n_ep} of {len(lengths)} epochs x all {C} "
                                              f"channels x all {S} scales ({done} coefficients), "
                                              f"{dt:.2f} s wall"}
        return line
    return None


def plain_fp32_batch(cw, w, x, batch_out, ep, lengths, flush, stream, chunk=8):
    """The plain FP32 GPU pipeline for the batching workload (cuFFT through
    torch.fft, the paper's own design): epochs grouped by their padded length
    N_e, `chunk` epochs at a time zero-padded to N_e, FFT, broadcast product
    with that length's FP32 bank, inverse FFT, crop, every d-th sample, |c|^2
    written to the same packed output layout.  Timed like the batch (CUDA
    events, L2 flushed), two steps after one warm-up; the largest per-row
    power difference from the batch kernel's result is reported."""
    import torch
    C, S, d = w.channels, w.scales, w.decimation
    groups = {}
    for e_, n in enumerate(lengths):
        groups.setdefault(padded_length(int(n), "pow2"), []).append(e_)
    banks = {}
    for Ne in groups:
        o = cw.cwt_options_init()
        p = cw.cwt_plan_create(1, Ne, w.fs, w.freqs, w.n_cycles, cw.CWT_WAVELET_MORLET,
                               cw.CWT_OUT_POWER, o)
        b, _, _ = cw.cwt_plan_bank(p)
        cw.cwt_plan_destroy(p)
        banks[Ne] = torch.from_numpy(b * Ne).cuda()  # the bank carries 1/N_e; ifft applies it
    out = torch.empty_like(batch_out)

    def step():
        for Ne, eps in groups.items():
            Wt = banks[Ne]
            for i0 in range(0, len(eps), chunk):
                sel = eps[i0:i0 + chunk]
                xs = torch.zeros((len(sel) * C, Ne), dtype=torch.float32, device="cuda")
                for j, e_ in enumerate(sel):
                    n = int(lengths[e_])
                    off = int(ep[e_].in_offset)
                    xs[j * C:(j + 1) * C, :n] = x[off:off + C * n].view(C, n)
                c = torch.fft.ifft(torch.fft.fft(xs)[:, None, :] * Wt[None])
                p = c.real * c.real + c.imag * c.imag
                for j, e_ in enumerate(sel):
                    n = int(lengths[e_])
                    no = -(-n // d)
                    off = int(ep[e_].out_offset)
                    out[off:off + C * S * no].view(C, S, no)[:] = p[j * C:(j + 1) * C, :, :n:d]
    step()
    torch.cuda.synchronize()
    ms = timed_steps(step, 2, flush, stream) / 2
    # compare the first epoch's rows
    n0 = int(lengths[0])
    no0 = -(-n0 // d)
    off0 = int(ep[0].out_offset)
    a = out[off0:off0 + C * S * no0].view(C * S, no0)
    b = batch_out[off0:off0 + C * S * no0].view(C * S, no0)
    diff = ((a - b).abs().amax(dim=-1) / b.amax(dim=-1).clamp_min(1e-30)).max().item()
    del out, banks
    torch.cuda.empty_cache()
    coeffs = int(batch_out.numel())
    return {"value": coeffs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": 2,
            "impl": f"torch.fft (cuFFT) per padded length, {chunk} epochs at a time: fft -> "
                    "broadcast product -> ifft -> crop, decimate -> |c|^2",
            "max_row_power_diff_vs_batch_first_epoch": diff}


def per_epoch_loop(cw, w, x_host, ep, lengths, stream, n_ep=256):
    """The plain alternative to the batch API: one cwt_execute per epoch (as the
    paper's software loops over recordings), plans created beforehand and
    cached per length, inputs resident.  First n_ep epochs of the batch, timed
    with CUDA events over two passes of the loop."""
    import torch
    C, S, d = w.channels, w.scales, w.decimation
    n_ep = min(n_ep, len(lengths))
    plans, xs, outs = {}, [], []
    coeffs = 0
    for e_ in range(n_ep):
        n = int(lengths[e_])
        if n not in plans:
            o = cw.cwt_options_init()
            o.decimation = d
            plans[n] = cw.cwt_plan_create(C, n, w.fs, w.freqs, w.n_cycles, cw.CWT_WAVELET_MORLET,
                                          cw.CWT_OUT_POWER, o)
        off = ep[e_].in_offset
        xs.append(torch.from_numpy(np.ascontiguousarray(x_host[off:off + C * n])).cuda())
        outs.append(torch.empty(C * S * (-(-n // d)), dtype=torch.float32, device="cuda"))
        coeffs += C * S * (-(-n // d))

    def run():
        for e_ in range(n_ep):
            cw.cwt_execute(plans[int(lengths[e_])], xs[e_], None, outs[e_], None, stream)
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run()
    run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 2
    for p in plans.values():
        cw.cwt_plan_destroy(p)
    return {"value": coeffs / (ms * 1e-3), "unit": UNIT, "ms": ms, "epochs": n_ep,
            "coefficients": coeffs, "plans": len(plans), "gpu_launches_per_pass": 2 * n_ep,
            "impl": "one cwt_execute (forward FFT + fused scale block) per epoch"}


def run_serving(args):
    """Serving workload: live streams arrive (Poisson, 2/s) and leave
    (exponential lifetimes, mean 16 s) against 32 slots and a device-memory
    budget; channels from {8,32,64,128,256}, fs from {250,...,4000} Hz, hop
    50 ms, window 2048, 64 log-spaced Morlet scales 1-100 Hz, power.  Samples
    are pushed in real time; every loop iteration steps the server (one batched
    launch of all ready hops) and pulls what is complete."""
    import torch
    import paper_2506_07793_gb300 as cw
    from eeg_synth import eeg, workload

    if int(os.environ.get("RANK", "0")) != 0:
        return  # a single serving process (one GPU) per node
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = workload("serving")
    S = w.scales
    rng = np.random.default_rng(np.random.SeedSequence([w.seed, 0]))
    C_choices, fs_choices = [8, 32, 64, 128, 256], [250.0, 500.0, 1000.0, 2000.0, 4000.0]
    blocks = {fs: eeg(w.seed, 256, int(2 * fs), fs, np.float32) for fs in fs_choices}
    o = cw.cwt_server_options_init()
    o.max_streams = 32
    o.mem_budget_bytes = 1 << 30
    srv = cw.cwt_server_create(w.freqs, w.n_cycles, cw.CWT_WAVELET_MORLET, o)
    T = float(args.serve_seconds)
    # arrivals: 24 streams at t = 0, then Poisson(2/s); lifetimes Exp(16 s)
    arrivals = [0.0] * 24
    t = 0.0
    while True:
        t += rng.exponential(0.5)
        if t >= T:
            break
        arrivals.append(t)
    plan = [(a, a + rng.exponential(16.0), int(rng.choice(C_choices)), float(rng.choice(fs_choices)))
            for a in arrivals]
    active = {}  # sid -> dict
    pending = sorted(plan)
    bufs = {}
    h2d = d2h = 0
    steps = 0
    t0 = time.perf_counter()
    # warm-up: one stream of each fs so that banks exist before the clock starts
    for fs in fs_choices:
        sid = cw.cwt_stream_open(srv, 8, fs)
        cw.cwt_stream_close(srv, sid)
    cw.cwt_server_reset_stats(srv)
    clocks = ClockSampler(torch.cuda.current_device())
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        if now >= T:
            break
        while pending and pending[0][0] <= now:
            a, dep, C, fs = pending.pop(0)
            try:
                sid = cw.cwt_stream_open(srv, C, fs)
            except cw.CWTError as e:
                if e.status != cw.CWT_EBUSY:
                    raise
                continue
            H = int(np.ceil(fs * 0.05))
            active[sid] = {"C": C, "fs": fs, "H": H, "t_open": now, "dep": dep, "pushed": 0,
                           "off": int(rng.integers(0, int(fs)))}
            bufs[sid] = np.empty((16, C, S, H), np.float32)
        for sid in [k for k, v in active.items() if v["dep"] <= now]:
            cw.cwt_stream_close(srv, sid)
            del active[sid]
        for sid, st in active.items():
            due = int((now - st["t_open"]) * st["fs"]) - st["pushed"]
            due = min(due, 4 * st["H"])
            if due <= 0:
                continue
            blk = blocks[st["fs"]]
            L = blk.shape[1]
            p0 = (st["off"] + st["pushed"]) % L
            idx = (p0 + np.arange(due)) % L
            chunk = np.ascontiguousarray(blk[:st["C"], idx])
            try:
                cw.cwt_stream_push(srv, sid, chunk)
            except cw.CWTError as e:
                if e.status != cw.CWT_EBUSY:
                    raise
                continue
            st["pushed"] += due
            h2d += chunk.nbytes
        cw.cwt_server_step(srv)
        steps += 1
        for sid in active:
            n, _ = cw.cwt_stream_pull(srv, sid, bufs[sid])
            d2h += n * bufs[sid][0].nbytes
    cw.cwt_server_sync(srv)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = cw.cwt_server_stats(srv)
    cw.cwt_server_destroy(srv)
    value = st.coefficients / wall
    hop_ms = 50.0
    line = {
        "metric": METRIC + "; stream p99", "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": steps, "warmup": 0, "ms_per_step": wall * 1e3 / max(steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.notes, "seconds": T, "admitted": st.admitted, "refused": st.refused,
                   "hops": st.hops, "launches": st.launches, "mem_budget_bytes": 1 << 30,
                   "arrivals": len(plan)},
        "latency": {"p50_ms": st.latency_p50_s * 1e3, "p99_ms": st.latency_p99_s * 1e3,
                    "max_ms": st.latency_max_s * 1e3, "mean_ms": st.latency_mean_s * 1e3,
                    "hop_interval_ms": hop_ms, "p99_below_hop": st.latency_p99_s * 1e3 < hop_ms},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d // max(steps, 1),
                "d2h_bytes_per_step": d2h // max(steps, 1)},
        "gpu_launches": int(st.launches), "clocks": clk,
        # a latency-bound path: the fraction of the hop interval (the deadline)
        # that the 99th-percentile hop takes
        "roofline": {"bound": "latency", "achieved": st.latency_p99_s * 1e3, "peak": hop_ms,
                     "unit": "ms (p99 hop latency vs hop interval)",
                     "frac": st.latency_p99_s * 1e3 / hop_ms, "traffic": None},
        "cpu_baseline": serving_cpu_baseline(w, blocks, min_seconds=getattr(args, "cpu_seconds", 5.0)),
    }
    return line


def serving_cpu_baseline(w, blocks, min_seconds=5.0):
    """The FP64 oracle on the serving definition: the cyclic CWT of one
    2048-sample window per hop (8 channels at 1000 Hz, all 64 scales), of
    which the H = 50 centred outputs are delivered; hops one after another
    until min_seconds of work."""
    import oracle
    cores = host_cores()
    fs, C, W, H = 1000.0, 8, 2048, 50
    rec = blocks[fs]
    rows = [(c, s) for c in range(C) for s in range(w.scales)]
    t0 = time.perf_counter()
    hops = 0
    while hops < 1 or time.perf_counter() - t0 < min_seconds:
        e = W + hops * H
        win = rec[:C, (np.arange(e - W, e)) % rec.shape[1]].astype(np.float64)
        oracle.cwt_rows(win, W, fs, w.freqs, w.n_cycles, rows, threads=cores)
        hops += 1
    dt = time.perf_counter() - t0
    delivered = hops * C * w.scales * H
    return {"value": delivered / dt, "unit": UNIT, "cores": cores, "cpu_model": host_cpu_model(),
            "kind": "oracle",
            "sample": f"{hops} hops of 8 channels at 1000 Hz x all {w.scales} scales: the "
                      f"2048-sample window's CWT, {H} outputs delivered per row, {dt:.2f} s wall"}


def rank_setup():
    """(world, rank, local_rank, torch.distributed or None) of this process.
    One process per GPU: RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* come from
    torchrun or from spawn_ranks.  The process group (NCCL on GPUs, gloo on a
    CPU-only host) carries only the barrier and the max-over-ranks timing."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            if torch.cuda.is_available():
                dist.init_process_group("nccl", device_id=torch.device("cuda", local))
            else:
                dist.init_process_group("gloo")
    return world, rank, local, dist


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_entry(local_rank, argv, world, port):
    os.environ.update({"RANK": str(local_rank), "LOCAL_RANK": str(local_rank),
                       "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    main(argv)


def spawn_ranks(argv, world):
    """--gpus N with no WORLD_SIZE in the environment: start N local ranks, one
    per GPU, each running this benchmark (rank 0 prints the line)."""
    import torch.multiprocessing as mp
    mp.spawn(_rank_entry, args=(argv, world, _free_port()), nprocs=world, join=True)


def launcher_selftest(args):
    """The multi-rank path without GPUs (gloo): each rank takes its block of a
    64 x N-channel recording with the shard helper, reports a rank-dependent
    time, and rank 0 prints the slowest rank's time and the blocks."""
    from paper_2506_07793_gb300.partition import max_over_ranks, shard_channels
    world, rank, local, dist = rank_setup()
    c0, c1 = shard_channels(64 * world, world, rank)
    ms = max_over_ranks(10.0 + rank, dist)
    blocks = [None] * world
    if dist:
        dist.all_gather_object(blocks, (c0, c1))
        dist.barrier()
    else:
        blocks = [(c0, c1)]
    if rank == 0:
        return {"metric": METRIC, "n_gpus": world, "ms_per_step": ms, "shards": blocks,
                "scaling": "weak", "launcher": "spawn" if "SPAWNED_BY_BENCH" in os.environ else "env"}
    return None


def sub_args(args, **kw):
    a = argparse.Namespace(**vars(args))
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def precision_suite(args):
    """The precision workload (256 ch x 122880 @2048 Hz, N = 131072, 128 scales,
    power + phase) in its three inverse-FFT arithmetics -- FP32 on clusters,
    tensor-core FP16 and BF16 hi/lo -- beside the plain FP32 cuFFT pipeline,
    each timed like the headline (CUDA events, L2 flushed between steps); and
    FP32 under the paper's smooth padding, where 122880 = 8 x 15360 needs none
    (mixed-radix clusters)."""
    out = {}
    for key, prec, pad in (("fp32", "fp32", "pow2"), ("tc_fp16", "tc_fp16", "pow2"),
                           ("tc_bf16", "tc_bf16", "pow2"), ("fp32_smooth", "fp32", "smooth")):
        main = key == "fp32"
        a = sub_args(args, workload="precision", precision=prec, pad=pad, steps=5, warmup=3,
                     no_e2e=not main, no_plain=not main, no_other=True,
                     no_cpu=not main, cpu_seconds=5.0, e2e_steps=1, channels=0)
        line = run_plan_workload(a, "precision")
        keep = {k: line[k] for k in ("value", "unit", "ms_per_step", "dtype", "roofline", "clocks",
                                     "gpu_launches", "e2e", "cpu_baseline", "plain_fp32_gpu",
                                     "error_vs_fp32_gpu", "steps", "warmup") if k in line}
        if not main:
            keep["fft_length"] = line["config"]["fft_length"]
        out[key] = keep
        if main:
            out["config"] = line["config"]
    plain = out["fp32"].pop("plain_fp32_gpu", None)
    if plain is not None:
        out["plain_fp32_gpu"] = plain
        for prec in ("fp32", "tc_fp16", "tc_bf16", "fp32_smooth"):
            out[prec]["speedup_over_plain_fp32_gpu"] = plain["ms_per_step"] / out[prec]["ms_per_step"]
    for prec in ("tc_fp16", "tc_bf16"):
        out[prec]["speedup_over_fp32_clusters"] = out["fp32"]["ms_per_step"] / out[prec]["ms_per_step"]
    out["error_bar"] = "2e-3 of each row's peak power (tests/test_gpu_tc.py checks it per frequency)"
    return out


def run_default(args):
    """The headline line (fused workload) and, on one GPU, the rest of the
    metric as sub-objects: precision (FP32 / TC FP16 / TC BF16 / plain cuFFT),
    batch and serving."""
    line = run_plan_workload(args, "fused")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if line is None or world > 1 or args.headline_only:
        return line
    line["precision"] = precision_suite(args)
    b = run_batch(sub_args(args, steps=5, warmup=3, e2e_steps=1, epochs=0, cpu_seconds=5.0))
    line["batch"] = {k: v for k, v in b.items() if k not in ("metric", "n_gpus", "scaling",
                                                             "higher_is_better", "vs_baseline",
                                                             "data")}
    s = run_serving(sub_args(args, serve_seconds=min(args.serve_seconds, 6.0)))
    line["serving"] = {k: v for k, v in s.items() if k not in ("metric", "n_gpus", "scaling",
                                                               "higher_is_better", "vs_baseline",
                                                               "data")}
    return line


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-channels", type=int, default=2)
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["fused", "batch", "serving", "precision", "sweep"])
    ap.add_argument("--headline-only", action="store_true",
                    help="fused workload only: leave out the precision, batch and serving "
                         "sub-objects of the default line")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--pad", default=None, choices=["pow2", "smooth"],
                    help="padding policy: the paper's 2,3,5,7-smooth length (default for the fused "
                         "workload) or the next power of two (default for the precision workload, "
                         "whose tensor-core forms need a power of two; its 122880 samples are "
                         "themselves smooth)")
    ap.add_argument("--channels", type=int, default=0,
                    help="override the workload's channel count (small profiling captures)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tc_fp16", "tc_bf16"],
                    help="inverse-FFT arithmetic of the precision workload: FP32, or the "
                         "tensor-core DFT stages with FP16 / BF16 hi/lo operands")
    ap.add_argument("--epochs", type=int, default=0,
                    help="batch workload: use only the first N epochs (small profiling captures)")
    ap.add_argument("--launcher-selftest", action="store_true", help=argparse.SUPPRESS)
    argv = sys.argv[1:] if argv is None else argv
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.pad is None:
        args.pad = "pow2" if args.workload == "precision" else "smooth"
    if args.gpus < 1:
        ap.error("--gpus must be >= 1")
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        os.environ["SPAWNED_BY_BENCH"] = "1"
        return spawn_ranks(argv, args.gpus)
    if int(os.environ.get("WORLD_SIZE", "1")) != args.gpus:
        ap.error(f"--gpus {args.gpus} but WORLD_SIZE={os.environ.get('WORLD_SIZE')}")
    if args.impl == "reference":
        return run_reference(args)
    if args.launcher_selftest:
        line = launcher_selftest(args)
    elif args.workload == "batch":
        line = run_batch(args)
    elif args.workload == "serving":
        line = run_serving(args)
    elif args.workload == "sweep":
        line = run_sweep(args)
    elif args.workload == "fused":
        line = run_default(args)
    else:
        line = run_plan_workload(args, args.workload)
    if line is not None:
        print(json.dumps(line), flush=True)
    import torch.distributed as tdist
    if tdist.is_available() and tdist.is_initialized():
        tdist.barrier()
        tdist.destroy_process_group()


SWEEP_LENGTHS = sorted(set(range(100, 2501, 100)) | {101, 127, 499, 509, 1009, 1021, 1024, 1499,
                                                      1999, 2048, 2039, 2477})


def run_sweep(args):
    """Time per CWT call against the signal length (the shape of Fig. 4) and
    wavelet-bank generation time (Table 2).

    Per length n (100..2500 samples at 1000 Hz, primes and powers of two
    included): 64 channels of seeded synthetic EEG, Morlet sigma = 7 at 30..90 Hz
    in 1 Hz steps (61 scales), complex64 output; padding to the next power of
    two and to the paper's 2,3,5,7-smooth length.  `device_us` is one
    cwt_execute on resident buffers (CUDA events, mean of --steps calls after
    --warmup); `e2e_us` is cwt_execute_host from pinned host memory, copies
    included.  `smooth_tuned` is the smooth padding with
    cwt_options.specialize = 2 (fixed-length kernels compiled at plan creation
    for candidate schedules of the length, the fastest on the plan's rows
    kept; `plan_ms` includes the compiles, cached per process).
    Bank generation: 61 scales, 1 s at 2048 Hz (N = 2048), Morlet and the GMW
    of Fig. 1 (beta 17.5, gamma 3), FP64 on the GPU."""
    import torch
    import paper_2506_07793_gb300 as cw
    from eeg_synth import eeg

    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    fs, C = 1000.0, 64
    freqs = np.arange(30.0, 91.0)
    cycles = np.full(len(freqs), 7.0)
    S = len(freqs)
    stream = torch.cuda.current_stream()
    points = []
    clocks = ClockSampler(torch.cuda.current_device())
    for n in SWEEP_LENGTHS:
        x_host = eeg(4000 + n, C, n, fs, np.float32)
        x = torch.from_numpy(x_host).cuda()
        out = torch.empty((C, S, n), dtype=torch.complex64, device="cuda")
        h_in = torch.from_numpy(x_host).pin_memory()
        h_out = torch.empty((C, S, n), dtype=torch.complex64).pin_memory()
        pt = {"samples": n}
        for pad in ("pow2", "smooth", "smooth_tuned"):
            o = cw.cwt_options_init()
            o.pad_policy = cw.CWT_PAD_POW2 if pad == "pow2" else cw.CWT_PAD_SMOOTH
            o.specialize = 2 if pad == "smooth_tuned" else 0
            t_plan = time.perf_counter()
            plan = cw.cwt_plan_create(C, n, fs, freqs, cycles, cw.CWT_WAVELET_MORLET,
                                      cw.CWT_OUT_COMPLEX, o)
            plan_ms = (time.perf_counter() - t_plan) * 1e3
            info = cw.cwt_plan_info(plan)
            for _ in range(args.warmup):
                cw.cwt_execute(plan, x, out, None, None, stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                cw.cwt_execute(plan, x, out, None, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            dev_us = e0.elapsed_time(e1) * 1e3 / args.steps
            cw.cwt_execute_host(plan, h_in, h_out, None, None, stream)
            torch.cuda.synchronize()
            reps = max(3, args.steps // 4)
            t0 = time.perf_counter()
            for _ in range(reps):
                cw.cwt_execute_host(plan, h_in, h_out, None, None, stream)
            e2e_us = (time.perf_counter() - t0) / reps * 1e6
            pt[pad] = {"N": info.fft_length, "device_us": dev_us, "e2e_us": e2e_us,
                       "bank_ms": info.bank_ms, "plan_ms": plan_ms, "fixed_kernel": info.fixed_kernel,
                       "specialized": info.specialized}
            cw.cwt_plan_destroy(plan)
        points.append(pt)
    clk = clocks.stop()

    bank = {}
    for name, wv, par in (("morlet", cw.CWT_WAVELET_MORLET, 7.0), ("gmw", cw.CWT_WAVELET_GMW, 17.5)):
        o = cw.cwt_options_init()
        o.gmw_gamma = 3.0
        times = []
        for _ in range(5):
            plan = cw.cwt_plan_create(1, 2048, 2048.0, freqs, np.full(S, par), wv, cw.CWT_OUT_POWER, o)
            times.append(cw.cwt_plan_info(plan).bank_ms)
            cw.cwt_plan_destroy(plan)
        bank[name] = {"ms_median": statistics.median(times[1:]), "scales": S, "fft_length": 2048}
    if rank == 0:
        coeffs = [C * S * p["samples"] for p in points]
        rate = [c / (p["pow2"]["device_us"] * 1e-6) for c, p in zip(coeffs, points)]
        print(json.dumps({
            "metric": "CWT time per call vs signal length (Fig. 4 shape)", "value": statistics.median(rate),
            "unit": "coeffs/s (median over lengths, pow2 padding)", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "none", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{C} ch @1000 Hz, n = 100..2500 (+ primes, powers of two), "
                                   "Morlet sigma 7, 30-90 Hz by 1 Hz (61 scales), complex64",
                       "l2": "not flushed (every length's working set is below the 129 MB L2)"},
            "points": points, "bank_generation": bank, "clocks": clk,
            "gpu_launches": 2 * args.steps * 3 * len(points),
        }), flush=True)


def run_plan_workload(args, name):
    """One cwt_execute per step over a resident [C][n] signal: the fused
    workload (complex64 + power, N = 16384) or the precision workload (power +
    phase, N = 131072, each row on a cluster of 8 CTAs)."""

    import torch
    import paper_2506_07793_gb300 as cw
    from eeg_synth import workload

    world, rank, local, dist = rank_setup()

    w = workload(name)
    if args.channels:
        w.channels = args.channels
    # weak scaling: the job is a recording of channels x world channels; each
    # rank transforms its contiguous block (the shard helper), no exchange
    from paper_2506_07793_gb300.partition import shard_channels
    c0, c1 = shard_channels(w.channels * world, world, rank)
    x_host = w.signal(channels=c1 - c0, first_channel=c0)
    x = torch.from_numpy(x_host).cuda()
    bits = {"complex": cw.CWT_OUT_COMPLEX, "power": cw.CWT_OUT_POWER, "phase": cw.CWT_OUT_PHASE}
    kinds = 0
    for o in w.outputs:
        kinds |= bits[o]
    popt = cw.cwt_options_init()
    popt.pad_policy = cw.CWT_PAD_SMOOTH if args.pad == "smooth" else cw.CWT_PAD_POW2
    popt.precision = {"fp32": cw.CWT_PREC_FP32, "tc_fp16": cw.CWT_PREC_TC_FP16,
                      "tc_bf16": cw.CWT_PREC_TC_BF16}[args.precision]
    plan = cw.cwt_plan_create(w.channels, w.samples, w.fs, w.freqs, w.n_cycles,
                              cw.CWT_WAVELET_MORLET, kinds, popt)
    info = cw.cwt_plan_info(plan)
    shape = (w.channels, w.scales, w.n_out)
    out_c = torch.empty(shape, dtype=torch.complex64, device="cuda") if "complex" in w.outputs else None
    out_p = torch.empty(shape, dtype=torch.float32, device="cuda")
    out_ph = torch.empty(shape, dtype=torch.float32, device="cuda") if "phase" in w.outputs else None
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        cw.cwt_execute(plan, x, out_c, out_p, out_ph, stream)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    cw.cwt_plan_set_profiling(plan, True)
    cw.cwt_plan_profile_read(plan, cw.CWT_KERNEL_SCALE_BLOCK, reset=True)
    cw.cwt_plan_profile_read(plan, cw.CWT_KERNEL_FORWARD_FFT, reset=True)
    clocks = ClockSampler(torch.cuda.current_device())
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        cw.cwt_execute(plan, x, out_c, out_p, out_ph, stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    n_sb, ms_sb = cw.cwt_plan_profile_read(plan, cw.CWT_KERNEL_SCALE_BLOCK, reset=True)
    n_fw, ms_fw = cw.cwt_plan_profile_read(plan, cw.CWT_KERNEL_FORWARD_FFT, reset=True)
    cw.cwt_plan_set_profiling(plan, False)
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())

    coeffs_rank = w.coefficients
    ms_step = total_ms / args.steps
    value = coeffs_rank * world / (ms_step * 1e-3)

    # roofline of the dominant kernel (fused scale block)
    peaks, peak_kind = measured_peaks()
    N = info.fft_length
    out_bytes_per_coef = 4 * (2 * ("complex" in w.outputs) + ("power" in w.outputs)
                              + ("phase" in w.outputs))
    alg_bytes = (w.channels * w.scales * w.n_out * out_bytes_per_coef  # requested outputs
                 + w.channels * N * 8                              # forward spectra, read once
                 + w.scales * N * 4)                               # wavelet bank, read once
    sb_s = ms_sb / max(n_sb, 1) * 1e-3
    achieved = alg_bytes / sb_s / 1e9
    traffic = profiled_traffic(args.pad)
    if N & (N - 1):
        pair = tuple(info.inlined_pair)
        rad = "x".join(str(r) for r in info.radices if r)
        if info.cluster > 1:
            kname = (f"cl_mr::scale_block_kernel<{info.cluster}, "
                     f"{'fixed' if info.fixed_kernel else 'generic'}> (cluster of {info.cluster} CTAs; "
                     f"N = {N} = {info.cluster} x {N // info.cluster}, local passes {rad})")
        elif info.fixed_kernel:
            kname = f"mr_fixed_scale_block_kernel (compiled for N = {N} = {rad})"
        elif pair[0]:
            kname = f"mr_scale_block_kernel<{pair[0]}, {pair[1]}> (inlined radix pair; N = {N} = {rad})"
        else:
            kname = f"mr_scale_block_kernel<0, 0> (generic mixed radix; N = {N} = {rad})"
    elif N <= 16384:
        kname = f"scale_block_kernel<{N},float>"
    elif args.precision != "fp32":
        kname = (f"tc_scale_block_cluster_kernel<{N // 16384}, {args.precision[3:]}> (cluster of "
                 f"{N // 16384} CTAs; radix-16 stages as mma.sync DFT products, hi/lo operands, "
                 "FP32 accumulation)")
    else:
        kname = f"cl_scale_block_kernel<{N},float> (cluster of {N // 16384} CTAs)"
    roofline = {"kernel": kname, "bound": "hbm",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_kind,
                "traffic": traffic if name == "fused" else None,
                "alg_bytes_per_launch": alg_bytes,
                "kernel_ms": sb_s * 1e3, "forward_fft_ms": ms_fw / max(n_fw, 1)}

    # end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if not getattr(args, "no_e2e", False):
        e2e = end_to_end(cw, plan, x_host, shape, out_c, out_ph, stream, w, world, dist,
                         args.e2e_steps if name == "fused" else 1, out_bytes_per_coef)
    if getattr(args, "no_plain", False):
        plain = None
    elif name == "fused":
        plain = plain_fp32_pipeline(cw, plan, x, out_p, w, args, flush, stream)
    elif name == "precision" and world == 1:
        plain = plain_fp32_chunked(cw, plan, x, out_p, out_ph, w, args, flush, stream)
    else:
        plain = None
    cw.cwt_plan_destroy(plan)
    tc_err = (tc_error_vs_fp32(cw, w, popt, x, out_p, stream)
              if name == "precision" and args.precision != "fp32" else None)
    other = (other_padding(cw, w, kinds, "pow2" if args.pad == "smooth" else "smooth", x,
                           (out_c, out_p, out_ph), flush, stream, args)
             if name == "fused" and world == 1 and not getattr(args, "no_other", False) else None)
    line = finish_plan_line(args, name, w, info, N, world, rank, value, ms_step, wall, clk, roofline,
                            e2e, plain, other, coeffs_rank, x_host)
    if line is not None and tc_err is not None:
        line["error_vs_fp32_gpu"] = tc_err
    return line


def tc_error_vs_fp32(cw, w, popt, x, tc_power, stream, channels=4):
    """The tensor-core result against the FP32 path on the same rows, per
    frequency: max over the first `channels` channels of each row's
    max_t |P_tc - P_fp32| / max_t P_fp32 (the FP32 path is itself within 1e-5
    of the FP64 oracle, which tests/test_gpu_tc.py checks per frequency)."""
    import torch
    o = cw.cwt_options_init()
    o.pad_policy = popt.pad_policy
    o.precision = cw.CWT_PREC_FP32
    plan = cw.cwt_plan_create(channels, w.samples, w.fs, w.freqs, w.n_cycles, cw.CWT_WAVELET_MORLET,
                              cw.CWT_OUT_POWER, o)
    ref = torch.empty((channels, w.scales, w.n_out), dtype=torch.float32, device="cuda")
    cw.cwt_execute(plan, x[:channels].contiguous(), None, ref, None, stream)
    torch.cuda.synchronize()
    cw.cwt_plan_destroy(plan)
    err = ((tc_power[:channels] - ref).abs().amax(dim=-1) / ref.amax(dim=-1)).amax(dim=0)
    err = [float(e) for e in err.cpu()]
    return {"channels": channels, "freqs_hz": [round(float(f), 4) for f in w.freqs],
            "power_err_per_frequency": [float(f"{e:.3g}") for e in err], "max": max(err), "bar": 2e-3}


def end_to_end(cw, plan, x_host, shape, out_c, out_ph, stream, w, world, dist, e2e_steps,
               out_bytes_per_coef):
    """The same metric through cwt_execute_host: pinned host input copied in and
    the outputs written to pinned host memory, inside the timed region."""
    import torch
    h_in = torch.from_numpy(x_host).pin_memory()
    h_c = torch.empty(shape, dtype=torch.complex64).pin_memory() if out_c is not None else None
    h_p = torch.empty(shape, dtype=torch.float32).pin_memory()
    h_ph = torch.empty(shape, dtype=torch.float32).pin_memory() if out_ph is not None else None
    cw.cwt_execute_host(plan, h_in, h_c, h_p, h_ph, stream)  # allocates staging
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        cw.cwt_execute_host(plan, h_in, h_c, h_p, h_ph, stream)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": w.coefficients * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(x_host.nbytes),
           "d2h_bytes_per_step": int(w.coefficients * out_bytes_per_coef),
           "ms_per_step": e2e_s * 1e3}
    del h_c, h_p, h_ph
    return e2e


def finish_plan_line(args, name, w, info, N, world, rank, value, ms_step, wall, clk, roofline,
                     e2e, plain, other, coeffs_rank, x_host):
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "tc_fp16": "f16 hi/lo, f32 accumulation",
                      "tc_bf16": "bf16 hi/lo, f32 accumulation"}[args.precision],
            "data": "synthetic",
            "config": {"workload": w.notes, "channels": w.channels, "samples": w.samples,
                       "scales": w.scales, "fft_length": N, "padding": args.pad,
                       "precision": args.precision,
                       "coefficients_per_step": coeffs_rank,
                       "l2": "256 MB buffer overwritten between timed steps (outside the events)",
                       "bank_ms": info.bank_ms, "wall_s_timed_region": wall,
                       "parallelism": f"weak x{world}, no collective"},
            "roofline": roofline,
            "e2e": e2e,
            "plain_fp32_gpu": plain,
            # forward FFT + scale block per step (+ the spectrum bounds of the tensor-core path)
            "gpu_launches": (3 if args.precision != "fp32" else 2) * args.steps,
            "clocks": clk,
        }
        if e2e is None:
            del line["e2e"]
        if other is not None:
            line["other_padding"] = other
        if world == 1 and not getattr(args, "no_cpu", False):
            line["cpu_baseline"] = cpu_baseline(w, x_host, args.cpu_channels if name == "fused" else 1, N,
                                                n_scales=None if name == "fused" else 8,
                                                min_seconds=getattr(args, "cpu_seconds", 10.0))
        if plain is not None:
            plain["speedup_of_fused"] = plain["ms_per_step"] / ms_step
        else:
            del line["plain_fp32_gpu"]
        return line
    return None


if __name__ == "__main__":
    main()
