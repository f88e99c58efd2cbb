"""Seeded synthetic EEG and the workload shapes used by tests and the benchmark.

This module only draws inputs: it holds none of the transform's arithmetic and
is shared, unchanged, by the oracle tests and the CUDA-path tests.

The paper measures on generated random EEG (Sections "Precision",
"Comparison between devices and software" and "Wavelength and flexibility"),
so synthetic signals stand in for it.  Each channel is the sum of
  * one sinusoid per EEG band centre (2, 6, 10, 20, 40 Hz), its frequency drawn
    from centre * U(0.9, 1.1), amplitude U(5, 30) uV, phase U(0, 2 pi);
  * 1/f ("pink") noise: white Gaussian noise whose spectrum is shaped by
    1/sqrt(f), DC removed, scaled to 10 uV rms;
  * white Gaussian noise, 2 uV rms.
Values are in microvolts.  Channel ch of workload seed s is drawn from
numpy.random.default_rng(SeedSequence([s, ch])), so any subset of channels can
be regenerated on its own.
"""
from dataclasses import dataclass, field

import numpy as np

BAND_CENTRES_HZ = (2.0, 6.0, 10.0, 20.0, 40.0)


def eeg_channel(seed, channel, n, fs):
    """One channel of synthetic EEG, float64 [n], microvolts."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(channel)]))
    t = np.arange(n) / float(fs)
    x = np.zeros(n)
    for centre in BAND_CENTRES_HZ:
        f = centre * rng.uniform(0.9, 1.1)
        amp = rng.uniform(5.0, 30.0)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        if f < fs / 2:
            x += amp * np.cos(2.0 * np.pi * f * t + ph)
    white = rng.standard_normal(n)
    if n > 2:
        spec = np.fft.rfft(white)
        f = np.fft.rfftfreq(n, d=1.0 / fs)
        shape = np.zeros_like(f)
        shape[1:] = 1.0 / np.sqrt(f[1:])
        pink = np.fft.irfft(spec * shape, n=n)
        rms = np.sqrt(np.mean(pink * pink))
        if rms > 0:
            x += pink * (10.0 / rms)
    x += 2.0 * rng.standard_normal(n)
    return x


def eeg(seed, channels, n, fs, dtype=np.float64, first_channel=0):
    """[channels][n] synthetic EEG of the given dtype."""
    out = np.empty((channels, n), dtype=dtype)
    for c in range(channels):
        out[c] = eeg_channel(seed, first_channel + c, n, fs)
    return out


@dataclass
class Workload:
    """One CWT workload: the signal shape, the scales and the requested outputs."""
    name: str
    channels: int
    samples: int
    fs: float
    freqs: np.ndarray
    n_cycles: np.ndarray
    outputs: tuple          # subset of ("complex", "power", "phase")
    dtype: str              # "f32" or "f64" input/output
    decimation: int = 1
    seed: int = 0
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def scales(self):
        return len(self.freqs)

    @property
    def n_out(self):
        return -(-self.samples // self.decimation)

    @property
    def coefficients(self):
        return self.channels * self.scales * self.n_out

    def signal(self, channels=None, first_channel=0):
        np_dtype = np.float64 if self.dtype == "f64" else np.float32
        C = self.channels if channels is None else channels
        return eeg(self.seed, C, self.samples, self.fs, np_dtype, first_channel)


def workload(name):
    """The five workload shapes: plain, fused, batch, precision, serving."""
    if name == "plain":
        # 8 ch x 500 samples (1 s at 500 Hz), f64, 40 linear freqs 1-40 Hz, sigma 7, power.
        f = np.linspace(1.0, 40.0, 40)
        return Workload("plain", 8, 500, 500.0, f, np.full(40, 7.0), ("power",), "f64", 1, 1,
                        "8 ch x 500 @500 Hz f64, 40 freqs 1-40 Hz, n_cycles 7, power")
    if name == "fused":
        # 64 ch x 10000 (10 s at 1000 Hz), f32, 100 log freqs 1-100 Hz, sigma 3->10.
        f = np.geomspace(1.0, 100.0, 100)
        return Workload("fused", 64, 10000, 1000.0, f, np.linspace(3.0, 10.0, 100),
                        ("complex", "power"), "f32", 1, 2,
                        "64 ch x 10000 @1000 Hz f32, 100 log freqs 1-100 Hz, n_cycles 3..10, "
                        "complex64 + power")
    if name == "batch":
        f = np.geomspace(2.0, 80.0, 64)
        w = Workload("batch", 64, 8192, 1000.0, f, np.clip(f / 2.0, 3.0, 12.0), ("power",), "f32",
                     4, 3, "2048 epochs, n_e ~ U{256..8192}, 64 ch @1000 Hz, 64 log freqs 2-80 Hz, "
                     "n_cycles clip(f/2,3,12), power decimated x4")
        rng = np.random.default_rng(np.random.SeedSequence([3, 1_000_000]))
        lengths = rng.integers(256, 8193, size=2048)
        w.extra["epoch_lengths"] = lengths
        # epochs are windows of one continuous recording (event-locked epochs)
        w.extra["recording_samples"] = 1 << 19
        w.extra["epoch_starts"] = rng.integers(0, (1 << 19) - lengths + 1)
        return w
    if name == "precision":
        f = np.geomspace(0.5, 200.0, 128)
        return Workload("precision", 256, 122880, 2048.0, f, np.full(128, 7.0), ("power", "phase"),
                        "f32", 1, 4, "256 ch x 122880 @2048 Hz, 128 log freqs 0.5-200 Hz, "
                        "n_cycles 7, power + phase")
    if name == "serving":
        f = np.geomspace(1.0, 100.0, 64)
        return Workload("serving", 0, 2048, 0.0, f, np.full(64, 7.0), ("power",), "f32", 1, 5,
                        "32 streams, C in {8,32,64,128,256}, fs in {250,500,1000,2000,4000}, "
                        "W=2048, 50 ms hop, 64 log freqs 1-100 Hz")
    raise KeyError(name)


def batch_signal(w, epochs=None):
    """Packed float32 input of the batching workload: epoch e is the window
    [start_e, start_e + n_e) of one continuous C-channel recording, laid out
    [C][n_e] and packed back to back in epoch order.  Returns (packed array,
    per-epoch element offsets, recording [C][L])."""
    lengths = np.asarray(w.extra["epoch_lengths"])
    starts = np.asarray(w.extra["epoch_starts"])
    if epochs is not None:
        lengths, starts = lengths[:epochs], starts[:epochs]
    rec = eeg(w.seed, w.channels, int(w.extra["recording_samples"]), w.fs, np.float32)
    offs = np.zeros(len(lengths), dtype=np.int64)
    offs[1:] = np.cumsum(w.channels * lengths[:-1])
    packed = np.empty(int(w.channels * lengths.sum()), dtype=np.float32)
    for e, (n, s0) in enumerate(zip(lengths, starts)):
        packed[offs[e]:offs[e] + w.channels * n] = rec[:, s0:s0 + n].reshape(-1)
    return packed, offs, rec
