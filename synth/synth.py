"""Seeded synthetic voltages for the X-engine, shared by the CUDA path's tests
and the oracle's tests.

This module only draws inputs; it holds none of the correlator's arithmetic.
The generator itself is plain C (``synth.c``): complex Gaussian noise from a
counter-based Philox4x32-10 stream plus injected tones, rounded half away
from zero, clipped to [-7, 7] and packed as one byte per complex sample with
the real part in the high nibble (the 4-bit + 4-bit format of Sec. 2.1).

Workload recipes (``workload(name)``) mirror the sizes of the paper's
system: 96 dual-polarisation feeds = 192 inputs (Sec. 1), 1024 channels
over 125 MHz (Sec. 2.2), and 64 blocks of 8192 samples per channel, which
at 122.07 kHz per channel is the ~4 s integration of Sec. 2.4.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

TWO_PI = 2.0 * np.pi


def build(force: bool = False) -> str:
    """Compile libsynth.so with gcc (portable C, no arch flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fno-math-errno", "-std=c99", "-fPIC", "-shared", "-pthread",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_block.restype = ctypes.c_int
            lib.synth_block.argtypes = [
                ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_int]
            lib.synth_philox4x32_10.restype = None
            lib.synth_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


def philox4x32_10(counter, key):
    """One Philox4x32-10 evaluation (for known-answer tests)."""
    c = np.array(counter, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    _load().synth_philox4x32_10(c.ctypes.data, k.ctypes.data)
    return [int(v) for v in c]


@dataclasses.dataclass
class Tones:
    """Injected tones: amplitude, frequency (cycles/sample), per-input start
    phase (rad) and per-input phase slope across channels (rad/channel)."""
    amp: np.ndarray      # [K]
    freq: np.ndarray     # [K]
    phase: np.ndarray    # [K][n_in]
    slope: np.ndarray    # [K][n_in]

    @staticmethod
    def none(n_in: int) -> "Tones":
        z = np.zeros((0, n_in))
        return Tones(np.zeros(0), np.zeros(0), z, z)


def random_phase_tone(n_in: int, seed: int, amp: float = 2.0, freq: float = 0.0) -> Tones:
    """One tone of amplitude `amp` with a uniform random phase per input."""
    rng = np.random.default_rng([seed, 0x70E])
    ph = rng.uniform(0.0, TWO_PI, size=(1, n_in))
    return Tones(np.array([amp]), np.array([freq]), ph, np.zeros((1, n_in)))


def gradient_tones(n_in: int, thetas, amps, freqs) -> Tones:
    """Tones whose phase grows linearly with the input index: phase_k[i] =
    theta_k * i (the index-space analogue of the delay law of Eq. 2)."""
    idx = np.arange(n_in, dtype=np.float64)
    ph = np.stack([th * idx for th in thetas])
    return Tones(np.asarray(amps, float), np.asarray(freqs, float), ph, np.zeros_like(ph))


def delay_tone(n_in: int, seed: int, amp: float, slopes) -> Tones:
    """One tone whose phase grows linearly with the channel index by a
    per-input slope (rad/channel), like a cable delay (Eq. 2)."""
    rng = np.random.default_rng([seed, 0xDE1A])
    ph = rng.uniform(0.0, TWO_PI, size=(1, n_in))
    return Tones(np.array([amp]), np.array([0.0]), ph,
                 np.asarray(slopes, float).reshape(1, n_in))


def make_block(n_in: int, n_chan: int, T: int, seed: int, block: int = 0,
               sigma: float = 2.5, tones: Tones | None = None, c0: int = 0,
               n_threads: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """Return uint8[n_chan][n_in][T] for channels c0..c0+n_chan-1 of `block`."""
    if tones is None:
        tones = Tones.none(n_in)
    if out is None:
        out = np.empty((n_chan, n_in, T), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.shape == (n_chan, n_in, T) and out.flags.c_contiguous
    amp = np.ascontiguousarray(tones.amp, dtype=np.float64)
    freq = np.ascontiguousarray(tones.freq, dtype=np.float64)
    ph = np.ascontiguousarray(tones.phase, dtype=np.float64).reshape(-1)
    sl = np.ascontiguousarray(tones.slope, dtype=np.float64).reshape(-1)
    k = len(amp)
    assert ph.size == k * n_in and sl.size == k * n_in
    if n_threads is None:
        n_threads = max(1, min(os.cpu_count() or 1, 32))
    rc = _load().synth_block(out.ctypes.data, n_in, n_chan, T, c0, seed & (2**64 - 1), block,
                             sigma, k, amp.ctypes.data, freq.ctypes.data, ph.ctypes.data,
                             sl.ctypes.data, n_threads)
    if rc != 0:
        raise ValueError("synth_block rejected its arguments")
    return out


def pack(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack integer real/imag parts in [-8, 7] into bytes (high nibble = real)."""
    re = np.asarray(re, dtype=np.int64)
    im = np.asarray(im, dtype=np.int64)
    if re.min(initial=0) < -8 or re.max(initial=0) > 7 or im.min(initial=0) < -8 or im.max(initial=0) > 7:
        raise ValueError("4-bit two's complement range is [-8, 7]")
    return (((re & 15) << 4) | (im & 15)).astype(np.uint8)


@dataclasses.dataclass
class Workload:
    name: str
    n_ant: int
    n_pol: int
    n_chan: int
    block_len: int
    n_blocks: int
    seed: int
    tones: Tones

    @property
    def n_in(self) -> int:
        return self.n_ant * self.n_pol

    @property
    def pairs(self) -> int:
        return self.n_in * (self.n_in + 1) // 2

    def block(self, b: int, c0: int = 0, n_chan: int | None = None, out=None, n_threads=None):
        n_chan = self.n_chan - c0 if n_chan is None else n_chan
        return make_block(self.n_in, n_chan, self.block_len, self.seed, b, 2.5, self.tones,
                          c0=c0, out=out, n_threads=n_threads)


def workload(name: str, seed: int = 1) -> Workload:
    """Named workloads with the shapes of the paper's system.

    tiny   : 8 dual-pol antennas (16 inputs), 64 channels, 2048 samples, 1 block
    paper  : 96 dual-pol antennas (192 inputs), 1024 channels, 8192 samples, 64 blocks
    large_n: 1024 dual-pol antennas (2048 inputs), 256 channels, 4096 samples, 16 blocks
    """
    if name == "tiny":
        n = 16
        return Workload(name, 8, 2, 64, 2048, 1, seed, random_phase_tone(n, seed))
    if name == "paper":
        n = 192
        return Workload(name, 96, 2, 1024, 8192, 64, seed, random_phase_tone(n, seed))
    if name == "large_n":
        n = 2048
        th = [2 * np.pi * 3 / n, 2 * np.pi * 40 / n, 2 * np.pi * 301 / n]
        # distinct tone frequencies (whole cycles per block) keep the tones
        # orthogonal over an integration
        return Workload(name, 1024, 2, 256, 4096, 16, seed,
                        gradient_tones(n, th, [1.2, 1.2, 1.2], [0.0, 17 / 4096, 101 / 4096]))
    raise KeyError(name)


# Input counts of the batched workload: arrays from 16 to 256 dual-pol antennas
BATCH_N = (32, 64, 128, 192, 256, 512)


def batched_instances(n_inst: int = 64, seed: int = 3):
    """Shapes of a batch of independent correlators: n_inst tuples
    (n_ant, n_pol, n_chan, block_len).  Input counts cycle through BATCH_N
    (dual-pol), channel counts are uniform in [16, 1024] and block lengths
    uniform in [256, 16384] on a 16-sample grid (so rows need no re-pitching,
    while most are not whole 64-sample chunks)."""
    rng = np.random.default_rng([seed, 0xBA7C])
    out = []
    for k in range(n_inst):
        n = BATCH_N[k % len(BATCH_N)]
        c = int(rng.integers(16, 1025))
        t = 16 * int(rng.integers(16, 1025))
        out.append((n // 2, 2, c, t))
    return out


def pool_offsets(sizes, pool_bytes: int, seed: int = 4):
    """Seeded 16-byte-aligned start offsets of windows of the given sizes in a
    byte pool of pool_bytes (every window fits)."""
    rng = np.random.default_rng([seed, 0x9001])
    out = []
    for sz in sizes:
        span = pool_bytes - int(sz)
        if span < 0:
            raise ValueError("window larger than the pool")
        out.append(16 * int(rng.integers(0, span // 16 + 1)))
    return out


# Input counts of the served workload: six arrays, dual polarisation
SERVED_N = (32, 96, 192, 192, 384, 512)


def served_arrays(seed: int = 6):
    """Shapes of the served arrays: (n_ant, n_pol, n_chan, block_len) with the
    input counts of SERVED_N, channel counts uniform in [64, 2048] and block
    lengths uniform in [1024, 8192] on a 16-sample grid."""
    rng = np.random.default_rng([seed, 0x5E4D])
    out = []
    for n in SERVED_N:
        c = int(rng.integers(64, 2049))
        t = 16 * int(rng.integers(64, 513))
        out.append((n // 2, 2, c, t))
    return out


def poisson_requests(n: int, rate_per_s: float, n_arrays: int, seed: int):
    """n requests (arrival time in s from the start, array index) of a Poisson
    process of the given rate, each for an array drawn uniformly."""
    rng = np.random.default_rng([seed, 0xA331])
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    a = rng.integers(0, n_arrays, size=n)
    return [(float(ti), int(ai)) for ti, ai in zip(t, a)]


def adc_streams(n_in: int, n_samples: int, seed: int, sigma: float = 20.0,
                tone_bins=(), tone_amp: float = 8.0, P: int = 2048) -> np.ndarray:
    """8-bit ADC samples int8[n_in][n_samples]: Gaussian noise of standard
    deviation sigma plus, for each entry of tone_bins, a sinusoid at that
    channel centre (bin b of a P-point transform) with a random phase per
    input; rounded half away from zero and clipped to [-128, 127]."""
    rng = np.random.default_rng([seed, 0xADC0])
    x = rng.normal(0.0, sigma, size=(n_in, n_samples))
    t = np.arange(n_samples)
    for b in tone_bins:
        ph = rng.uniform(0.0, 2 * np.pi, size=(n_in, 1))
        x += tone_amp * np.cos(2 * np.pi * b * t[None, :] / P + ph)
    r = np.sign(x) * np.floor(np.abs(x) + 0.5)
    return np.clip(r, -128, 127).astype(np.int8)


def eq_for_noise(n_in: int, sigma: float, target_rms: float = 2.5,
                 proto_sq_sum: float | None = None) -> np.ndarray:
    """EQ gains float32[n_in][1024] that scale white noise of standard
    deviation sigma to target_rms per real component after the filter bank
    (rms per component = sigma sqrt(sum h^2 / 2))."""
    if proto_sq_sum is None:
        L = 4 * 2048
        m = np.arange(L)
        h = (0.54 - 0.46 * np.cos(2 * np.pi * m / (L - 1))) * np.sinc((m - L / 2) / 2048)
        proto_sq_sum = float((h * h).sum())
    g = target_rms / (sigma * np.sqrt(proto_sq_sum / 2.0))
    return np.full((n_in, 1024), g, dtype=np.float32)
