"""Oracle of the F-engine (test infrastructure only: imported by tests,
``__graft_entry__.smoke`` and ``bench.py``'s CPU baseline, never by the
product path).

What the F-engine computes (Sec. 2.1; the paper gives the parameters and
names the CASPER blocks, not the formulas, so the formulas below are the
standard polyphase filter bank that those parameters describe):

- Input: 8-bit ADC samples, one stream per input.
- Polyphase FIR (``pfb_fir``): P = 2048 points ("PFB size 2^11"), 4 taps,
  Hamming window.  The prototype filter has L = 4 P coefficients,
      h[m] = w[m] sinc((m - L/2) / P),   w[m] = 0.54 - 0.46 cos(2 pi m / (L - 1)),
  with sinc(x) = sin(pi x) / (pi x).  Spectrum k is formed from samples
  [k P, (k + 4) P) as
      v_k[n] = sum_{j=0..3} h[j P + n] x[(k + j) P + n],   n = 0 .. P-1.
- Real FFT of size P (``fft_biplex_real_2x``, "FFT size 2^11"), keeping
  channels 0 .. P/2 - 1 (1024 channels):
      X_k[c] = sum_n v_k[n] exp(-2 pi j n c / P).
  The FPGA's fixed-point widths and shift schedule only scale the result;
  the scale is absorbed by the EQ gains, so no normalisation is applied.
- EQ: each (input, channel) has its own real gain g[i][c]; the quantiser
  sees g X.
- Requantisation to 4-bit real and 4-bit imaginary parts: round half away
  from zero, clip to [-7, 7] (the symmetric range keeps conj exact), packed
  one byte per sample with the real part in the high nibble.
- Corner turn (Transpose): out[c][i][k], the X-engine's input order.

Everything here is numpy in float64; numpy's FFT serves as the library
step for the DFT sum above (pinned against the direct sum in the tests).
"""
from __future__ import annotations

import numpy as np

P = 2048          # PFB / FFT size
TAPS = 4
N_CHAN = P // 2   # channels kept


def prototype(P: int = P, taps: int = TAPS) -> np.ndarray:
    """The Hamming-windowed sinc prototype filter h[m], m = 0 .. taps P - 1."""
    L = taps * P
    m = np.arange(L, dtype=np.float64)
    w = 0.54 - 0.46 * np.cos(2.0 * np.pi * m / (L - 1))
    return w * np.sinc((m - L / 2) / P)


def pfb_fir(x: np.ndarray, P: int = P, taps: int = TAPS) -> np.ndarray:
    """v[i][k][n] = sum_j h[j P + n] x[i][(k + j) P + n] for every spectrum k
    whose samples [k P, (k + taps) P) lie inside the stream.
    x: [n_in][n_samples] (any real dtype)."""
    x = np.asarray(x, dtype=np.float64)
    n_in, n_samp = x.shape
    n_spec = n_samp // P - taps + 1
    h = prototype(P, taps).reshape(taps, P)
    seg = x[:, :(n_spec + taps - 1) * P].reshape(n_in, n_spec + taps - 1, P)
    v = np.zeros((n_in, n_spec, P), dtype=np.float64)
    for j in range(taps):
        v += h[j][None, None, :] * seg[:, j:j + n_spec, :]
    return v


def spectra(x: np.ndarray, P: int = P, taps: int = TAPS) -> np.ndarray:
    """X[i][k][c], c = 0 .. P/2 - 1: the DFT of each FIR output."""
    v = pfb_fir(x, P, taps)
    return np.fft.fft(v, axis=2)[:, :, :P // 2]


def quantize(z: np.ndarray) -> np.ndarray:
    """Complex values -> packed 4+4-bit bytes (round half away from zero,
    clip to [-7, 7], real part in the high nibble)."""
    def q(a):
        r = np.sign(a) * np.floor(np.abs(a) + 0.5)
        return np.clip(r, -7, 7).astype(np.int64)
    re, im = q(np.real(z)), q(np.imag(z))
    return (((re & 15) << 4) | (im & 15)).astype(np.uint8)


def fengine(x: np.ndarray, eq: np.ndarray | None = None, P: int = P,
            taps: int = TAPS) -> np.ndarray:
    """Packed channel samples in X-engine order, uint8[P/2][n_in][n_spec].
    x: int8 [n_in][n_samples]; eq: float [n_in][P/2] gains (1 if None)."""
    X = spectra(x, P, taps)
    n_in = X.shape[0]
    g = np.ones((n_in, P // 2)) if eq is None else np.asarray(eq, dtype=np.float64)
    codes = quantize(X * g[:, None, :])            # [n_in][n_spec][P/2]
    return np.ascontiguousarray(np.transpose(codes, (2, 0, 1)))


def prequant(x: np.ndarray, eq: np.ndarray | None = None, P: int = P,
             taps: int = TAPS) -> np.ndarray:
    """g X in X-engine order, complex [P/2][n_in][n_spec] (what the quantiser
    sees), for tolerance checks near rounding boundaries."""
    X = spectra(x, P, taps)
    n_in = X.shape[0]
    g = np.ones((n_in, P // 2)) if eq is None else np.asarray(eq, dtype=np.float64)
    return np.ascontiguousarray(np.transpose(X * g[:, None, :], (2, 0, 1)))
