"""Pins of the F-engine oracle (oracle/fengine.py) against facts that its
definitions fix: an impulse through the filter bank (closed form, which fixes
the FIR indexing and the DFT sign), the prototype's textbook values (Hamming
end and centre, sinc zeros), the channel response of a polyphase filter bank
to a tone at a channel centre, superposition, the DC gain, and hand-worked
quantiser values."""
import numpy as np
import pytest

from oracle import fengine as F

P = F.P


def test_prototype_textbook_values():
    h = F.prototype()
    L = 4 * P
    assert h.shape == (L,)
    # Hamming end value 0.08 times sinc(-2) = 0; centre: sinc(0) = 1, w ~ 1
    assert abs(h[0]) < 1e-12
    assert abs(h[L // 2] - (0.54 - 0.46 * np.cos(2 * np.pi * (L // 2) / (L - 1)))) < 1e-15
    assert abs(h[L // 2] - 1.0) < 1e-6
    # sinc zeros whole channel-widths from the centre (inside the filter)
    for q in (-2, -1, 1):
        assert abs(h[L // 2 + q * P]) < 1e-12
    # the window is 0.08 at both ends and 1 in the middle (textbook Hamming)
    w = h[1:L // 2] / np.sinc((np.arange(1, L // 2) - L / 2) / P)
    assert abs(w[0] - (0.54 - 0.46 * np.cos(2 * np.pi / (L - 1)))) < 1e-12


@pytest.mark.parametrize("k0,j0,n0", [(0, 0, 0), (0, 3, 5), (2, 1, 1000), (1, 2, 2047)])
def test_impulse_closed_form(k0, j0, n0):
    # x = delta at sample (k0 + j0) P + n0: spectrum k0 sees only tap j0 at
    # position n0, so X_k0[c] = h[j0 P + n0] exp(-2 pi j n0 c / P)
    n_spec = 3
    x = np.zeros((1, (n_spec + 3) * P))
    x[0, (k0 + j0) * P + n0] = 1.0
    X = F.spectra(x)[0]
    h = F.prototype()
    c = np.arange(P // 2)
    want = h[j0 * P + n0] * np.exp(-2j * np.pi * n0 * c / P)
    assert np.allclose(X[k0], want, atol=1e-12, rtol=0)


def test_tone_at_a_channel_centre_stays_in_its_channel():
    # a 4-tap Hamming PFB passes a centred tone into its own channel and keeps
    # the rest below -45 dB (adjacent) and -65 dB (two or more channels away)
    f0 = 321
    t = np.arange(8 * P)
    x = (90 * np.cos(2 * np.pi * f0 * t / P))[None, :]
    m = np.abs(F.spectra(x)[0]).max(axis=0)
    assert int(np.argmax(m)) == f0
    assert max(m[f0 - 1], m[f0 + 1]) / m[f0] < 10 ** (-45 / 20)
    far = np.concatenate([m[:f0 - 1], m[f0 + 2:]])
    assert far.max() / m[f0] < 10 ** (-65 / 20)


def test_superposition_and_dc_gain():
    rng = np.random.default_rng(0)
    a = rng.integers(-128, 128, size=(2, 6 * P)).astype(np.float64)
    b = rng.integers(-128, 128, size=(2, 6 * P)).astype(np.float64)
    assert np.allclose(F.spectra(a + b), F.spectra(a) + F.spectra(b), atol=1e-6, rtol=0)
    # a constant input: channel 0 is the constant times the sum of all taps
    dc = F.spectra(np.full((1, 5 * P), 3.0))[0]
    assert np.allclose(dc[:, 0].real, 3.0 * F.prototype().sum(), atol=1e-9, rtol=0)
    assert np.allclose(dc[:, 0].imag, 0.0, atol=1e-9)


def test_quantize_handworked():
    z = np.array([0.49, 0.5, -0.5, 1.5, -2.5, 6.9, 7.5, -100, 3 - 2j, -7.49 + 0.51j])
    codes = F.quantize(z)
    # (re, im) -> high, low nibble, two's complement
    want = [(0, 0), (1, 0), (-1, 0), (2, 0), (-3, 0), (7, 0), (7, 0), (-7, 0), (3, -2), (-7, 1)]
    assert codes.tolist() == [((r & 15) << 4) | (i & 15) for r, i in want]
    assert codes[8] == 0x3E


def test_fengine_layout_and_eq():
    rng = np.random.default_rng(1)
    x = rng.integers(-20, 21, size=(3, 5 * P)).astype(np.int8)
    eq = rng.uniform(0.001, 0.01, size=(3, P // 2))
    out = F.fengine(x, eq)
    assert out.shape == (P // 2, 3, 2) and out.dtype == np.uint8
    z = F.prequant(x, eq)
    assert np.array_equal(out, F.quantize(z))
    # X-engine order: out[c][i][k] is spectrum k of input i in channel c
    X = F.spectra(x)
    assert np.allclose(z[17, 2, 1], X[2, 1, 17] * eq[2, 17])
