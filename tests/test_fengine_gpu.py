"""The GPU F-engine (corr_fengine_*) against the oracle of oracle/fengine.py.

The kernel computes in fp32 and the oracle in fp64, so:
- The spectra must agree within 1e-5 of the largest |g X| of the run.  The
  rounding error of a P = 2048 fp32 filter bank and FFT is of order
  eps32 log2(P) max|X|, about 1e-6 of the maximum.
- Each 4-bit code must equal the oracle's, except where the oracle's g X lies
  within 1e-3 (quantiser units) of a rounding boundary.  There it may differ
  by one step.
Also covered: the channel response to a tone, and the chain from F-engine
output to the X-engine."""
import numpy as np
import pytest

from oracle import fengine as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def corr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19013_gb300 import build
    build.build()
    from paper_2406_19013_gb300 import corr as c
    return c


def _run(corr, x, eq, n_spec):
    import torch
    n_in = x.shape[0]
    with corr.FEngine(n_in, n_spec, eq=eq) as fe:
        d = torch.from_numpy(x).cuda()
        codes = fe.run(d).cpu().numpy()
        spec = fe.spectra(d).cpu().numpy()
    return codes, spec[..., 0] + 1j * spec[..., 1]


def _signed(nib):
    nib = nib.astype(np.int64)
    return np.where(nib >= 8, nib - 16, nib)


def _check_codes(codes, z, tau=1e-3, max_frac=1e-3):
    """GPU codes vs the oracle's: equal, or one step apart in a component
    whose exact value lies within tau of a rounding boundary (k + 1/2)."""
    want = F.quantize(z)
    bad = codes != want
    assert bad.mean() <= max_frac
    if not bad.any():
        return
    for shift, part in ((4, np.real(z[bad])), (0, np.imag(z[bad]))):
        d = np.abs(_signed((codes[bad] >> shift) & 15) - _signed((want[bad] >> shift) & 15))
        a = np.abs(part)
        near = np.abs(a - np.floor(a) - 0.5) < tau
        assert d.max() <= 1
        assert np.all((d == 0) | near)


@pytest.mark.parametrize("n_in,n_spec", [(1, 1), (3, 40), (5, 33), (2, 64)])
def test_fengine_matches_oracle(corr, synth_mod, n_in, n_spec):
    x = synth_mod.adc_streams(n_in, (n_spec + 3) * F.P, seed=n_in * 100 + n_spec,
                              tone_bins=(37, 500))
    rng = np.random.default_rng(n_spec)
    eq = (synth_mod.eq_for_noise(n_in, 20.0) * rng.uniform(0.5, 2.0, size=(n_in, 1024))
          ).astype(np.float32)
    codes, spec = _run(corr, x, eq, n_spec)
    z = F.prequant(x, eq.astype(np.float64))
    assert np.abs(spec - z).max() <= 1e-5 * np.abs(z).max()
    assert codes.shape == (1024, n_in, n_spec)
    _check_codes(codes, z)


def test_fengine_tone_response(corr):
    # a tone at a channel centre through the kernel stays in its channel
    f0, n_spec = 257, 8
    t = np.arange((n_spec + 3) * F.P)
    x = np.round(90 * np.cos(2 * np.pi * f0 * t / F.P)).astype(np.int8)[None, :]
    _, spec = _run(corr, x, np.ones((1, 1024), np.float32), n_spec)
    m = np.abs(spec[:, 0, :]).max(axis=1)
    assert int(np.argmax(m)) == f0
    assert max(m[f0 - 1], m[f0 + 1]) / m[f0] < 10 ** (-45 / 20)


def test_fengine_feeds_the_xengine(corr, oracle_mod, synth_mod):
    # F-engine codes go straight into a correlator context: the visibilities
    # equal the X-engine oracle on the same codes
    import torch
    n_ant, n_spec = 8, 256
    n_in = 2 * n_ant
    x = synth_mod.adc_streams(n_in, (n_spec + 3) * F.P, seed=7, tone_bins=(100,))
    eq = synth_mod.eq_for_noise(n_in, 20.0)
    with corr.FEngine(n_in, n_spec, eq=eq) as fe:
        codes = fe.run(torch.from_numpy(x).cuda())
    with corr.Correlator(n_ant, 2, 1024, n_spec) as xc:
        xc.push_block(codes)
        vis, st = xc.dump()
        xc.check()
    c = codes.cpu().numpy()
    want = oracle_mod.xcorr(c)
    assert np.array_equal(vis.cpu().numpy(), want)
    assert np.array_equal(st.cpu().numpy(), oracle_mod.stokes(want, n_ant))
    _check_codes(c, F.prequant(x, eq.astype(np.float64)))


def test_fengine_paper_size_sampled(corr, synth_mod):
    # 192 inputs x 8192 spectra (3.2 GB of ADC samples): two inputs' first
    # and last 32 spectra against the oracle
    import torch
    n_in, n_spec = 192, 8192
    n_samp = (n_spec + 3) * F.P
    rng = np.random.default_rng(3)
    x = rng.integers(-40, 41, size=(n_in, n_samp), dtype=np.int8)
    eq = synth_mod.eq_for_noise(n_in, 23.7)
    with corr.FEngine(n_in, n_spec, eq=eq) as fe:
        codes = fe.run(torch.from_numpy(x).cuda())
        for i in (0, 191):
            for k0 in (0, n_spec - 32):
                seg = x[i:i + 1, k0 * F.P:(k0 + 32 + 3) * F.P]
                z = F.prequant(seg, eq[i:i + 1].astype(np.float64))
                _check_codes(codes[:, i:i + 1, k0:k0 + 32].cpu().numpy(), z)


def test_fengine_rejects_unaligned_samples(corr):
    # the samples are copied into shared memory in 16-byte pieces: a stream
    # that does not start on a 16-byte boundary is refused before any launch
    import torch
    n_in, n_spec = 1, 4
    n = n_in * (n_spec + 3) * F.P
    base = torch.zeros(n + 16, dtype=torch.int8, device="cuda")
    with corr.FEngine(n_in, n_spec) as fe:
        for off in (8, 4, 1):
            with pytest.raises(corr.CorrError) as ei:
                fe.run(base[off:off + n])
            assert ei.value.code == corr.CORR_EINVAL
            with pytest.raises(corr.CorrError) as ei:
                fe.spectra(base[off:off + n])
            assert ei.value.code == corr.CORR_EINVAL
        fe.run(base[16:16 + n])
        torch.cuda.synchronize()
