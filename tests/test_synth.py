"""The seeded input generator: known answers, determinism and ranges."""
import numpy as np


def test_philox_known_answers(synth_mod):
    # Philox4x32-10 known-answer vectors (Salmon et al., SC'11; Random123)
    assert synth_mod.philox4x32_10([0, 0, 0, 0], [0, 0]) == [
        0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert synth_mod.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert synth_mod.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                                   [0xA4093822, 0x299F31D0]) == [
        0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_deterministic_and_thread_independent(synth_mod):
    tones = synth_mod.random_phase_tone(12, 3)
    a = synth_mod.make_block(12, 9, 333, seed=3, tones=tones, n_threads=1)
    b = synth_mod.make_block(12, 9, 333, seed=3, tones=tones, n_threads=5)
    assert np.array_equal(a, b)
    # a channel subset equals the same channels of the full block
    c = synth_mod.make_block(12, 3, 333, seed=3, tones=tones, c0=4)
    assert np.array_equal(c, a[4:7])
    # another block or seed differs
    assert not np.array_equal(a, synth_mod.make_block(12, 9, 333, seed=3, block=1, tones=tones))
    assert not np.array_equal(a, synth_mod.make_block(12, 9, 333, seed=4, tones=tones))


def test_range_and_noise_level(synth_mod):
    x = synth_mod.make_block(8, 16, 4096, seed=1)
    re = (x.astype(np.int8) >> 4).astype(np.int64)
    im = ((x << 4).astype(np.uint8).astype(np.int8) >> 4).astype(np.int64)
    assert re.min() >= -7 and re.max() <= 7 and im.min() >= -7 and im.max() <= 7
    # sigma 2.5 noise rounded to integers: var ~ 6.25 + 1/12, clipping trims a little
    assert abs(re.std() - 2.5) < 0.1 and abs(im.std() - 2.5) < 0.1
    assert abs(re.mean()) < 0.02 and abs(im.mean()) < 0.02
    assert abs(np.corrcoef(re.ravel(), im.ravel())[0, 1]) < 0.01


def test_pack_roundtrip(synth_mod):
    v = np.arange(-8, 8)
    re, im = np.meshgrid(v, v, indexing="ij")
    b = synth_mod.pack(re, im)
    assert len(set(b.ravel().tolist())) == 256
    back_re = (b.astype(np.int8) >> 4)
    back_im = ((b << 4).astype(np.uint8).astype(np.int8) >> 4)
    assert np.array_equal(back_re, re) and np.array_equal(back_im, im)
