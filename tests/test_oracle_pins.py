"""Pins of the CPU oracle to things other than itself.

Each test checks the oracle against what the paper or the mathematics fixes:
hand-worked values (tests/golden), brute force with Python's own complex
arithmetic, a library matrix product, Hermitian symmetry, closed forms for
autos, bilinearity, conjugation under re<->im exchange, and the phase law of
Eq. 2 for injected tones and delays.
"""
import os

import numpy as np
import pytest

from conftest import GOLDEN


def _nib(v):
    v = int(v) & 15
    return v - 16 if v >= 8 else v


def _decode_py(b):
    return complex(_nib(int(b) >> 4), _nib(int(b)))


def _split(x):
    """Decoded integer real / imaginary parts via numpy's signed shifts."""
    s = x.astype(np.int8)
    re = (s >> 4).astype(np.int64)
    im = ((x << 4).astype(np.uint8).astype(np.int8) >> 4).astype(np.int64)
    return re, im


def _read_cmac_golden():
    d = {"bytes": {}, "vis": {}}
    with open(os.path.join(GOLDEN, "cmac_handworked.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] in ("n_in", "T"):
                d[line[0]] = int(line[1])
            elif line[0] == "bytes":
                d["bytes"][int(line[1])] = [int(v, 16) for v in line[2:]]
            elif line[0] == "vis":
                d["vis"][(int(line[1]), int(line[2]))] = (int(line[3]), int(line[4]))
    return d


def _read_stokes_golden():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "stokes_handworked.txt")) as f:
        for line in f:
            tok = line.split("#")[0].split()
            if not tok:
                continue
            if tok[0] == "case":
                cur = {"name": tok[1], "samples": [], "stokes": {}}
            elif tok[0] in ("n_ant", "T"):
                cur[tok[0]] = int(tok[1])
            elif tok[0] == "sample":
                cur["samples"].append(tuple(int(v) for v in tok[1:]))
            elif tok[0] == "stokes":
                cur["stokes"][(int(tok[1]), int(tok[2]))] = [int(v) for v in tok[3:]]
            elif tok[0] == "end":
                cases.append(cur)
    return cases


def test_decode_all_bytes(oracle_mod):
    # Sec. 2.1: 4-bit real (high nibble) + 4-bit imaginary (low nibble)
    for b in range(256):
        z = _decode_py(b)
        assert oracle_mod.decode(b) == (int(z.real), int(z.imag))


def test_golden_handworked(oracle_mod):
    g = _read_cmac_golden()
    n, T = g["n_in"], g["T"]
    x = np.array([g["bytes"][i] for i in range(n)], dtype=np.uint8).reshape(1, n, T)
    vis = oracle_mod.xcorr(x)
    assert vis.shape == (1, n * (n + 1) // 2, 2)
    for (i, j), (re, im) in g["vis"].items():
        p = oracle_mod.pair_index(i, j)
        assert tuple(vis[0, p]) == (re, im), (i, j)
        assert oracle_mod.xcorr_pair(x, 0, i, j) == (re, im)


def test_all_byte_pairs_brute_force(oracle_mod):
    # every (x0, x1) byte combination, one sample, as 65536 channels of N = 2
    b0 = np.arange(65536) & 255
    b1 = np.arange(65536) >> 8
    x = np.stack([b0, b1], axis=1).astype(np.uint8).reshape(65536, 2, 1)
    vis = oracle_mod.xcorr(x)
    lut = np.array([_decode_py(b) for b in range(256)])
    z0, z1 = lut[b0], lut[b1]
    want = np.stack([z0 * np.conj(z0), z1 * np.conj(z0), z1 * np.conj(z1)], axis=1)
    assert np.array_equal(vis[:, :, 0], want.real.astype(np.int64))
    assert np.array_equal(vis[:, :, 1], want.imag.astype(np.int64))


def test_python_complex_brute_force_small(oracle_mod, synth_mod):
    x = synth_mod.make_block(5, 3, 7, seed=11)
    vis = oracle_mod.xcorr(x)
    for c in range(3):
        for i in range(5):
            for j in range(i + 1):
                acc = 0j
                for t in range(7):
                    acc += _decode_py(x[c, i, t]) * _decode_py(x[c, j, t]).conjugate()
                p = oracle_mod.pair_index(i, j)
                assert (vis[c, p, 0], vis[c, p, 1]) == (int(acc.real), int(acc.imag))


@pytest.mark.parametrize("n_in,T", [(1, 5), (7, 33), (24, 300), (40, 1024)])
def test_library_matmul_crosscheck(oracle_mod, synth_mod, n_in, T):
    # Re V = A A^T + B B^T, Im V = B A^T - A B^T with A, B the integer real
    # and imaginary parts (a library int64 matrix product, exact)
    x = synth_mod.make_block(n_in, 4, T, seed=5 + n_in, tones=synth_mod.random_phase_tone(n_in, 3))
    vis = oracle_mod.xcorr(x, n_threads=2)
    A, B = _split(x)
    ii, jj = np.tril_indices(n_in)
    for c in range(4):
        re = A[c] @ A[c].T + B[c] @ B[c].T
        im = B[c] @ A[c].T - A[c] @ B[c].T
        assert np.array_equal(vis[c, :, 0], re[ii, jj])
        assert np.array_equal(vis[c, :, 1], im[ii, jj])
    # tril_indices enumerates (i, j) in the same row-major order as i(i+1)/2 + j
    assert all(oracle_mod.pair_index(i, j) == k for k, (i, j) in enumerate(zip(ii, jj)))


def test_hermitian_and_autos(oracle_mod, synth_mod):
    x = synth_mod.make_block(9, 2, 257, seed=3)
    full = oracle_mod.xcorr_full(x)
    tri = oracle_mod.xcorr(x)
    A, B = _split(x)
    for c in range(2):
        for i in range(9):
            # autos are real and equal the summed power
            assert full[c, i, i, 1] == 0
            assert full[c, i, i, 0] == int((A[c, i] ** 2 + B[c, i] ** 2).sum())
            assert full[c, i, i, 0] >= 0
            for j in range(9):
                assert full[c, i, j, 0] == full[c, j, i, 0]
                assert full[c, i, j, 1] == -full[c, j, i, 1]
                if j <= i:
                    assert tuple(tri[c, oracle_mod.pair_index(i, j)]) == tuple(full[c, i, j])


def test_extremes_and_empty(oracle_mod, synth_mod):
    # -8-8j everywhere: every product is (-8-8j)(-8+8j) = 128
    x = np.full((2, 3, 100), 0x88, dtype=np.uint8)
    vis = oracle_mod.xcorr(x)
    assert np.all(vis[..., 0] == 12800) and np.all(vis[..., 1] == 0)
    # -8 real against 7 imaginary: (-8)(-7j) ... check a mixed pair by hand
    x = np.zeros((1, 2, 1), dtype=np.uint8)
    x[0, 0, 0] = 0x80          # -8 + 0j
    x[0, 1, 0] = 0x07          #  0 + 7j
    vis = oracle_mod.xcorr(x)
    # V10 = (7j)(-8) = -56j
    assert tuple(vis[0, 1]) == (0, -56)
    # T = 0: nothing accumulates
    vis = oracle_mod.xcorr(np.zeros((2, 4, 0), dtype=np.uint8))
    assert not vis.any()


def test_accumulates_over_blocks(oracle_mod, synth_mod):
    b0 = synth_mod.make_block(6, 3, 64, seed=9, block=0)
    b1 = synth_mod.make_block(6, 3, 64, seed=9, block=1)
    acc = oracle_mod.xcorr(b0)
    oracle_mod.xcorr(b1, vis=acc)
    both = oracle_mod.xcorr(np.concatenate([b0, b1], axis=2))
    assert np.array_equal(acc, both)


def test_bilinear_and_swap(oracle_mod, synth_mod):
    rng = np.random.default_rng(4)
    re = rng.integers(-3, 4, size=(2, 6, 50))
    im = rng.integers(-3, 4, size=(2, 6, 50))
    v1 = oracle_mod.xcorr(synth_mod.pack(re, im))
    v2 = oracle_mod.xcorr(synth_mod.pack(2 * re, 2 * im))
    assert np.array_equal(v2, 4 * v1)
    vn = oracle_mod.xcorr(synth_mod.pack(-re, -im))
    assert np.array_equal(vn, v1)
    # x -> j conj(x) swaps re and im and conjugates every product
    vs = oracle_mod.xcorr(synth_mod.pack(im, re))
    assert np.array_equal(vs[..., 0], v1[..., 0]) and np.array_equal(vs[..., 1], -v1[..., 1])
    # x -> j x leaves every x_i conj(x_j) unchanged
    vj = oracle_mod.xcorr(synth_mod.pack(-im, re))
    assert np.array_equal(vj, v1)


def test_tone_phase_per_input(oracle_mod, synth_mod):
    # a common tone with phase phi_i per input: arg V_ij -> phi_i - phi_j (Eq. 2)
    n = 16
    tones = synth_mod.random_phase_tone(n, seed=21)
    x = synth_mod.make_block(n, 64, 2048, seed=21, tones=tones)
    vis = oracle_mod.xcorr(x, n_threads=4)
    v = (vis[..., 0] + 1j * vis[..., 1]).sum(axis=0)
    phi = tones.phase[0]
    for i in range(n):
        for j in range(i):
            want = phi[i] - phi[j]
            err = np.angle(v[oracle_mod.pair_index(i, j)] * np.exp(-1j * want))
            assert abs(err) < 0.2, (i, j, err)


def test_delay_phase_slope(oracle_mod, synth_mod):
    # Eq. 2: the visibility phase of a delayed copy grows linearly with
    # frequency, slope 2 pi tau.  Here tau is a per-input phase slope per
    # channel; the fitted slope of arg V_ij across channels is s_i - s_j.
    n, C = 4, 48
    slopes = np.array([0.0, 0.05, -0.08, 0.11])
    tones = synth_mod.delay_tone(n, seed=2, amp=3.0, slopes=slopes)
    x = synth_mod.make_block(n, C, 1024, seed=2, tones=tones, sigma=1.0)
    vis = oracle_mod.xcorr(x)
    ch = np.arange(C)
    for i in range(n):
        for j in range(i):
            ph = np.unwrap(np.angle(vis[:, oracle_mod.pair_index(i, j), 0]
                                    + 1j * vis[:, oracle_mod.pair_index(i, j), 1]))
            k = np.polyfit(ch, ph, 1)[0]
            assert abs(k - (slopes[i] - slopes[j])) < 2e-3, (i, j, k)


def test_gradient_tones_peak(oracle_mod, synth_mod):
    # tones with phase theta_k * i: summing V_ij exp(-j theta (i - j)) over
    # baselines peaks at each injected gradient
    n, T = 64, 2048
    th = [2 * np.pi * 3 / n, 2 * np.pi * 20 / n]
    tones = synth_mod.gradient_tones(n, th, [2.0, 2.0], [0.0, 37 / T])
    x = synth_mod.make_block(n, 2, T, seed=8, tones=tones)
    vis = oracle_mod.xcorr(x)
    v = (vis[..., 0] + 1j * vis[..., 1]).sum(axis=0)
    ii, jj = np.tril_indices(n, -1)
    vv = v[ii * (ii + 1) // 2 + jj]
    grid = 2 * np.pi * np.arange(n) / n
    power = np.array([abs((vv * np.exp(-1j * g * (ii - jj))).sum()) for g in grid])
    top = set(np.argsort(power)[-2:])
    assert top == {3, 20}


def test_stokes_golden(oracle_mod, synth_mod):
    for case in _read_stokes_golden():
        n_ant, T = case["n_ant"], case["T"]
        re = np.zeros((1, 2 * n_ant, T), dtype=np.int64)
        im = np.zeros_like(re)
        for i, t, a, b in case["samples"]:
            re[0, i, t], im[0, i, t] = a, b
        vis = oracle_mod.xcorr(synth_mod.pack(re, im))
        st = oracle_mod.stokes(vis, n_ant)
        for (p, q), want in case["stokes"].items():
            a = p * (p + 1) // 2 + q
            assert list(st[0, a].reshape(-1)) == want, (case["name"], p, q)


def test_stokes_closed_forms(oracle_mod, synth_mod):
    rng = np.random.default_rng(7)
    T = 200
    a = rng.integers(-7, 8, size=T)
    b = rng.integers(-7, 8, size=T)
    power = int((a * a + b * b).sum())
    zeros = np.zeros(T, dtype=np.int64)
    # X only: I = Q = |X|^2, U = V = 0
    st = oracle_mod.stokes(oracle_mod.xcorr(synth_mod.pack(np.stack([a, zeros])[None], np.stack([b, zeros])[None])), 1)
    assert list(st[0, 0].reshape(-1)) == [power, 0, power, 0, 0, 0, 0, 0]
    # Y only: I = |Y|^2, Q = -|Y|^2
    st = oracle_mod.stokes(oracle_mod.xcorr(synth_mod.pack(np.stack([zeros, a])[None], np.stack([zeros, b])[None])), 1)
    assert list(st[0, 0].reshape(-1)) == [power, 0, -power, 0, 0, 0, 0, 0]
    # Y = -X (linear at -45 deg): U = -2|X|^2
    st = oracle_mod.stokes(oracle_mod.xcorr(synth_mod.pack(np.stack([a, -a])[None], np.stack([b, -b])[None])), 1)
    assert list(st[0, 0].reshape(-1)) == [2 * power, 0, 0, 0, -2 * power, 0, 0, 0]
    # Y = j X (circular): V = -2|X|^2 ; Y = -j X: V = +2|X|^2
    st = oracle_mod.stokes(oracle_mod.xcorr(synth_mod.pack(np.stack([a, -b])[None], np.stack([b, a])[None])), 1)
    assert list(st[0, 0].reshape(-1)) == [2 * power, 0, 0, 0, 0, 0, -2 * power, 0]
    st = oracle_mod.stokes(oracle_mod.xcorr(synth_mod.pack(np.stack([a, b])[None], np.stack([b, -a])[None])), 1)
    assert list(st[0, 0].reshape(-1)) == [2 * power, 0, 0, 0, 0, 0, 2 * power, 0]


def test_stokes_auto_identities(oracle_mod, synth_mod):
    # for integrated autos the 2x2 coherency matrix is Hermitian PSD:
    # I, Q, U, V real; I >= |Q|; I^2 >= Q^2 + U^2 + V^2
    n_ant = 5
    x = synth_mod.make_block(2 * n_ant, 6, 512, seed=13, tones=synth_mod.random_phase_tone(2 * n_ant, 1))
    st = oracle_mod.stokes(oracle_mod.xcorr(x), n_ant)
    for c in range(6):
        for p in range(n_ant):
            s = st[c, p * (p + 1) // 2 + p]
            assert (s[:, 1] == 0).all()
            I, Q, U, V = (int(v) for v in s[:, 0])
            assert I >= abs(Q)
            assert I * I >= Q * Q + U * U + V * V


def test_stokes_cross_pairs_from_full_matrix(oracle_mod, synth_mod):
    # cross-antenna Stokes equal the same combinations of the full Hermitian
    # matrix read directly (both triangles from the full-matrix variant)
    n_ant = 4
    x = synth_mod.make_block(2 * n_ant, 2, 64, seed=17)
    full = oracle_mod.xcorr_full(x)
    st = oracle_mod.stokes(oracle_mod.xcorr(x), n_ant)
    F = full[..., 0] + 1j * full[..., 1]
    for c in range(2):
        for p in range(n_ant):
            for q in range(p + 1):
                XX, YY = F[c, 2 * p, 2 * q], F[c, 2 * p + 1, 2 * q + 1]
                XY, YX = F[c, 2 * p, 2 * q + 1], F[c, 2 * p + 1, 2 * q]
                want = [XX + YY, XX - YY, XY + YX, -1j * (XY - YX)]
                got = st[c, p * (p + 1) // 2 + q]
                for s in range(4):
                    assert complex(got[s, 0], got[s, 1]) == want[s]


def test_corner_turn_handworked(oracle_mod):
    # 3 samples x 2 channels x 2 inputs, every byte distinct: byte (t, c, i)
    # = 16 t + 4 c + i; the turned block holds input i's samples of channel c
    # in time order
    x = np.array([[[16 * t + 4 * c + i for i in range(2)] for c in range(2)] for t in range(3)],
                 dtype=np.uint8)
    out = oracle_mod.corner_turn(x)
    assert out.shape == (2, 2, 3)
    assert out[1, 0].tolist() == [4, 20, 36]
    assert out[0, 1].tolist() == [1, 17, 33]
    assert np.array_equal(out, np.transpose(x, (1, 2, 0)))


def test_corner_turn_feeds_the_correlation(oracle_mod, synth_mod):
    # the turned F-engine-order block correlates exactly like the block
    # generated in X-engine order
    x = synth_mod.make_block(6, 3, 40, seed=8)
    x_tcn = np.ascontiguousarray(np.transpose(x, (2, 0, 1)))
    assert np.array_equal(oracle_mod.corner_turn(x_tcn), x)
    assert np.array_equal(oracle_mod.xcorr(oracle_mod.corner_turn(x_tcn)), oracle_mod.xcorr(x))
