"""The X-engine at full workload shapes, compared with the CPU oracle on samples
it computes one by one.

- The paper's 192-input system exactly as the benchmark times it: eight
  distinct 1024-channel blocks of 8192 samples in one corr_push_blocks call
  (one CMAC launch and one int64 fold), then a dump with visibilities and
  Stokes.
- The large-N configuration at its own shape: 1024 dual-pol antennas (2048
  inputs), 256 channels, 16 blocks of 4096 samples (two launches of eight
  blocks) into an 8.6 GB int64 integration buffer, with three injected tones
  whose phases grow linearly with the input index at distinct gradients.

Drawing every block with the seeded generator would take minutes on the host,
so each test draws two base blocks and derives the others from them: a
per-input rotation of every sample by a power of j (paper shape), which turns
each visibility by j^(m_i - m_j), or a shift along time (large-N shape),
which leaves a block's visibilities unchanged but its bytes distinct.  A
kernel that read one block in place of another, or skipped one, would give a
different sum.  All comparisons are exact (integer arithmetic).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_THREADS = max(1, min(os.cpu_count() or 1, 64))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def corr(torch_cuda):
    from paper_2406_19013_gb300 import build
    build.build()
    from paper_2406_19013_gb300 import corr as c
    return c


def _rotation_tables():
    """tables[q][byte]: the sample multiplied by j^q (values in [-7, 7] only)."""
    b = np.arange(256)
    re = ((b >> 4) ^ 8) - 8
    im = ((b & 15) ^ 8) - 8
    out = []
    for q in range(4):
        r, i = re.copy(), im.copy()
        for _ in range(q):
            r, i = -i, r
        out.append((((r & 15) << 4) | (i & 15)).astype(np.uint8))
    return out


def _rotate_inputs(x, quarter_turns, tables):
    """Input i of every channel multiplied by j^quarter_turns[i]."""
    out = np.empty_like(x)
    for i, q in enumerate(quarter_turns):
        out[:, i, :] = tables[int(q)][x[:, i, :]]
    return out


def _autos(x):
    """sum_t |x_i(t)|^2 per channel and input, int64[C][N], in channel chunks."""
    C, N, T = x.shape
    chunk = max(1, (1 << 26) // (N * T))
    out = np.empty((C, N), dtype=np.int64)
    for c0 in range(0, C, chunk):
        s = x[c0:c0 + chunk].view(np.int8)
        re = (s >> 4).astype(np.int32)
        im = ((s << 4).astype(np.int8) >> 4).astype(np.int32)
        out[c0:c0 + chunk] = (re * re + im * im).sum(axis=2)
    return out


def _diag_index(n):
    return np.arange(n) * (np.arange(n) + 3) // 2


def test_paper_workload_as_benchmarked(corr, torch_cuda, oracle_mod, synth_mod):
    torch = torch_cuda
    w = synth_mod.workload("paper", seed=1)
    N, C, T = w.n_in, w.n_chan, w.block_len
    base = [w.block(b) for b in range(2)]
    tables = _rotation_tables()
    rng = np.random.default_rng(8)
    turns = [np.zeros(N, dtype=np.int64)] * 2 + [rng.integers(0, 4, size=N) for _ in range(6)]
    chans = [0, 1, 511, 777, 1023]
    dev, sub = [], []
    for k in range(8):
        xk = base[k % 2] if k < 2 else _rotate_inputs(base[k % 2], turns[k], tables)
        dev.append(torch.from_numpy(xk).cuda())
        sub.append(np.ascontiguousarray(xk[chans]))
        del xk
    with corr.Correlator(w.n_ant, w.n_pol, C, T) as xc:
        n0 = xc.launch_count()
        xc.push_blocks(dev)  # one CMAC launch of eight blocks, as in the benchmark
        assert xc.launch_count() - n0 == 1
        assert xc.samples_integrated() == 8 * T
        vis, st = xc.dump()
        xc.check()
    del dev
    vis = vis.cpu().numpy()
    st = st.cpu().numpy()
    # whole channels, visibilities and Stokes
    ov = None
    for s in sub:
        ov = oracle_mod.xcorr(s, vis=ov, n_threads=N_THREADS)
    assert np.array_equal(vis[chans], ov)
    assert np.array_equal(st[chans], oracle_mod.stokes(ov, w.n_ant))
    # random pairs of random channels, summed over the eight blocks one by one
    for _ in range(64):
        c = int(rng.integers(0, C))
        i = int(rng.integers(0, N))
        j = int(rng.integers(0, i + 1))
        want = [0, 0]
        for k in range(8):
            # V_k[i][j] = j^(m_i - m_j) V_base[i][j]
            re, im = oracle_mod.xcorr_pair(base[k % 2], c, i, j)
            for _ in range((int(turns[k][i]) - int(turns[k][j])) % 4):
                re, im = -im, re
            want[0] += re
            want[1] += im
        assert list(vis[c, i * (i + 1) // 2 + j]) == want, (c, i, j)
    # every auto-correlation of every channel (rotations leave autos unchanged)
    autos = 4 * (_autos(base[0]) + _autos(base[1]))
    diag = _diag_index(N)
    assert np.array_equal(vis[:, diag, 0], autos)
    assert not vis[:, diag, 1].any()


def test_large_n_at_full_shape(corr, torch_cuda, oracle_mod, synth_mod):
    torch = torch_cuda
    w = synth_mod.workload("large_n", seed=1)
    N, C, T = w.n_in, w.n_chan, w.block_len
    assert (N, C, T, w.n_blocks) == (2048, 256, 4096, 16)
    base = [w.block(b) for b in range(2)]
    with corr.Correlator(w.n_ant, w.n_pol, C, T) as xc:
        for g in range(2):  # two launches of eight distinct device blocks
            dev = []
            for k in range(8):
                b = 8 * g + k
                xk = base[b % 2] if b < 2 else np.roll(base[b % 2], 64 * b + 16, axis=2)
                dev.append(torch.from_numpy(np.ascontiguousarray(xk)).cuda())
                del xk
            xc.push_blocks(dev)
            torch.cuda.synchronize()
            del dev
        assert xc.samples_integrated() == 16 * T
        vis, _ = xc.dump(want_stokes=False)
        xc.check()
    vis = vis.cpu().numpy()
    # two whole channels against the oracle (eight copies of each base block)
    for c in (0, C - 1):
        ov = None
        for b in base:
            ov = oracle_mod.xcorr(np.ascontiguousarray(b[c:c + 1]), vis=ov, n_threads=N_THREADS)
        assert np.array_equal(vis[c:c + 1], 8 * ov), c
    # sampled pairs across the triangle's tiles
    rng = np.random.default_rng(5)
    for _ in range(64):
        c = int(rng.integers(0, C))
        i = int(rng.integers(0, N))
        j = int(rng.integers(0, i + 1))
        want = [8 * (a + b) for a, b in zip(oracle_mod.xcorr_pair(base[0], c, i, j),
                                            oracle_mod.xcorr_pair(base[1], c, i, j))]
        assert list(vis[c, i * (i + 1) // 2 + j]) == want, (c, i, j)
    # every auto of every channel
    diag = _diag_index(N)
    assert np.array_equal(vis[:, diag, 0], 8 * (_autos(base[0]) + _autos(base[1])))
    assert not vis[:, diag, 1].any()
    # the three injected tones: summing V_ij exp(-j g (i - j)) over the
    # baselines peaks at each tone's phase gradient g (the phase law of
    # Eq. 2 in input-index space); diagonal sums turn it into one FFT
    v = vis.sum(axis=0)
    ii = np.repeat(np.arange(N), np.arange(1, N + 1))
    jj = np.arange(ii.size) - ii * (ii + 1) // 2
    d = ii - jj
    s_re = np.bincount(d, weights=v[:, 0].astype(np.float64), minlength=N)
    s_im = np.bincount(d, weights=v[:, 1].astype(np.float64), minlength=N)
    s = s_re + 1j * s_im
    s[0] = 0.0  # autos carry no phase
    power = np.abs(np.fft.fft(s))
    top = set(int(k) for k in np.argsort(power)[-3:])
    assert top == {3, 40, 301}
