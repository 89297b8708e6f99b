"""Parity of the CUDA X-engine with the CPU oracle, through the C ABI.

Integer arithmetic end to end: every comparison is exact (bit-for-bit int64
visibilities and Stokes products); no tolerance applies anywhere.
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


def _run(corr, torch, blocks, n_ant, n_pol, want_stokes=True):
    C, N, T = blocks[0].shape
    with corr.Correlator(n_ant, n_pol, C, T) as xc:
        for b in blocks:
            xc.push_block(torch.from_numpy(b).cuda())
        vis, st = xc.dump(want_stokes=want_stokes and n_pol == 2)
        xc.check()
        assert xc.samples_integrated() == 0
        return vis.cpu().numpy(), (st.cpu().numpy() if st is not None else None)


def _oracle(oracle_mod, blocks, n_ant, n_pol):
    vis = None
    for b in blocks:
        vis = oracle_mod.xcorr(b, vis=vis, n_threads=N_THREADS)
    st = oracle_mod.stokes(vis, n_ant) if n_pol == 2 else None
    return vis, st


def test_tiny_workload(corr, torch_cuda, oracle_mod, synth_mod):
    # 8 dual-pol antennas, 64 channels, 2048 samples, noise + tone
    w = synth_mod.workload("tiny")
    x = w.block(0)
    vis, st = _run(corr, torch_cuda, [x], w.n_ant, w.n_pol)
    ov, ost = _oracle(oracle_mod, [x], w.n_ant, w.n_pol)
    assert np.array_equal(vis, ov)
    assert np.array_equal(st, ost)


@pytest.mark.parametrize("n_ant,n_pol,C,T,nb", [
    (1, 1, 3, 16, 1),        # one input
    (33, 1, 4, 48, 3),       # ragged N, T not a multiple of the 32-sample chunk
    (64, 2, 3, 4096, 1),     # N = 128: two full row tiles
    (96, 2, 7, 8192, 2),     # the paper's 192 inputs, few channels
    (100, 2, 5, 1000, 2),    # N = 200: two units; T % 16 != 0 (pitched staging)
    (128, 2, 2, 512, 1),     # N = 256: largest single window
    (150, 2, 3, 512, 1),     # N = 300: row-tile pairs against 256-column pieces
    (320, 2, 2, 256, 1),     # N = 640: off-diagonal pieces
    (17, 2, 9, 2056, 1),     # N = 34, T % 32 = 8
    (5, 2, 11, 1024, 2),     # N = 10: tiles of four 16-row channels, 11 channels (last unit partial)
    (10, 2, 9, 2048, 1),     # N = 20: tiles of two 32-row channels, ragged rows
    (16, 2, 3, 256, 1),      # N = 32: tiles of two full 32-row channels, 3 channels
    (8, 1, 17, 512, 2),      # N = 8 single-pol, 17 channels
])
def test_ragged_shapes(corr, torch_cuda, oracle_mod, synth_mod, n_ant, n_pol, C, T, nb):
    N = n_ant * n_pol
    tones = synth_mod.random_phase_tone(N, 5)
    blocks = [synth_mod.make_block(N, C, T, seed=100 + N, block=b, tones=tones) for b in range(nb)]
    vis, st = _run(corr, torch_cuda, blocks, n_ant, n_pol)
    ov, ost = _oracle(oracle_mod, blocks, n_ant, n_pol)
    assert np.array_equal(vis, ov)
    if n_pol == 2:
        assert np.array_equal(st, ost)


@pytest.mark.parametrize("n_ant,n_pol,C,T,nb", [
    (20, 2, 3, 20000, 7),    # 6 blocks per launch (6 * 20000 <= 131071), then 1
    (96, 2, 4, 8192, 9),     # 8 blocks per launch, then 1
    (9, 1, 5, 1000, 3),      # pitched staging: one block per launch
])
def test_push_blocks_groups(corr, torch_cuda, oracle_mod, synth_mod, n_ant, n_pol, C, T, nb):
    torch = torch_cuda
    N = n_ant * n_pol
    blocks = [synth_mod.make_block(N, C, T, seed=7, block=b) for b in range(nb)]
    dev = [torch.from_numpy(b).cuda() for b in blocks]
    with corr.Correlator(n_ant, n_pol, C, T) as xc:
        n0 = xc.launch_count()
        xc.push_blocks(dev)
        assert xc.samples_integrated() == nb * T
        vis, st = xc.dump()
        xc.check()
        launches = xc.launch_count() - n0
    ov, ost = _oracle(oracle_mod, blocks, n_ant, n_pol)
    assert np.array_equal(vis.cpu().numpy(), ov)
    if n_pol == 2:
        assert np.array_equal(st.cpu().numpy(), ost)
    per = 1 if T % 16 else min(8, 131071 // T)
    cmac_launches = -(-nb // per)
    assert launches == cmac_launches + (nb if T % 16 else 0) + 1


def test_push_blocks_rejects(corr, torch_cuda):
    torch = torch_cuda
    with corr.Correlator(4, 2, 2, 64) as xc:
        with pytest.raises(corr.CorrError) as e:
            xc.push_blocks([])
        assert e.value.code == corr.CORR_EINVAL
        good = torch.zeros(2 * 8 * 64 + 16, dtype=torch.uint8, device="cuda")
        with pytest.raises(corr.CorrError) as e:
            xc.push_blocks([good.data_ptr(), good.data_ptr() + 8])  # misaligned second block
        assert e.value.code == corr.CORR_EINVAL
        with pytest.raises(corr.CorrError):
            xc.push_blocks([good.data_ptr(), 0])
        # nothing was enqueued by the rejected calls
        assert xc.samples_integrated() == 0
        v, _ = xc.dump()
        assert not v.cpu().numpy().any()


def test_extremes_at_max_block_len(corr, torch_cuda, oracle_mod, synth_mod):
    # The largest block keeps every fp32 partial an exact integer: -8-8j on
    # every sample gives autos of 128 * 131071 = 16777088 (< 2^24).  The
    # second block adds small values after a large running sum, which an
    # accumulator that dropped low-order bits would lose.
    T = 131071
    n_ant, C = 8, 2
    N = 2 * n_ant
    x0 = np.full((C, N, T), 0x88, dtype=np.uint8)
    rng = np.random.default_rng(3)
    re = rng.integers(-8, 8, size=(C, N, T))
    im = rng.integers(-8, 8, size=(C, N, T))
    x1 = synth_mod.pack(re, im)
    x1[:, :, : 3 * T // 4] = 0x88
    small = rng.integers(-1, 2, size=(C, N, T // 4))
    x1[:, :, 3 * T // 4: 3 * T // 4 + T // 4] = synth_mod.pack(small, -small)
    for blocks in ([x0], [x1], [x0, x1]):
        vis, st = _run(corr, torch_cuda, blocks, n_ant, 2)
        ov, ost = _oracle(oracle_mod, blocks, n_ant, 2)
        assert np.array_equal(vis, ov)
        assert np.array_equal(st, ost)
        if len(blocks) == 1 and blocks[0] is x0:
            assert (vis[..., 0] == 128 * T).all() and not vis[..., 1].any()


@pytest.mark.parametrize("T,nb", [(300000, 1), (200001, 2)])
def test_blocks_longer_than_the_fold_window(corr, torch_cuda, oracle_mod, synth_mod, T, nb):
    # Runs of -8-8j longer than 131071 samples: an auto reaches 128 x the run
    # length > 2^24, which stays exact only if every item folds its fp32
    # partials into int64 within the window.  T = 200001 also takes the
    # pitched staging path (T % 16 != 0).
    n_ant, C = 8, 2
    N = 2 * n_ant
    rng = np.random.default_rng(T)
    blocks = []
    for b in range(nb):
        x = synth_mod.make_block(N, C, T, seed=40 + b, tones=synth_mod.random_phase_tone(N, 40))
        x[:, :, : 2 * T // 3] = 0x88
        x[:, 3, T // 3: T // 3 + 4096] = rng.integers(0, 256, size=(C, 4096), dtype=np.uint8)
        blocks.append(x)
    vis, st = _run(corr, torch_cuda, blocks, n_ant, 2)
    ov, ost = _oracle(oracle_mod, blocks, n_ant, 2)
    assert np.array_equal(vis, ov)
    assert np.array_equal(st, ost)
    assert ov[:, 0, 0].min() > 2 ** 24  # the check above is beyond one fp32 partial


def test_all_byte_values(corr, torch_cuda, oracle_mod):
    # every byte value against every other, 16 inputs x 256 samples
    N, T = 16, 256
    x = np.empty((2, N, T), dtype=np.uint8)
    for i in range(N):
        x[0, i] = (np.arange(T) * (2 * i + 1) + i) % 256
        x[1, i] = (np.arange(T) * 7 + 31 * i) % 256
    vis, st = _run(corr, torch_cuda, [x], 8, 2)
    ov, ost = _oracle(oracle_mod, [x], 8, 2)
    assert np.array_equal(vis, ov)
    assert np.array_equal(st, ost)


def test_dump_semantics(corr, torch_cuda, oracle_mod, synth_mod):
    torch = torch_cuda
    n_ant, C, T = 12, 6, 320
    N = 2 * n_ant
    b0 = synth_mod.make_block(N, C, T, seed=1, block=0)
    b1 = synth_mod.make_block(N, C, T, seed=1, block=1)
    with corr.Correlator(n_ant, 2, C, T) as xc:
        xc.push_block(torch.from_numpy(b0).cuda())
        assert xc.samples_integrated() == T
        v0, _ = xc.dump(want_stokes=False)
        assert np.array_equal(v0.cpu().numpy(), oracle_mod.xcorr(b0))
        # the integration restarted at zero
        v, s = xc.dump()
        assert not v.cpu().numpy().any() and not s.cpu().numpy().any()
        # blocks accumulate; a dump with no outputs still resets
        xc.push_block(torch.from_numpy(b0).cuda())
        xc.push_block(torch.from_numpy(b1).cuda())
        assert xc.samples_integrated() == 2 * T
        _, s01 = xc.dump(want_vis=False)
        ov = oracle_mod.xcorr(b1, vis=oracle_mod.xcorr(b0))
        assert np.array_equal(s01.cpu().numpy(), oracle_mod.stokes(ov, n_ant))
        xc.push_block(torch.from_numpy(b1).cuda())
        xc.dump(want_vis=False, want_stokes=False)
        v, _ = xc.dump(want_stokes=False)
        assert not v.cpu().numpy().any()
        xc.check()
    with corr.Correlator(N, 1, C, T) as xs:
        xs.push_block(torch.from_numpy(b0).cuda())
        with pytest.raises(corr.CorrError) as e:
            xs.dump(want_stokes=True)
        assert e.value.code == corr.CORR_EINVAL
        v, s = xs.dump()
        assert s is None and np.array_equal(v.cpu().numpy(), oracle_mod.xcorr(b0))


def test_host_buffer_api(corr, torch_cuda, oracle_mod, synth_mod):
    w = synth_mod.workload("tiny")
    blocks = [w.block(b) for b in range(3)]
    with corr.Correlator(w.n_ant, w.n_pol, w.n_chan, w.block_len) as xc:
        for b in blocks:
            xc.push_block_host(b)
        vis, st = xc.dump_host()
        xc.check()
    ov, ost = _oracle(oracle_mod, blocks, w.n_ant, w.n_pol)
    assert np.array_equal(vis, ov)
    assert np.array_equal(st, ost)


def test_independent_contexts(corr, torch_cuda, oracle_mod, synth_mod):
    torch = torch_cuda
    xa = synth_mod.make_block(40, 3, 256, seed=2)
    xb = synth_mod.make_block(10, 5, 96, seed=3)
    a = corr.Correlator(20, 2, 3, 256)
    b = corr.Correlator(10, 1, 5, 96)
    try:
        a.push_block(torch.from_numpy(xa).cuda())
        b.push_block(torch.from_numpy(xb).cuda())
        a.push_block(torch.from_numpy(xa).cuda())
        va, _ = a.dump()
        vb, _ = b.dump()
        assert np.array_equal(va.cpu().numpy(), 2 * oracle_mod.xcorr(xa))
        assert np.array_equal(vb.cpu().numpy(), oracle_mod.xcorr(xb))
    finally:
        a.close()
        b.close()


def test_channel_bands_on_two_streams(corr, torch_cuda, oracle_mod, synth_mod):
    # The multi-GPU layout on one GPU: two contexts, each on its own stream,
    # integrate the two bands of one workload; stitched, they equal the
    # oracle over the whole band (and the Stokes of a whole-band context).
    torch = torch_cuda
    from paper_2406_19013_gb300 import shard
    w = synth_mod.workload("tiny", seed=21)
    n_chan, T = 37, 512
    blocks = [synth_mod.make_block(w.n_in, n_chan, T, seed=21, block=b, tones=w.tones)
              for b in range(2)]
    want = oracle_mod.xcorr(blocks[0]) + oracle_mod.xcorr(blocks[1])
    parts, parts_st = [], []
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ctxs = []
    try:
        for r in range(2):
            c0, n = shard.band(r, 2, n_chan)
            xc = corr.Correlator(w.n_ant, w.n_pol, n, T)
            ctxs.append(xc)
            with torch.cuda.stream(streams[r]):
                for b in blocks:
                    xc.push_block(torch.from_numpy(np.ascontiguousarray(b[c0:c0 + n])).cuda(),
                                  streams[r])
                v, st = xc.dump(stream=streams[r])
            parts.append(v)
            parts_st.append(st)
        torch.cuda.synchronize()
        got = np.concatenate([v.cpu().numpy() for v in parts])
        assert np.array_equal(got, want)
        got_st = np.concatenate([s.cpu().numpy() for s in parts_st])
        assert np.array_equal(got_st, oracle_mod.stokes(want, w.n_ant))
    finally:
        for xc in ctxs:
            xc.close()


def test_device_wait_timeout_is_reported_and_the_context_recovers(corr, torch_cuda, oracle_mod,
                                                                   synth_mod):
    # A launch whose accumulator-draining warps wait on a barrier that nothing
    # completes: the bounded wait gives up after 200 ms, the kernel winds down
    # and reports through the status word; the context keeps integrating.
    import time
    torch = torch_cuda
    x0 = synth_mod.make_block(16, 8, 1024, seed=90, tones=synth_mod.random_phase_tone(16, 90))
    x1 = synth_mod.make_block(16, 8, 1024, seed=91, tones=synth_mod.random_phase_tone(16, 91))
    with corr.Correlator(8, 2, 8, 1024) as xc:
        d0, d1 = torch.from_numpy(x0).cuda(), torch.from_numpy(x1).cuda()
        xc.push_block(d0)
        xc.check()
        t0 = time.time()
        xc.selftest_timeout(d1, timeout_ms=200)
        with pytest.raises(corr.CorrError) as err:
            xc.check()
        elapsed = time.time() - t0
        assert err.value.code == corr.CORR_ETIMEOUT
        assert 0.15 < elapsed < 10.0
        xc.check()  # the status was cleared
        assert xc.samples_integrated() == 1024  # nothing of the aborted launch counted
        xc.push_block(d1)
        vis, _ = xc.dump()
        xc.check()
    assert np.array_equal(vis.cpu().numpy(), oracle_mod.xcorr(x0) + oracle_mod.xcorr(x1))


def _autos_numpy(x):
    s = x.astype(np.int8)
    re = (s >> 4).astype(np.int64)
    im = ((x << 4).astype(np.uint8).astype(np.int8) >> 4).astype(np.int64)
    return (re * re + im * im).sum(axis=2)


def test_paper_scale_sampled(corr, torch_cuda, oracle_mod, synth_mod):
    # 96 dual-pol antennas, 1024 channels, 8192-sample blocks: the launch the
    # benchmark times.  Whole channels and random pairs against the oracle,
    # and every auto-correlation of every channel against numpy.
    torch = torch_cuda
    w = synth_mod.workload("paper")
    x = w.block(0)
    with corr.Correlator(w.n_ant, w.n_pol, w.n_chan, w.block_len) as xc:
        xc.push_block(torch.from_numpy(x).cuda())
        vis, st = xc.dump()
        xc.check()
    vis = vis.cpu().numpy()
    st = st.cpu().numpy()
    chans = [0, 1, 511, 1023]
    ov = oracle_mod.xcorr(np.ascontiguousarray(x[chans]), n_threads=N_THREADS)
    assert np.array_equal(vis[chans], ov)
    assert np.array_equal(st[chans], oracle_mod.stokes(ov, w.n_ant))
    rng = np.random.default_rng(0)
    for _ in range(64):
        c = int(rng.integers(0, w.n_chan))
        i = int(rng.integers(0, w.n_in))
        j = int(rng.integers(0, i + 1))
        assert tuple(vis[c, i * (i + 1) // 2 + j]) == oracle_mod.xcorr_pair(x, c, i, j)
    autos = _autos_numpy(x)
    diag = np.arange(w.n_in) * (np.arange(w.n_in) + 3) // 2
    assert np.array_equal(vis[:, diag, 0], autos)
    assert not vis[:, diag, 1].any()


@pytest.mark.parametrize("kernel", ["default", "pair"])
def test_large_n_sampled(corr, torch_cuda, oracle_mod, synth_mod, monkeypatch, kernel):
    # 1024 dual-pol antennas (2048 inputs), 2 channels of 4096 samples, on
    # one-CTA units (the default) and on CTA pairs
    if kernel != "default":
        monkeypatch.setenv("CORR_CMAC_KERNEL", kernel)
    torch = torch_cuda
    w = synth_mod.workload("large_n")
    x = w.block(0, c0=0, n_chan=2)
    with corr.Correlator(w.n_ant, w.n_pol, 2, w.block_len) as xc:
        xc.push_block(torch.from_numpy(x).cuda())
        vis, _ = xc.dump(want_stokes=False)
        xc.check()
    vis = vis.cpu().numpy()
    rng = np.random.default_rng(1)
    for c in range(2):
        for i in [0, 63, 64, 255, 256, 257, 1000, 2047]:
            for j in sorted(set([0, i // 2, max(0, i - 1), i] + list(rng.integers(0, i + 1, 4)))):
                assert tuple(vis[c, i * (i + 1) // 2 + j]) == oracle_mod.xcorr_pair(x, c, i, int(j))
    autos = _autos_numpy(x)
    diag = np.arange(w.n_in) * (np.arange(w.n_in) + 3) // 2
    assert np.array_equal(vis[:, diag, 0], autos)


@pytest.mark.parametrize("T,C,N", [(1, 1, 1), (5, 3, 10), (128, 2, 128), (129, 3, 130),
                                   (100, 7, 192), (1000, 2, 301), (2048, 4, 64), (257, 1, 1030)])
def test_corner_turn_matches_oracle(corr, torch_cuda, oracle_mod, T, C, N):
    torch = torch_cuda
    rng = np.random.default_rng(T * 7 + C * 3 + N)
    x_tcn = rng.integers(0, 256, size=(T, C, N), dtype=np.uint8)
    got = corr.corner_turn(torch.from_numpy(x_tcn).cuda())
    assert np.array_equal(got.cpu().numpy(), oracle_mod.corner_turn(x_tcn))


@pytest.mark.parametrize("n_ant,n_pol,C,T,fused", [
    (8, 2, 16, 1024, True),    # 16 inputs: tiles of four channels, boxes of 16 inputs x 4 channels
    (16, 2, 5, 512, True),     # 32 inputs: tiles of two channels
    (32, 2, 4, 4096, True),    # 64 inputs
    (48, 2, 5, 1000, True),    # 96 inputs: two-channel units of two row tiles, last channel alone
    (64, 2, 4, 2048, True),    # 128 inputs: two-channel units of two row tiles
    (96, 2, 5, 2048, True),    # the paper's 192 inputs: three row tiles
    (96, 2, 3, 1000, True),    # ragged block length
    (128, 2, 3, 1000, True),   # 256 inputs: two window units
    (160, 2, 2, 256, True),    # 320 inputs: row-tile pairs, plain column regions
    (65, 2, 3, 1000, False),   # 130 inputs: strides not multiples of 16 -> turned in HBM
    (5, 1, 4, 33, False),      # 5 inputs
])
def test_push_block_tcn_matches_oracle(corr, torch_cuda, oracle_mod, synth_mod, monkeypatch, n_ant,
                                       n_pol, C, T, fused):
    # Blocks in F-engine order ([time][channel][input], Sec. 2.1's Transpose
    # input).  Inputs counts that are multiples of 16 are staged straight from
    # that order by the CMAC kernel (one launch per block, transposed on chip);
    # the others are corner-turned in HBM first (two launches).
    torch = torch_cuda
    monkeypatch.setenv("CORR_CMAC_KERNEL", "smem")
    n = n_ant * n_pol
    blocks = [synth_mod.make_block(n, C, T, seed=30 + b, tones=synth_mod.random_phase_tone(n, 30))
              for b in range(2)]
    blocks[1][:, :, : T // 3] = 0x88
    with corr.Correlator(n_ant, n_pol, C, T) as xc:
        n0 = xc.launch_count()
        for x in blocks:
            x_tcn = np.ascontiguousarray(np.transpose(x, (2, 0, 1)))  # F-engine order
            xc.push_block_tcn(torch.from_numpy(x_tcn).cuda())
        launches = xc.launch_count() - n0
        vis, st = xc.dump()
        xc.check()
    ov, ost = _oracle(oracle_mod, blocks, n_ant, n_pol)
    assert np.array_equal(vis.cpu().numpy(), ov)
    if n_pol == 2:
        assert np.array_equal(st.cpu().numpy(), ost)
    assert launches == (2 if fused else 4)


def test_push_block_tcn_all_byte_values(corr, torch_cuda, oracle_mod):
    # every byte value against every other through the fused F-engine-order path
    torch = torch_cuda
    N, T = 64, 512
    x = np.empty((3, N, T), dtype=np.uint8)
    for c in range(3):
        for i in range(N):
            x[c, i] = (np.arange(T) * (2 * i + 1) + 7 * c + i) % 256
    with corr.Correlator(N // 2, 2, 3, T) as xc:
        xc.push_block_tcn(torch.from_numpy(np.ascontiguousarray(np.transpose(x, (2, 0, 1)))).cuda())
        vis, st = xc.dump()
        xc.check()
    ov, ost = _oracle(oracle_mod, [x], N // 2, 2)
    assert np.array_equal(vis.cpu().numpy(), ov)
    assert np.array_equal(st.cpu().numpy(), ost)


def test_corner_turn_paper_block(corr, torch_cuda, oracle_mod, synth_mod):
    # the full 1.61 GB block of the 192-input workload, in F-engine order
    torch = torch_cuda
    w = synth_mod.workload("paper", seed=12)
    x = w.block(0)
    x_tcn = np.ascontiguousarray(np.transpose(x, (2, 0, 1)))
    got = corr.corner_turn(torch.from_numpy(x_tcn).cuda()).cpu().numpy()
    assert np.array_equal(got, oracle_mod.corner_turn(x_tcn))


@pytest.mark.parametrize("kernel", ["tm", "smem"])
@pytest.mark.parametrize("n_ant,n_pol,C,T,nb", [
    (1, 1, 2, 64, 1),        # one input, one row tile
    (9, 1, 3, 100, 2),       # ragged N and T (pitched staging)
    (32, 2, 4, 2048, 3),     # N = 64: one full row tile
    (65, 1, 3, 512, 2),      # N = 65: a second, almost empty row tile
    (64, 2, 3, 4096, 2),     # N = 128: two row tiles, the second from TMEM
    (75, 2, 5, 1024, 3),     # N = 150: three row tiles, the last ragged
    (96, 2, 6, 8192, 2),     # N = 192: the paper's inputs
])
def test_both_cmac_kernels_match_oracle(corr, torch_cuda, oracle_mod, synth_mod, monkeypatch,
                                        kernel, n_ant, n_pol, C, T, nb):
    # CORR_CMAC_KERNEL=tm selects, at corr_create, the kernel that keeps row
    # tile 0's row operand in TMEM (up to three row tiles); =smem the
    # all-shared-memory kernel.  Both must give the oracle's visibilities
    # exactly.
    monkeypatch.setenv("CORR_CMAC_KERNEL", kernel)
    N = n_ant * n_pol
    tones = synth_mod.random_phase_tone(N, 17)
    blocks = [synth_mod.make_block(N, C, T, seed=300 + N, block=b, tones=tones) for b in range(nb)]
    blocks[0][:, :, : T // 2] = 0x88  # -8-8j runs: the largest products
    vis, st = _run(corr, torch_cuda, blocks, n_ant, n_pol)
    ov, ost = _oracle(oracle_mod, blocks, n_ant, n_pol)
    assert np.array_equal(vis, ov)
    if n_pol == 2:
        assert np.array_equal(st, ost)


@pytest.mark.parametrize("kernel", ["pair", "smem"])
@pytest.mark.parametrize("n_ant,n_pol,C,T,nb", [
    (150, 2, 2, 2048, 2),    # N = 300: the odd CTA of the last row block is empty
    (256, 2, 3, 1024, 2),    # N = 512: two row blocks, one piece below the diagonal
    (300, 2, 2, 1008, 2),    # N = 600: ragged inputs and a ragged last chunk
    (512, 2, 2, 512, 3),     # N = 1024: four row blocks
])
def test_cta_pair_kernel_matches_oracle(corr, torch_cuda, oracle_mod, synth_mod, monkeypatch,
                                        kernel, n_ant, n_pol, C, T, nb):
    # CORR_CMAC_KERNEL=pair runs contexts of more than 256 inputs on CTA
    # pairs (the quad cover: M = 256 MMAs whose B rows are split between the
    # two CTAs of a cluster); =smem on one-CTA pairs units.  Both must give
    # the oracle's visibilities and Stokes products exactly.
    monkeypatch.setenv("CORR_CMAC_KERNEL", kernel)
    N = n_ant * n_pol
    tones = synth_mod.random_phase_tone(N, 23)
    blocks = [synth_mod.make_block(N, C, T, seed=500 + N, block=b, tones=tones) for b in range(nb)]
    blocks[0][:, :, : T // 2] = 0x88  # -8-8j runs: the largest products
    vis, st = _run(corr, torch_cuda, blocks, n_ant, n_pol)
    ov, ost = _oracle(oracle_mod, blocks, n_ant, n_pol)
    assert np.array_equal(vis, ov)
    assert np.array_equal(st, ost)


def test_cta_pair_wait_timeout_is_reported_and_the_context_recovers(corr, torch_cuda, oracle_mod,
                                                                    synth_mod, monkeypatch):
    # The same self-test on the CTA-pair kernel: both CTAs of every cluster
    # give up their waits, meet at the cluster barrier and release TMEM; the
    # context then integrates exactly.
    import time
    monkeypatch.setenv("CORR_CMAC_KERNEL", "pair")
    torch = torch_cuda
    x0 = synth_mod.make_block(300, 4, 1024, seed=92, tones=synth_mod.random_phase_tone(300, 92))
    x1 = synth_mod.make_block(300, 4, 1024, seed=93, tones=synth_mod.random_phase_tone(300, 93))
    with corr.Correlator(150, 2, 4, 1024) as xc:
        d0, d1 = torch.from_numpy(x0).cuda(), torch.from_numpy(x1).cuda()
        xc.push_block(d0)
        xc.check()
        t0 = time.time()
        xc.selftest_timeout(d1, timeout_ms=200)
        with pytest.raises(corr.CorrError) as err:
            xc.check()
        assert err.value.code == corr.CORR_ETIMEOUT
        assert 0.15 < time.time() - t0 < 10.0
        xc.check()
        assert xc.samples_integrated() == 1024
        xc.push_block(d1)
        vis, _ = xc.dump()
        xc.check()
    assert np.array_equal(vis.cpu().numpy(), oracle_mod.xcorr(x0) + oracle_mod.xcorr(x1))
