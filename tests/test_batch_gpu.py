"""Batches of independent correlators (corr_batch_*) against the oracle.

Every instance of a batch must equal, bit for bit, the oracle on its own
blocks: sums are exact integers, so sharing launches with other instances
(of other sizes, in other launch groups) may change nothing.  Covers mixed
input counts (one and two launch groups, the cover for N > 256), ragged
block lengths (the pitched staging path), dumps of one instance while the
others integrate on, the autotuner, and a CUDA-graph capture of a push."""
import numpy as np
import pytest

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


# (n_ant, n_pol, n_chan, block_len): N = 16, 40, 10, 130, 192, 300, 64 inputs,
# block lengths with and without a 16-sample tail
SHAPES = [(8, 2, 11, 2048), (20, 2, 3, 1000), (10, 1, 5, 96), (65, 2, 4, 512),
          (96, 2, 6, 1024), (150, 2, 2, 256), (32, 2, 40, 300)]


def _blocks(synth_mod, shapes, seed, block):
    out = []
    for k, (na, npol, nc, T) in enumerate(shapes):
        n = na * npol
        out.append(synth_mod.make_block(n, nc, T, seed=seed + k, block=block,
                                        tones=synth_mod.random_phase_tone(n, seed + k)))
    return out


def test_batch_matches_oracle_per_instance(corr, oracle_mod, synth_mod):
    import torch
    b0 = _blocks(synth_mod, SHAPES, 100, 0)
    b1 = _blocks(synth_mod, SHAPES, 100, 1)
    with corr.Batch(SHAPES) as bt:
        groups = {bt.info(k)[1] for k in range(len(SHAPES))}
        assert len(groups) == bt.info(0)[2] and len(groups) >= 2
        for blocks in (b0, b1):
            bt.push([torch.from_numpy(x).cuda() for x in blocks])
        bt.check()
        for k, (na, npol, nc, T) in enumerate(SHAPES):
            assert bt.samples_integrated(k) == 2 * T
            vis, st = bt.dump(k)
            want = oracle_mod.xcorr(b0[k]) + oracle_mod.xcorr(b1[k])
            assert np.array_equal(vis.cpu().numpy(), want), f"instance {k}"
            if npol == 2:
                assert np.array_equal(st.cpu().numpy(), oracle_mod.stokes(want, na))
            assert bt.samples_integrated(k) == 0
        bt.check()


def test_dump_of_one_instance_leaves_the_others_integrating(corr, oracle_mod, synth_mod):
    import torch
    shapes = SHAPES[:3]
    b0 = _blocks(synth_mod, shapes, 200, 0)
    b1 = _blocks(synth_mod, shapes, 200, 1)
    with corr.Batch(shapes) as bt:
        bt.push([torch.from_numpy(x).cuda() for x in b0])
        v1, _ = bt.dump(1)
        bt.push([torch.from_numpy(x).cuda() for x in b1])
        assert np.array_equal(v1.cpu().numpy(), oracle_mod.xcorr(b0[1]))
        v0, _ = bt.dump(0)
        v1b, _ = bt.dump(1)
        v2, _ = bt.dump(2)
        assert np.array_equal(v0.cpu().numpy(), oracle_mod.xcorr(b0[0]) + oracle_mod.xcorr(b1[0]))
        assert np.array_equal(v1b.cpu().numpy(), oracle_mod.xcorr(b1[1]))
        assert np.array_equal(v2.cpu().numpy(), oracle_mod.xcorr(b0[2]) + oracle_mod.xcorr(b1[2]))
        bt.check()


def test_autotuned_batch_is_identical(corr, oracle_mod, synth_mod):
    import torch
    shapes = [(96, 2, 5, 1024), (8, 2, 9, 4096), (150, 2, 2, 512)]
    blocks = _blocks(synth_mod, shapes, 300, 0)
    with corr.Batch(shapes, autotune=True) as bt:
        for k, (na, npol, nc, T) in enumerate(shapes):
            cv = corr.tuned_cover(na * npol, T)
            assert cv in (corr.CORR_COVER_WINDOW, corr.CORR_COVER_STRIPS, corr.CORR_COVER_PAIRS)
            assert bt.info(k)[0] == cv
        assert corr.tuned_cover(300, 512) == corr.CORR_COVER_PAIRS  # the only cover above 256
        bt.push([torch.from_numpy(x).cuda() for x in blocks])
        bt.check()
        for k in range(len(shapes)):
            vis, _ = bt.dump(k)
            assert np.array_equal(vis.cpu().numpy(), oracle_mod.xcorr(blocks[k]))


def test_batch_push_in_a_cuda_graph(corr, oracle_mod, synth_mod):
    import torch
    shapes = [(96, 2, 4, 512), (8, 2, 7, 256)]
    blocks = _blocks(synth_mod, shapes, 400, 0)
    dev = [torch.from_numpy(x).cuda() for x in blocks]
    with corr.Batch(shapes) as bt:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bt.push(dev, stream=s)
        torch.cuda.synchronize()
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        bt.check()
        for k in range(len(shapes)):
            vis, _ = bt.dump(k)
            assert np.array_equal(vis.cpu().numpy(), 3 * oracle_mod.xcorr(blocks[k]))


def test_batch_rejects(corr):
    import torch
    with pytest.raises(corr.CorrError):
        corr.Batch([(8, 3, 4, 64)])
    with pytest.raises(corr.CorrError):
        corr.Batch([(8, 2, 4, corr.CORR_MAX_BLOCK_LEN + 1)])
    with corr.Batch([(8, 2, 4, 64)]) as bt:
        x = torch.zeros(4 * 16 * 64 + 16, dtype=torch.uint8, device="cuda")
        lib = corr.load()
        arr = (corr._vp * 1)(x.data_ptr() + 8)
        assert lib.corr_batch_push(bt._h, arr, None) == corr.CORR_EINVAL
        assert lib.corr_batch_dump(bt._h, 1, None, None, None) == corr.CORR_EINVAL
        assert lib.corr_batch_dump(bt._h, -1, None, None, None) == corr.CORR_EINVAL


def test_batched_workload_sampled(corr, oracle_mod, synth_mod):
    # The 64-correlator batch at full size (32..512 inputs, up to 1024
    # channels, up to 16384 samples), autotuned.  Inputs are seeded windows of
    # a device pool of synthetic samples; the oracle recomputes the first, the
    # last and one seeded middle channel of every instance from the same bytes.
    import os

    import torch
    shapes = synth_mod.batched_instances()
    sizes = [c * na * npol * t for na, npol, c, t in shapes]
    base = synth_mod.make_block(192, 64, 8192, seed=77,
                                tones=synth_mod.random_phase_tone(192, 77)).reshape(-1)
    reps = -(-(max(sizes) + (1 << 20)) // base.size)
    dbase = torch.from_numpy(base).cuda()
    pool = torch.empty(reps * base.size, dtype=torch.uint8, device="cuda")
    for r in range(reps):
        pool[r * base.size:(r + 1) * base.size].copy_(dbase)
    offs = synth_mod.pool_offsets(sizes, pool.numel())
    rng = np.random.default_rng(5)
    with corr.Batch(shapes, autotune=True) as bt:
        bt.push([pool[o:o + sz] for o, sz in zip(offs, sizes)])
        bt.check()
        threads = min(16, os.cpu_count() or 1)
        for k, (na, npol, C, T) in enumerate(shapes):
            n = na * npol
            vis, _ = bt.dump(k, want_stokes=False)
            chans = sorted({0, C - 1, int(rng.integers(0, C))})
            got = vis[chans].cpu().numpy()
            x = np.empty((len(chans), n, T), dtype=np.uint8)
            for q, c in enumerate(chans):
                start = offs[k] + c * n * T
                x[q] = base[(start + np.arange(n * T)) % base.size].reshape(n, T)
            want = oracle_mod.xcorr(x, n_threads=threads)
            assert np.array_equal(got, want), f"instance {k} {shapes[k]}"
        bt.check()
