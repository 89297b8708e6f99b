"""The served loop (corr_server_*).

Without a GPU, dry mode runs the admission and ordering policy with
instantaneous device steps: integrations close and complete as documented
under reordering, duplicates, drops, late blocks, a full arena and held
results.  On the GPU, every returned integration must equal the oracle over
exactly the blocks its mask names, whatever the arrival order and faults."""
import time

import numpy as np
import pytest


@pytest.fixture(scope="module")
def corr():
    from paper_2406_19013_gb300 import corr as c
    c.load()
    return c


def _drain(srv, n_expected, timeout_s=10.0):
    got = []
    t0 = time.time()
    while len(got) < n_expected and time.time() - t0 < timeout_s:
        got += srv.poll(timeout_ms=50)
    return got


SMALL = (4, 2, 3, 64, 4)  # 8 inputs, 3 channels, 64 samples, L = 4
BLOCK = 3 * 8 * 64


def test_in_order_integrations(corr):
    with corr.Server([SMALL, SMALL], arena_bytes=8 * BLOCK, dry=True) as srv:
        for seq in range(12):
            srv.submit(0, seq)
        for seq in range(4):
            srv.submit(1, seq)
        res = _drain(srv, 4)
        assert sorted((r["array"], r["integration"]) for r in res) == [(0, 0), (0, 1), (0, 2),
                                                                      (1, 0)]
        assert all(r["n_blocks"] == 4 and r["block_mask"] == 0xF for r in res)
        st = srv.stats()
        assert st["integrated"] == 16 and st["integrations"] == 4
        assert st["incomplete_integrations"] == 0 and st["error"] == 0
        assert st["latency_samples"] == 16


def test_reordered_blocks_within_the_window(corr):
    with corr.Server([SMALL], arena_bytes=16 * BLOCK, window=2, dry=True) as srv:
        for seq in [1, 0, 5, 3, 2, 4, 7, 6]:
            srv.submit(0, seq)
        res = _drain(srv, 2)
        assert [(r["integration"], r["n_blocks"], r["block_mask"]) for r in res] == \
            [(0, 4, 0xF), (1, 4, 0xF)]


def test_duplicates_and_late_blocks_are_discarded(corr):
    with corr.Server([SMALL], arena_bytes=16 * BLOCK, dry=True) as srv:
        for seq in [0, 0, 1, 2, 2, 3]:
            srv.submit(0, seq)
        res = _drain(srv, 1)
        assert res[0]["n_blocks"] == 4
        srv.submit(0, 1)  # integration 0 is finished
        time.sleep(0.05)
        st = srv.stats()
        assert st["duplicates"] == 2 and st["late"] == 1 and st["integrated"] == 4


def test_drop_closes_an_integration_when_the_window_moves_on(corr):
    with corr.Server([SMALL], arena_bytes=16 * BLOCK, window=2, dry=True) as srv:
        for seq in [0, 1, 3]:  # 2 is lost
            srv.submit(0, seq)
        time.sleep(0.05)
        assert srv.poll() == []  # still waiting for block 2
        srv.submit(0, 8)  # integration 2: integration 0 can no longer complete
        res = _drain(srv, 1)
        assert (res[0]["integration"], res[0]["n_blocks"], res[0]["block_mask"]) == (0, 3, 0b1011)
        srv.submit(0, 2)   # too late now
        srv.submit(0, 5)   # integration 1 is still open: the window is {1, 2}
        srv.submit(0, 17)  # integration 4 closes those below 3; the window is {3, 4}
        res = _drain(srv, 2)
        assert [(r["integration"], r["n_blocks"], r["block_mask"]) for r in res] == \
            [(1, 1, 0b0010), (2, 1, 0b0001)]
        srv.submit(0, 13)  # integration 3
        srv.submit(0, 25)  # integration 6 closes 3 (one block) and 4 (one block), 5 is empty
        res = _drain(srv, 2)
        assert [(r["integration"], r["n_blocks"], r["block_mask"]) for r in res] == \
            [(3, 1, 0b0010), (4, 1, 0b0010)]
        srv.submit(0, 21)  # integration 5 is open (window {5, 6})
        srv.submit(0, 33)  # integration 8 closes 5 and 6; 7 is skipped when it closes
        srv.submit(0, 29)  # integration 7 is still open (window {7, 8})
        srv.flush()        # everything open completes
        res = _drain(srv, 4)
        assert [(r["integration"], r["n_blocks"], r["block_mask"]) for r in res] == \
            [(5, 1, 0b0010), (6, 1, 0b0010), (7, 1, 0b0010), (8, 1, 0b0010)]
        srv.submit(0, 30)  # integration 7 is finished
        time.sleep(0.05)
        st = srv.stats()
        assert st["late"] == 2 and st["incomplete_integrations"] == 9
        assert st["integrations"] == 9 and st["integrated"] == 11


def test_an_integration_closed_while_empty_is_skipped(corr):
    with corr.Server([SMALL], arena_bytes=16 * BLOCK, window=2, dry=True) as srv:
        srv.submit(0, 0)
        srv.submit(0, 12)  # integration 3 closes 0 and 1 (1 is empty): window {2, 3}
        res = _drain(srv, 1)
        assert [(r["integration"], r["n_blocks"]) for r in res] == [(0, 1)]
        srv.submit(0, 5)   # integration 1 was closed while empty
        srv.submit(0, 9)   # integration 2 is open
        srv.flush()
        res = _drain(srv, 2)
        assert [(r["integration"], r["block_mask"]) for r in res] == [(2, 0b0010), (3, 0b0001)]
        st = srv.stats()
        assert st["late"] == 1 and st["integrations"] == 3


def test_arena_bounds_blocks_in_flight(corr):
    # room for two blocks only: the rest wait in arrival order, all complete
    with corr.Server([SMALL, SMALL], arena_bytes=2 * 1536 + 100, dry=True) as srv:
        for seq in range(8):
            srv.submit(seq % 2, seq // 2)
        res = _drain(srv, 2)
        assert len(res) == 2
        assert srv.stats()["arena_peak_bytes"] <= 2 * 1536


def test_a_held_result_holds_back_the_next(corr):
    lib = corr.load()
    with corr.Server([(4, 2, 3, 64, 1)], arena_bytes=8 * BLOCK, dry=True) as srv:
        for seq in range(3):
            srv.submit(0, seq)
        out = (corr.ServerResult * 4)()
        n = lib.corr_server_poll(srv._h, out, 4, 1000)
        assert n == 1 and out[0].integration == 0
        time.sleep(0.05)
        assert lib.corr_server_poll(srv._h, out, 4, 0) == 0  # not released yet
        assert lib.corr_server_release(srv._h, 0) == 0
        n = lib.corr_server_poll(srv._h, out, 4, 1000)
        assert n == 1 and out[0].integration == 1


def test_server_rejects(corr):
    with pytest.raises(corr.CorrError):
        corr.Server([(4, 2, 3, 64, 65)], arena_bytes=1 << 20, dry=True)  # L > 64
    with pytest.raises(corr.CorrError):
        corr.Server([(4, 2, 3, 64, 4)], arena_bytes=100, dry=True)  # block does not fit
    with pytest.raises(corr.CorrError):
        corr.Server([(4, 2, 3, 64, 4)], arena_bytes=1 << 20, window=0, dry=True)
    with corr.Server([SMALL], arena_bytes=1 << 20, dry=True) as srv:
        with pytest.raises(corr.CorrError):
            srv.submit(1, 0)
        with pytest.raises(corr.CorrError):
            srv.submit(0, -1)


# ---------------------------------------------------------------- GPU

@pytest.mark.gpu
@pytest.mark.gpu
def test_served_results_match_oracle_under_faults(corr, oracle_mod, synth_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19013_gb300 import build
    build.build()
    arrays = [(8, 2, 5, 512, 3), (20, 2, 3, 1000, 2)]
    blocks = {}
    for a, (na, npol, nc, T, L) in enumerate(arrays):
        n = na * npol
        for seq in range(3 * L):
            x = synth_mod.make_block(n, nc, T, seed=50 + a, block=seq,
                                     tones=synth_mod.random_phase_tone(n, 50 + a))
            blocks[(a, seq)] = torch.from_numpy(x).pin_memory()
    # array 0: reordered, one duplicate, seq 4 dropped; array 1: in order
    order = [(0, 2), (0, 0), (1, 0), (0, 1), (0, 1), (1, 1), (0, 5), (0, 3), (1, 2), (1, 3),
             (0, 7), (0, 8), (0, 6), (1, 4), (1, 5)]
    with corr.Server(arrays, arena_bytes=4 * 3 * 40 * 1000, window=2) as srv:
        for a, seq in order:
            srv.submit(a, seq, blocks[(a, seq)])
        srv.flush()
        res = _drain(srv, 6, timeout_s=60)
        st = srv.stats()
    assert st["error"] == 0 and st["duplicates"] == 1
    assert len(res) == 6
    for r in res:
        a, k = r["array"], r["integration"]
        L = arrays[a][4]
        seqs = [k * L + s for s in range(L) if r["block_mask"] >> s & 1]
        assert len(seqs) == r["n_blocks"]
        want = sum(oracle_mod.xcorr(blocks[(a, q)].numpy()) for q in seqs)
        assert np.array_equal(r["vis"], want), (a, k, seqs)
    masks = {(r["array"], r["integration"]): r["block_mask"] for r in res}
    assert masks[(0, 1)] == 0b101  # seq 4 never came
    assert masks[(0, 0)] == 0b111 and masks[(1, 2)] == 0b11
    assert st["latency_samples"] == st["integrated"] == 14
    assert 0 < st["latency_p50_ms"] <= st["latency_p99_ms"] <= st["latency_max_ms"]


@pytest.mark.gpu
def test_served_mix_equals_each_array_alone(corr, oracle_mod, synth_mod):
    # Four arrays of different sizes submit their blocks interleaved and
    # back to back, so their CMAC launches overlap on the device (each array
    # has its own compute stream).  Every integration must equal, bit for bit,
    # the same array's integration served alone and the oracle.
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19013_gb300 import build
    build.build()
    arrays = [(16, 2, 96, 2048, 2), (48, 2, 40, 4096, 2), (96, 2, 64, 1024, 2), (8, 1, 200, 512, 2)]
    n_int = 3
    blocks = {}
    for a, (na, npol, nc, T, L) in enumerate(arrays):
        n = na * npol
        for seq in range(n_int * L):
            x = synth_mod.make_block(n, nc, T, seed=70 + a, block=seq,
                                     tones=synth_mod.random_phase_tone(n, 70 + a))
            blocks[(a, seq)] = torch.from_numpy(x).pin_memory()
    arena = 6 * max(b.numel() for b in blocks.values())

    def serve(which):
        order = [(a, seq) for seq in range(n_int * 2) for a in which]
        with corr.Server(arrays, arena_bytes=arena, window=2) as srv:
            for a, seq in order:
                srv.submit(a, seq, blocks[(a, seq)])
            srv.flush()
            res = _drain(srv, n_int * len(which), timeout_s=60)
            st = srv.stats()
        assert st["error"] == 0 and len(res) == n_int * len(which)
        return {(r["array"], r["integration"]): r["vis"].copy() for r in res}

    mixed = serve(range(len(arrays)))
    for a in range(len(arrays)):
        alone = serve([a])
        for k in range(n_int):
            assert np.array_equal(mixed[(a, k)], alone[(a, k)]), (a, k)
            want = sum(oracle_mod.xcorr(blocks[(a, 2 * k + q)].numpy()) for q in range(2))
            assert np.array_equal(mixed[(a, k)], want), (a, k)
