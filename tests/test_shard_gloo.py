"""Multi-process host logic of the channel-band sharding, on the CPU with the
gloo backend at world size 2 (and 3 for a ragged split).

Each rank correlates its own band of one global workload (the oracle stands
in for the GPU here). Rank 0 then gathers the bands. The stitched result
must equal the single-process oracle over the whole band, bit for bit. The
timing reductions and the failure of a rank that leaves are checked too."""
import datetime
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=60):
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=timeout_s))
    return dist


def _band_worker(rank, world, port, n_chan, q):
    try:
        dist = _init(rank, world, port)
        import torch
        from oracle import oracle
        from paper_2406_19013_gb300 import shard
        from synth import synth
        w = synth.workload("tiny", seed=9)
        c0, n = shard.band(rank, world, n_chan)
        x = w.block(0, c0=c0, n_chan=n)
        vis = torch.from_numpy(oracle.xcorr(x))
        full = shard.gather_bands(vis, n_chan)
        t_max = shard.max_over_ranks(10.0 + rank)
        work = shard.sum_over_ranks(float(n))
        if rank == 0:
            q.put(("ok", full.numpy(), t_max, work))
        else:
            q.put(("ok", None, t_max, work))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the test, which fails on it
        q.put(("error", repr(e), None, None))


def _leaver_worker(rank, world, port, q):
    """Rank 1 leaves between steps; rank 0's next collective must end in an
    error within the process group's short timeout, not hang."""
    try:
        dist = _init(rank, world, port, timeout_s=5)
        from paper_2406_19013_gb300 import shard
        shard.max_over_ranks(1.0)  # one step in which both ranks take part
        if rank == 1:
            dist.destroy_process_group()
            q.put(("left", None))
            return
        try:
            shard.max_over_ranks(2.0)
            q.put(("no error", None))
        except Exception as e:
            q.put(("raised", type(e).__name__))
    except Exception as e:
        q.put(("error", repr(e)))


def _run(target, world, *args, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port) + args + (q,)) for r in range(world)]
    for p in procs:
        p.start()
    out = []
    try:
        for _ in range(world):
            out.append(q.get(timeout=timeout))
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    return out


def test_band_partition_covers_every_channel_once():
    from paper_2406_19013_gb300 import shard
    for n_chan in (0, 1, 7, 64, 1024, 1031):
        for world in (1, 2, 3, 8):
            spans = [shard.band(r, world, n_chan) for r in range(world)]
            assert sum(n for _, n in spans) == n_chan
            pos = 0
            for c0, n in spans:
                assert c0 == pos and n >= 0
                pos += n
            assert max(n for _, n in spans) - min(n for _, n in spans) <= 1
    with pytest.raises(ValueError):
        shard.band(2, 2, 10)


@pytest.mark.parametrize("world,n_chan", [(2, 64), (2, 7), (3, 8)])
def test_gloo_bands_gather_to_the_full_band(oracle_mod, synth_mod, world, n_chan):
    out = _run(_band_worker, world, n_chan)
    errors = [o for o in out if o[0] != "ok"]
    assert not errors, errors
    full = next(o[1] for o in out if o[1] is not None)
    from synth import synth
    w = synth.workload("tiny", seed=9)
    want = oracle_mod.xcorr(w.block(0, c0=0, n_chan=n_chan))
    assert full.shape == want.shape
    assert np.array_equal(full, want)
    for o in out:
        assert o[2] == 10.0 + (world - 1)  # the slowest rank's time
        assert o[3] == float(n_chan)       # every channel counted once


def test_gloo_rank_leaving_ends_the_next_collective_with_an_error():
    out = _run(_leaver_worker, 2, timeout=90)
    kinds = sorted(o[0] for o in out)
    assert kinds == ["left", "raised"], out
