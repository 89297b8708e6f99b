"""corr_xcorr_static, the entry point for callers that must not allocate device
memory: code inside a framework that owns the device memory pool (an
allocation outside it can break the pool's budget) and code on a real-time
path, where cudaMalloc's implicit synchronisation would stall queued work.
Its scratch lives in a fixed device array inside the library.

Its visibilities must equal the CPU oracle's exactly, and the context API's on
the same bytes, call after call; once the device is warm a call must not
change the device's free memory.  This file is collected last so that a run
stopping at the first failure has already run every other test."""
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


def _context_vis(corr, block, n_ant, n_pol):
    C, N, T = block.shape
    with corr.Correlator(n_ant, n_pol, C, T) as xc:
        xc.push_block(block)
        vis, _ = xc.dump(want_stokes=False)
        xc.check()
    return vis.cpu().numpy()


# (n_ant, n_pol, channels, block_len, seed)
CASES = [
    (96, 2, 48, 2048, 11),   # the paper's 192 inputs
    (100, 2, 5, 1008, 12),   # 200 inputs: two units
    (128, 2, 3, 512, 13),    # 256 inputs: the largest accepted
    (8, 2, 64, 2048, 14),    # the tiny 16-input workload
    (9, 1, 3, 64, 15),       # 9 inputs: one partial row tile, one chunk
    (33, 1, 4, 48, 16),      # 33 inputs, a block shorter than one chunk
]


@pytest.mark.parametrize("n_ant,n_pol,C,T,seed", CASES)
def test_static_entry_matches_oracle_two_calls(corr, oracle_mod, synth_mod, n_ant, n_pol, C, T,
                                                seed):
    import torch
    N = n_ant * n_pol
    blocks = [synth_mod.make_block(N, C, T, seed=seed, block=b,
                                   tones=synth_mod.random_phase_tone(N, seed)) for b in range(2)]
    vis = torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, device="cuda")
    for b in blocks:  # two calls in a row, the second on different bytes
        x = torch.from_numpy(b).cuda()
        corr.xcorr_static(x, n_ant, n_pol, vis=vis)
        torch.cuda.synchronize()
        got = vis.cpu().numpy()
        assert np.array_equal(got, oracle_mod.xcorr(b))
        assert np.array_equal(got, _context_vis(corr, x, n_ant, n_pol))


def test_warm_calls_leave_free_memory_unchanged(corr, oracle_mod, synth_mod):
    import torch
    n_ant, n_pol, C, T = 96, 2, 16, 1024
    N = n_ant * n_pol
    x = torch.from_numpy(synth_mod.make_block(N, C, T, seed=21)).cuda()
    vis = torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int64, device="cuda")
    corr.xcorr_static(x, n_ant, n_pol, vis=vis)  # first call: device set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        corr.xcorr_static(x, n_ant, n_pol, vis=vis)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(vis.cpu().numpy(), oracle_mod.xcorr(x.cpu().numpy()))


def test_static_entry_rejects_out_of_limit_sizes(corr):
    import torch
    lib = corr.load()
    x = torch.zeros(2 * 300 * 64, dtype=torch.uint8, device="cuda")
    v = torch.zeros(2 * 300 * 301 // 2 * 2, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    # more inputs than the scratch schedule holds
    assert lib.corr_xcorr_static(x.data_ptr(), 150, 2, 2, 64, v.data_ptr(), s) == corr.CORR_EINVAL
    # block_len not a multiple of 16
    assert lib.corr_xcorr_static(x.data_ptr(), 8, 2, 2, 40, v.data_ptr(), s) == corr.CORR_EINVAL
    # misaligned pointers, bad n_pol, NULL
    assert lib.corr_xcorr_static(x.data_ptr() + 8, 8, 2, 2, 64, v.data_ptr(), s) == corr.CORR_EINVAL
    assert lib.corr_xcorr_static(x.data_ptr(), 8, 3, 2, 64, v.data_ptr(), s) == corr.CORR_EINVAL
    assert lib.corr_xcorr_static(None, 8, 2, 2, 64, v.data_ptr(), s) == corr.CORR_EINVAL
    assert not v.any().item()  # nothing was written
