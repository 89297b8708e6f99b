"""Counters, checkpoint/resume and the debug build, on the GPU.

A resumed integration must end bit-identical to one that never stopped (the
accumulators are integers), and the debug build's address checks and guard
bands must stay silent on correct runs and report a guard band that was
overwritten from the host.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from conftest import ROOT

pytestmark = pytest.mark.gpu


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


def test_stats_count_blocks_samples_dumps(corr, torch_cuda, synth_mod):
    torch = torch_cuda
    n_ant, n_pol, C, T = 12, 2, 3, 4096
    blocks = [torch.from_numpy(synth_mod.make_block(n_ant * n_pol, C, T, seed=3, block=b)).cuda()
              for b in range(5)]
    with corr.Correlator(n_ant, n_pol, C, T) as xc:
        s0 = xc.stats()
        assert s0["blocks_pushed"] == 0 and s0["dumps"] == 0 and s0["samples_total"] == 0
        xc.push_blocks(blocks[:3])
        xc.push_block(blocks[3])
        s1 = xc.stats()
        assert s1["blocks_pushed"] == 4 and s1["samples_pending"] == 4 * T
        assert s1["samples_total"] == 4 * T and s1["launches"] == xc.launch_count()
        xc.dump()
        xc.push_block(blocks[4])
        s2 = xc.stats()
        assert s2["dumps"] == 1 and s2["samples_pending"] == T and s2["samples_total"] == 5 * T
        xc.check()


@pytest.mark.parametrize("n_ant,n_pol,C,T", [(96, 2, 4, 8192), (40, 2, 3, 1000), (70, 1, 2, 2048)])
def test_snapshot_restore_resumes_bit_exact(corr, torch_cuda, oracle_mod, synth_mod,
                                            n_ant, n_pol, C, T):
    """Blocks 0-1 into one context, a snapshot, blocks 2-3 into a second
    context restored from it: the second context's dump is the oracle's sum
    of all four blocks."""
    torch = torch_cuda
    N = n_ant * n_pol
    host = [synth_mod.make_block(N, C, T, seed=11, block=b) for b in range(4)]
    dev = [torch.from_numpy(b).cuda() for b in host]
    with corr.Correlator(n_ant, n_pol, C, T) as a:
        a.push_block(dev[0])
        a.push_block(dev[1])
        acc, samples = a.snapshot()
        assert samples == 2 * T
        a.check()
    with corr.Correlator(n_ant, n_pol, C, T) as b:
        b.push_block(dev[3])          # discarded by the restore
        b.restore(acc, samples)
        assert b.samples_integrated() == 2 * T
        b.push_block(dev[2])
        b.push_block(dev[3])
        vis, st = b.dump(want_stokes=n_pol == 2)
        b.check()
    ov = None
    for blk in host:
        ov = oracle_mod.xcorr(blk, vis=ov, n_threads=max(1, min(os.cpu_count() or 1, 64)))
    assert np.array_equal(vis.cpu().numpy(), ov)
    if n_pol == 2:
        assert np.array_equal(st.cpu().numpy(), oracle_mod.stokes(ov, n_ant))
    # the snapshot itself is the oracle's two-block sum
    ov2 = None
    for blk in host[:2]:
        ov2 = oracle_mod.xcorr(blk, vis=ov2, n_threads=max(1, min(os.cpu_count() or 1, 64)))
    assert np.array_equal(acc, ov2)


def test_restore_rejects(corr, torch_cuda):
    with corr.Correlator(4, 2, 2, 64) as xc:
        acc = np.zeros((2, xc.n_pairs, 2), dtype=np.int64)
        with pytest.raises(corr.CorrError) as e:
            xc.restore(acc, -1)
        assert e.value.code == corr.CORR_EINVAL
        with pytest.raises(ValueError):
            xc.restore(acc[:1], 0)


# Runs in a fresh process, so that the binding loads the debug library.
_DEBUG_SCRIPT = r'''
import os, sys
import numpy as np
import torch
sys.path.insert(0, os.environ["REPO_ROOT"])
from paper_2406_19013_gb300 import build
build.build(debug=True)
from paper_2406_19013_gb300 import corr
from oracle import oracle
from synth import synth
oracle.build(); synth.build()
assert corr.LIB_PATH.endswith("libcorr_debug.so") and corr.debug_build()
def run(n_ant, n_pol, C, T, nb, tcn=False):
    N = n_ant * n_pol
    host = [synth.make_block(N, C, T, seed=5, block=b) for b in range(nb)]
    with corr.Correlator(n_ant, n_pol, C, T) as xc:
        for h in host:
            d = torch.from_numpy(h).cuda()
            if tcn:
                xc.push_block_tcn(d.permute(2, 0, 1).contiguous())
            else:
                xc.push_block(d)
        vis, st = xc.dump(want_stokes=n_pol == 2)
        xc.check()   # no address check or guard band fired
    ov = None
    for h in host:
        ov = oracle.xcorr(h, vis=ov)
    assert np.array_equal(vis.cpu().numpy(), ov), (n_ant, n_pol, C, T)
    if n_pol == 2:
        assert np.array_equal(st.cpu().numpy(), oracle.stokes(ov, n_ant))
run(96, 2, 3, 8192, 2)          # shared-memory kernel, 192 inputs
run(64, 2, 2, 4096, 2)          # TMEM-operand kernel, 128 inputs
run(16, 2, 5, 2048, 3)          # two-channel units, 32 inputs
run(21, 1, 3, 1000, 2)          # ragged inputs and samples, pitched staging
run(96, 2, 2, 4096, 1, tcn=True)  # F-engine-order staging
os.environ["CORR_CMAC_KERNEL"] = "pair"
run(150, 2, 2, 1024, 2)         # CTA pairs, 300 inputs
del os.environ["CORR_CMAC_KERNEL"]
for side in (0, 1):
    with corr.Correlator(8, 2, 2, 256) as xc:
        xc.check()
        xc.debug_corrupt_guard(side)
        try:
            xc.check()
        except corr.CorrError as e:
            assert e.code == corr.CORR_EBOUNDS, e
        else:
            raise AssertionError("corrupted guard band not reported")
print("debug build ok")
'''


def test_debug_build_checks(torch_cuda):
    env = dict(os.environ, CORR_LIB_VARIANT="debug", REPO_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", _DEBUG_SCRIPT], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok" in r.stdout


def test_release_build_has_no_debug_hooks(corr, torch_cuda):
    assert not corr.debug_build()
    with corr.Correlator(8, 2, 2, 256) as xc:
        with pytest.raises(corr.CorrError) as e:
            xc.debug_corrupt_guard(0)
        assert e.value.code == corr.CORR_ESTATE


def test_mma_rate_measures_a_plausible_fp8_rate(corr, torch_cuda):
    """The roofline's denominator: a short run of the dense E5M2 MMA loop
    (N = 256, A from TMEM) finishes with a clear status and lands between
    half and 1.2x the nominal dense fp8 rate of the part (4.5 PFLOP/s), at
    a cycle count per MMA near 128 x 256 x 32 MACs / 8192 per clock."""
    tflops, ms, cyc = corr.mma_rate(n=256, issuers=1, iters=2000, a_from_tmem=True, reps=2)
    assert 2250 < tflops < 5400, tflops
    assert 100 < cyc < 300, cyc
    assert ms > 0
