"""The C-ABI library without a GPU: it loads, exports every declared symbol,
validates arguments before touching a device, and its tile schedule covers
the lower triangle exactly once."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def corr():
    from paper_2406_19013_gb300 import build
    build.build()
    from paper_2406_19013_gb300 import corr as c
    return c


def _declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(corr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(corr):
    lib = corr.load()
    declared = _declared_functions()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wires every declared function
    assert sorted(n for n, _, _ in corr.ABI) == declared


def test_strerror(corr):
    assert corr.strerror(0) == "ok"
    for code in range(-6, 0):
        assert corr.strerror(code) != "unknown error"
    assert corr.strerror(-99) == "unknown error"


@pytest.mark.parametrize("args", [
    (0, 2, 4, 64), (4, 3, 4, 64), (4, 0, 4, 64), (4, 2, 0, 64), (4, 2, 4, 0),
    (4, 2, 4, -5), (4, 2, 4, 16777216), (8193, 1, 1, 16), (4097, 2, 1, 16)])
def test_create_rejects_bad_sizes(corr, args):
    with pytest.raises(corr.CorrError) as e:
        corr.Correlator(*args)
    assert e.value.code == corr.CORR_EINVAL


def test_null_context_calls(corr):
    lib = corr.load()
    assert lib.corr_push_block(None, None, None) == corr.CORR_EINVAL
    assert lib.corr_dump(None, None, None, None) == corr.CORR_EINVAL
    assert lib.corr_check(None, None) == corr.CORR_EINVAL
    assert lib.corr_sizes(None, None, None, None) == corr.CORR_EINVAL
    assert lib.corr_launch_count(None) == 0
    lib.corr_destroy(None)


@pytest.mark.parametrize("n", [1, 2, 7, 16, 17, 63, 64, 65, 100, 127, 128, 129, 191, 192, 193,
                               200, 255, 256, 257, 300, 383, 384, 385, 511, 512, 513, 640, 1000,
                               1025, 2048])
def test_plan_covers_lower_triangle_once(corr, n):
    n_units, issued, cover = corr.plan(n, with_cover=True)
    assert np.array_equal(cover, np.tril(np.ones((n, n), dtype=np.uint8)))
    assert n_units >= 1
    assert issued >= n * (n + 1) // 2


def test_plan_efficiency_at_paper_scale(corr):
    # 192 inputs: 64-input row tiles against their strips, 75.4 % of the
    # issued complex MACs are lower-triangle ones
    n_units, issued, _ = corr.plan(192)
    assert n_units == 1
    assert issued == 64 * (64 + 128 + 192)
    assert abs(192 * 193 / 2 / issued - 0.754) < 1e-3


def test_plan_rejects(corr):
    with pytest.raises(corr.CorrError):
        corr.plan(0)
    with pytest.raises(corr.CorrError):
        corr.plan(8193)


@pytest.mark.parametrize("cover", [0, 1, 2, 3])
@pytest.mark.parametrize("n", [1, 16, 40, 64, 65, 127, 128, 192, 200, 256, 257, 300, 384, 512,
                               600, 1000, 1024, 2048])
def test_every_cover_covers_lower_triangle_once(corr, n, cover):
    _, issued, got = corr.plan_cover(n, cover, with_cover=True)
    assert np.array_equal(got, np.tril(np.ones((n, n), dtype=np.uint8)))
    assert issued >= n * (n + 1) // 2


def _chans_per_unit(n_in):
    """Channels one window-cover unit holds: two 64-row tiles of 64 / n16
    channels each up to 32 inputs, two channels up to two row tiles."""
    if n_in <= 32:
        return 2 * (64 // (-(-n_in // 16) * 16))
    return 2 if n_in <= 128 else 1


def _check_split(corr, n_in, n_chan, block_len, n_blocks, grid, cover=0, min_split=16):
    items, first = corr.plan_items(n_in, n_chan, block_len, n_blocks, grid, cover)
    n_tpl = corr.plan_cover(n_in, cover)[0]
    ppb = -(-block_len // 128)
    npk = ppb * n_blocks
    used = len(first) - 1
    assert 1 <= used <= grid
    assert first[0] == 0 and first[-1] == len(items)
    assert np.all(np.diff(first) >= 1)  # no empty CTA
    # every (template, channel, stage) exactly once; with a single row tile
    # the window cover's unit holds two channels (the item names the first)
    per_unit = _chans_per_unit(n_in) if cover == 0 else 1
    seen = np.zeros((n_tpl, n_chan, npk), dtype=np.int32)
    for prob, tpl, chan, pk0, n in items:
        assert prob == 0 and n >= 1 and 0 <= pk0 and pk0 + n <= npk
        assert chan % per_unit == 0
        for c in range(chan, min(chan + per_unit, n_chan)):
            seen[tpl, c, pk0:pk0 + n] += 1
    assert np.all(seen == 1)
    # a unit is split only into pieces of >= min_split stages
    pieces = {}
    for prob, tpl, chan, pk0, n in items:
        pieces.setdefault((tpl, chan), []).append(n)
    for ns in pieces.values():
        if len(ns) > 1:
            assert min(ns) >= min(min_split, npk)
    return items, first


@pytest.mark.parametrize("n_in,n_chan,block_len,n_blocks", [
    (16, 3, 300000, 1), (16, 2, 200001, 1), (192, 4, 16777215, 1), (64, 5, 65536, 2)])
def test_items_stay_inside_the_fold_window(corr, n_in, n_chan, block_len, n_blocks):
    # a block longer than the fp32 fold window is cut into items of at most
    # 1023 stages (130944 samples), each folded on its own; coverage stays exact
    items, _ = _check_split(corr, n_in, n_chan, block_len, n_blocks, 152)
    assert items[:, 4].max() <= corr.CORR_FOLD_SAMPLES // 128
    npk = -(-block_len // 128) * n_blocks
    n_tpl = corr.plan_cover(n_in, 0)[0]
    per_unit = _chans_per_unit(n_in)  # channels per window unit
    assert len(items) >= n_tpl * -(-n_chan // per_unit) * -(-npk // 1023)


def test_item_split_balances_the_paper_launch(corr):
    # 192 inputs, 1024 channels, 8 blocks of 8192 samples over 152 SMs:
    # whole units would give some SMs 7 units and others 6
    items, first = _check_split(corr, 192, 1024, 8192, 8, 152)
    stages = np.zeros(len(first) - 1)
    for b in range(len(first) - 1):
        stages[b] = items[first[b]:first[b + 1], 4].sum()
    # stages differ only by the modelled fold cost of an extra item
    assert stages.max() / stages.mean() < 1.02
    # dealing whole units would leave 7 x 512 stages on the busiest SM
    assert stages.max() < 0.98 * 7 * 512
    assert len(first) - 1 == 152


@pytest.mark.parametrize("args", [(16, 64, 2048, 1, 152), (192, 5, 1008, 1, 152),
                                  (40, 3, 256, 2, 152), (512, 37, 4096, 1, 152),
                                  (2048, 4, 4096, 2, 152), (100, 1, 100, 1, 4),
                                  (192, 1024, 8192, 1, 152), (64, 16, 16384, 1, 7)])
def test_item_split_covers_every_unit_stage_once(corr, args):
    _check_split(corr, *args)


@pytest.mark.parametrize("cover", [1, 2])
def test_item_split_other_covers(corr, cover):
    _check_split(corr, 192, 300, 4096, 2, 152, cover)


@pytest.mark.parametrize("args", [(2048, 4, 4096, 2, 76), (1000, 300, 8192, 1, 76),
                                  (512, 16, 16384, 1, 76)])
def test_item_split_quad_cover(corr, args):
    """With CTA pairs the items are dealt to clusters (76 on 152 SMs)."""
    _check_split(corr, *args, cover=3)


def test_quad_cover_units_are_pair_units(corr):
    """Each quad unit's 256 rows are covered by its two CTAs (the cover view
    reads the odd CTA's rows and the column blocks the way the epilogue
    does), and 2048 inputs need 36 units (8 row blocks x up to 8 column
    pieces).  The 28 below the diagonal issue two N = 256 MMAs per CTA; the 8
    on it pair row tiles T0 and T1 against 128 columns and T3 and T2 against
    256, three quarters of that work."""
    n_units, issued, got = corr.plan_cover(2048, 3, with_cover=True)
    assert n_units == 36
    # units x CTAs x (row tiles x 64 inputs x columns)
    assert issued == 28 * 2 * (2 * 64 * 256) + 8 * 2 * (64 * 128 + 64 * 256)
    assert np.array_equal(got, np.tril(np.ones((2048, 2048), dtype=np.uint8)))


@pytest.mark.parametrize("n", [257, 300, 384, 512, 600, 1000])
def test_quad_cover_is_the_triangle_once(corr, n):
    # ragged sizes too: rows and columns past N are staged as zeros and never folded
    _, issued, got = corr.plan_cover(n, 3, with_cover=True)
    assert np.array_equal(got, np.tril(np.ones((n, n), dtype=np.uint8)))
    blocks = (n + 255) // 256
    assert issued == (blocks * (blocks - 1) // 2) * 2 * (2 * 64 * 256) + blocks * 2 * (64 * 128 + 64 * 256)


def test_plan_items_rejects(corr):
    with pytest.raises(corr.CorrError):
        corr.plan_items(192, 10, 8192, 17, 152)  # 17 x 8192 samples exceed one fold
    with pytest.raises(corr.CorrError):
        corr.plan_items(192, 10, 8192, 1, 0)
    with pytest.raises(corr.CorrError):
        corr.plan_items(192, 10, 8192, 1, 152, cover=4)


def test_tuned_cover_is_empty_without_a_gpu(corr):
    assert corr.tuned_cover(192, 8192) == -1


def test_stats_snapshot_restore_reject_null(corr):
    lib = corr.load()
    st = corr.Stats()
    n = corr._ll()
    assert lib.corr_get_stats(None, corr.ctypes.byref(st)) == corr.CORR_EINVAL
    assert lib.corr_snapshot(None, None, corr.ctypes.byref(n), None) == corr.CORR_EINVAL
    assert lib.corr_restore(None, None, 0, None) == corr.CORR_EINVAL
    assert lib.corr_debug_corrupt_guard(None, 0) == corr.CORR_EINVAL
    assert lib.corr_debug_build() == 0
    assert corr.strerror(corr.CORR_EBOUNDS).startswith("an address check")


def test_debug_variant_builds_and_exports(corr):
    """The debug build (CORR_DEBUG) compiles and exports the same symbols, and
    says that it is the debug build."""
    import ctypes
    from paper_2406_19013_gb300 import build
    path = build.build(debug=True)
    assert path.endswith("libcorr_debug.so")
    lib = ctypes.CDLL(path)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    lib.corr_debug_build.restype = ctypes.c_int
    assert lib.corr_debug_build() == 1


@pytest.mark.parametrize("n,issuers,iters,a_tmem", [
    (8, 1, 10, 0), (264, 1, 10, 0), (100, 1, 10, 0),   # N outside 16..256 or not a multiple of 16
    (256, 0, 10, 0), (256, 5, 10, 0),                   # issuing threads outside 1..4
    (256, 1, 0, 0), (256, 1, 10, 2),                    # no iterations; A source not 0/1
    (256, 2, 10, 1),                                    # 2 x 256 + 32 TMEM columns > 512
])
def test_mma_rate_rejects_before_any_device_work(corr, n, issuers, iters, a_tmem):
    status = np.zeros(1, dtype=np.int32)  # never touched: the call fails its checks first
    rc = corr.load().corr_mma_rate(n, issuers, iters, a_tmem, status.ctypes.data, None, None)
    assert rc == corr.CORR_EINVAL
    assert corr.load().corr_mma_rate(256, 1, 10, 0, None, None, None) == corr.CORR_EINVAL
