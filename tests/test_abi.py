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
    (4, 2, 4, -5), (4, 2, 4, 131072), (8193, 1, 1, 16), (4097, 2, 1, 16)])
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
