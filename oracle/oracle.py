"""Python binding of the CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module; the library package
never does.  The oracle shares no code with the CUDA path.

Every function here is the plain definition of the X-engine (Sec. 2.3: CMAC
per channel over all baselines; Eq. 1: N(N+1)/2 products with autos; Eq. 2:
V = <S1^* S2>, stored as V[i][j] = sum_t x_i conj(x_j) for i >= j) and the
full-Stokes reading documented in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C99, no architecture flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread", _SRC,
                        "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, ci = ctypes.c_void_p, ctypes.c_int
            lib.oracle_xcorr.argtypes = [vp, ci, ci, ci, vp, ci]
            lib.oracle_xcorr_pair.argtypes = [vp, ci, ci, ci, ci, ci, vp]
            lib.oracle_xcorr_full.argtypes = [vp, ci, ci, ci, vp]
            lib.oracle_stokes.argtypes = [vp, ci, ci, vp]
            lib.oracle_decode.argtypes = [ctypes.c_uint8, vp, vp]
            for f in (lib.oracle_xcorr, lib.oracle_xcorr_pair, lib.oracle_xcorr_full,
                      lib.oracle_stokes):
                f.restype = ci
            lib.oracle_decode.restype = None
            _lib = lib
    return _lib


def n_pairs(n_in: int) -> int:
    return n_in * (n_in + 1) // 2


def decode(b: int) -> tuple[int, int]:
    re, im = ctypes.c_int64(), ctypes.c_int64()
    _load().oracle_decode(b, ctypes.byref(re), ctypes.byref(im))
    return re.value, im.value


def _check_x(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x)
    if x.dtype != np.uint8 or x.ndim != 3:
        raise ValueError("x must be uint8[n_chan][n_in][T]")
    return x


def xcorr(x: np.ndarray, vis: np.ndarray | None = None, n_threads: int = 1) -> np.ndarray:
    """Lower-triangle visibilities int64[n_chan][P][2]; accumulates into `vis`."""
    x = _check_x(x)
    C, N, T = x.shape
    if vis is None:
        vis = np.zeros((C, n_pairs(N), 2), dtype=np.int64)
    assert vis.dtype == np.int64 and vis.shape == (C, n_pairs(N), 2) and vis.flags.c_contiguous
    if _load().oracle_xcorr(x.ctypes.data, N, C, T, vis.ctypes.data, n_threads) != 0:
        raise ValueError("oracle_xcorr rejected its arguments")
    return vis


def xcorr_pair(x: np.ndarray, c: int, i: int, j: int) -> tuple[int, int]:
    """V[i][j] of channel c (any i, j)."""
    x = _check_x(x)
    C, N, T = x.shape
    out = np.zeros(2, dtype=np.int64)
    if _load().oracle_xcorr_pair(x.ctypes.data, N, T, c, i, j, out.ctypes.data) != 0:
        raise ValueError("oracle_xcorr_pair rejected its arguments")
    return int(out[0]), int(out[1])


def xcorr_full(x: np.ndarray) -> np.ndarray:
    """Every V[i][j], int64[n_chan][n_in][n_in][2]."""
    x = _check_x(x)
    C, N, T = x.shape
    full = np.zeros((C, N, N, 2), dtype=np.int64)
    if _load().oracle_xcorr_full(x.ctypes.data, N, C, T, full.ctypes.data) != 0:
        raise ValueError("oracle_xcorr_full rejected its arguments")
    return full


def stokes(vis: np.ndarray, n_ant: int) -> np.ndarray:
    """Full-Stokes int64[n_chan][A][4][2] (I, Q, U, V) from dual-pol visibilities."""
    vis = np.ascontiguousarray(vis, dtype=np.int64)
    C = vis.shape[0]
    assert vis.shape == (C, n_pairs(2 * n_ant), 2)
    out = np.zeros((C, n_pairs(n_ant), 4, 2), dtype=np.int64)
    if _load().oracle_stokes(vis.ctypes.data, n_ant, C, out.ctypes.data) != 0:
        raise ValueError("oracle_stokes rejected its arguments")
    return out


def pair_index(i: int, j: int) -> int:
    """Row-major lower-triangle index of (i, j), i >= j (Eq. 1's N(N+1)/2 count)."""
    assert i >= j >= 0
    return i * (i + 1) // 2 + j


def corner_turn(x_tcn: np.ndarray) -> np.ndarray:
    """The Transpose step of Sec. 2.1: uint8[T][C][N] (one spectrum per time
    step) to uint8[C][N][T] (each input's samples contiguous per channel),
    out[c][i][t] = x[t][c][i]."""
    x = np.asarray(x_tcn)
    assert x.dtype == np.uint8 and x.ndim == 3
    T, C, N = x.shape
    out = np.empty((C, N, T), dtype=np.uint8)
    for t in range(T):
        out[:, :, t] = x[t]
    return out
