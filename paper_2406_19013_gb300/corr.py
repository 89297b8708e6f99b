"""Python binding of libcorr (include/corr.h): argument marshalling only.

Every step of the X-engine runs in the library's CUDA kernels; this module
passes device pointers (torch tensors' ``data_ptr()``), host pointers (numpy
arrays) and the current CUDA stream, and turns negative return codes into
exceptions.  There is no fallback: if the library is missing the import of
this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# CORR_LIB_VARIANT=debug loads the debug build (libcorr_debug.so: address
# checks in the kernels, guard bands around the integration buffers).
LIB_PATH = os.path.join(_HERE, "libcorr_debug.so" if os.environ.get("CORR_LIB_VARIANT") == "debug"
                        else "libcorr.so")

CORR_OK = 0
CORR_EINVAL = -1
CORR_ENOMEM = -2
CORR_ECUDA = -3
CORR_EARCH = -4
CORR_ETIMEOUT = -5
CORR_ESTATE = -6
CORR_EBOUNDS = -7
CORR_MAX_BLOCK_LEN = 16777215
CORR_FOLD_SAMPLES = 131071
CORR_STATIC_MAX_BLOCK_LEN = 131056
CORR_MAX_INPUTS = 8192
CORR_COVER_WINDOW = 0
CORR_COVER_STRIPS = 1
CORR_COVER_PAIRS = 2
CORR_COVER_QUADS = 3
CORR_BATCH_AUTOTUNE = 1

# (name, restype, argtypes) of every function include/corr.h declares
_vp, _ci, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
ABI = [
    ("corr_create", _ci, [_ci, _ci, _ci, _ci, ctypes.POINTER(_vp)]),
    ("corr_push_block", _ci, [_vp, _vp, _vp]),
    ("corr_push_blocks", _ci, [_vp, ctypes.POINTER(_vp), _ci, _vp]),
    ("corr_dump", _ci, [_vp, _vp, _vp, _vp]),
    ("corr_push_block_host", _ci, [_vp, _vp, _vp]),
    ("corr_dump_host", _ci, [_vp, _vp, _vp, _vp]),
    ("corr_sizes", _ci, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                         ctypes.POINTER(_ll)]),
    ("corr_check", _ci, [_vp, _vp]),
    ("corr_plan", _ci, [_ci, _vp, ctypes.POINTER(_ci), ctypes.POINTER(_ll)]),
    ("corr_plan_cover", _ci, [_ci, _ci, _vp, ctypes.POINTER(_ci), ctypes.POINTER(_ll)]),
    ("corr_plan_items", _ci, [_ci, _ci, _ci, _ci, _ci, _ci, _vp, _ci, ctypes.POINTER(_ci), _vp,
                              ctypes.POINTER(_ci)]),
    ("corr_batch_create", _ci, [_ci, _vp, _vp, _vp, _vp, _ci, ctypes.POINTER(_vp)]),
    ("corr_batch_push", _ci, [_vp, ctypes.POINTER(_vp), _vp]),
    ("corr_batch_dump", _ci, [_vp, _ci, _vp, _vp, _vp]),
    ("corr_batch_sizes", _ci, [_vp, _ci, ctypes.POINTER(ctypes.c_size_t),
                               ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_ll)]),
    ("corr_batch_info", _ci, [_vp, _ci, ctypes.POINTER(_ci), ctypes.POINTER(_ci),
                              ctypes.POINTER(_ci)]),
    ("corr_batch_check", _ci, [_vp, _vp]),
    ("corr_batch_launch_count", _ll, [_vp]),
    ("corr_batch_destroy", None, [_vp]),
    ("corr_tuned_cover", _ci, [_ci, _ci]),
    ("corr_corner_turn", _ci, [_vp, _vp, _ci, _ci, _ci, _vp]),
    ("corr_push_block_tcn", _ci, [_vp, _vp, _vp]),
    ("corr_selftest_timeout", _ci, [_vp, _vp, _ci, _vp]),
    ("corr_xcorr_static", _ci, [_vp, _ci, _ci, _ci, _ci, _vp, _vp]),
    ("corr_mma_rate", _ci, [_ci, _ci, _ci, _ci, _vp, _vp, _vp]),
    ("corr_launch_count", _ll, [_vp]),
    ("corr_get_stats", _ci, [_vp, _vp]),
    ("corr_snapshot", _ci, [_vp, _vp, ctypes.POINTER(_ll), _vp]),
    ("corr_restore", _ci, [_vp, _vp, _ll, _vp]),
    ("corr_debug_build", _ci, []),
    ("corr_debug_corrupt_guard", _ci, [_vp, _ci]),
    ("corr_destroy", None, [_vp]),
    ("corr_strerror", ctypes.c_char_p, [_ci]),
]

class Stats(ctypes.Structure):
    _fields_ = [("blocks_pushed", _ll), ("samples_total", _ll), ("samples_pending", _ll),
                ("dumps", _ll), ("launches", _ll)]


def debug_build() -> bool:
    """Whether the loaded library is the debug build."""
    return bool(load().corr_debug_build())


class ArrayDesc(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int), ("n_pol", ctypes.c_int), ("n_chan", ctypes.c_int),
                ("block_len", ctypes.c_int), ("blocks_per_integration", ctypes.c_int)]


class ServerResult(ctypes.Structure):
    _fields_ = [("array", ctypes.c_int), ("integration", ctypes.c_longlong),
                ("n_blocks", ctypes.c_int), ("block_mask", ctypes.c_uint64),
                ("vis", ctypes.c_void_p), ("t_first_arrival_ms", ctypes.c_double),
                ("t_last_arrival_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("integrated", ctypes.c_longlong),
                ("duplicates", ctypes.c_longlong), ("late", ctypes.c_longlong),
                ("integrations", ctypes.c_longlong),
                ("incomplete_integrations", ctypes.c_longlong),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_max_ms", ctypes.c_double), ("latency_samples", ctypes.c_longlong),
                ("arena_peak_bytes", ctypes.c_size_t), ("error", ctypes.c_int)]


ABI += [
    ("corr_server_create", _ci, [_ci, ctypes.POINTER(ArrayDesc), ctypes.c_size_t, _ci, _ci,
                                 ctypes.POINTER(_vp)]),
    ("corr_server_submit", _ci, [_vp, _ci, _ll, _vp]),
    ("corr_server_poll", _ci, [_vp, ctypes.POINTER(ServerResult), _ci, _ci]),
    ("corr_server_release", _ci, [_vp, _ci]),
    ("corr_server_flush", _ci, [_vp]),
    ("corr_server_stats", _ci, [_vp, ctypes.POINTER(ServerInfo)]),
    ("corr_server_destroy", None, [_vp]),
]
CORR_SERVER_DRY = 1
ABI += [
    ("corr_fengine_create", _ci, [_ci, _ci, ctypes.POINTER(_vp)]),
    ("corr_fengine_set_eq", _ci, [_vp, _vp]),
    ("corr_fengine_run", _ci, [_vp, _vp, _vp, _vp]),
    ("corr_fengine_spectra", _ci, [_vp, _vp, _vp, _vp]),
    ("corr_fengine_destroy", None, [_vp]),
]

_lock = threading.Lock()
_lib = None


class CorrError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


def load(path: str = LIB_PATH):
    """Loads libcorr.so (built by ``paper_2406_19013_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: run paper_2406_19013_gb300.build.build()")
            lib = ctypes.CDLL(path)
            for name, res, args in ABI:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def strerror(code: int) -> str:
    return load().corr_strerror(code).decode()


def _ck(rc: int, what: str):
    if rc != CORR_OK:
        raise CorrError(rc, what)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def plan(n_in: int, with_cover: bool = False):
    """(units per channel, issued CMACs per channel-sample, cover or None)."""
    cover = np.zeros((n_in, n_in), dtype=np.uint8) if with_cover else None
    nu, iss = _ci(), _ll()
    _ck(load().corr_plan(n_in, cover.ctypes.data if with_cover else None, ctypes.byref(nu),
                         ctypes.byref(iss)), "corr_plan")
    return nu.value, iss.value, cover


def plan_cover(n_in: int, cover: int, with_cover: bool = False):
    """As ``plan`` for the given CORR_COVER_* cover."""
    out = np.zeros((n_in, n_in), dtype=np.uint8) if with_cover else None
    nu, iss = _ci(), _ll()
    _ck(load().corr_plan_cover(n_in, cover, out.ctypes.data if with_cover else None,
                               ctypes.byref(nu), ctypes.byref(iss)), "corr_plan_cover")
    return nu.value, iss.value, out


def plan_items(n_in: int, n_chan: int, block_len: int, n_blocks: int, grid: int,
               cover: int = CORR_COVER_WINDOW):
    """The per-CTA item split of one launch: (items int32[n][5] as (problem,
    template, channel, first stage, stages), cta_first int32[used_grid + 1])."""
    lib = load()
    n, used = _ci(), _ci()
    _ck(lib.corr_plan_items(n_in, n_chan, block_len, n_blocks, cover, grid, None, 0,
                            ctypes.byref(n), None, ctypes.byref(used)), "corr_plan_items")
    items = np.zeros((n.value, 5), dtype=np.int32)
    first = np.zeros(grid + 1, dtype=np.int32)
    _ck(lib.corr_plan_items(n_in, n_chan, block_len, n_blocks, cover, grid, items.ctypes.data,
                            n.value, ctypes.byref(n), first.ctypes.data, ctypes.byref(used)),
        "corr_plan_items")
    return items, first[:used.value + 1]


def tuned_cover(n_in: int, block_len: int) -> int:
    """The autotuner's cached cover for (n_in, block_len), or -1."""
    rc = load().corr_tuned_cover(n_in, block_len)
    if rc < -1:
        _ck(rc, "corr_tuned_cover")
    return rc


def corner_turn(x_tcn, out=None, stream=None):
    """F-engine order uint8[block_len][n_chan][n_inputs] (CUDA tensor) to
    X-engine order uint8[n_chan][n_inputs][block_len] via corr_corner_turn."""
    import torch
    if not (x_tcn.is_cuda and x_tcn.dtype == torch.uint8 and x_tcn.is_contiguous()
            and x_tcn.dim() == 3):
        raise ValueError("x_tcn must be a contiguous uint8 CUDA tensor [block_len][n_chan][n_inputs]")
    T, C, N = x_tcn.shape
    if out is None:
        out = torch.empty((C, N, T), dtype=torch.uint8, device=x_tcn.device)
    _ck(load().corr_corner_turn(x_tcn.data_ptr(), out.data_ptr(), N, C, T,
                                _stream_handle(stream)), "corr_corner_turn")
    return out


def xcorr_static(block, n_ant: int, n_pol: int, vis=None, stream=None):
    """One block's visibilities through corr_xcorr_static (no allocation in the
    library): block is a uint8[n_chan][n_inputs][block_len] CUDA tensor, vis an
    int64[n_chan][P][2] CUDA tensor to overwrite (allocated here by torch if
    not given, outside the library call)."""
    import torch
    n_chan, n_in, block_len = block.shape
    if n_in != n_ant * n_pol or not (block.is_cuda and block.dtype == torch.uint8
                                      and block.is_contiguous()):
        raise ValueError("block must be a contiguous uint8 CUDA tensor [n_chan][n_inputs][block_len]")
    if vis is None:
        vis = torch.empty((n_chan, n_pairs(n_in), 2), dtype=torch.int64, device=block.device)
    _ck(load().corr_xcorr_static(block.data_ptr(), n_ant, n_pol, n_chan, block_len, vis.data_ptr(),
                                 _stream_handle(stream)), "corr_xcorr_static")
    return vis


def mma_rate(n: int = 256, issuers: int = 1, iters: int = 10000, a_from_tmem: bool = False,
             reps: int = 3, stream=None):
    """Dense E5M2 tcgen05 MMA rate (corr_mma_rate), best of `reps` launches
    timed with CUDA events: returns (TFLOP/s, ms per launch, median cycles per
    MMA per issuing thread)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    cycles = torch.zeros(n_sm, dtype=torch.int64, device=dev)
    st = torch.cuda.current_stream() if stream is None else stream
    h = _stream_handle(st)
    lib = load()
    best_ms, best_cyc = None, None
    for _ in range(max(1, reps) + 1):  # the first launch is a warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        _ck(lib.corr_mma_rate(n, issuers, iters, int(a_from_tmem), status.data_ptr(),
                              cycles.data_ptr(), h), "corr_mma_rate")
        b.record(st)
        b.synchronize()
        ms = a.elapsed_time(b)
        if int(status.item()) != 0:
            raise CorrError(CORR_ETIMEOUT, "corr_mma_rate")
        cyc = float(cycles.float().median().item()) / (4 * iters)
        if best_ms is None or ms < best_ms:
            best_ms, best_cyc = ms, cyc
    flop = n_sm * issuers * iters * 4 * 2 * 128 * n * 32
    return flop / (best_ms / 1e3) / 1e12, best_ms, best_cyc


def n_pairs(n_in: int) -> int:
    return n_in * (n_in + 1) // 2


class Correlator:
    """One X-engine integration context on the current CUDA device.

    ``push_block`` integrates a uint8[n_chan][n_inputs][block_len] device
    tensor; ``dump`` returns (vis int64[n_chan][P][2], stokes
    int64[n_chan][A][4][2] or None) and restarts the integration.
    """

    def __init__(self, n_ant: int, n_pol: int, n_chan: int, block_len: int):
        self._lib = load()
        h = _vp()
        _ck(self._lib.corr_create(n_ant, n_pol, n_chan, block_len, ctypes.byref(h)), "corr_create")
        self._h = h
        self.n_ant, self.n_pol, self.n_chan, self.block_len = n_ant, n_pol, n_chan, block_len
        self.n_in = n_ant * n_pol
        self.n_pairs = n_pairs(self.n_in)
        self.n_apairs = n_pairs(n_ant)

    # ---------------------------------------------------------------- device
    def push_block(self, block, stream=None):
        import torch
        if isinstance(block, torch.Tensor):
            if not (block.is_cuda and block.dtype == torch.uint8 and block.is_contiguous()):
                raise ValueError("block must be a contiguous uint8 CUDA tensor")
            if block.numel() != self.n_chan * self.n_in * self.block_len:
                raise ValueError("block has the wrong number of samples")
            ptr = block.data_ptr()
        else:
            ptr = int(block)
        _ck(self._lib.corr_push_block(self._h, ptr, _stream_handle(stream)), "corr_push_block")

    def push_block_tcn(self, block_tcn, stream=None):
        """Integrates a block in F-engine order, uint8[block_len][n_chan][n_inputs]
        (corner-turned on the device by the library)."""
        import torch
        if not (block_tcn.is_cuda and block_tcn.dtype == torch.uint8 and block_tcn.is_contiguous()
                and block_tcn.numel() == self.n_chan * self.n_in * self.block_len):
            raise ValueError("block_tcn must be a contiguous uint8 CUDA tensor of the context's size")
        _ck(self._lib.corr_push_block_tcn(self._h, block_tcn.data_ptr(), _stream_handle(stream)),
            "corr_push_block_tcn")

    def push_blocks(self, blocks, stream=None):
        """Integrates several blocks (device tensors or pointers) with shared folds."""
        ptrs = []
        for blk in blocks:
            if hasattr(blk, "data_ptr"):
                if not (blk.is_cuda and blk.is_contiguous() and
                        blk.numel() == self.n_chan * self.n_in * self.block_len):
                    raise ValueError("each block must be a contiguous uint8 CUDA tensor of one block")
                ptrs.append(blk.data_ptr())
            else:
                ptrs.append(int(blk))
        arr = (_vp * max(1, len(ptrs)))(*ptrs)
        _ck(self._lib.corr_push_blocks(self._h, arr, len(ptrs), _stream_handle(stream)),
            "corr_push_blocks")

    def dump(self, vis=None, stokes=None, want_vis: bool = True, want_stokes: bool | None = None,
             stream=None):
        import torch
        if want_stokes is None:
            want_stokes = self.n_pol == 2
        dev = torch.device("cuda", torch.cuda.current_device())
        if vis is None and want_vis:
            vis = torch.empty((self.n_chan, self.n_pairs, 2), dtype=torch.int64, device=dev)
        if stokes is None and want_stokes:
            stokes = torch.empty((self.n_chan, self.n_apairs, 4, 2), dtype=torch.int64, device=dev)
        _ck(self._lib.corr_dump(self._h, vis.data_ptr() if vis is not None else None,
                                stokes.data_ptr() if stokes is not None else None,
                                _stream_handle(stream)), "corr_dump")
        return vis, stokes

    # ---------------------------------------------------------------- host
    @staticmethod
    def _host_ptr(a, dtype, n, what):
        """Address of a contiguous host buffer (numpy array or CPU torch tensor)."""
        if isinstance(a, np.ndarray):
            if a.dtype != dtype or a.size != n or not a.flags.c_contiguous:
                raise ValueError(f"{what} must be a contiguous {np.dtype(dtype).name}[{n}] array")
            return a.ctypes.data
        if a.device.type != "cpu" or not a.is_contiguous() or a.numel() != n or \
                a.element_size() != np.dtype(dtype).itemsize:
            raise ValueError(f"{what} must be a contiguous host tensor of {n} elements")
        return a.data_ptr()

    def push_block_host(self, block, stream=None):
        """block: uint8[n_chan][n_inputs][block_len] numpy array or CPU tensor (pinned is faster)."""
        if isinstance(block, np.ndarray):
            block = np.ascontiguousarray(block)
        ptr = self._host_ptr(block, np.uint8, self.n_chan * self.n_in * self.block_len, "block")
        _ck(self._lib.corr_push_block_host(self._h, ptr, _stream_handle(stream)),
            "corr_push_block_host")

    def dump_host(self, vis=None, stokes=None, want_stokes: bool | None = None, stream=None):
        if want_stokes is None:
            want_stokes = self.n_pol == 2 or stokes is not None
        if vis is None:
            vis = np.empty((self.n_chan, self.n_pairs, 2), dtype=np.int64)
        if stokes is None and want_stokes:
            stokes = np.empty((self.n_chan, self.n_apairs, 4, 2), dtype=np.int64)
        pv = self._host_ptr(vis, np.int64, self.n_chan * self.n_pairs * 2, "vis")
        ps = (self._host_ptr(stokes, np.int64, self.n_chan * self.n_apairs * 8, "stokes")
              if stokes is not None else None)
        _ck(self._lib.corr_dump_host(self._h, pv, ps, _stream_handle(stream)), "corr_dump_host")
        return vis, stokes

    # ---------------------------------------------------------------- misc
    def selftest_timeout(self, block, timeout_ms: int = 200, stream=None):
        """Enqueues the failure-detection self-test (corr_selftest_timeout); the
        next check() raises CorrError with CORR_ETIMEOUT."""
        _ck(self._lib.corr_selftest_timeout(self._h, block.data_ptr(), timeout_ms,
                                            _stream_handle(stream)), "corr_selftest_timeout")

    def check(self, stream=None):
        _ck(self._lib.corr_check(self._h, _stream_handle(stream)), "corr_check")

    def samples_integrated(self) -> int:
        s = _ll()
        _ck(self._lib.corr_sizes(self._h, None, None, ctypes.byref(s)), "corr_sizes")
        return s.value

    def launch_count(self) -> int:
        return int(self._lib.corr_launch_count(self._h))

    def stats(self) -> dict:
        """The context's counters (corr_get_stats)."""
        st = Stats()
        _ck(self._lib.corr_get_stats(self._h, ctypes.byref(st)), "corr_get_stats")
        return {name: int(getattr(st, name)) for name, _ in Stats._fields_}

    def snapshot(self, stream=None):
        """(acc int64[n_chan][P][2] numpy array, samples): the integration in
        progress, for corr_restore."""
        acc = np.empty((self.n_chan, self.n_pairs, 2), dtype=np.int64)
        n = _ll()
        _ck(self._lib.corr_snapshot(self._h, acc.ctypes.data, ctypes.byref(n),
                                    _stream_handle(stream)), "corr_snapshot")
        return acc, n.value

    def restore(self, acc, samples: int, stream=None):
        """Replaces the integration in progress with a snapshot."""
        pa = self._host_ptr(acc, np.int64, self.n_chan * self.n_pairs * 2, "acc")
        _ck(self._lib.corr_restore(self._h, pa, int(samples), _stream_handle(stream)),
            "corr_restore")

    def debug_corrupt_guard(self, side: int):
        """Debug builds: overwrites a byte of a guard band (corr_debug_corrupt_guard)."""
        _ck(self._lib.corr_debug_corrupt_guard(self._h, side), "corr_debug_corrupt_guard")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.corr_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent correlators integrated by shared launches (corr_batch_*).

    ``shapes`` is a list of (n_ant, n_pol, n_chan, block_len).  ``push``
    takes one uint8[n_chan][n_inputs][block_len] CUDA tensor per instance;
    ``dump(k)`` returns instance k's (vis, stokes or None) and restarts its
    integration.
    """

    def __init__(self, shapes, autotune: bool = False):
        self._lib = load()
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        n = len(self.shapes)
        arr = [np.array([sh[k] for sh in self.shapes], dtype=np.int32) for k in range(4)]
        h = _vp()
        _ck(self._lib.corr_batch_create(n, *(a.ctypes.data for a in arr),
                                        CORR_BATCH_AUTOTUNE if autotune else 0, ctypes.byref(h)),
            "corr_batch_create")
        self._h = h

    def __len__(self):
        return len(self.shapes)

    def push(self, blocks, stream=None):
        import torch
        if len(blocks) != len(self.shapes):
            raise ValueError("one block per instance")
        ptrs = []
        for blk, (na, npol, nc, T) in zip(blocks, self.shapes):
            if isinstance(blk, torch.Tensor):
                if not (blk.is_cuda and blk.dtype == torch.uint8 and blk.is_contiguous()
                        and blk.numel() == nc * na * npol * T):
                    raise ValueError("each block must be a contiguous uint8 CUDA tensor of its "
                                     "instance's size")
                ptrs.append(blk.data_ptr())
            else:
                ptrs.append(int(blk))
        arr = (_vp * len(ptrs))(*ptrs)
        _ck(self._lib.corr_batch_push(self._h, arr, _stream_handle(stream)), "corr_batch_push")

    def dump(self, k: int, vis=None, stokes=None, want_stokes: bool | None = None, stream=None):
        import torch
        na, npol, nc, _ = self.shapes[k]
        if want_stokes is None:
            want_stokes = npol == 2
        dev = torch.device("cuda", torch.cuda.current_device())
        if vis is None:
            vis = torch.empty((nc, n_pairs(na * npol), 2), dtype=torch.int64, device=dev)
        if stokes is None and want_stokes:
            stokes = torch.empty((nc, n_pairs(na), 4, 2), dtype=torch.int64, device=dev)
        _ck(self._lib.corr_batch_dump(self._h, k, vis.data_ptr(),
                                      stokes.data_ptr() if stokes is not None else None,
                                      _stream_handle(stream)), "corr_batch_dump")
        return vis, stokes

    def info(self, k: int):
        """(cover, launch group, number of launch groups) of instance k."""
        cv, g, ng = _ci(), _ci(), _ci()
        _ck(self._lib.corr_batch_info(self._h, k, ctypes.byref(cv), ctypes.byref(g),
                                      ctypes.byref(ng)), "corr_batch_info")
        return cv.value, g.value, ng.value

    def samples_integrated(self, k: int) -> int:
        s = _ll()
        _ck(self._lib.corr_batch_sizes(self._h, k, None, None, ctypes.byref(s)),
            "corr_batch_sizes")
        return s.value

    def check(self, stream=None):
        _ck(self._lib.corr_batch_check(self._h, _stream_handle(stream)), "corr_batch_check")

    def launch_count(self) -> int:
        return int(self._lib.corr_batch_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.corr_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A served X-engine (corr_server_*): blocks of several arrays arrive one by
    one from host memory; completed integrations come back from ``poll``.

    ``arrays`` is a list of (n_ant, n_pol, n_chan, block_len,
    blocks_per_integration).  ``submit(array, seq, block)`` takes a uint8
    numpy array or CPU torch tensor of the array's block size (pinned memory
    copies fastest); the Server keeps a reference until it is closed.
    ``poll`` returns dicts with the integration's metadata and, unless dry, a
    copy of its visibilities (int64[n_chan][P][2]); the server-side buffer is
    released at once.
    """

    def __init__(self, arrays, arena_bytes: int, window: int = 2, dry: bool = False):
        self._lib = load()
        self.arrays = [tuple(int(v) for v in a) for a in arrays]
        self.dry = dry
        descs = (ArrayDesc * len(self.arrays))(*[ArrayDesc(*a) for a in self.arrays])
        h = _vp()
        _ck(self._lib.corr_server_create(len(self.arrays), descs, int(arena_bytes), window,
                                         CORR_SERVER_DRY if dry else 0, ctypes.byref(h)),
            "corr_server_create")
        self._h = h
        self._keep = []

    def submit(self, array: int, seq: int, block=None):
        ptr = None
        if block is not None:
            na, npol, nc, T, _ = self.arrays[array]
            nbytes = nc * na * npol * T
            if hasattr(block, "data_ptr"):
                if block.is_cuda or block.numel() * block.element_size() != nbytes:
                    raise ValueError("block must be a host tensor of the array's block size")
                ptr = block.data_ptr()
            else:
                arr = np.asarray(block)
                if arr.dtype != np.uint8 or arr.nbytes != nbytes or not arr.flags.c_contiguous:
                    raise ValueError("block must be a contiguous uint8 array of the array's "
                                     "block size")
                ptr = arr.ctypes.data
            self._keep.append(block)
        _ck(self._lib.corr_server_submit(self._h, array, seq, ptr), "corr_server_submit")

    def poll(self, max_results: int = 64, timeout_ms: int = 0, copy: bool = True):
        """Completed integrations, oldest first.  With copy=False the
        visibilities are not copied out ("vis" is None) and the server-side
        buffer is released at once."""
        out = (ServerResult * max_results)()
        n = self._lib.corr_server_poll(self._h, out, max_results, timeout_ms)
        if n < 0:
            _ck(n, "corr_server_poll")
        res = []
        for r in out[:n]:
            d = {"array": r.array, "integration": r.integration, "n_blocks": r.n_blocks,
                 "block_mask": r.block_mask, "t_first_arrival_ms": r.t_first_arrival_ms,
                 "t_last_arrival_ms": r.t_last_arrival_ms, "t_done_ms": r.t_done_ms, "vis": None}
            if r.vis and copy:
                na, npol, nc, T, _ = self.arrays[r.array]
                shape = (nc, n_pairs(na * npol), 2)
                buf = (ctypes.c_int64 * (shape[0] * shape[1] * 2)).from_address(r.vis)
                d["vis"] = np.frombuffer(buf, dtype=np.int64).reshape(shape).copy()
            _ck(self._lib.corr_server_release(self._h, r.array), "corr_server_release")
            res.append(d)
        return res

    def flush(self):
        _ck(self._lib.corr_server_flush(self._h), "corr_server_flush")

    def stats(self) -> dict:
        info = ServerInfo()
        _ck(self._lib.corr_server_stats(self._h, ctypes.byref(info)), "corr_server_stats")
        return {name: getattr(info, name) for name, _ in ServerInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.corr_server_destroy(self._h)
            self._h = None
            self._keep = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FEngine:
    """The GPU F-engine (corr_fengine_*): int8 ADC streams
    [n_in][(n_spectra + 3) * 2048] (starting on a 16-byte boundary) -> packed
    channel samples uint8[1024][n_in][n_spectra], the X-engine's input order."""

    def __init__(self, n_in: int, n_spectra: int, eq=None):
        self._lib = load()
        h = _vp()
        _ck(self._lib.corr_fengine_create(n_in, n_spectra, ctypes.byref(h)), "corr_fengine_create")
        self._h = h
        self.n_in, self.n_spectra = n_in, n_spectra
        if eq is not None:
            self.set_eq(eq)

    def set_eq(self, eq):
        g = np.ascontiguousarray(eq, dtype=np.float32)
        if g.shape != (self.n_in, 1024):
            raise ValueError("eq must be float[n_in][1024]")
        _ck(self._lib.corr_fengine_set_eq(self._h, g.ctypes.data), "corr_fengine_set_eq")

    def _check_adc(self, adc):
        import torch
        if not (adc.is_cuda and adc.dtype == torch.int8 and adc.is_contiguous()
                and adc.numel() == self.n_in * (self.n_spectra + 3) * 2048):
            raise ValueError("adc must be a contiguous int8 CUDA tensor [n_in][(n_spectra+3)*2048]")

    def run(self, adc, out=None, stream=None):
        import torch
        self._check_adc(adc)
        if out is None:
            out = torch.empty((1024, self.n_in, self.n_spectra), dtype=torch.uint8,
                              device=adc.device)
        _ck(self._lib.corr_fengine_run(self._h, adc.data_ptr(), out.data_ptr(),
                                       _stream_handle(stream)), "corr_fengine_run")
        return out

    def spectra(self, adc, stream=None):
        import torch
        self._check_adc(adc)
        out = torch.empty((1024, self.n_in, self.n_spectra, 2), dtype=torch.float32,
                          device=adc.device)
        _ck(self._lib.corr_fengine_spectra(self._h, adc.data_ptr(), out.data_ptr(),
                                           _stream_handle(stream)), "corr_fengine_spectra")
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.corr_fengine_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
