"""GB300-native TPC sector tracking (standalone TPC tracking of arXiv:2009.07515, Sec. 6).

The tracking runs entirely in ``libtpctrack.so`` (hand-written sm_103a CUDA kernels behind the
C-ABI of ``include/tpctrack.h``). This package is its thin Python binding: ``_lib`` mirrors the
C entry points one to one; ``Tracker`` marshals numpy arrays or torch CUDA tensors (PyTorch serves
only device memory and streams) into those calls.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import TpcError, cf_default_params, default_params, load, tracks_to_numpy

__all__ = ["Tracker", "TpcError", "default_params", "cf_default_params", "load", "build"]


def build(force: bool = False) -> str:
    """Compile libtpctrack.so in-tree (nvcc, sm_103a)."""
    from . import build_ext
    return build_ext.build(force=force)


def _ptr(a):
    """Host numpy array or torch tensor -> (address, on_device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def make_clusters(sector, row, y, w, keep: list) -> _lib.tpc_clusters:
    """Fill a tpc_clusters descriptor; ``keep`` holds references that must outlive the call."""
    arrs = []
    for a, dt in ((sector, np.uint8), (row, np.uint8), (y, np.float32), (w, np.float32)):
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=dt)
        arrs.append(a)
    keep.extend(arrs)
    ptrs = [_ptr(a) for a in arrs]
    on_dev = {p[1] for p in ptrs}
    if len(on_dev) != 1:
        raise ValueError("cluster arrays must all be on the host or all on the device")
    n = int(arrs[2].shape[0])
    return _lib.tpc_clusters(ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], n, on_dev.pop())


class Tracker:
    """One library context on the current CUDA device."""

    def __init__(self, params: _lib.tpc_params | None = None, **overrides):
        self.lib = load()
        self.params = params if params is not None else default_params(**overrides)
        self.params.struct_size = ctypes.sizeof(_lib.tpc_params)
        ctx = ctypes.c_void_p()
        _lib.check(self.lib.tpc_create(ctypes.byref(self.params), ctypes.byref(ctx)))
        self.ctx = ctx
        self._keep: dict[int, list] = {}

    def close(self):
        if self.ctx:
            self.lib.tpc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        return _lib.check(rc, self.ctx)

    # --------------------------------------------------------------- plain path
    def load(self, sector, row, y, w) -> int:
        keep: list = []
        cl = make_clusters(sector, row, y, w, keep)
        h = ctypes.c_uint64()
        self._check(self.lib.tpc_load_clusters(self.ctx, ctypes.byref(cl), ctypes.byref(h)))
        if cl.on_device:
            self._keep[h.value] = keep
        return h.value

    def track(self, frame: int, stream=None) -> None:
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream)
        self._check(self.lib.tpc_track_sectors(self.ctx, ctypes.c_uint64(frame), s))

    def track_batch(self, frames, stream=None) -> None:
        arr = (ctypes.c_uint64 * len(frames))(*frames)
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream)
        self._check(self.lib.tpc_track_batch(self.ctx, arr, len(frames), s))

    TUNE_KEYS = ("bin_occupancy", "k2_warps", "k2_tma", "k5_block", "k5_regs", "k5_blocks_per_sm", "k5_order",
                 "k5_ilp", "sel_lanes", "ms", "total_ms", "stage")

    def autotune(self, frames, reps: int = 3) -> dict:
        """Time launch shapes on a batch (tpc_autotune) and keep the fastest. Returns the timed
        configurations (``entries``, in timing order) and the chosen one (``best``)."""
        frames = [frames] if isinstance(frames, int) else list(frames)
        arr = (ctypes.c_uint64 * len(frames))(*frames)
        rep = _lib.tpc_tune_report()
        self._check(self.lib.tpc_autotune(self.ctx, arr, len(frames), int(reps), ctypes.byref(rep)))
        entries = [{k: getattr(rep.entries[i], k) for k in self.TUNE_KEYS} for i in range(rep.n_entries)]
        return {"entries": entries, "best": entries[rep.best] if rep.best >= 0 else None}

    def tracks(self, frame: int, copy: bool = True) -> dict:
        """The frame's tracks (tpc_get_tracks). copy=False returns views of the library's result
        block, valid until the frame is released."""
        t = _lib.tpc_tracks()
        self._check(self.lib.tpc_get_tracks(self.ctx, ctypes.c_uint64(frame), ctypes.byref(t)))
        return tracks_to_numpy(t, copy=copy)

    def merged(self, frame: int, copy: bool = True) -> dict:
        """The frame's merged and refit tracks (tpc_get_merged_tracks; needs merge=1)."""
        t = _lib.tpc_merged_tracks()
        self._check(self.lib.tpc_get_merged_tracks(self.ctx, ctypes.c_uint64(frame), ctypes.byref(t)))
        return _lib.merged_to_numpy(t, copy=copy)

    def links(self, frame: int, what: int, n: int) -> np.ndarray:
        out = np.empty(n, np.int32)
        self._check(self.lib.tpc_get_links(self.ctx, ctypes.c_uint64(frame), what, out.ctypes.data, n))
        return out

    def keep_mask(self, frame: int, n: int) -> np.ndarray:
        """Strategy-B keep mask of a tracked frame (1 = kept), in the caller's cluster order."""
        out = np.empty(n, np.uint8)
        self._check(self.lib.tpc_get_keep_mask(self.ctx, ctypes.c_uint64(frame), out.ctypes.data, n))
        return out

    def counts(self, frame: int):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.tpc_get_counts(self.ctx, ctypes.c_uint64(frame), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    STAT_NAMES = ("clusters", "sorted", "bins", "starts", "tracklets", "steps", "tracklet_hits", "tracks",
                  "track_hits", "err")

    def stats(self, frame: int) -> dict:
        out = (ctypes.c_int64 * len(self.STAT_NAMES))()
        n = self._check(self.lib.tpc_get_stats(self.ctx, ctypes.c_uint64(frame), out, len(self.STAT_NAMES)))
        return {self.STAT_NAMES[i]: int(out[i]) for i in range(min(n, len(self.STAT_NAMES)))}

    def release(self, frame: int) -> None:
        self._check(self.lib.tpc_release_frame(self.ctx, ctypes.c_uint64(frame)))
        self._keep.pop(frame, None)

    def run(self, sector, row, y, w) -> dict:
        """Load, track and return one frame's tracks (and release it)."""
        f = self.load(sector, row, y, w)
        try:
            self.track(f)
            return self.tracks(f)
        finally:
            self.release(f)

    # --------------------------------------------------------------- cluster finding
    def find_clusters(self, sector, row, pad, time, adc, n_time: int, *, to_host: bool = True,
                      cf_params: _lib.tpc_cf_params | None = None, stream=None, copy: bool = True):
        """Clusters of one frame's digits (tpc_find_clusters). Digit arrays: numpy (host) or torch
        CUDA tensors (device). to_host=True returns numpy arrays (copies, or with copy=False views
        valid until the next call); to_host=False returns the raw tpc_cluster_list of device arrays,
        valid until the next call (see load_cluster_list)."""
        keep = []
        arrs = []
        for a, dt in ((sector, np.uint8), (row, np.uint8), (pad, np.uint16), (time, np.uint16), (adc, np.uint16)):
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=dt)
            arrs.append(a)
        keep.extend(arrs)
        ptrs = [_ptr(a) for a in arrs]
        on_dev = {p[1] for p in ptrs}
        if len(on_dev) != 1:
            raise ValueError("digit arrays must all be on the host or all on the device")
        d = _lib.tpc_digits(*(p[0] for p in ptrs), int(arrs[4].shape[0]), int(n_time), on_dev.pop())
        out = _lib.tpc_cluster_list()
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream)
        cp = ctypes.byref(cf_params) if cf_params is not None else None
        self._check(self.lib.tpc_find_clusters(self.ctx, cp, ctypes.byref(d), 1 if to_host else 0, ctypes.byref(out), s))
        return _lib.clusters_to_numpy(out, copy=copy) if to_host else out

    def load_cluster_list(self, cl: _lib.tpc_cluster_list) -> int:
        """Load the device clusters of find_clusters(to_host=False) as a frame (borrowed: track it
        before the next find_clusters call)."""
        if not cl.on_device:
            raise ValueError("expected a device cluster list")
        c = _lib.tpc_clusters(cl.sector, cl.row, cl.y, cl.w, int(cl.n_clusters), 1)
        h = ctypes.c_uint64()
        self._check(self.lib.tpc_load_clusters(self.ctx, ctypes.byref(c), ctypes.byref(h)))
        return h.value

    def cf_kernel_times(self, launches: bool = False) -> dict:
        kt = _lib.tpc_kernel_times()
        self._check(self.lib.tpc_get_cf_kernel_times(self.ctx, ctypes.byref(kt)))
        if launches:
            return {kt.names[i].decode(): int(kt.launches[i]) for i in range(kt.n_kernels)}
        return {kt.names[i].decode(): float(kt.ms[i]) for i in range(kt.n_kernels)}

    # --------------------------------------------------------------- serving
    def submit(self, sector, row, y, w, borrow: bool = False) -> int:
        """Serving: admit a frame (tpc_submit_frame). borrow=True lends page-locked host arrays
        (on_device = 2): no copy is made; they must stay unchanged until the frame's tracks are read."""
        keep: list = []
        cl = make_clusters(sector, row, y, w, keep)
        if borrow:
            if cl.on_device:
                raise ValueError("borrow=True takes host arrays")
            cl.on_device = 2
        h = ctypes.c_uint64()
        self._check(self.lib.tpc_submit_frame(self.ctx, ctypes.byref(cl), ctypes.byref(h)))
        if cl.on_device:
            self._keep[h.value] = keep
        return h.value

    def poll(self, max_done: int = 64, timeout_us: int = 0) -> list[int]:
        arr = (ctypes.c_uint64 * max(1, max_done))()
        n = self._check(self.lib.tpc_poll(self.ctx, arr, max_done, timeout_us))
        return [arr[i] for i in range(n)]

    # --------------------------------------------------------------- timing
    def set_timing(self, on: bool) -> None:
        self._check(self.lib.tpc_set_timing(self.ctx, 1 if on else 0))

    def kernel_times(self, launches: bool = False) -> dict:
        kt = _lib.tpc_kernel_times()
        self._check(self.lib.tpc_get_kernel_times(self.ctx, ctypes.byref(kt)))
        if launches:
            return {kt.names[i].decode(): int(kt.launches[i]) for i in range(kt.n_kernels)}
        return {kt.names[i].decode(): float(kt.ms[i]) for i in range(kt.n_kernels)}
