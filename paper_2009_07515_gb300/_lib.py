"""ctypes binding of libtpctrack.so — argument marshalling only.

Every function here has the name and meaning of the C entry point in ``include/tpctrack.h``; all
tracking work runs in the library's CUDA kernels. The library must have been built (``build_ext.py``);
loading fails loudly otherwise, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtpctrack.so")

TPC_OK = 0
TPC_E_INVAL = -1
TPC_E_NOMEM = -2
TPC_E_BUDGET = -3
TPC_E_CAPACITY = -4
TPC_E_TIMEOUT = -5
TPC_E_CUDA = -6
TPC_E_STATE = -7
ERROR_NAMES = {0: "TPC_OK", -1: "TPC_E_INVAL", -2: "TPC_E_NOMEM", -3: "TPC_E_BUDGET", -4: "TPC_E_CAPACITY",
               -5: "TPC_E_TIMEOUT", -6: "TPC_E_CUDA", -7: "TPC_E_STATE"}

NSECTORS = 36
NROWS = 152


class tpc_params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("bz", ctypes.c_double),
        ("ky", ctypes.c_double), ("kw", ctypes.c_double), ("eps", ctypes.c_double),
        ("chi_n_max", ctypes.c_double),
        ("lmin", ctypes.c_int32),
        ("sigma_y", ctypes.c_double), ("sigma_w", ctypes.c_double),
        ("chi2_hit_max", ctypes.c_double),
        ("n_miss_max", ctypes.c_int32),
        ("win_nsig", ctypes.c_double), ("win_add", ctypes.c_double),
        ("x0_per_row", ctypes.c_double),
        ("max_sin", ctypes.c_double),
        ("y_margin", ctypes.c_double),
        ("nmin", ctypes.c_int32),
        ("cov0", ctypes.c_double * 5),
        ("ext_stop", ctypes.c_int32),
        ("drift_length", ctypes.c_double),
        ("drift_velocity", ctypes.c_double),
        ("keep_vy", ctypes.c_double),
        ("keep_vw", ctypes.c_double),
        ("keep_qpt_max", ctypes.c_double),
        ("packed", ctypes.c_int32),
        ("bin_occupancy", ctypes.c_float),
        ("tracklet_capacity", ctypes.c_float),
        ("hbm_budget", ctypes.c_int64),
        ("max_batch_frames", ctypes.c_int32),
        ("use_graphs", ctypes.c_int32),
        ("compress", ctypes.c_int32),
        ("k2_warps", ctypes.c_int32),
        ("k2_tma", ctypes.c_int32),
        ("k5_block", ctypes.c_int32),
        ("k5_regs", ctypes.c_int32),
        ("k5_blocks_per_sm", ctypes.c_int32),
        ("k5_order", ctypes.c_int32),
        ("sel_lanes", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("merge", ctypes.c_int32),
        ("merge_gap_rows", ctypes.c_int32),
        ("merge_dw", ctypes.c_double),
        ("merge_chi2_max", ctypes.c_double),
        ("refit_passes", ctypes.c_int32),
        ("refit_scale", ctypes.c_double),
        ("k5_ilp", ctypes.c_int32),
        ("wide_votes", ctypes.c_int32),
    ]


class tpc_clusters(ctypes.Structure):
    _fields_ = [
        ("sector", ctypes.c_void_p),
        ("row", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("on_device", ctypes.c_int32),
    ]


class tpc_merged_tracks(ctypes.Structure):
    _fields_ = [
        ("n_merged", ctypes.c_int64),
        ("sector", ctypes.POINTER(ctypes.c_int32)),
        ("n_seg", ctypes.POINTER(ctypes.c_int32)),
        ("head", ctypes.POINTER(ctypes.c_int32)),
        ("x_ref", ctypes.POINTER(ctypes.c_float)),
        ("param", ctypes.POINTER(ctypes.c_float)),
        ("cov", ctypes.POINTER(ctypes.c_float)),
        ("chi2", ctypes.POINTER(ctypes.c_float)),
        ("ndf", ctypes.POINTER(ctypes.c_int32)),
        ("n_fit", ctypes.POINTER(ctypes.c_int32)),
        ("hit_offset", ctypes.POINTER(ctypes.c_int64)),
        ("hit_index", ctypes.POINTER(ctypes.c_uint32)),
        ("n_tracks", ctypes.c_int64),
        ("track_next", ctypes.POINTER(ctypes.c_int32)),
        ("track_merge_chi2", ctypes.POINTER(ctypes.c_float)),
    ]


class tpc_tracks(ctypes.Structure):
    _fields_ = [
        ("n_tracks", ctypes.c_int64),
        ("sector", ctypes.POINTER(ctypes.c_int32)),
        ("x_ref", ctypes.POINTER(ctypes.c_float)),
        ("param", ctypes.POINTER(ctypes.c_float)),
        ("cov", ctypes.POINTER(ctypes.c_float)),
        ("chi2", ctypes.POINTER(ctypes.c_float)),
        ("ndf", ctypes.POINTER(ctypes.c_int32)),
        ("hit_offset", ctypes.POINTER(ctypes.c_int64)),
        ("hit_index", ctypes.POINTER(ctypes.c_uint32)),
        ("beam", ctypes.POINTER(ctypes.c_float)),
        ("residual", ctypes.POINTER(ctypes.c_int32)),
        ("n_pred", ctypes.POINTER(ctypes.c_int32)),
    ]


class tpc_kernel_times(ctypes.Structure):
    _fields_ = [
        ("n_kernels", ctypes.c_int32),
        ("names", ctypes.POINTER(ctypes.c_char_p)),
        ("ms", ctypes.POINTER(ctypes.c_float)),
        ("launches", ctypes.POINTER(ctypes.c_int64)),
    ]


class tpc_tune_entry(ctypes.Structure):
    _fields_ = [
        ("bin_occupancy", ctypes.c_float),
        ("k2_warps", ctypes.c_int32), ("k2_tma", ctypes.c_int32), ("k5_block", ctypes.c_int32),
        ("k5_regs", ctypes.c_int32), ("k5_blocks_per_sm", ctypes.c_int32), ("k5_order", ctypes.c_int32),
        ("sel_lanes", ctypes.c_int32),
        ("ms", ctypes.c_float),
        ("total_ms", ctypes.c_float),
        ("stage", ctypes.c_int32),
        ("k5_ilp", ctypes.c_int32),
    ]


class tpc_tune_report(ctypes.Structure):
    _fields_ = [
        ("n_entries", ctypes.c_int32),
        ("entries", ctypes.POINTER(tpc_tune_entry)),
        ("best", ctypes.c_int32),
    ]


class tpc_cf_params(ctypes.Structure):
    _fields_ = [
        ("pad_pitch", ctypes.c_double),
        ("time_bin_w", ctypes.c_double),
        ("q_peak_min", ctypes.c_int32),
        ("q_total_min", ctypes.c_int32),
    ]


class tpc_digits(ctypes.Structure):
    _fields_ = [
        ("sector", ctypes.c_void_p),
        ("row", ctypes.c_void_p),
        ("pad", ctypes.c_void_p),
        ("time", ctypes.c_void_p),
        ("adc", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("n_time", ctypes.c_int32),
        ("on_device", ctypes.c_int32),
    ]


class tpc_cluster_list(ctypes.Structure):
    _fields_ = [
        ("n_clusters", ctypes.c_int64),
        ("on_device", ctypes.c_int32),
        ("sector", ctypes.c_void_p),
        ("row", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("q_tot", ctypes.c_void_p),
        ("q_max", ctypes.c_void_p),
        ("sigma_pad", ctypes.c_void_p),
        ("sigma_time", ctypes.c_void_p),
        ("digit", ctypes.c_void_p),
    ]


CLUSTER_FIELDS = (("sector", np.uint8), ("row", np.uint8), ("y", np.float32), ("w", np.float32),
                  ("q_tot", np.uint32), ("q_max", np.uint16), ("sigma_pad", np.float32),
                  ("sigma_time", np.float32), ("digit", np.uint32))


def clusters_to_numpy(c: tpc_cluster_list, copy: bool = True) -> dict:
    """numpy arrays of a host cluster list (to_host = 1): copies, or (copy=False) views of the
    context's page-locked block, valid until its next tpc_find_clusters call."""
    if c.on_device:
        raise ValueError("the cluster list holds device pointers")
    n = int(c.n_clusters)
    out = {"n_clusters": n}
    for name, dt in CLUSTER_FIELDS:
        ptr = getattr(c, name)
        if n == 0 or not ptr:
            out[name] = np.zeros(0, dt)
        else:
            buf = (ctypes.c_char * (n * np.dtype(dt).itemsize)).from_address(ptr)
            a = np.frombuffer(buf, dtype=dt)
            out[name] = a.copy() if copy else a
    return out


def cf_default_params(**overrides) -> tpc_cf_params:
    p = tpc_cf_params()
    load().tpc_cf_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


_ctx_p = ctypes.c_void_p
_frame = ctypes.c_uint64

# (name, restype, argtypes) of every entry point declared in include/tpctrack.h
SIGNATURES = [
    ("tpc_default_params", None, [ctypes.POINTER(tpc_params)]),
    ("tpc_create", ctypes.c_int, [ctypes.POINTER(tpc_params), ctypes.POINTER(_ctx_p)]),
    ("tpc_destroy", None, [_ctx_p]),
    ("tpc_last_error", ctypes.c_char_p, [_ctx_p]),
    ("tpc_version", ctypes.c_char_p, []),
    ("tpc_load_clusters", ctypes.c_int, [_ctx_p, ctypes.POINTER(tpc_clusters), ctypes.POINTER(_frame)]),
    ("tpc_track_sectors", ctypes.c_int, [_ctx_p, _frame, ctypes.c_void_p]),
    ("tpc_track_batch", ctypes.c_int, [_ctx_p, ctypes.POINTER(_frame), ctypes.c_int32, ctypes.c_void_p]),
    ("tpc_get_tracks", ctypes.c_int, [_ctx_p, _frame, ctypes.POINTER(tpc_tracks)]),
    ("tpc_get_merged_tracks", ctypes.c_int, [_ctx_p, _frame, ctypes.POINTER(tpc_merged_tracks)]),
    ("tpc_release_frame", ctypes.c_int, [_ctx_p, _frame]),
    ("tpc_submit_frame", ctypes.c_int, [_ctx_p, ctypes.POINTER(tpc_clusters), ctypes.POINTER(_frame)]),
    ("tpc_poll", ctypes.c_int, [_ctx_p, ctypes.POINTER(_frame), ctypes.c_int32, ctypes.c_int32]),
    ("tpc_get_links", ctypes.c_int, [_ctx_p, _frame, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64]),
    ("tpc_get_keep_mask", ctypes.c_int, [_ctx_p, _frame, ctypes.c_void_p, ctypes.c_int64]),
    ("tpc_get_counts", ctypes.c_int, [_ctx_p, _frame, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("tpc_get_stats", ctypes.c_int, [_ctx_p, _frame, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]),
    ("tpc_autotune", ctypes.c_int, [_ctx_p, ctypes.POINTER(_frame), ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(tpc_tune_report)]),
    ("tpc_check_wait_timeout", ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p]),
    ("tpc_set_timing", ctypes.c_int, [_ctx_p, ctypes.c_int32]),
    ("tpc_get_kernel_times", ctypes.c_int, [_ctx_p, ctypes.POINTER(tpc_kernel_times)]),
    ("tpc_cf_default_params", None, [ctypes.POINTER(tpc_cf_params)]),
    ("tpc_find_clusters", ctypes.c_int, [_ctx_p, ctypes.POINTER(tpc_cf_params), ctypes.POINTER(tpc_digits),
                                         ctypes.c_int32, ctypes.POINTER(tpc_cluster_list), ctypes.c_void_p]),
    ("tpc_get_cf_kernel_times", ctypes.c_int, [_ctx_p, ctypes.POINTER(tpc_kernel_times)]),
    ("tpc_links_static", ctypes.c_int, [ctypes.POINTER(tpc_params), ctypes.POINTER(tpc_clusters), ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
]

STATIC_MAX_CLUSTERS = 262144

_lib = None


def load(path: str = LIB_PATH):
    """Load the library (no build, no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libtpctrack.so is not built ({path}); run paper_2009_07515_gb300/build_ext.py")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TpcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, ctx=None) -> int:
    if code < 0:
        msg = load().tpc_last_error(ctx).decode() if ctx else ""
        raise TpcError(code, msg)
    return code


def default_params(**overrides) -> tpc_params:
    p = tpc_params()
    load().tpc_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "cov0":
            for i in range(5):
                p.cov0[i] = float(v[i])
        else:
            setattr(p, k, v)
    return p


def tracks_to_numpy(t: tpc_tracks, copy: bool = True) -> dict:
    """numpy arrays of a tpc_tracks view: copies (default), or views of the library's page-locked
    result block that stay valid until the frame is released."""
    n = int(t.n_tracks)

    def arr(ptr, count, dtype, shape=None):
        if count == 0:
            return np.zeros(shape if shape else (0,), dtype)
        a = np.ctypeslib.as_array(ptr, shape=(count,))
        if copy:
            a = a.copy()
        return a.reshape(shape) if shape else a

    off = arr(t.hit_offset, n + 1, np.int64) if n else np.zeros(1, np.int64)
    return dict(n_tracks=n, sector=arr(t.sector, n, np.int32), x_ref=arr(t.x_ref, n, np.float32),
                param=arr(t.param, 5 * n, np.float32, (n, 5)), cov=arr(t.cov, 15 * n, np.float32, (n, 15)),
                chi2=arr(t.chi2, n, np.float32), ndf=arr(t.ndf, n, np.int32), hit_offset=off,
                hit_index=arr(t.hit_index, int(off[-1]), np.uint32),
                beam=arr(t.beam, 5 * n, np.float32, (n, 5)),
                **({} if not t.residual else
                   dict(residual=arr(t.residual, 2 * int(off[-1]), np.int32, (int(off[-1]), 2)),
                        n_pred=arr(t.n_pred, n, np.int32))))


def merged_to_numpy(t: tpc_merged_tracks, copy: bool = True) -> dict:
    """numpy arrays of a tpc_merged_tracks view (copies, or views valid until the frame is released)."""
    n, nt = int(t.n_merged), int(t.n_tracks)

    def arr(ptr, count, dtype, shape=None):
        if count == 0:
            return np.zeros(shape if shape else (0,), dtype)
        a = np.ctypeslib.as_array(ptr, shape=(count,))
        if copy:
            a = a.copy()
        return a.reshape(shape) if shape else a

    off = arr(t.hit_offset, n + 1, np.int64) if n else np.zeros(1, np.int64)
    return dict(n_merged=n, sector=arr(t.sector, n, np.int32), n_seg=arr(t.n_seg, n, np.int32),
                head=arr(t.head, n, np.int32), x_ref=arr(t.x_ref, n, np.float32),
                param=arr(t.param, 5 * n, np.float32, (n, 5)), cov=arr(t.cov, 15 * n, np.float32, (n, 15)),
                chi2=arr(t.chi2, n, np.float32), ndf=arr(t.ndf, n, np.int32), n_fit=arr(t.n_fit, n, np.int32),
                hit_offset=off, hit_index=arr(t.hit_index, int(off[-1]), np.uint32),
                track_next=arr(t.track_next, nt, np.int32), track_merge_chi2=arr(t.track_merge_chi2, nt, np.float32))
