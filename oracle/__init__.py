"""CPU oracle for TPC sector tracking — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this
package. The product path (``paper_2009_07515_gb300``) never imports it and shares no code with it.

``tpc_oracle.c`` (sector tracking) and ``cf_oracle.c`` (cluster finding from digits) are compiled
three times with gcc (``-ffp-contract=off``, no fast-math): REAL = double (``precision="f64"``), REAL =
float with the kernels' arithmetic form (``precision="f32"``: explicit fused multiply-adds,
reciprocals formed once) and REAL = float in plain form (``precision="f32plain"``: no fused
multiply-add, true divisions). The step-by-step definition of what each computes is in its header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpc_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "cf_oracle.c")]
_lock = threading.Lock()
_libs: dict = {}

BRUTE_FORCE = 1
PACKED = 2
MERGE = 4


PRECISIONS = ("f32", "f64", "f32plain")


def _lib_path(precision: str) -> str:
    return os.path.join(_HERE, f"libtpcoracle_{precision}.so")


def build(force: bool = False) -> None:
    """Compile every precision beside the source (a checker build; nothing on the product path):
    ``f64``, ``f32`` (the kernels' arithmetic form: fused multiply-adds, reciprocals formed once) and
    ``f32plain`` (plain FP32: every product and sum rounded, true divisions)."""
    with _lock:
        for prec in PRECISIONS:
            out = _lib_path(prec)
            if (not force and os.path.exists(out)
                    and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in _SRCS)):
                continue
            tmp = out + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                   "-fPIC", "-shared"] + _SRCS + ["-o", tmp, "-lm"]
            if prec in ("f32", "f32plain"):
                cmd.insert(1, "-DORACLE_F32")
            if prec == "f32plain":
                cmd.insert(1, "-DORACLE_PLAIN")
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)


class Params(ctypes.Structure):
    _fields_ = [
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
        ("keep_vy", ctypes.c_double), ("keep_vw", ctypes.c_double),
        ("keep_qpt_max", ctypes.c_double),
        ("merge_gap_rows", ctypes.c_int32),
        ("merge_dw", ctypes.c_double),
        ("merge_chi2_max", ctypes.c_double),
        ("refit_passes", ctypes.c_int32),
        ("refit_scale", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "cov0"}
        d["cov0"] = list(self.cov0)
        return d


_P = ctypes.POINTER
_i32p, _i64p, _f64p = _P(ctypes.c_int32), _P(ctypes.c_int64), _P(ctypes.c_double)


class _Merge(ctypes.Structure):
    _fields_ = [
        ("n_tracks", ctypes.c_int64), ("n_merged", ctypes.c_int64),
        ("mt_head", _i32p), ("mt_nseg", _i32p), ("mt_sector", _i32p), ("mt_ndf", _i32p), ("mt_nfit", _i32p),
        ("mt_xref", _f64p), ("mt_param", _f64p), ("mt_cov", _f64p), ("mt_chi2", _f64p),
        ("mt_hit_off", _i64p), ("mt_hits", _i32p),
        ("tr_next", _i32p), ("tr_merge_chi2", _f64p), ("tr_outer", _f64p),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("n_clusters", ctypes.c_int64),
        ("up", _i32p), ("down", _i32p), ("up_c", _i32p), ("down_c", _i32p),
        ("nb_margin", _f64p),
        ("n_start", ctypes.c_int64), ("start", _i32p),
        ("n_tracklets", ctypes.c_int64),
        ("tl_sector", _i32p), ("tl_start", _i32p), ("tl_nhits", _i32p), ("tl_ndf", _i32p),
        ("tl_row_ref", _i32p), ("tl_row_top", _i32p), ("tl_ok", _i32p),
        ("tl_xref", _f64p), ("tl_param", _f64p), ("tl_cov", _f64p), ("tl_chi2", _f64p),
        ("tl_margin", _f64p),
        ("tl_hit_off", _i64p), ("tl_hits", _i32p),
        ("n_tracks", ctypes.c_int64),
        ("tr_sector", _i32p), ("tr_ndf", _i32p), ("tr_nhits", _i32p), ("tr_tracklet", _i32p),
        ("tr_xref", _f64p), ("tr_param", _f64p), ("tr_cov", _f64p), ("tr_chi2", _f64p),
        ("tr_beam", _f64p),
        ("tr_res", _i32p), ("tr_npred", _i32p), ("keep", _P(ctypes.c_uint8)),
        ("tr_hit_off", _i64p), ("tr_hits", _i32p),
        ("merged", _P(_Merge)),
    ]


class CFParams(ctypes.Structure):
    _fields_ = [
        ("pad_pitch", ctypes.c_double), ("time_bin_w", ctypes.c_double),
        ("q_peak_min", ctypes.c_int32), ("q_total_min", ctypes.c_int32),
    ]


class _CFResult(ctypes.Structure):
    _fields_ = [
        ("n_clusters", ctypes.c_int64),
        ("sector", _i32p), ("row", _i32p), ("pad", _i32p), ("time", _i32p), ("digit", _i64p),
        ("q_tot", _i64p), ("q_max", _i32p),
        ("y", _f64p), ("w", _f64p), ("sigma_pad", _f64p), ("sigma_time", _f64p),
    ]


def _load(precision: str):
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {PRECISIONS}")
    if precision in _libs:
        return _libs[precision]
    build()
    lib = ctypes.CDLL(_lib_path(precision))
    pre = f"oracle_{precision}_"
    f = getattr(lib, pre + "default_params"); f.argtypes = [_P(Params)]; f.restype = None
    f = getattr(lib, pre + "track")
    f.argtypes = [_P(Params), ctypes.c_int64, _P(ctypes.c_uint8), _P(ctypes.c_uint8), _f64p, _f64p,
                  ctypes.c_int, ctypes.c_int, _P(_P(_Result))]
    f.restype = ctypes.c_int
    f = getattr(lib, pre + "free_result"); f.argtypes = [_P(_Result)]; f.restype = None
    f = getattr(lib, pre + "propagate")
    f.argtypes = [_P(Params), _f64p, _f64p, ctypes.c_double, ctypes.c_double, _f64p]
    f.restype = ctypes.c_int
    f = getattr(lib, pre + "update"); f.argtypes = [_P(Params), _f64p, _f64p, ctypes.c_double, ctypes.c_double]
    f.restype = ctypes.c_double
    f = getattr(lib, pre + "seed"); f.argtypes = [_P(Params), _f64p, _f64p]; f.restype = ctypes.c_int
    f = getattr(lib, pre + "asin"); f.argtypes = [ctypes.c_double]; f.restype = ctypes.c_double
    f = getattr(lib, pre + "pack"); f.argtypes = [_f64p, _f64p]; f.restype = None
    f = getattr(lib, pre + "row_x"); f.argtypes = [ctypes.c_int]; f.restype = ctypes.c_double
    f = getattr(lib, pre + "beamline")
    f.argtypes = [_P(Params), _f64p, _f64p, ctypes.c_double, ctypes.c_int, _f64p]
    f.restype = None
    f = getattr(lib, pre + "merge")
    f.argtypes = [_P(Params), ctypes.c_int64, _P(ctypes.c_uint8), _f64p, _f64p, ctypes.c_int64, _i32p, _i32p,
                  _f64p, _f64p, _i64p, _i32p, ctypes.c_int, _P(_P(_Merge))]
    f.restype = ctypes.c_int
    f = getattr(lib, pre + "free_merge"); f.argtypes = [_P(_Merge)]; f.restype = None
    f = getattr(lib, pre + "rotate")
    f.argtypes = [_P(Params), _f64p, _f64p, _f64p, ctypes.c_int, ctypes.c_int]
    f.restype = ctypes.c_int
    f = getattr(lib, pre + "select")
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _i32p, _i32p,
                  _P(ctypes.c_uint64)]
    f.restype = ctypes.c_int
    f = getattr(lib, pre + "cf_default_params"); f.argtypes = [_P(CFParams)]; f.restype = None
    f = getattr(lib, pre + "n_pads"); f.argtypes = [ctypes.c_double, ctypes.c_int]; f.restype = ctypes.c_int
    f = getattr(lib, pre + "find_clusters")
    f.argtypes = [_P(CFParams), ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.c_int32, ctypes.c_int,
                                                                           _P(_P(_CFResult))]
    f.restype = ctypes.c_int
    f = getattr(lib, pre + "free_cf_result"); f.argtypes = [_P(_CFResult)]; f.restype = None
    _libs[precision] = lib
    return lib


def default_params(precision: str = "f64", **overrides) -> Params:
    p = Params()
    getattr(_load(precision), f"oracle_{precision}_default_params")(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "cov0":
            for i in range(5):
                p.cov0[i] = float(v[i])
        else:
            setattr(p, k, v)
    return p


@dataclass
class Result:
    """Oracle output. Link arrays are in caller index space; tracks are in canonical order
    (sector, smallest original cluster index); hit lists are in ascending row order."""
    up: np.ndarray
    down: np.ndarray
    up_c: np.ndarray
    down_c: np.ndarray
    nb_margin: np.ndarray
    start: np.ndarray
    tl_sector: np.ndarray
    tl_start: np.ndarray
    tl_nhits: np.ndarray
    tl_ndf: np.ndarray
    tl_row_ref: np.ndarray
    tl_row_top: np.ndarray
    tl_ok: np.ndarray
    tl_xref: np.ndarray
    tl_param: np.ndarray
    tl_cov: np.ndarray
    tl_chi2: np.ndarray
    tl_margin: np.ndarray
    tl_hit_off: np.ndarray
    tl_hits: np.ndarray
    tr_sector: np.ndarray
    tr_ndf: np.ndarray
    tr_nhits: np.ndarray
    tr_tracklet: np.ndarray
    tr_xref: np.ndarray
    tr_param: np.ndarray
    tr_cov: np.ndarray
    tr_chi2: np.ndarray
    tr_beam: np.ndarray     # [n_tracks, 5]: y0, w0, var(w0), t0 (us), z_ref (NaN: no transport)
    tr_res: np.ndarray      # [track hits, 2] int32: q(hit) - q(prediction), or q(hit) past n_pred
    tr_npred: np.ndarray    # [n_tracks] hits stored as residuals
    keep: np.ndarray        # [n_clusters] uint8: 1 = kept by strategy B
    tr_hit_off: np.ndarray
    tr_hits: np.ndarray
    merged: "Merged | None" = None   # step 9 (track(..., merge=True))

    @property
    def n_tracks(self) -> int:
        return int(self.tr_sector.shape[0])

    def track_hits(self, i: int) -> np.ndarray:
        return self.tr_hits[self.tr_hit_off[i]:self.tr_hit_off[i + 1]]

    def tracklet_hits(self, i: int) -> np.ndarray:
        return self.tl_hits[self.tl_hit_off[i]:self.tl_hit_off[i + 1]]


@dataclass
class Merged:
    """Step 9: merged tracks in canonical order (their innermost sector track's index), each a chain
    of sector tracks refit over all its hits; per sector track its outer partner, the merge chi2 and
    the outer state used for matching."""
    head: np.ndarray        # [m] sector-track index of the innermost segment
    nseg: np.ndarray        # [m] segments
    sector: np.ndarray      # [m] frame of the refit result (the innermost segment reached)
    ndf: np.ndarray         # [m] 2 * fitted hits - 5
    nfit: np.ndarray        # [m] hits the refit used
    xref: np.ndarray        # [m] x of the innermost fitted hit
    param: np.ndarray       # [m, 5]
    cov: np.ndarray         # [m, 15]
    chi2: np.ndarray        # [m]
    hit_off: np.ndarray     # [m + 1]
    hits: np.ndarray        # cluster indices: the segments' hits, inner segment first
    tr_next: np.ndarray     # [n_tracks] outer partner or -1
    tr_merge_chi2: np.ndarray
    tr_outer: np.ndarray    # [n_tracks, 5]

    @property
    def n(self) -> int:
        return int(self.head.shape[0])

    def track_hits(self, i: int) -> np.ndarray:
        return self.hits[self.hit_off[i]:self.hit_off[i + 1]]


def _merged(M) -> Merged:
    nt, m = int(M.n_tracks), int(M.n_merged)
    off = _copy(M.mt_hit_off, m + 1, np.int64)
    return Merged(head=_copy(M.mt_head, m, np.int32), nseg=_copy(M.mt_nseg, m, np.int32),
                  sector=_copy(M.mt_sector, m, np.int32), ndf=_copy(M.mt_ndf, m, np.int32),
                  nfit=_copy(M.mt_nfit, m, np.int32), xref=_copy(M.mt_xref, m, np.float64),
                  param=_copy(M.mt_param, 5 * m, np.float64, (m, 5)), cov=_copy(M.mt_cov, 15 * m, np.float64, (m, 15)),
                  chi2=_copy(M.mt_chi2, m, np.float64), hit_off=off, hits=_copy(M.mt_hits, int(off[-1]), np.int32),
                  tr_next=_copy(M.tr_next, nt, np.int32), tr_merge_chi2=_copy(M.tr_merge_chi2, nt, np.float64),
                  tr_outer=_copy(M.tr_outer, 5 * nt, np.float64, (nt, 5)))


def _copy(ptr, n, dtype, shape=None):
    if n == 0:
        return np.zeros(shape if shape else (0,), dtype=dtype)
    a = np.ctypeslib.as_array(ptr, shape=(n,)).copy().astype(dtype, copy=False)
    return a.reshape(shape) if shape else a


def track(sector, row, y, w, *, precision: str = "f32", params: Params | None = None,
          brute_force: bool = False, packed: bool = False, merge: bool = False, n_threads: int = 0) -> Result:
    """Run the oracle tracker on one frame (clusters in caller order); merge=True adds step 9."""
    lib = _load(precision)
    pre = f"oracle_{precision}_"
    if params is None:
        params = default_params(precision)
    sector = np.ascontiguousarray(sector, dtype=np.uint8)
    row = np.ascontiguousarray(row, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n = int(y.shape[0])
    if n_threads <= 0:
        n_threads = 1
    rp = _P(_Result)()
    rc = getattr(lib, pre + "track")(
        ctypes.byref(params), n, sector.ctypes.data_as(_P(ctypes.c_uint8)),
        row.ctypes.data_as(_P(ctypes.c_uint8)), y.ctypes.data_as(_f64p), w.ctypes.data_as(_f64p),
        (BRUTE_FORCE if brute_force else 0) | (PACKED if packed else 0) | (MERGE if merge else 0), int(n_threads),
        ctypes.byref(rp))
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    try:
        R = rp.contents
        nt, ntr = int(R.n_tracklets), int(R.n_tracks)
        tl_off = _copy(R.tl_hit_off, nt + 1, np.int64)
        tr_off = _copy(R.tr_hit_off, ntr + 1, np.int64)
        res = Result(
            up=_copy(R.up, n, np.int32), down=_copy(R.down, n, np.int32),
            up_c=_copy(R.up_c, n, np.int32), down_c=_copy(R.down_c, n, np.int32),
            nb_margin=_copy(R.nb_margin, n, np.float64),
            start=_copy(R.start, int(R.n_start), np.int32),
            tl_sector=_copy(R.tl_sector, nt, np.int32), tl_start=_copy(R.tl_start, nt, np.int32),
            tl_nhits=_copy(R.tl_nhits, nt, np.int32), tl_ndf=_copy(R.tl_ndf, nt, np.int32),
            tl_row_ref=_copy(R.tl_row_ref, nt, np.int32), tl_row_top=_copy(R.tl_row_top, nt, np.int32),
            tl_ok=_copy(R.tl_ok, nt, np.int32), tl_xref=_copy(R.tl_xref, nt, np.float64),
            tl_param=_copy(R.tl_param, 5 * nt, np.float64, (nt, 5)),
            tl_cov=_copy(R.tl_cov, 15 * nt, np.float64, (nt, 15)),
            tl_chi2=_copy(R.tl_chi2, nt, np.float64), tl_margin=_copy(R.tl_margin, nt, np.float64),
            tl_hit_off=tl_off, tl_hits=_copy(R.tl_hits, int(tl_off[-1]), np.int32),
            tr_sector=_copy(R.tr_sector, ntr, np.int32), tr_ndf=_copy(R.tr_ndf, ntr, np.int32),
            tr_nhits=_copy(R.tr_nhits, ntr, np.int32), tr_tracklet=_copy(R.tr_tracklet, ntr, np.int32),
            tr_xref=_copy(R.tr_xref, ntr, np.float64),
            tr_param=_copy(R.tr_param, 5 * ntr, np.float64, (ntr, 5)),
            tr_cov=_copy(R.tr_cov, 15 * ntr, np.float64, (ntr, 15)),
            tr_chi2=_copy(R.tr_chi2, ntr, np.float64),
            tr_beam=_copy(R.tr_beam, 5 * ntr, np.float64, (ntr, 5)),
            tr_res=_copy(R.tr_res, 2 * int(tr_off[-1]), np.int32, (int(tr_off[-1]), 2)),
            tr_npred=_copy(R.tr_npred, ntr, np.int32),
            keep=_copy(R.keep, n, np.uint8),
            tr_hit_off=tr_off, tr_hits=_copy(R.tr_hits, int(tr_off[-1]), np.int32),
            merged=_merged(R.merged.contents) if R.merged else None)
    finally:
        getattr(lib, pre + "free_result")(rp)
    return res


# ---------------------------------------------------------------- unit entry points (pins)

def propagate(P, C, x0, x1, *, precision="f64", params: Params | None = None):
    lib = _load(precision)
    params = params or default_params(precision)
    P = np.array(P, dtype=np.float64).copy()
    C = np.array(C, dtype=np.float64).reshape(5, 5).copy()
    J = np.zeros((5, 5))
    rc = getattr(lib, f"oracle_{precision}_propagate")(ctypes.byref(params), P.ctypes.data_as(_f64p),
                                                       C.ctypes.data_as(_f64p), float(x0), float(x1),
                                                       J.ctypes.data_as(_f64p))
    return rc, P, C, J


def update(P, C, ym, wm, *, precision="f64", params: Params | None = None):
    lib = _load(precision)
    params = params or default_params(precision)
    P = np.array(P, dtype=np.float64).copy()
    C = np.array(C, dtype=np.float64).reshape(5, 5).copy()
    chi2 = getattr(lib, f"oracle_{precision}_update")(ctypes.byref(params), P.ctypes.data_as(_f64p),
                                                      C.ctypes.data_as(_f64p), float(ym), float(wm))
    return chi2, P, C


def seed(h, *, precision="f64", params: Params | None = None):
    """h: 3x3 array of (x, y, w) for the first, middle and last chain hits."""
    lib = _load(precision)
    params = params or default_params(precision)
    h = np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(9))
    P = np.zeros(5)
    rc = getattr(lib, f"oracle_{precision}_seed")(ctypes.byref(params), h.ctypes.data_as(_f64p),
                                                  P.ctypes.data_as(_f64p))
    return rc, P


def asin(t: float, *, precision="f64") -> float:
    return getattr(_load(precision), f"oracle_{precision}_asin")(float(t))


def pack(y: float, w: float, *, precision="f32"):
    """(y, w) read back through the 16-bit cluster storage format."""
    a, b = ctypes.c_double(y), ctypes.c_double(w)
    getattr(_load(precision), f"oracle_{precision}_pack")(ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def beamline(P, C, x_ref: float, sector: int, *, precision="f64", params: Params | None = None) -> np.ndarray:
    """Step 7 for one fit (P, full 5x5 C at x_ref): (y0, w0, var(w0), t0, z_ref), NaN if the
    transport to x = 0 fails."""
    lib = _load(precision)
    params = params or default_params(precision)
    P = np.ascontiguousarray(np.asarray(P, dtype=np.float64).reshape(5))
    C = np.ascontiguousarray(np.asarray(C, dtype=np.float64).reshape(25))
    out = np.zeros(5)
    getattr(lib, f"oracle_{precision}_beamline")(ctypes.byref(params), P.ctypes.data_as(_f64p),
                                                 C.ctypes.data_as(_f64p), float(x_ref), int(sector),
                                                 out.ctypes.data_as(_f64p))
    return out


def merge(row, y, w, sector, row_ref, param, cov, hit_off, hits, *, precision: str = "f32",
          params: Params | None = None, brute_force: bool = False) -> Merged:
    """Step 9 alone on given sector tracks: sector, row of x_ref, fit (param [n, 5], cov [n, 15]) and
    kept hits (hit_off, hits: cluster indices in ascending row) of each; row, y, w of the clusters."""
    lib = _load(precision)
    params = params or default_params(precision)
    row = np.ascontiguousarray(row, dtype=np.uint8)
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    sector = np.ascontiguousarray(sector, dtype=np.int32)
    row_ref = np.ascontiguousarray(row_ref, dtype=np.int32)
    param = np.ascontiguousarray(param, dtype=np.float64).reshape(-1)
    cov = np.ascontiguousarray(cov, dtype=np.float64).reshape(-1)
    hit_off = np.ascontiguousarray(hit_off, dtype=np.int64)
    hits = np.ascontiguousarray(hits, dtype=np.int32)
    mp = _P(_Merge)()
    rc = getattr(lib, f"oracle_{precision}_merge")(
        ctypes.byref(params), int(y.shape[0]), row.ctypes.data_as(_P(ctypes.c_uint8)), y.ctypes.data_as(_f64p),
        w.ctypes.data_as(_f64p), int(sector.shape[0]), sector.ctypes.data_as(_i32p), row_ref.ctypes.data_as(_i32p),
        param.ctypes.data_as(_f64p), cov.ctypes.data_as(_f64p), hit_off.ctypes.data_as(_i64p),
        hits.ctypes.data_as(_i32p), 1 if brute_force else 0, ctypes.byref(mp))
    if rc != 0:
        raise ValueError(f"oracle rejected the tracks (code {rc})")
    try:
        return _merged(mp.contents)
    finally:
        getattr(lib, f"oracle_{precision}_free_merge")(mp)


def rotate(P, C, x: float, sector_from: int, sector_to: int, *, precision="f64", params: Params | None = None):
    """One rotation of a state (P, full 5x5 C at x) from a sector's frame into its phi neighbour's:
    (rc, P', C', x')."""
    lib = _load(precision)
    params = params or default_params(precision)
    P = np.array(P, dtype=np.float64).copy()
    C = np.array(C, dtype=np.float64).reshape(5, 5).copy()
    xx = ctypes.c_double(x)
    rc = getattr(lib, f"oracle_{precision}_rotate")(ctypes.byref(params), P.ctypes.data_as(_f64p),
                                                    C.ctypes.data_as(_f64p), ctypes.byref(xx), int(sector_from),
                                                    int(sector_to))
    return rc, P, C, xx.value


def select(rank, slots, n_hits: int, *, nmin: int = 10, precision: str = "f32"):
    """Step 6 (tracklet selection) alone on caller-given tracklets of one sector: rank[t] the unique
    start-hit rank of tracklet t, slots[t, r] its hit in row r (an index < n_hits) or -1. Returns
    (accepted bool[nt], kept int[nt], weight uint64[n_hits])."""
    lib = _load(precision)
    rank = np.ascontiguousarray(rank, dtype=np.int32)
    slots = np.ascontiguousarray(slots, dtype=np.int32).reshape(-1, 152)
    nt = int(rank.shape[0])
    assert slots.shape[0] == nt
    acc = np.zeros(max(nt, 1), np.int32)
    kept = np.zeros(max(nt, 1), np.int32)
    weight = np.zeros(max(n_hits, 1), np.uint64)
    rc = getattr(lib, f"oracle_{precision}_select")(
        int(nmin), int(n_hits), nt, rank.ctypes.data_as(_i32p), slots.ctypes.data_as(_i32p),
        acc.ctypes.data_as(_i32p), kept.ctypes.data_as(_i32p), weight.ctypes.data_as(_P(ctypes.c_uint64)))
    if rc != 0:
        raise ValueError(f"oracle rejected the tracklets (code {rc})")
    return acc[:nt].astype(bool), kept[:nt], weight[:n_hits]


def row_x(r: int, *, precision="f64") -> float:
    return getattr(_load(precision), f"oracle_{precision}_row_x")(int(r))


# ---------------------------------------------------------------- cluster finding (cf_oracle.c)

def cf_default_params(precision: str = "f64", **overrides) -> CFParams:
    p = CFParams()
    getattr(_load(precision), f"oracle_{precision}_cf_default_params")(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def n_pads(r: int, pad_pitch: float = 0.4) -> int:
    return getattr(_load("f64"), "oracle_f64_n_pads")(float(pad_pitch), int(r))


def find_clusters(sector, row, pad, time, adc, n_time: int, *, precision: str = "f32",
                  params: CFParams | None = None, n_threads: int = 0) -> dict:
    """Clusters of a frame's digits, in the input order of their peak digits (arrays of a dict).
    Raises ValueError when the oracle rejects the input (a cell out of range, a zero charge or two
    digits in one cell)."""
    lib = _load(precision)
    pre = f"oracle_{precision}_"
    params = params or cf_default_params(precision)
    a = [np.ascontiguousarray(x, dtype=dt) for x, dt in
         ((sector, np.uint8), (row, np.uint8), (pad, np.uint16), (time, np.uint16), (adc, np.uint16))]
    n = int(a[0].shape[0])
    rp = _P(_CFResult)()
    rc = getattr(lib, pre + "find_clusters")(ctypes.byref(params), n, *(x.ctypes.data for x in a), int(n_time),
                                             int(n_threads), ctypes.byref(rp))
    if rc != 0:
        raise ValueError(f"oracle rejected the digits (code {rc})")
    try:
        R = rp.contents
        m = int(R.n_clusters)
        out = dict(n_clusters=m, sector=_copy(R.sector, m, np.int32), row=_copy(R.row, m, np.int32),
                   pad=_copy(R.pad, m, np.int32), time=_copy(R.time, m, np.int32),
                   digit=_copy(R.digit, m, np.int64), q_tot=_copy(R.q_tot, m, np.int64),
                   q_max=_copy(R.q_max, m, np.int32), y=_copy(R.y, m, np.float64), w=_copy(R.w, m, np.float64),
                   sigma_pad=_copy(R.sigma_pad, m, np.float64), sigma_time=_copy(R.sigma_time, m, np.float64))
    finally:
        getattr(lib, pre + "free_cf_result")(rp)
    return out
