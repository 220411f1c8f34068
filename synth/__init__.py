"""Seeded synthetic TPC time frames (input generator shared by the oracle tests and the CUDA path).

This package holds no tracker arithmetic. It wraps ``tpcsynth.c`` (compiled on first use with gcc)
and names the workloads of this project:

* ``pp_500``        — one pp-like event, 500 primaries, t = 0, no scattering (small parity case);
* ``pbpb_2x10000``  — two central-like collisions of 10000 primaries each at random drift times,
                      3% X0 scattering, about 3 M clusters;
* ``batch16``       — frame ``f`` (0..15) of the batched workload: Poisson(5) collisions with
                      exponential multiplicity (mean 2500, capped at 12000);
* ``full_570``      — full-size synchronous frame: 570 collisions over 128 orbits (11.44 ms),
                      exponential multiplicity, about 1.7e8 clusters;
* ``slice_80``      — an 18-orbit slice of the synchronous frame (80 collisions, about 2.5e7 clusters);
* ``serve``         — a serving-stream frame with ``n_collisions`` given by the caller.

``digitize`` turns a frame's clusters into the zero-suppressed pad x time-bin digits a cluster finder
starts from (``DIGIT_DEFAULTS``: 0.4 cm pads, 0.2 us time bins, 0.3 cm charge spread, log-normal
cluster charge, 2-ADC threshold, 10-bit saturation).

Common laws (Sec. 2 and 7.1 of the paper describe the continuous-readout frames these stand in for):
pT log-uniform in [0.1, 10] GeV, |eta| < 0.9, phi uniform, q = +-1, Bz = 0.5 T, sigma_y = sigma_w =
0.1 cm, 2% row-crossing inefficiency, 5% uniform noise clusters per (sector, row).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpcsynth.c")
_LIB = os.path.join(_HERE, "libtpcsynth.so")
_lock = threading.Lock()
_lib = None

ORBIT_US = 89.4
VDRIFT_CM_PER_US = 250.0 / 90.0


class SynthParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("frame_id", ctypes.c_uint64),
        ("n_collisions", ctypes.c_int32),
        ("poisson_mean", ctypes.c_double),
        ("mult_fixed", ctypes.c_int32),
        ("mult_mean", ctypes.c_double),
        ("mult_cap", ctypes.c_int32),
        ("pt_min", ctypes.c_double),
        ("pt_max", ctypes.c_double),
        ("eta_max", ctypes.c_double),
        ("bz", ctypes.c_double),
        ("sigma_y", ctypes.c_double),
        ("sigma_w", ctypes.c_double),
        ("dropout", ctypes.c_double),
        ("noise_frac", ctypes.c_double),
        ("x0_total", ctypes.c_double),
        ("frame_us", ctypes.c_double),
        ("tail_us", ctypes.c_double),
        ("t_zero", ctypes.c_int32),
        ("shuffle", ctypes.c_int32),
        ("want_truth", ctypes.c_int32),
        ("n_threads", ctypes.c_int32),
    ]


class _Frame(ctypes.Structure):
    _fields_ = [
        ("n_clusters", ctypes.c_int64),
        ("n_tracks", ctypes.c_int64),
        ("n_collisions", ctypes.c_int64),
        ("sector", ctypes.POINTER(ctypes.c_uint8)),
        ("row", ctypes.POINTER(ctypes.c_uint8)),
        ("y", ctypes.POINTER(ctypes.c_float)),
        ("w", ctypes.POINTER(ctypes.c_float)),
        ("truth_track", ctypes.POINTER(ctypes.c_int32)),
        ("truth_state", ctypes.POINTER(ctypes.c_double)),
        ("trk_coll", ctypes.POINTER(ctypes.c_int32)),
        ("trk_q", ctypes.POINTER(ctypes.c_int8)),
        ("trk_pt", ctypes.POINTER(ctypes.c_double)),
        ("trk_eta", ctypes.POINTER(ctypes.c_double)),
        ("trk_phi0", ctypes.POINTER(ctypes.c_double)),
        ("trk_tc", ctypes.POINTER(ctypes.c_double)),
        ("trk_ncl", ctypes.POINTER(ctypes.c_int32)),
        ("coll_tc", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile ``tpcsynth.c`` into ``libtpcsynth.so`` beside it (gcc, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.synth_generate.argtypes = [ctypes.POINTER(SynthParams), ctypes.POINTER(ctypes.POINTER(_Frame))]
        lib.synth_generate.restype = ctypes.c_int
        lib.synth_free.argtypes = [ctypes.POINTER(_Frame)]
        lib.synth_free.restype = None
        lib.synth_digitize.argtypes = [ctypes.POINTER(SynthDigitParams), ctypes.c_int64] + [ctypes.c_void_p] * 4 + \
            [ctypes.POINTER(ctypes.POINTER(_Digits))]
        lib.synth_digitize.restype = ctypes.c_int
        lib.synth_free_digits.argtypes = [ctypes.POINTER(_Digits)]
        lib.synth_free_digits.restype = None
        lib.synth_npads.argtypes = [ctypes.c_double, ctypes.c_int]
        lib.synth_npads.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Frame:
    """One time frame of clusters in caller order (SoA), plus generator truth."""
    sector: np.ndarray          # uint8 [n]: 0..35 (0..17 side A, 18..35 side C)
    row: np.ndarray             # uint8 [n]: 0..151
    y: np.ndarray               # float32 [n]: local y along the pad row, cm
    w: np.ndarray               # float32 [n]: drift coordinate v_d * t_arrival, cm
    truth_track: np.ndarray     # int32 [n]: generating track, -1 for noise
    truth_state: np.ndarray | None  # float64 [n,5]: (y, w, sin phi, dw/ds, q/pT) before smearing
    tracks: dict = field(default_factory=dict)  # per-track arrays (coll, q, pt, eta, phi0, tc, ncl)
    coll_tc: np.ndarray | None = None
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.y.shape[0])


BASE = dict(seed=1, frame_id=0, n_collisions=1, poisson_mean=0.0, mult_fixed=500, mult_mean=2500.0,
            mult_cap=12000, pt_min=0.1, pt_max=10.0, eta_max=0.9, bz=0.5, sigma_y=0.1, sigma_w=0.1,
            dropout=0.02, noise_frac=0.05, x0_total=0.0, frame_us=90.0, tail_us=90.0, t_zero=1, shuffle=1,
            want_truth=0, n_threads=0)

CONFIGS = {
    # one pp-like event of 500 primaries at t = 0 (small parity case)
    "pp_500": dict(seed=1, n_collisions=1, mult_fixed=500, t_zero=1, frame_us=90.0, x0_total=0.0),
    # two central-like collisions of 10000 primaries, each at a random drift time, 3% X0 scattering
    "pbpb_2x10000": dict(seed=2, n_collisions=2, mult_fixed=10000, t_zero=0, frame_us=90.0,
                         x0_total=0.03),
    # one frame of the batched workload: Poisson(5) collisions within 100 us, exponential multiplicity
    "batch16": dict(seed=3, n_collisions=-1, poisson_mean=5.0, mult_fixed=0, t_zero=0,
                    frame_us=100.0, x0_total=0.03),
    # full-size synchronous frame: 570 collisions over 128 orbits; the frame ends with the last orbit,
    # so tracks of collisions in its last 90 us are cut (Sec. 2); clusters in generation order
    "full_570": dict(seed=4, n_collisions=570, mult_fixed=0, t_zero=0, frame_us=128 * ORBIT_US,
                     tail_us=0.0, x0_total=0.03, shuffle=0),
    # an 18-orbit slice of the synchronous frame: 80 collisions over 18 orbits (1.6 ms), cut like it
    "slice_80": dict(seed=4, n_collisions=80, mult_fixed=0, t_zero=0, frame_us=18 * ORBIT_US,
                     tail_us=0.0, x0_total=0.03, shuffle=0),
    # serving stream frame: n_collisions set by the caller, 20 us per collision at 50 kHz
    "serve": dict(seed=5, n_collisions=1, mult_fixed=0, t_zero=0, frame_us=20.0, x0_total=0.03),
}


DIGIT_DEFAULTS = dict(seed=11, pad_pitch=0.4, time_bin_w=VDRIFT_CM_PER_US * 0.2, sigma_pad=0.3, sigma_time=0.3,
                      q_median=60.0, q_log_sigma=0.4, adc_threshold=2, adc_max=1023, shuffle=0, n_threads=0)


class SynthDigitParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("pad_pitch", ctypes.c_double), ("time_bin_w", ctypes.c_double),
        ("sigma_pad", ctypes.c_double), ("sigma_time", ctypes.c_double),
        ("q_median", ctypes.c_double), ("q_log_sigma", ctypes.c_double),
        ("adc_threshold", ctypes.c_int32), ("adc_max", ctypes.c_int32),
        ("shuffle", ctypes.c_int32), ("n_threads", ctypes.c_int32),
    ]


class _Digits(ctypes.Structure):
    _fields_ = [
        ("n_digits", ctypes.c_int64),
        ("n_time", ctypes.c_int32),
        ("sector", ctypes.POINTER(ctypes.c_uint8)),
        ("row", ctypes.POINTER(ctypes.c_uint8)),
        ("pad", ctypes.POINTER(ctypes.c_uint16)),
        ("time", ctypes.POINTER(ctypes.c_uint16)),
        ("adc", ctypes.POINTER(ctypes.c_uint16)),
        ("truth_cluster", ctypes.POINTER(ctypes.c_int32)),
    ]


@dataclass
class Digits:
    """Zero-suppressed digits of one frame (SoA, caller order) and the generator's truth."""
    sector: np.ndarray          # uint8 [n]
    row: np.ndarray             # uint8 [n]
    pad: np.ndarray             # uint16 [n]: 0 .. n_pads(row) - 1
    time: np.ndarray            # uint16 [n]: time bin, 0 .. n_time - 1
    adc: np.ndarray             # uint16 [n]: charge, >= adc_threshold
    truth_cluster: np.ndarray   # int32 [n]: cluster with the largest deposit in the cell
    n_time: int
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.adc.shape[0])


def n_pads(row: int, pad_pitch: float = DIGIT_DEFAULTS["pad_pitch"]) -> int:
    """Pads of a row: 2 ceil(x_r tan(10 deg) / pitch) (the generator's geometry)."""
    return int(_load().synth_npads(ctypes.c_double(pad_pitch), int(row)))


def digitize(frame: Frame, **overrides) -> Digits:
    """Digits of a frame's clusters (each cluster spreads its charge over pads x time bins)."""
    p = dict(DIGIT_DEFAULTS)
    p.update(overrides)
    lib = _load()
    sp = SynthDigitParams(**{k: p[k] for k, _ in SynthDigitParams._fields_})
    dp = ctypes.POINTER(_Digits)()
    c = [np.ascontiguousarray(a) for a in (frame.sector, frame.row, frame.y, frame.w)]
    rc = lib.synth_digitize(ctypes.byref(sp), frame.n, *(a.ctypes.data for a in c), ctypes.byref(dp))
    if rc != 0:
        raise RuntimeError(f"synth_digitize failed ({rc})")
    try:
        d = dp.contents
        n = int(d.n_digits)

        def arr(ptr, dtype):
            if n == 0:
                return np.zeros(0, dtype)
            return np.ctypeslib.as_array(ptr, shape=(n,)).view(dtype).copy()

        return Digits(sector=arr(d.sector, np.uint8), row=arr(d.row, np.uint8), pad=arr(d.pad, np.uint16),
                      time=arr(d.time, np.uint16), adc=arr(d.adc, np.uint16),
                      truth_cluster=arr(d.truth_cluster, np.int32), n_time=int(d.n_time), params=p)
    finally:
        lib.synth_free_digits(dp)


def generate_digits(config: str | None = None, *, digit_overrides: dict | None = None, **overrides):
    """(frame, digits) of a named workload: the frame's clusters digitized with ``DIGIT_DEFAULTS``."""
    f = generate(config, **overrides)
    return f, digitize(f, **(digit_overrides or {}))


def params_for(config: str | None = None, **overrides) -> dict:
    p = dict(BASE)
    if config is not None:
        p.update(CONFIGS[config])
    p.update(overrides)
    if config == "serve" and "frame_us" not in overrides:
        p["frame_us"] = 20.0 * max(1, int(p["n_collisions"]))
    return p


def generate(config: str | None = None, *, truth: bool = False, **overrides) -> Frame:
    """Generate one frame. ``config`` names a workload above; keyword overrides change any parameter."""
    p = params_for(config, **overrides)
    p["want_truth"] = 1 if truth else 0
    lib = _load()
    sp = SynthParams(**{k: p[k] for k, _ in SynthParams._fields_})
    fp = ctypes.POINTER(_Frame)()
    rc = lib.synth_generate(ctypes.byref(sp), ctypes.byref(fp))
    if rc != 0:
        raise RuntimeError(f"synth_generate failed ({rc})")
    try:
        f = fp.contents
        n, nt, nc = int(f.n_clusters), int(f.n_tracks), int(f.n_collisions)

        def arr(ptr, count, dtype, shape=None):
            if count == 0:
                return np.zeros(shape or (0,), dtype=dtype)
            a = np.ctypeslib.as_array(ptr, shape=(count,)).view(dtype).copy()
            return a.reshape(shape) if shape else a

        frame = Frame(
            sector=arr(f.sector, n, np.uint8), row=arr(f.row, n, np.uint8),
            y=arr(f.y, n, np.float32), w=arr(f.w, n, np.float32),
            truth_track=arr(f.truth_track, n, np.int32),
            truth_state=(arr(f.truth_state, 5 * n, np.float64, (n, 5)) if truth else None),
            tracks=dict(coll=arr(f.trk_coll, nt, np.int32), q=arr(f.trk_q, nt, np.int8),
                        pt=arr(f.trk_pt, nt, np.float64), eta=arr(f.trk_eta, nt, np.float64),
                        phi0=arr(f.trk_phi0, nt, np.float64), tc=arr(f.trk_tc, nt, np.float64),
                        ncl=arr(f.trk_ncl, nt, np.int32)),
            coll_tc=arr(f.coll_tc, nc, np.float64), params=p)
    finally:
        lib.synth_free(fp)
    return frame
