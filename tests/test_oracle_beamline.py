"""Pins of the oracle's beam-line step (Sec. 6: track seeds are extrapolated to the beam line and the
most likely z is computed for a primary from a vertex at the origin).

The step transports each track's fit from x_ref to the plane x = 0 without material and reads
(y0, w0, var(w0)); for a primary from z = 0 it gives the collision time t0 = (w0 - L) / v_d and the
track's z at x_ref. These tests check it against a closed form (zero field: straight lines), against
the generator's exact construction (every primary starts at the origin at its collision time, and
its clusters have w = v_d t_c + L - |z|), and statistically (pulls of t0 against its variance).
"""
import math

import numpy as np
import pytest

import oracle
import synth

L_DRIFT = 250.0
V_DRIFT = 250.0 / 90.0


def _full(cov15):
    C = np.zeros((5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            C[i, j] = C[j, i] = cov15[k]
            k += 1
    return C


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_straight_line_closed_form(prec, tol):
    """B = 0: y0 = y - x tan(phi), w0 = w - t x / cos(phi), var(w0) = J C J^T with J = dw0/dstate."""
    p = oracle.default_params(prec, bz=0.0)
    rng = np.random.default_rng(3)
    for _ in range(50):
        x = float(rng.uniform(85.0, 245.0))
        s, t = float(rng.uniform(-0.8, 0.8)), float(rng.uniform(-1.2, 1.2))
        P = np.array([rng.uniform(-20, 20), rng.uniform(10, 500), s, t, 0.0])
        A = rng.normal(size=(5, 5)) * 0.05
        C = A @ A.T + np.eye(5) * 1e-3
        sector = int(rng.integers(0, 36))
        out = oracle.beamline(P, C, x, sector, precision=prec, params=p)
        c = math.sqrt(1.0 - s * s)
        y0 = P[0] - x * s / c
        w0 = P[1] - t * x / c
        # w0 = w - t x (1 - s^2)^(-1/2): dw0/dw = 1, dw0/ds = -t x s / c^3, dw0/dt = -x / c
        J = np.array([0.0, 1.0, -t * x * s / c**3, -x / c, 0.0])
        var = J @ C @ J
        z = (w0 - P[1]) * (1.0 if sector < 18 else -1.0)
        want = np.array([y0, w0, var, (w0 - L_DRIFT) / V_DRIFT, z])
        scale = np.maximum(np.abs(want), [1.0, 1.0, 1e-3, 1.0, 1.0])
        assert np.all(np.abs(out - want) <= tol * scale * 50), (out, want)


def _primaries(seed):
    """Noise-free primaries at random collision times (exact double coordinates of the generator)."""
    return synth.generate("pp_500", truth=True, sigma_y=0.0, sigma_w=0.0, dropout=0.0, noise_frac=0.0,
                          x0_total=0.0, t_zero=0, frame_us=90.0, n_collisions=3, mult_fixed=200, seed=seed)


@pytest.mark.parametrize("seed", [31, 32])
def test_noise_free_primaries_give_collision_time_and_z(seed):
    """Each primary starts at the origin at its collision time: y0 = 0, t0 = t_c, and z at x_ref
    equals the generator's |z| = L - (w - v_d t_c) with the side's sign."""
    f = _primaries(seed)
    p = oracle.default_params("f64", x0_per_row=0.0)
    ts = f.truth_state
    res = oracle.track(f.sector, f.row, ts[:, 0], ts[:, 1], precision="f64", params=p)
    tt = f.truth_track
    checked = 0
    for i in range(res.n_tracks):
        hl = res.tracklet_hits(res.tr_tracklet[i])
        if len(np.unique(tt[hl])) != 1:
            continue
        trk = int(tt[hl[0]])
        tc = f.tracks["tc"][trk]
        y0, w0, var, t0, z = res.tr_beam[i]
        assert abs(y0) < 1e-7, y0
        assert abs(t0 - tc) < 1e-8, (t0, tc)
        ref = hl[0]
        side = 1.0 if f.sector[ref] < 18 else -1.0
        z_true = side * (L_DRIFT - (ts[ref, 1] - V_DRIFT * tc))
        assert abs(z - z_true) < 1e-7, (z, z_true)
        assert var > 0
        checked += 1
    assert checked >= 0.9 * res.n_tracks and checked > 100
    assert len(np.unique(f.tracks["tc"])) == 3


@pytest.mark.parametrize("prec,tol_us", [("f64", 5e-3), ("f32", 2e-2)])
def test_float_clusters_within_resolution(prec, tol_us):
    """The same primaries from the float32 cluster coordinates: t0 within a tiny fraction of the
    0.1 cm / v_d = 0.036 us that one cluster's resolution corresponds to."""
    f = _primaries(33)
    p = oracle.default_params(prec, x0_per_row=0.0)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision=prec, params=p)
    tt = f.truth_track
    errs = []
    for i in range(res.n_tracks):
        hl = res.tracklet_hits(res.tr_tracklet[i])
        if len(np.unique(tt[hl])) != 1:
            continue
        errs.append(res.tr_beam[i, 3] - f.tracks["tc"][int(tt[hl[0]])])
    errs = np.array(errs)
    assert len(errs) > 100
    assert np.all(np.abs(errs) < tol_us), np.abs(errs).max()


def test_t0_pulls_are_standard_normal():
    """Smeared clusters with scattering: (t0 - t_c) / sigma(t0), sigma(t0) = sqrt(var(w0)) / v_d, has
    mean ~0 and the spread of a unit normal (median |pull| 0.674)."""
    f = synth.generate("pbpb_2x10000", truth=True, mult_fixed=600, seed=34)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision="f64", n_threads=8)
    tt = f.truth_track
    pulls = []
    for i in range(res.n_tracks):
        h = res.track_hits(i)
        t = tt[h]
        if len(h) < 20 or np.mean(t == t[0]) < 1.0 or t[0] < 0:
            continue
        y0, w0, var, t0, z = res.tr_beam[i]
        if not np.isfinite(t0):
            continue
        pulls.append((t0 - f.tracks["tc"][int(t[0])]) / (math.sqrt(var) / V_DRIFT))
    pulls = np.array(pulls)
    assert len(pulls) > 500
    assert abs(pulls.mean()) < 0.1, pulls.mean()
    med = float(np.median(np.abs(pulls)))
    assert 0.6 < med < 0.85, med


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_transport_failure_gives_nan(prec):
    """A track that turns back before x = 0 (|sin phi| would pass max_sin) has no beam-line point."""
    # d(sin phi)/dx = kq q/pT = -0.0015 * 5 per cm: over dx = -120 cm sin(phi) would reach 0.95 + 0.9
    P = np.array([10.0, 100.0, 0.95, -0.5, 5.0])
    out = oracle.beamline(P, np.eye(5) * 0.01, 120.0, 3, precision=prec)
    assert np.all(np.isnan(out))
    P[4] = 0.001
    out = oracle.beamline(P, np.eye(5) * 0.01, 120.0, 3, precision=prec)
    assert np.all(np.isfinite(out))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_unit_entry_matches_tracker_output(prec):
    f = synth.generate("pp_500", seed=35)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision=prec)
    assert res.n_tracks > 100
    for i in range(0, res.n_tracks, 7):
        out = oracle.beamline(res.tr_param[i], _full(res.tr_cov[i]), res.tr_xref[i], int(res.tr_sector[i]),
                              precision=prec)
        assert np.array_equal(out, res.tr_beam[i], equal_nan=True), (i, out, res.tr_beam[i])
