"""Input generator checks: determinism, detector geometry, exact helix geometry, workload sizes."""
import math

import numpy as np

import synth


def test_deterministic_and_thread_independent():
    a = synth.generate("pp_500", truth=True)
    b = synth.generate("pp_500", truth=True, n_threads=1)
    for k in ("sector", "row", "y", "w", "truth_track"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    c = synth.generate("pp_500", frame_id=1)
    assert c.n != a.n or not np.array_equal(c.y, a.y)


def test_detector_geometry():
    f = synth.generate("pbpb_2x10000", truth=True, mult_fixed=1000)
    assert f.sector.max() < 36 and f.row.max() < 152
    x = 85.0 + f.row * (160.0 / 151.0)
    sig = f.truth_track >= 0
    assert np.all(np.abs(f.truth_state[sig, 0]) <= x[sig] * math.tan(math.radians(10)) + 1e-9)
    # one cluster per (track, row): the first outgoing leg crosses each row once
    key = f.truth_track[sig].astype(np.int64) * 152 + f.row[sig]
    assert len(np.unique(key)) == len(key)
    # drift side follows the sign of eta
    side = f.sector[sig] // 18
    eta = f.tracks["eta"][f.truth_track[sig]]
    assert np.all(side == (eta < 0))


def test_clusters_on_exact_helix():
    f = synth.generate("pp_500", truth=True, sigma_y=0.0, sigma_w=0.0, x0_total=0.0, noise_frac=0.0)
    kappa = 0.0029979246 * 0.5
    for t in range(0, 500, 7):
        sel = np.where(f.truth_track == t)[0]
        if len(sel) < 3:
            continue
        q, pt, phi0, eta = f.tracks["q"][t], f.tracks["pt"][t], f.tracks["phi0"][t], f.tracks["eta"][t]
        k = -kappa * q / pt
        cx, cy = -math.sin(phi0) / k, math.cos(phi0) / k
        alpha = (f.sector[sel] % 18 + 0.5) * math.pi / 9
        x = 85.0 + f.row[sel] * (160.0 / 151.0)
        yl = f.truth_state[sel, 0]
        gx = x * np.cos(alpha) - yl * np.sin(alpha)
        gy = x * np.sin(alpha) + yl * np.cos(alpha)
        assert np.allclose(np.hypot(gx - cx, gy - cy), 1 / abs(k), rtol=0, atol=1e-8)
        # drift coordinate: w = 250 - |z|, z = sinh(eta) * arc length from the origin
        chord = np.hypot(gx, gy)
        arc = 2 * np.arcsin(np.clip(chord * abs(k) / 2, 0, 1)) / abs(k)
        assert np.allclose(f.truth_state[sel, 1], 250 - np.abs(math.sinh(eta)) * arc, atol=1e-8)
        assert np.allclose(f.truth_state[sel, 3], -abs(math.sinh(eta)))
        assert np.allclose(f.truth_state[sel, 4], q / pt)


def test_workload_sizes():
    f = synth.generate("pbpb_2x10000")
    assert 2.7e6 < f.n < 3.3e6
    g = synth.generate("pp_500")
    assert 6e4 < g.n < 9e4
    b = [synth.generate("batch16", frame_id=i).n for i in range(4)]
    assert len(set(b)) == 4           # uneven frame sizes
