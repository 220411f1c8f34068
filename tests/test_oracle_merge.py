"""Pins of the oracle's step 9: merging of sector tracks across sector boundaries and the global refit.

Each pin checks the step against something outside it: the geometry of a rotation in global
coordinates, finite differences, generator truth of noise-free helices that cross a sector
boundary, an independent least-squares helix fit of the merged hits in global coordinates (scipy),
invariance under the order of the tracks, the brute-force candidate search, and the generator's
track labels.
"""
import math

import numpy as np
import pytest

import oracle
import synth

KQ = -0.0029979246 * 0.5
ALPHA = lambda s: ((s % 18) + 0.5) * math.pi / 9.0  # noqa: E731  sector frame angle


def _global(P, x, s):
    """Global (X, Y) and direction angle of a local state at x in sector s's frame."""
    a = ALPHA(s)
    X = x * math.cos(a) - P[0] * math.sin(a)
    Y = x * math.sin(a) + P[0] * math.cos(a)
    d = a + math.asin(P[2])
    return X, Y, math.cos(d), math.sin(d)


def _rand_state(rng):
    A = rng.normal(size=(5, 5))
    C = A @ A.T * 0.01 + 0.01 * np.eye(5)
    return np.array([rng.uniform(10, 18), rng.uniform(50, 400), rng.uniform(0.1, 0.5), rng.uniform(-1, 1),
                     rng.choice([-1, 1]) / rng.uniform(0.2, 3)]), C


def test_rotation_keeps_the_point_and_the_direction():
    rng = np.random.default_rng(1)
    for _ in range(200):
        P, C = _rand_state(rng)
        x = rng.uniform(85, 245)
        s = int(rng.integers(0, 36))
        sb = (s // 18) * 18 + (s % 18 + 1) % 18
        rc, P1, C1, x1 = oracle.rotate(P, C, x, s, sb)
        assert rc == 0
        g0, g1 = _global(P, x, s), _global(P1, x1, sb)
        assert np.allclose(g0, g1, rtol=0, atol=1e-10), (g0, g1)
        assert P1[1] == P[1] and P1[3] == P[3] and P1[4] == P[4]


def test_rotation_round_trip_is_the_identity():
    rng = np.random.default_rng(2)
    for _ in range(100):
        P, C = _rand_state(rng)
        x = rng.uniform(85, 245)
        rc, P1, C1, x1 = oracle.rotate(P, C, x, 4, 5)
        rc2, P2, C2, x2 = oracle.rotate(P1, C1, x1, 5, 4)
        assert rc == 0 and rc2 == 0
        assert abs(x2 - x) < 1e-11 and np.allclose(P2, P, rtol=1e-12, atol=1e-12)
        assert np.allclose(C2, C, rtol=1e-10, atol=1e-12)


def test_rotation_jacobian_matches_finite_differences():
    """The covariance is carried by the derivative of (rotate, then propagate to a fixed x in the new
    frame) with respect to the state at fixed x: compared with central differences of the exact map."""
    rng = np.random.default_rng(3)
    p = oracle.default_params("f64", x0_per_row=0.0)
    for _ in range(40):
        P, _ = _rand_state(rng)
        x = rng.uniform(100, 230)
        _, P1, _, x1 = oracle.rotate(P, np.eye(5), x, 7, 8, params=p)
        xt = x1 + 4.0

        def f(Q):
            rc, Qr, _, xr = oracle.rotate(Q, np.eye(5), x, 7, 8, params=p)
            assert rc == 0
            rc, Qp, _, _ = oracle.propagate(Qr, np.eye(5), xr, xt, params=p)
            assert rc == 0
            return Qp

        # analytic: C' = J C J^T with C = e_i e_j^T recovers J; use a full propagation of unit C
        Jn = np.zeros((5, 5))
        for j in range(5):
            h = 1e-6 * max(1.0, abs(P[j]))
            a, b = P.copy(), P.copy()
            a[j] += h
            b[j] -= h
            Jn[:, j] = (f(a) - f(b)) / (2 * h)
        _, Pr, Cr, xr = oracle.rotate(P, np.eye(5), x, 7, 8, params=p)
        # J_rot from the rotated unit covariance is not unique (J J^T); build it column by column
        Jr = np.zeros((5, 5))
        for j in range(5):
            E = np.zeros((5, 5))
            E[j, j] = 1.0
            _, _, Cj, _ = oracle.rotate(P, E, x, 7, 8, params=p)
            Jr[:, j] = Cj[:, j] / math.sqrt(Cj[j, j]) if Cj[j, j] > 0 else 0.0
            # sign: the diagonal element of J_rot is positive for y and sin(phi), 1 for the rest
        _, _, _, Jp = oracle.propagate(Pr, np.eye(5), xr, xt, params=p)
        Ja = Jp @ Jr
        assert np.allclose(Ja, Jn, rtol=2e-5, atol=2e-6), (Ja - Jn)


def _noise_free(seed):
    return synth.generate("pp_500", truth=True, sigma_y=0.0, sigma_w=0.0, dropout=0.0, noise_frac=0.0,
                          x0_total=0.0, seed=seed)


def _truth_of(tt, hits):
    v, c = np.unique(tt[hits], return_counts=True)
    j = int(np.argmax(c))
    return int(v[j]) if c[j] == len(hits) else -1


@pytest.mark.parametrize("seed", [11, 12])
def test_noise_free_boundary_crossing_helices_merge_to_truth(seed):
    """Noise-free helices from the origin: every track whose clusters fall in two or more sectors
    with at least 15 in each (a sector track keeps at least 10) is one merged track holding exactly
    its clusters, and the refit equals the generator's truth at its innermost cluster to 1e-9 (FP64)."""
    f = _noise_free(seed)
    ts = f.truth_state
    p = oracle.default_params("f64", x0_per_row=0.0)
    res = oracle.track(f.sector, f.row, ts[:, 0], ts[:, 1], precision="f64", params=p, merge=True)
    M = res.merged
    tt = f.truth_track
    want = {}
    for t in np.unique(tt[tt >= 0]):
        secs, cnt = np.unique(f.sector[tt == t], return_counts=True)
        if len(secs) >= 2 and np.all(cnt >= 15):
            want[int(t)] = int(np.sum(tt == t))
    assert len(want) > 100
    got, exact = 0, 0
    for i in range(M.n):
        h = M.track_hits(i)
        t = _truth_of(tt, h)
        if t not in want or M.nseg[i] < 2:
            continue
        got += 1
        if len(h) != want[t]:
            continue
        exact += 1
        inner = h[0]   # the inner segment's hits come first, in ascending row
        assert M.sector[i] == f.sector[inner]
        assert math.isclose(M.xref[i], oracle.row_x(int(f.row[inner])), rel_tol=1e-15)
        d = np.abs(M.param[i] - ts[inner]) / np.maximum(1e-3, np.abs(ts[inner]))
        assert d.max() < 1e-9, (i, d)
        assert M.ndf[i] == 2 * len(h) - 5
    assert got >= 0.95 * len(want) and exact >= 0.95 * got


def _helix_residuals(q, hits, f, x_in, s_in):
    """Residuals of hits (sector frames, row planes) against a helix given at the innermost hit:
    q = (y0, w0, sin phi0, t, q/pT) at x_in in sector s_in's frame; hits in order of arc length."""
    y0, w0, sp, t, qpt = q
    k = KQ * qpt
    a = ALPHA(s_in)
    X0, Y0 = x_in * math.cos(a) - y0 * math.sin(a), x_in * math.sin(a) + y0 * math.cos(a)
    F0 = a + math.asin(max(-0.999999, min(0.999999, sp)))

    def pos(s):
        if abs(k) < 1e-12:
            return X0 + s * math.cos(F0), Y0 + s * math.sin(F0)
        return X0 + (math.sin(F0 + k * s) - math.sin(F0)) / k, Y0 - (math.cos(F0 + k * s) - math.cos(F0)) / k

    out = []
    s_prev = 0.0
    for c in hits:
        ah = ALPHA(int(f.sector[c]))
        xh = oracle.row_x(int(f.row[c]))
        g = lambda s: pos(s)[0] * math.cos(ah) + pos(s)[1] * math.sin(ah) - xh  # noqa: E731
        lo = s_prev - 1.0
        hi = lo + 0.5
        for _ in range(2000):   # a bracket within 1000 cm of arc (a trial helix may never get there)
            if g(hi) >= 0:
                break
            hi += 0.5
        else:
            out += [1e3, 1e3]
            continue
        for _ in range(80):  # bisection: the local x grows along the outgoing leg
            mid = 0.5 * (lo + hi)
            if g(mid) < 0:
                lo = mid
            else:
                hi = mid
        s = 0.5 * (lo + hi)
        s_prev = s
        X, Y = pos(s)
        yl = -X * math.sin(ah) + Y * math.cos(ah)
        out += [(f.y[c] - yl) / 0.1, (f.w[c] - (w0 + t * s)) / 0.1]
    return np.array(out)


def test_refit_of_merged_hits_equals_a_least_squares_helix_fit():
    """Smeared clusters without scattering: the Kalman refit of a merged track (rotated between the
    sector frames) equals a least-squares fit of one helix to all its hits in global coordinates,
    within 5% of the fit's sigma, and its chi2 is the least-squares minimum (the passes start from
    the previous pass's covariance scaled by 100, a prior worth 1% of the hits)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    f = synth.generate("pp_500", truth=True, noise_frac=0.0, dropout=0.0, x0_total=0.0, seed=31)
    p = oracle.default_params("f64", x0_per_row=0.0)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision="f64", params=p, merge=True)
    M = res.merged
    tt = f.truth_track
    checked = 0
    for i in np.flatnonzero(M.nseg >= 2):
        h = M.track_hits(i)
        if _truth_of(tt, h) < 0 or M.nfit[i] != len(h):
            continue
        inner = h[0]
        x_in = oracle.row_x(int(f.row[inner]))
        assert math.isclose(M.xref[i], x_in, rel_tol=1e-12)
        fit = scipy_opt.least_squares(_helix_residuals, M.param[i] * (1 + 1e-3), args=(h, f, x_in, int(f.sector[inner])),
                                      xtol=1e-14, ftol=1e-14, gtol=1e-14)
        cov = M.cov[i]
        sig = np.sqrt([cov[0], cov[2], cov[5], cov[9], cov[14]])
        pull = np.abs(fit.x - M.param[i]) / sig
        assert pull.max() < 0.05, (i, pull)
        r_kf = _helix_residuals(M.param[i], h, f, x_in, int(f.sector[inner]))
        assert r_kf @ r_kf - fit.fun @ fit.fun < 0.05   # the refit's chi2 is the optimum's
        checked += 1
        if checked == 25:
            break
    assert checked == 25


def _tracks_of(res):
    rref = res.tl_row_ref[res.tr_tracklet]
    return (res.tr_sector, rref, res.tr_param, res.tr_cov, res.tr_hit_off, res.tr_hits)


def test_merging_is_invariant_to_the_order_of_the_tracks_and_equals_brute_force():
    f = synth.generate("pbpb_2x10000", mult_fixed=3000)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", n_threads=8)
    sec, rref, par, cov, off, hits = _tracks_of(res)
    y, w = f.y.astype(np.float64), f.w.astype(np.float64)
    a = oracle.merge(f.row, y, w, sec, rref, par, cov, off, hits)
    b = oracle.merge(f.row, y, w, sec, rref, par, cov, off, hits, brute_force=True)
    for k in ("head", "nseg", "sector", "ndf", "xref", "param", "cov", "chi2", "hit_off", "hits", "tr_next"):
        assert np.array_equal(getattr(a, k), getattr(b, k), equal_nan=True), k
    assert np.sum(a.nseg >= 2) > 500
    # the tracks given in another order (sectors reversed, tracks shuffled within)
    rng = np.random.default_rng(4)
    perm = np.lexsort((rng.random(len(sec)), -sec))
    hl = [hits[off[i]:off[i + 1]] for i in perm]
    off2 = np.concatenate([[0], np.cumsum([len(x) for x in hl])])
    c = oracle.merge(f.row, y, w, sec[perm], rref[perm], par[perm], cov[perm], off2, np.concatenate(hl))
    key_a = {tuple(a.track_hits(i)): i for i in range(a.n)}
    key_c = {tuple(c.track_hits(i)): i for i in range(c.n)}
    assert set(key_a) == set(key_c)
    for k, i in key_a.items():
        j = key_c[k]
        assert np.array_equal(a.param[i], c.param[j], equal_nan=True) and np.array_equal(a.cov[i], c.cov[j], equal_nan=True)
        assert a.nseg[i] == c.nseg[j] and a.chi2[i] == c.chi2[j] or (np.isnan(a.chi2[i]) and np.isnan(c.chi2[j]))


def test_merges_join_segments_of_one_generated_track(n_threads):
    """On the Pb-Pb-like frame: more than 99.5% of the merges join two segments of one generated
    track, and more than 95% of the pairs of segments of one track in neighbouring sectors (as found
    by the sector tracking) are merged."""
    f = synth.generate("pbpb_2x10000")
    res = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", merge=True, n_threads=n_threads)
    M = res.merged
    tt = f.truth_track

    def maj(h):
        v, c = np.unique(tt[h], return_counts=True)
        j = int(np.argmax(c))
        return int(v[j]) if c[j] > 0.9 * len(h) else -1

    seg = np.array([maj(res.track_hits(i)) for i in range(res.n_tracks)])
    linked = np.flatnonzero(M.tr_next >= 0)
    good = (seg[linked] >= 0) & (seg[linked] == seg[M.tr_next[linked]])
    assert len(linked) > 5000 and good.mean() > 0.995
    first_row = np.array([f.row[res.track_hits(i)[0]] for i in range(res.n_tracks)])
    should = found = 0
    for t in np.unique(seg[seg >= 0]):
        idx = sorted(np.flatnonzero(seg == t), key=lambda i: first_row[i])
        for a, b in zip(idx[:-1], idx[1:]):
            sa, sb = res.tr_sector[a], res.tr_sector[b]
            if sa // 18 == sb // 18 and (sa % 18 - sb % 18) % 18 in (1, 17):
                should += 1
                found += M.tr_next[a] == b
    assert should > 5000 and found > 0.95 * should
    # every merged track's hits: its segments' hits, inner segment first, each in ascending row
    for i in np.flatnonzero(M.nseg >= 2)[:500]:
        segs = [M.head[i]]
        while M.tr_next[segs[-1]] >= 0:
            segs.append(M.tr_next[segs[-1]])
        assert len(segs) == M.nseg[i]
        assert np.array_equal(M.track_hits(i), np.concatenate([res.track_hits(s) for s in segs]))
