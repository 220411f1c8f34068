"""Pins of the oracle's compression inputs (Sec. 4: hits of good tracks are stored as residuals to
the extrapolated track position; strategy B removes every hit not in the vicinity of a good track).

Each track's fit is transported (state only, no scattering) from x_ref directly to every row it
spans, one exact helix step per row; a hit is stored as q(hit) - q(prediction), q(v) = rint(512 v);
a good track (|q/pT| <= 20) protects the clusters within +-(1 cm, 1 cm) of its prediction at every
row it spans. These tests check the residuals
against exact tracks, the entropy claim, the keep mask against brute force over all clusters, and
the decoding of the residuals.
"""
import numpy as np
import pytest

import oracle
import synth

Q = 512.0


def _entropy_bits(v):
    _, c = np.unique(v, return_counts=True)
    p = c / c.sum()
    return float(-(p * np.log2(p)).sum())


def _noise_free(seed):
    return synth.generate("pp_500", truth=True, sigma_y=0.0, sigma_w=0.0, dropout=0.0, noise_frac=0.0,
                          x0_total=0.0, seed=seed)


def test_exact_tracks_have_zero_residuals():
    """Exact helix clusters, no scattering: every prediction is the cluster itself (FP64, the
    generator's exact coordinates), so the residuals vanish up to the quantum's rounding."""
    f = _noise_free(41)
    p = oracle.default_params("f64", x0_per_row=0.0)
    ts = f.truth_state
    res = oracle.track(f.sector, f.row, ts[:, 0], ts[:, 1], precision="f64", params=p)
    assert res.n_tracks > 300
    assert np.array_equal(res.tr_npred, np.diff(res.tr_hit_off))
    r = res.tr_res
    assert np.all(np.abs(r) <= 1)
    assert np.mean(r == 0) > 0.99


def test_residuals_have_lower_entropy_than_positions():
    """The paper's claim: residuals to the extrapolated track carry fewer bits than the absolute
    positions of the same hits, in both coordinates (smeared clusters with scattering)."""
    f = synth.generate("pbpb_2x10000", mult_fixed=1500, seed=42)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", n_threads=8)
    npred = res.tr_npred
    pred = np.concatenate([np.arange(o, o + k) for o, k in zip(res.tr_hit_off[:-1], npred)])
    hits = res.tr_hits[pred]
    for c, coord in ((0, f.y), (1, f.w)):
        h_abs = _entropy_bits(np.rint(coord[hits].astype(np.float64) * Q).astype(np.int64))
        h_res = _entropy_bits(res.tr_res[pred, c])
        assert h_res < h_abs - 3.0, (c, h_res, h_abs)


def _full(cov15):
    C = np.zeros((5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            C[i, j] = C[j, i] = cov15[k]
            k += 1
    return C


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_keep_mask_and_decoding_match_brute_force(prec):
    """On a small frame: predictions by one transport from x_ref to each row (the unit entry point),
    every cluster tested against every good track's window at its rows (brute force over the
    whole frame), and the residuals decoded back to the hits' quantized positions."""
    f = synth.generate("pp_500", mult_fixed=60, seed=43)
    p = oracle.default_params(prec)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision=prec, params=p)
    assert res.n_tracks > 30
    rows_x = np.array([oracle.row_x(r, precision=prec) for r in range(152)])
    y = f.y.astype(np.float64)
    w = f.w.astype(np.float64)
    if prec == "f32":
        y, w = f.y, f.w
    keep = np.zeros(f.n, np.uint8)
    p_noms = oracle.default_params(prec, x0_per_row=0.0)
    for i in range(res.n_tracks):
        hits = res.track_hits(i)
        hrows = f.row[hits].astype(int)
        r0 = int(round((res.tr_xref[i] - 85.0) / (160.0 / 151.0)))
        assert abs(rows_x[r0] - res.tr_xref[i]) < 1e-9
        P0 = res.tr_param[i].copy()
        good = abs(P0[4]) <= 20.0
        ok, n = True, 0
        for r in range(r0, hrows[-1] + 1):
            P = P0
            if ok and r > r0:
                rc, P, _, _ = oracle.propagate(P0, np.eye(5), rows_x[r0], rows_x[r], precision=prec, params=p_noms)
                ok = rc == 0
            if ok and good:
                m = (f.sector == res.tr_sector[i]) & (f.row == r)
                near = m & (np.abs(w - P[1]) <= 1.0) & (np.abs(y - P[0]) <= 1.0)
                keep[near] = 1
            if n < len(hits) and hrows[n] == r:
                h = hits[n]
                if good:
                    keep[h] = 1
                q = np.rint(np.array([y[h], w[h]], dtype=np.float64) * Q).astype(np.int64)
                if ok:
                    qp = np.rint(np.array([P[0], P[1]]) * Q).astype(np.int64)
                    assert np.array_equal(qp + res.tr_res[res.tr_hit_off[i] + n], q)
                else:
                    assert np.array_equal(res.tr_res[res.tr_hit_off[i] + n], q)
                n += 1
        assert n == len(hits)
    assert np.array_equal(keep, res.keep)


def test_strategy_b_keeps_good_tracks_and_drops_noise():
    f = synth.generate("pp_500", truth=True, seed=44)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision="f32")
    good = np.abs(res.tr_param[:, 4]) <= 20.0
    for i in np.flatnonzero(good):
        assert np.all(res.keep[res.track_hits(i)] == 1)
    noise = f.truth_track < 0
    assert noise.sum() > 1000
    assert res.keep[noise].mean() < 0.2
    assert res.keep[~noise].mean() > 0.9
