"""Shared test helpers: efficiency against generator truth and canonical track comparison."""
from __future__ import annotations

import numpy as np


def segments(frame):
    """Truth segments: (track, sector) -> number of clusters."""
    tt = frame.truth_track.astype(np.int64)
    key = np.where(tt >= 0, tt * 36 + frame.sector.astype(np.int64), -1)
    keys, counts = np.unique(key[key >= 0], return_counts=True)
    return key, dict(zip(keys.tolist(), counts.tolist()))


def efficiency(frame, tracks_hits, *, pt_min=0.2, min_clusters=30):
    """Efficiency definitions used throughout the tests.

    A truth segment is a (primary, sector) pair with >= min_clusters clusters. A reconstructed track
    is matched to the segment that holds > 90% of its clusters; a segment is found if a matched
    track holds >= 50% of the segment's clusters. Returns (efficiency, n_segments, clones, fakes).
    """
    key, segs = segments(frame)
    found, clones, fakes = set(), 0, 0
    for h in tracks_hits:
        h = np.asarray(h)
        if len(h) == 0:
            continue
        vals, cnt = np.unique(key[h], return_counts=True)
        j = int(np.argmax(cnt))
        if vals[j] >= 0 and cnt[j] > 0.9 * len(h):
            if cnt[j] >= 0.5 * segs[int(vals[j])]:
                if int(vals[j]) in found:
                    clones += 1
                found.add(int(vals[j]))
        else:
            fakes += 1
    pt = frame.tracks["pt"]
    good = [k for k, c in segs.items() if c >= min_clusters and pt[k // 36] > pt_min]
    eff = float(np.mean([k in found for k in good])) if good else 1.0
    return eff, len(good), clones, fakes


def oracle_track_list(res):
    return [res.track_hits(i) for i in range(res.n_tracks)]


def track_sets(gpu, orc):
    """(sector, hit tuple) -> index, for the GPU tracks and the oracle's tracks."""
    g = {}
    for i in range(gpu["n_tracks"]):
        h = gpu["hit_index"][gpu["hit_offset"][i]:gpu["hit_offset"][i + 1]]
        g[(int(gpu["sector"][i]), tuple(h.tolist()))] = i
    o = {}
    for i in range(orc.n_tracks):
        o[(int(orc.tr_sector[i]), tuple(orc.track_hits(i).tolist()))] = i
    return g, o


def trace_margins(orc, tracks):
    """For each disagreeing track (a hit tuple), the smallest relative margin of a decision near it in
    the oracle's run: the neighbour decisions of its hits and every decision of each oracle tracklet
    that holds one of its hits (a tracklet whose outcome changed takes or leaves hits of the tracks
    it overlaps, so the deciding comparison may sit in an overlapping tracklet)."""
    if not tracks:
        return []
    want = np.unique(np.concatenate([np.asarray(h, np.int64) for h in tracks]))
    tl_of = np.repeat(np.arange(len(orc.tl_start)), np.diff(orc.tl_hit_off))
    sel = np.isin(orc.tl_hits, want)
    by_hit = {}
    for h, t in zip(orc.tl_hits[sel].tolist(), tl_of[sel].tolist()):
        by_hit.setdefault(h, set()).add(t)
    out = []
    for hits in tracks:
        tls = set()
        for h in hits:
            tls |= by_hit.get(h, set())
        m = [float(orc.nb_margin[h]) for h in hits] + [float(orc.tl_margin[t]) for t in tls]
        out.append(min(m) if m else float("inf"))
    return out


def compare_tracks(gpu, orc, *, frac=0.999, margin=1e-5, report=None, fit="same_form"):
    """Check the parity bar and return the matched (gpu, oracle) index pairs, in canonical order.

    Integer results identical on at least `frac` of the tracks; every disagreeing track (on either
    side) traced to a decision within `margin` relative of its cut (trace_margins); the tracks both
    sides find in the same canonical order. Fits of the tracks both find: with fit="same_form" (an
    oracle evaluating the kernels' sequence of FP32 operations) parameters within 1e-4 relative,
    covariances within 1e-3, beam-line results likewise (NaN where the transport fails on both);
    with fit="sigma" (an oracle in another arithmetic form) the parameter differences in units of
    the oracle fit's sigma have median < 0.01 and 99th percentile < 0.2, as for the FP64 oracle, and
    beam-line failures (NaN) differ on at most 0.1% of the tracks. `report`, a dict, receives the
    counts, the largest traced margin and, with fit="sigma", the pull quantiles."""
    g, o = track_sets(gpu, orc)
    common = sorted(set(g) & set(o), key=lambda k: o[k])
    n = max(len(g), len(o), 1)
    assert len(common) >= frac * n, f"{len(common)} identical of {len(g)} GPU / {len(o)} oracle tracks"
    only = [k for k in set(o) ^ set(g)]
    margins = trace_margins(orc, [k[1] for k in only])
    for k, m in zip(only, margins):
        side = "oracle" if k in o else "GPU"
        assert m < margin, f"untraced disagreement: {side}-only track of {len(k[1])} hits, nearest margin {m:.3g}"
    gi = np.array([g[k] for k in common], dtype=np.int64)
    oi = np.array([o[k] for k in common], dtype=np.int64)
    assert np.all(np.diff(gi) > 0), "the tracks both sides find come in a different order"
    if report is not None:
        report.update(n_gpu=len(g), n_oracle=len(o), n_common=len(common), n_disagree=len(only),
                      identical_frac=len(common) / n, max_traced_margin=max(margins) if margins else None)
    if len(common) and fit == "sigma":
        assert np.array_equal(gpu["ndf"][gi], orc.tr_ndf[oi])
        np.testing.assert_allclose(gpu["x_ref"][gi], orc.tr_xref[oi], rtol=1e-6)
        sig = np.sqrt(orc.tr_cov[oi][:, [0, 2, 5, 9, 14]])
        pull = np.abs(gpu["param"][gi] - orc.tr_param[oi]) / sig
        assert np.all(np.median(pull, axis=0) < 0.01) and np.all(np.quantile(pull, 0.99, axis=0) < 0.2)
        gb, ob = gpu["beam"][gi].astype(np.float64), orc.tr_beam[oi]
        nan_diff = int(np.sum(np.isnan(gb[:, 0]) != np.isnan(ob[:, 0])))
        assert nan_diff <= 1e-3 * len(gi)
        if report is not None:
            report.update(pull_median=np.median(pull, axis=0).tolist(), pull_q99=np.quantile(pull, 0.99, axis=0).tolist(),
                          pull_max=pull.max(axis=0).tolist(), beam_nan_differ=nan_diff)
    elif len(common):
        assert np.array_equal(gpu["ndf"][gi], orc.tr_ndf[oi])
        np.testing.assert_allclose(gpu["x_ref"][gi], orc.tr_xref[oi], rtol=1e-6)
        np.testing.assert_allclose(gpu["param"][gi], orc.tr_param[oi], rtol=1e-4, atol=1e-6)
        np.testing.assert_allclose(gpu["cov"][gi], orc.tr_cov[oi], rtol=1e-3, atol=1e-9)
        np.testing.assert_allclose(gpu["chi2"][gi], orc.tr_chi2[oi], rtol=1e-3, atol=1e-5)
        # beam line (y0, w0, var(w0), t0, z_ref): same transport of the same fit, NaN where it fails
        gb, ob = gpu["beam"][gi].astype(np.float64), orc.tr_beam[oi]
        assert np.array_equal(np.isnan(gb), np.isnan(ob))
        for c, (rtol, atol) in enumerate(((1e-4, 1e-4), (1e-4, 1e-4), (1e-3, 1e-9), (1e-4, 1e-4), (1e-4, 1e-4))):
            np.testing.assert_allclose(gb[:, c], ob[:, c], rtol=rtol, atol=atol, equal_nan=True)
    return gi, oi
