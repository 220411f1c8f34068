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
