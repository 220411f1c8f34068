"""Pins of the oracle's control flow: start-hit chain length, the extension stop, the consecutive-miss
stop and the selection rule.

Each case is built by hand so that the method's readings fix the outcome before the oracle runs:
noise-free straight tracks (zero field, no scattering) laid on chosen rows of one sector, and
tracklet sets given directly to the selection step. The expected hit sets, start hits and tracks are
worked out from the readings (start hit: a cleaned chain of at least 6 hits; an outward extension
ends right after it accepts another tracklet's start hit; an extension ends after 5 consecutive rows
without a hit; each hit goes to the voter with the largest (hits, -start rank) key, and a tracklet
with >= 10 hits keeping >= 10 and at least half of them becomes a track). The constants are written
here, not read from the oracle's defaults, so a changed default fails these pins.
"""
import numpy as np
import pytest

import oracle

LMIN = 6        # minimum cleaned-chain length of a start hit
N_MISS = 5      # consecutive rows without a hit that end an extension
NMIN = 10       # minimum hits of a voting tracklet and of a track
NROW = 152


def _line(rows, sector=3, y0=1.5, w0=120.0, dydx=0.08, dwdx=0.35, x_at=100.0):
    """Clusters of a straight track (zero field) on the given rows of one sector."""
    x = np.array([oracle.row_x(r) for r in rows])
    y = y0 + dydx * (x - x_at)
    w = w0 + dwdx * (x - x_at)
    n = len(rows)
    return (np.full(n, sector, np.uint8), np.array(rows, np.uint8), y, w)


def _track(clusters, **over):
    p = oracle.default_params("f64", bz=0.0, x0_per_row=0.0, **over)
    s, r, y, w = clusters
    return oracle.track(s, r, y, w, precision="f64", params=p)


def _rows_of(res, hits, row):
    return sorted(int(row[h]) for h in hits)


def _chain_len(res, h):
    n = 0
    while h >= 0:
        n += 1
        h = res.up_c[h]
    return n


@pytest.mark.parametrize("n_rows,chain,starts", [(7, 5, 0), (8, 6, 1), (9, 7, 1)])
def test_start_hit_needs_a_cleaned_chain_of_lmin_hits(n_rows, chain, starts):
    """A track on n consecutive rows: the first and last clusters have no (down, up) pair, so the
    cleaned chain holds the n - 2 inner clusters and starts at the second. Chains of 5, 6 and 7 hits
    give 0, 1 and 1 start hits."""
    rows = list(range(40, 40 + n_rows))
    cl = _line(rows)
    res = _track(cl)
    second = 1
    assert res.down_c[second] < 0 and res.up_c[second] == 2
    assert _chain_len(res, second) == chain
    assert len(res.start) == starts
    if starts:
        assert res.start[0] == second


def test_start_hits_of_the_pbpb_like_frame_head_chains_of_at_least_lmin():
    import synth
    f = synth.generate("pbpb_2x10000", mult_fixed=1500)
    res = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", n_threads=8)
    assert len(res.start) > 1000
    lens = np.array([_chain_len(res, int(s)) for s in res.start])
    assert lens.min() == LMIN
    for s in res.start:
        assert res.up_c[s] >= 0 and res.down_c[s] < 0
    # every chain head of at least LMIN hits is a start hit
    heads = np.flatnonzero((res.up_c >= 0) & (res.down_c < 0))
    long_heads = [h for h in heads if _chain_len(res, int(h)) >= LMIN]
    assert sorted(long_heads) == sorted(res.start.tolist())


def test_extension_stops_after_accepting_another_start_hit():
    """One straight track on rows 10-40 and 42-100 (row 41 empty): two cleaned chains, rows 11-39
    and 43-99, so two start hits (rows 11 and 43). The lower tracklet follows its chain, extends
    through rows 40 and 42, accepts the start hit at row 43 and stops there; inward it adds row 10:
    33 hits. The upper tracklet runs out to row 100 and inward through every row down to 10: 90 hits.
    It takes every shared hit (more hits), so the upper tracklet is the one track, of 90 hits.
    Without the stop the lower tracklet runs to row 100 too, and wins the tie on hits by its smaller
    start rank."""
    rows = list(range(10, 41)) + list(range(42, 101))
    cl = _line(rows)
    row = cl[1]
    res = _track(cl)
    assert [int(row[s]) for s in res.start] == [11, 43]
    lo, hi = 0, 1
    assert _rows_of(res, res.tracklet_hits(lo), row) == list(range(10, 41)) + [42, 43]
    assert res.tl_row_top[lo] == 43 and res.tl_nhits[lo] == 33
    assert _rows_of(res, res.tracklet_hits(hi), row) == rows
    assert res.tl_row_top[hi] == 100 and res.tl_nhits[hi] == 90
    assert res.n_tracks == 1 and res.tr_tracklet[0] == hi
    assert _rows_of(res, res.track_hits(0), row) == rows
    # the same frame without the stop (ext_stop = 0)
    off = _track(cl, ext_stop=0)
    assert _rows_of(off, off.tracklet_hits(lo), row) == rows and off.tl_row_top[lo] == 100
    assert off.n_tracks == 1 and off.tr_tracklet[0] == lo


def test_extension_continues_through_hits_that_are_not_start_hits():
    """Hits beyond a one-row gap that head no chain of LMIN hits (rows 42-46: chain 43-45 of 3) are
    picked up by the outward extension, which then runs until N_MISS empty rows."""
    rows = list(range(10, 41)) + list(range(42, 47))
    cl = _line(rows)
    res = _track(cl)
    assert len(res.start) == 1
    assert _rows_of(res, res.tracklet_hits(0), cl[1]) == rows
    assert res.tl_row_top[0] == 46


@pytest.mark.parametrize("gap", [N_MISS - 1, N_MISS])
def test_outward_extension_crosses_fewer_than_n_miss_empty_rows(gap):
    """Chain on rows 20-60, then `gap` empty rows, then 5 hits (their cleaned chain of 3 heads no
    tracklet). A gap of N_MISS - 1 rows is crossed and the 5 hits join; a gap of N_MISS ends the
    extension."""
    beyond = list(range(61 + gap, 66 + gap))
    rows = list(range(20, 61)) + beyond
    cl = _line(rows)
    res = _track(cl)
    assert len(res.start) == 1
    got = _rows_of(res, res.tracklet_hits(0), cl[1])
    want = rows if gap < N_MISS else list(range(20, 61))
    assert got == want


@pytest.mark.parametrize("gap", [N_MISS - 1, N_MISS])
def test_inward_extension_crosses_fewer_than_n_miss_empty_rows(gap):
    """5 hits on rows 30-34, then `gap` empty rows, then a chain up to row 80. Inward from its start
    the tracklet crosses a gap of N_MISS - 1 rows and picks up the 5 hits, but not a gap of N_MISS."""
    below = list(range(30, 35))
    upper = list(range(35 + gap, 81))
    cl = _line(below + upper)
    res = _track(cl)
    assert len(res.start) == 1
    got = _rows_of(res, res.tracklet_hits(0), cl[1])
    want = below + upper if gap < N_MISS else upper
    assert got == want


# ------------------------------------------------------------------ selection (tracklets given)

def _slots(tracklets):
    """tracklets: list of hit lists; hit j of a tracklet goes to row j (rows only order the hits)."""
    s = np.full((len(tracklets), NROW), -1, np.int32)
    for t, hits in enumerate(tracklets):
        s[t, :len(hits)] = hits
    return s


def _select(tracklets, ranks, n_hits):
    return oracle.select(np.array(ranks), _slots(tracklets), n_hits, nmin=NMIN)


def test_selection_equal_hits_go_to_the_smaller_start_rank():
    """Two tracklets of 20 hits sharing 12: the one with the smaller start rank keeps all 20; the
    other keeps 8 < 10 and is no track. The order in which they are given does not matter."""
    a = list(range(0, 20))
    b = list(range(8, 28))
    acc, kept, _ = _select([b, a], [9, 5], 28)
    assert acc.tolist() == [False, True] and kept.tolist() == [0, 20]
    acc, kept, _ = _select([a, b], [5, 9], 28)
    assert acc.tolist() == [True, False] and kept.tolist() == [20, 0]


def test_selection_more_hits_win_and_half_is_enough():
    """25 hits (rank 9) against 20 hits (rank 5) sharing 10: the larger keeps its 25; the smaller
    keeps 10, which is both >= 10 and exactly half of its hits, so it is a track."""
    big = list(range(0, 25))
    small = list(range(15, 35))
    acc, kept, w = _select([big, small], [9, 5], 35)
    assert acc.tolist() == [True, True] and kept.tolist() == [25, 10]
    key_big = (25 << 32) | (0xFFFFFFFF - 9)
    assert np.all(w[:25] == key_big)


def test_selection_fewer_than_half_kept_is_no_track():
    """21 hits keeping 10 (less than half) are no track; 15 hits keeping 9 (>= half, < 10) are none
    either."""
    big = list(range(0, 30))
    t21 = list(range(19, 40))            # shares 11 with big, keeps 10 of 21
    t15 = list(range(50, 59)) + list(range(0, 6))   # shares 6 with big, keeps 9 of 15
    acc, kept, _ = _select([big, t21, t15], [20, 1, 2], 60)
    assert acc.tolist() == [True, False, False] and kept.tolist() == [30, 0, 0]


def test_selection_short_tracklets_do_not_vote():
    """A tracklet of 9 hits (fewer than 10) with the largest key holds no hit: the 12-hit tracklet
    sharing 5 of its hits keeps all 12."""
    short = list(range(0, 9))
    t12 = list(range(4, 16))
    acc, kept, w = _select([short, t12], [1, 7], 16)
    assert acc.tolist() == [False, True] and kept.tolist() == [0, 12]
    assert np.all(w[:4] == 0)


@pytest.mark.parametrize("seed", range(40))
def test_selection_equals_brute_force_on_tiny_random_sets(seed):
    """Random tracklets over a few dozen hits: every hit's owner found by comparing all voters that
    hold it, then the acceptance rule, gives the oracle's tracks and kept counts."""
    rng = np.random.default_rng(1000 + seed)
    n_hits = int(rng.integers(12, 60))
    nt = int(rng.integers(1, 12))
    ranks = rng.permutation(200)[:nt]
    tls = [sorted(rng.choice(n_hits, size=int(rng.integers(6, min(n_hits, 30) + 1)), replace=False).tolist())
           for _ in range(nt)]
    acc, kept, w = _select(tls, ranks, n_hits)
    key = [(len(h), -int(r)) for h, r in zip(tls, ranks)]
    owner = {}
    for h in range(n_hits):
        best = None
        for t in range(nt):
            if len(tls[t]) >= NMIN and h in tls[t] and (best is None or key[t] > key[best]):
                best = t
        owner[h] = best
    for t in range(nt):
        k = sum(owner[h] == t for h in tls[t])
        ok = len(tls[t]) >= NMIN and k >= NMIN and 2 * k >= len(tls[t])
        assert bool(acc[t]) == ok, (seed, t)
        assert int(kept[t]) == (k if ok else 0)
    for h in range(n_hits):
        t = owner[h]
        want = 0 if t is None else (len(tls[t]) << 32) | (0xFFFFFFFF - int(ranks[t]))
        assert int(w[h]) == want
