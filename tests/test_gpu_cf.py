"""GPU parity of the cluster finder (tpc_find_clusters) with the FP32 oracle (cf_oracle.c).

Every decision is an integer one (peaks, included cells, sums) and every value a fixed sequence of
IEEE FP32 operations on both sides, so the clusters must agree bit for bit: same count, same order
(input order of the peak digits), same bits in every field. Cases: the small pp frame in readout and
in shuffled order, the Pb-Pb frame of the tracking benchmark, another pad pitch and thresholds,
edge cells, empty input, malformed input (refused, and the next call still correct), a sequence of
frames of different lengths on one context, device-resident digits, and digits -> clusters -> tracks
against the oracle's tracker on the oracle's clusters.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.test_gpu_parity import compare_tracks

pytestmark = pytest.mark.gpu

FIELDS = ("sector", "row", "y", "w", "q_tot", "q_max", "sigma_pad", "sigma_time", "digit")


@pytest.fixture(scope="module")
def tpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_07515_gb300 as t
    t.build()
    return t


@pytest.fixture(scope="module")
def tracker(tpc):
    tr = tpc.Tracker()
    yield tr
    tr.close()


def oracle_cf(d, n_time=None, **kw):
    p = oracle.cf_default_params("f32", **kw)
    return oracle.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time if n_time is None else n_time,
                                precision="f32", params=p, n_threads=8)


def assert_same(gpu, orc):
    assert gpu["n_clusters"] == orc["n_clusters"]
    for k in FIELDS:
        g = gpu[k]
        o = orc[k]
        if g.dtype == np.float32:
            assert np.array_equal(g.view(np.uint32), o.astype(np.float32).view(np.uint32)), k
        else:
            assert np.array_equal(g.astype(np.int64), o.astype(np.int64)), k


@pytest.mark.parametrize("shuffle", [0, 1])
def test_pp_frame_bit_exact(tracker, shuffle):
    f = synth.generate("pp_500")
    d = synth.digitize(f, shuffle=shuffle)
    gpu = tracker.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time)
    orc = oracle_cf(d)
    assert orc["n_clusters"] > 70000
    assert_same(gpu, orc)


def test_pbpb_frame_bit_exact(tracker):
    f, d = synth.generate_digits("pbpb_2x10000")
    gpu = tracker.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time)
    orc = oracle_cf(d)
    assert orc["n_clusters"] > 2_500_000
    assert_same(gpu, orc)


def test_other_pitch_and_thresholds(tpc, tracker):
    f = synth.generate("pp_500", mult_fixed=200, seed=9)
    d = synth.digitize(f, pad_pitch=0.6, time_bin_w=0.5, sigma_pad=0.4)
    cp = tpc.cf_default_params(pad_pitch=0.6, time_bin_w=0.5, q_peak_min=6, q_total_min=25)
    gpu = tracker.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time, cf_params=cp)
    orc = oracle_cf(d, pad_pitch=0.6, time_bin_w=0.5, q_peak_min=6, q_total_min=25)
    assert orc["n_clusters"] > 1000
    assert_same(gpu, orc)


def _cells(cells):
    a = np.array(cells, dtype=np.int64).reshape(-1, 5)
    return [a[:, i] for i in range(5)]


def test_edge_cells_and_small_inputs(tracker):
    n151 = oracle.n_pads(151)
    cells = [(35, 151, 0, 0, 20), (35, 151, 1, 0, 10), (35, 151, n151 - 1, 99, 20), (0, 0, 75, 50, 7),
             (0, 0, 74, 50, 7), (17, 3, 10, 10, 5), (17, 3, 12, 10, 9), (17, 3, 11, 10, 2), (18, 1, 5, 5, 3)]
    cols = _cells(cells)
    gpu = tracker.find_clusters(*cols, 100)
    orc = oracle.find_clusters(*cols, 100, precision="f32")
    assert orc["n_clusters"] >= 3
    assert_same(gpu, orc)
    empty = [np.zeros(0, t) for t in (np.uint8, np.uint8, np.uint16, np.uint16, np.uint16)]
    assert tracker.find_clusters(*empty, 100)["n_clusters"] == 0
    one = _cells([(4, 4, 4, 4, 44)])
    g = tracker.find_clusters(*one, 5)
    assert_same(g, oracle.find_clusters(*one, 5, precision="f32"))


@pytest.mark.parametrize("bad", [(36, 0, 0, 0, 5), (0, 152, 0, 0, 5), (0, 0, 76, 0, 5), (0, 0, 0, 64, 5),
                                 (0, 0, 0, 0, 0), (0, 0, 3, 3, 4)])
def test_malformed_digits_are_refused_and_leave_the_map_clean(tpc, tracker, bad):
    cols = _cells([(0, 0, 3, 3, 9), (0, 0, 4, 3, 30), bad])
    with pytest.raises(tpc.TpcError) as e:
        tracker.find_clusters(*cols, 64)
    assert e.value.code == -1
    ok = _cells([(0, 0, 3, 3, 9), (0, 0, 4, 3, 30)])
    assert_same(tracker.find_clusters(*ok, 64), oracle.find_clusters(*ok, 64, precision="f32"))


def test_frames_of_different_lengths_on_one_context(tracker):
    for seed, frame_us in ((21, 20.0), (22, 90.0), (23, 5.0)):
        f = synth.generate("serve", n_collisions=2, mult_fixed=300, frame_us=frame_us, seed=seed)
        d = synth.digitize(f, shuffle=1, seed=seed)
        assert_same(tracker.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time + 3), oracle_cf(d, d.n_time + 3))


def test_device_digits_and_tracking_of_found_clusters(tpc, tracker):
    import torch
    f, d = synth.generate_digits("pp_500", seed=12)
    dev = torch.device("cuda", 0)
    t = [torch.from_numpy(a.astype(np.int32)).to(dev) for a in (d.sector, d.row, d.pad, d.time, d.adc)]
    t = [t[0].to(torch.uint8), t[1].to(torch.uint8)] + [x.to(torch.uint16) for x in t[2:]]
    gpu = tracker.find_clusters(*t, d.n_time)
    orc = oracle_cf(d)
    assert_same(gpu, orc)
    cl = tracker.find_clusters(*t, d.n_time, to_host=False)
    assert cl.on_device == 1 and cl.n_clusters == orc["n_clusters"]
    h = tracker.load_cluster_list(cl)
    try:
        tracker.track(h)
        res = tracker.tracks(h)
    finally:
        tracker.release(h)
    trk = oracle.track(orc["sector"], orc["row"], orc["y"].astype(np.float32), orc["w"].astype(np.float32),
                       precision="f32")
    assert trk.n_tracks > 300
    gi, oi = compare_tracks(res, trk)
    assert len(gi) == trk.n_tracks == res["n_tracks"]


def test_long_frame(tracker):
    """A frame of several thousand time bins (a long drift window at low occupancy)."""
    f = synth.generate("serve", n_collisions=3, mult_fixed=200, frame_us=900.0, seed=31)
    d = synth.digitize(f, shuffle=1, seed=31)
    assert d.n_time > 4000
    assert_same(tracker.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time), oracle_cf(d))


LINE_BYTES = 36 * 152 * 224 * 2   # one time line of the charge map (widest row 218 pads + guards)


def test_charge_map_beyond_the_budget_is_refused(tpc):
    """Half of the HBM budget must hold the map of a window of at least 16 time bins."""
    f = synth.generate("pp_500", mult_fixed=20, seed=32)
    d = synth.digitize(f)
    tr = tpc.Tracker(hbm_budget=2 * 19 * LINE_BYTES)
    try:
        with pytest.raises(tpc.TpcError) as e:
            tr.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time)
        assert e.value.code == -3
    finally:
        tr.close()


def _windowed(tpc, window_bins):
    """A context whose budget holds the map of a window of window_bins time bins."""
    return tpc.Tracker(hbm_budget=2 * (window_bins + 4) * LINE_BYTES + LINE_BYTES // 2)


def test_long_frame_in_time_windows_equals_one_pass_and_oracle(tpc, tracker):
    """A frame of 4400 time bins processed in five windows of about 1000 bins (the map of the whole
    frame exceeds the budget): the same clusters, in the same order, bit for bit, as one pass over
    the whole frame and as the oracle."""
    f = synth.generate("serve", n_collisions=3, mult_fixed=200, frame_us=900.0, seed=31)
    d = synth.digitize(f, shuffle=1, seed=31)
    assert d.n_time > 4000
    one = tracker.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time)
    tw = _windowed(tpc, 1000)
    try:
        win = tw.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time)
        assert_same(win, oracle_cf(d))
        for k in FIELDS:
            assert np.array_equal(np.asarray(win[k]), np.asarray(one[k])), k
    finally:
        tw.close()


def test_pbpb_digits_in_small_windows_match_oracle(tpc):
    """The Pb-Pb-like frame's 2.3e7 digits in windows of 40 time bins (19 windows, halos crossing
    every window edge)."""
    f, d = synth.generate_digits("pbpb_2x10000")
    tw = _windowed(tpc, 40)
    try:
        assert_same(tw.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time), oracle_cf(d))
    finally:
        tw.close()


def test_full_length_frame_in_windows_at_the_default_budget(tpc):
    """A frame as long as the full-size synchronous frame (128 orbits, about 55,000 time bins) at low
    occupancy (16 collisions, 4.4e7 digits). Its charge map, about 135 GB, exceeds half of the default
    80 GB budget, so the default context clusters it in time windows; the clusters of sectors 0-2
    equal the oracle's on those sectors' digits, bit for bit and in order."""
    f = synth.generate("full_570", n_collisions=16, seed=41)
    d = synth.digitize(f)
    assert d.n_time > 50000 and (d.n_time + 4) * LINE_BYTES > 40 * (1 << 30)
    tr = tpc.Tracker()
    try:
        tr.set_timing(True)
        g = tr.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time)
        nl = tr.cf_kernel_times(launches=True)
        # the windowed passes ran: fill, flag, clear and fill, emit, clear per window, at least 4 windows
        assert nl["cf_peaks"] == 0 and nl["cf_fill"] == nl["cf_copy"] >= 12 and nl["cf_fill"] % 3 == 0
    finally:
        tr.close()
    m = d.sector < 3
    idx = np.flatnonzero(m)
    o = oracle.find_clusters(d.sector[m], d.row[m], d.pad[m], d.time[m], d.adc[m], d.n_time, precision="f32",
                             n_threads=8)
    sel = np.asarray(g["sector"]) < 3
    assert int(sel.sum()) == o["n_clusters"] > 0
    for k in FIELDS:
        gk = np.asarray(g[k])[sel]
        ok = idx[o[k].astype(np.int64)] if k == "digit" else o[k]
        if gk.dtype == np.float32:
            assert np.array_equal(gk.view(np.uint32), ok.astype(np.float32).view(np.uint32)), k
        else:
            assert np.array_equal(gk.astype(np.int64), ok.astype(np.int64)), k


def test_windowed_mode_refuses_malformed_input_and_stays_exact(tpc):
    tw = _windowed(tpc, 20)
    try:
        ok = _cells([(0, 0, 3, 3, 9), (0, 0, 4, 3, 30), (0, 0, 2, 4, 7), (5, 9, 10, 50, 12), (5, 9, 10, 51, 20)])
        for bad in ([(0, 0, 2, 3, 40000), (0, 0, 2, 3, 40000)], [(0, 152, 0, 0, 5)], [(0, 0, 3, 80, 5)]):
            cols = _cells([(0, 0, 6, 3, 20), (4, 4, 4, 40, 30)] + bad)
            with pytest.raises(tpc.TpcError) as e:
                tw.find_clusters(*cols, 64)
            assert e.value.code == -1
            assert_same(tw.find_clusters(*ok, 64), oracle.find_clusters(*ok, 64, precision="f32"))
    finally:
        tw.close()


def test_tracks_from_found_clusters_match_tracks_from_generated_clusters(tracker):
    """Physics check of the whole chain on the Pb-Pb frame: the tracks of the found clusters are as
    many as the tracks of the generator's clusters (within 3%), and nearly every track found from
    the digits has its peaks from one generated track."""
    f, d = synth.generate_digits("pbpb_2x10000", truth=True)
    c = tracker.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time)
    t_dig = tracker.run(c["sector"], c["row"], c["y"], c["w"])
    t_gen = tracker.run(f.sector, f.row, f.y, f.w)
    assert abs(t_dig["n_tracks"] - t_gen["n_tracks"]) < 0.03 * t_gen["n_tracks"]
    src = f.truth_track[d.truth_cluster[c["digit"]]]
    off, hits = t_dig["hit_offset"], t_dig["hit_index"]
    pure = 0
    for i in range(t_dig["n_tracks"]):
        tt = src[hits[off[i]:off[i + 1]]]
        vals, cnt = np.unique(tt, return_counts=True)
        pure += cnt.max() >= 0.9 * len(tt) and vals[cnt.argmax()] >= 0
    assert pure >= 0.95 * t_dig["n_tracks"]


def test_two_large_digits_in_one_cell_carry_and_the_next_call_is_exact(tpc, tracker):
    """Two digits of 40000 in one cell add up past 16 bits and carry into the next pad's cell; the
    call is refused, and the next call (which re-clears the whole map) sees only its own digits."""
    bad = _cells([(0, 0, 2, 3, 40000), (0, 0, 2, 3, 40000), (0, 0, 6, 3, 20)])
    with pytest.raises(tpc.TpcError) as e:
        tracker.find_clusters(*bad, 64)
    assert e.value.code == -1
    ok = _cells([(0, 0, 3, 3, 9), (0, 0, 4, 3, 30), (0, 0, 2, 4, 7)])
    assert_same(tracker.find_clusters(*ok, 64), oracle.find_clusters(*ok, 64, precision="f32"))


def test_malformed_digit_beside_a_carrying_pair_leaves_the_map_clean(tpc, tracker):
    """A frame with a malformed digit and, beside it, two digits of 40000 in one cell (their sum
    carries into the next pad's cell) is refused; the next call sees only its own digits."""
    bad = _cells([(0, 0, 2, 3, 40000), (0, 0, 2, 3, 40000), (0, 0, 6, 3, 20), (0, 152, 0, 0, 5)])
    with pytest.raises(tpc.TpcError) as e:
        tracker.find_clusters(*bad, 64)
    assert e.value.code == -1
    ok = _cells([(0, 0, 3, 3, 9), (0, 0, 4, 3, 30), (0, 0, 2, 4, 7)])
    assert_same(tracker.find_clusters(*ok, 64), oracle.find_clusters(*ok, 64, precision="f32"))


def test_digits_whose_sum_wraps_to_their_own_charge_are_refused(tpc, tracker):
    """Three digits of 32768 in one cell leave 32768 in the cell (the sum wraps) and carry 1 into the
    next pad's cell: the cell still holds each digit's charge, yet the call is refused and the next
    call is exact."""
    bad = _cells([(0, 0, 2, 3, 32768)] * 3 + [(0, 0, 6, 3, 20)])
    with pytest.raises(tpc.TpcError) as e:
        tracker.find_clusters(*bad, 64)
    assert e.value.code == -1
    ok = _cells([(0, 0, 3, 3, 9), (0, 0, 4, 3, 30), (0, 0, 2, 4, 7)])
    assert_same(tracker.find_clusters(*ok, 64), oracle.find_clusters(*ok, 64, precision="f32"))
