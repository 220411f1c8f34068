"""GPU parity: the CUDA path (through the C-ABI) against the FP32 oracle on the same seeded inputs.

Bar: integer results (neighbour links, cluster-to-track assignments, track counts) identical on at
least 99.9% of tracks, each disagreement traced to a decision within 1e-5 relative of its cut;
track parameters within 1e-4 relative and covariances within 1e-3. The error of the GPU fit against
the FP64 oracle is reported per parameter.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import compare_tracks, track_sets  # noqa: F401 (compare_tracks is imported from here too)

pytestmark = pytest.mark.gpu

PARAM_NAMES = ("y", "w", "sin_phi", "dw_ds", "q_pt")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def tracker(torch_cuda):
    import paper_2009_07515_gb300 as tpc
    tpc.build()
    t = tpc.Tracker()
    yield t
    t.close()


def run_gpu(tracker, f):
    h = tracker.load(f.sector, f.row, f.y, f.w)
    tracker.track(h)
    res = tracker.tracks(h)
    links = [tracker.links(h, k, f.n) for k in range(4)]
    tracker.release(h)
    return res, links


@pytest.fixture(scope="module")
def tracker16(torch_cuda):
    import paper_2009_07515_gb300 as tpc
    tpc.build()
    t = tpc.Tracker(packed=1)
    yield t
    t.close()


@pytest.mark.parametrize("cfg", ["pp_500", "pbpb_2x10000"])
def test_links_and_tracks_match_fp32_oracle(tracker, cfg, n_threads):
    f = synth.generate(cfg)
    gpu, links = run_gpu(tracker, f)
    orc = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", n_threads=n_threads)
    names = ("up", "down", "up_c", "down_c")
    for k, name in enumerate(names):
        ref = getattr(orc, name)
        diff = np.flatnonzero(links[k] != ref)
        assert np.all(orc.nb_margin[diff] < 1e-5), f"{name}: {len(diff)} untraced link differences"
        assert len(diff) <= 1e-4 * f.n
    gi, oi = compare_tracks(gpu, orc)
    assert gpu["n_tracks"] > 500


@pytest.mark.parametrize("packed", [0, 1], ids=["fp32", "16bit"])
def test_dense_windows_match_oracle(tracker, tracker16, packed, n_threads):
    """Six central-like collisions at one drift time (8.9e6 clusters, so the grid is placed by the
    per-segment passes): the neighbour windows of the inner rows hold 16-19 candidates on average and
    up to about 37, so the neighbour search runs both its listed pairs (up to 16 positions per window)
    and its nested walk beyond them; links and tracks against the FP32 oracle as above."""
    f = synth.generate("pbpb_2x10000", n_collisions=6, t_zero=1)
    assert f.n > (1 << 23)
    gpu, links = run_gpu(tracker16 if packed else tracker, f)
    orc = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", packed=bool(packed), n_threads=n_threads)
    for k, name in enumerate(("up", "down", "up_c", "down_c")):
        diff = np.flatnonzero(links[k] != getattr(orc, name))
        assert np.all(orc.nb_margin[diff] < 1e-5), f"{name}: {len(diff)} untraced link differences"
        assert len(diff) <= 1e-4 * f.n
    compare_tracks(gpu, orc)
    assert gpu["n_tracks"] > 10000


@pytest.mark.parametrize("cfg", ["pp_500", "pbpb_2x10000", "batch16"])
def test_16bit_storage_matches_oracle_on_read_back_clusters(tracker16, cfg, n_threads):
    """16-bit cluster storage: the GPU equals the FP32 oracle run on the read-back coordinates."""
    f = synth.generate(cfg)
    gpu, links = run_gpu(tracker16, f)
    orc = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", packed=True, n_threads=n_threads)
    for k, name in enumerate(("up", "down", "up_c", "down_c")):
        diff = np.flatnonzero(links[k] != getattr(orc, name))
        assert np.all(orc.nb_margin[diff] < 1e-5), f"{name}: {len(diff)} untraced link differences"
    compare_tracks(gpu, orc)


def test_error_against_fp64_oracle(tracker, n_threads):
    """Per-parameter error of the GPU fit against the FP64 oracle, in units of the fitted sigma."""
    f = synth.generate("pbpb_2x10000", mult_fixed=4000)
    gpu, _ = run_gpu(tracker, f)
    o64 = oracle.track(f.sector, f.row, f.y, f.w, precision="f64", n_threads=n_threads)
    g, o = track_sets(gpu, o64)
    common = sorted(set(g) & set(o))
    assert len(common) >= 0.99 * max(len(g), len(o))
    gi = np.array([g[k] for k in common])
    oi = np.array([o[k] for k in common])
    diag = [0, 2, 5, 9, 14]
    sig = np.sqrt(o64.tr_cov[oi][:, diag])
    pull = np.abs(gpu["param"][gi] - o64.tr_param[oi]) / sig
    rel = np.abs(gpu["param"][gi] - o64.tr_param[oi]) / np.maximum(np.abs(o64.tr_param[oi]), 1e-12)
    report = {n: (float(np.median(rel[:, k])), float(np.max(pull[:, k]))) for k, n in enumerate(PARAM_NAMES)}
    print("FP32 GPU vs FP64 oracle (median relative error, max |error|/sigma):", report)
    # FP32 rounding only: far below the fit's own uncertainty
    assert np.all(np.median(pull, axis=0) < 0.01)
    assert np.all(np.quantile(pull, 0.99, axis=0) < 0.2)
    # beam-line collision time: FP32 error far below its own uncertainty sqrt(var(w0)) / v_d
    ok = np.isfinite(o64.tr_beam[oi, 3]) & np.isfinite(gpu["beam"][gi, 3])
    assert ok.mean() > 0.95
    t_pull = np.abs(gpu["beam"][gi, 3][ok] - o64.tr_beam[oi, 3][ok]) / (np.sqrt(o64.tr_beam[oi, 2][ok]) / (250.0 / 90.0))
    assert np.median(t_pull) < 0.01 and np.quantile(t_pull, 0.99) < 0.2


def test_edge_cases(tracker):
    import paper_2009_07515_gb300 as tpc
    z8, zf = np.zeros(0, np.uint8), np.zeros(0, np.float32)
    res = tracker.run(z8, z8, zf, zf)
    assert res["n_tracks"] == 0
    one = tracker.run(np.array([3], np.uint8), np.array([40], np.uint8), np.array([1.0], np.float32),
                      np.array([50.0], np.float32))
    assert one["n_tracks"] == 0
    # every cluster in one row: no links, no tracks
    f = synth.generate("pp_500")
    row = np.full(f.n, 77, np.uint8)
    assert tracker.run(f.sector, row, f.y, f.w)["n_tracks"] == 0
    # noise only
    g = synth.generate("pp_500", seed=9)
    noise = g.truth_track < 0
    res = tracker.run(g.sector[noise], g.row[noise], g.y[noise], g.w[noise])
    orc = oracle.track(g.sector[noise], g.row[noise], g.y[noise], g.w[noise], precision="f32")
    assert res["n_tracks"] == orc.n_tracks
    # malformed input is reported, not tracked
    for bad in ((np.array([36], np.uint8), np.array([1], np.uint8), [0.0], [0.0]),
                (np.array([1], np.uint8), np.array([152], np.uint8), [0.0], [0.0]),
                (np.array([1], np.uint8), np.array([1], np.uint8), [np.nan], [0.0]),
                (np.array([1], np.uint8), np.array([1], np.uint8), [0.0], [np.inf])):
        with pytest.raises(tpc.TpcError) as e:
            tracker.run(bad[0], bad[1], np.array(bad[2], np.float32), np.array(bad[3], np.float32))
        assert e.value.code == tpc._lib.TPC_E_INVAL


def test_ragged_subsets_span_tiles(tracker):
    """Random subsets (ragged row occupancies, several bins and chunks per row) match exactly."""
    f = synth.generate("pbpb_2x10000", mult_fixed=3000)
    rng = np.random.default_rng(5)
    for frac in (0.37, 0.81):
        keep = np.flatnonzero(rng.random(f.n) < frac)
        s, r, y, w = f.sector[keep], f.row[keep], f.y[keep], f.w[keep]
        gpu = tracker.run(s, r, y, w)
        orc = oracle.track(s, r, y, w, precision="f32", n_threads=8)
        compare_tracks(gpu, orc)


def test_batch_alone_vs_in_the_mix(tracker):
    frames = [synth.generate("batch16", frame_id=i) for i in range(5)]
    alone = [tracker.run(f.sector, f.row, f.y, f.w) for f in frames]
    hs = [tracker.load(f.sector, f.row, f.y, f.w) for f in frames]
    tracker.track_batch(hs)
    for h, a in zip(hs, alone):
        b = tracker.tracks(h)
        for k in a:
            assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]), equal_nan=True), k
        tracker.release(h)


@pytest.mark.parametrize("borrow", [False, True], ids=["copied", "borrowed"])
def test_serving_results_equal_plain(tracker, torch_cuda, borrow):
    """Continuous batching: each frame's tracks are identical alone and in the mix, with the input
    copied at submit or borrowed (page-locked host arrays uploaded at admission)."""
    import paper_2009_07515_gb300 as tpc
    torch = torch_cuda
    frames = [synth.generate("serve", n_collisions=int(c), frame_id=i) for i, c in enumerate([3, 1, 7, 2, 5, 1, 4, 6])]
    plain = [tracker.run(f.sector, f.row, f.y, f.w) for f in frames]
    if borrow:
        for f in frames:
            for k in ("sector", "row", "y", "w"):
                setattr(f, k, torch.from_numpy(np.ascontiguousarray(getattr(f, k))).pin_memory().numpy())
    srv = tpc.Tracker(hbm_budget=3 << 30, max_batch_frames=3)
    tickets = []
    done = []
    for f in frames:  # arrivals interleaved with polls: later frames join while earlier ones run
        tickets.append(srv.submit(f.sector, f.row, f.y, f.w, borrow=borrow))
        done += srv.poll(64, 0)
    for _ in range(10000):
        done += srv.poll(64, 100000)
        if len(done) == len(tickets):
            break
    assert sorted(done) == sorted(tickets)
    for t, p in zip(tickets, plain):
        s = srv.tracks(t)
        for k in p:
            assert np.array_equal(np.asarray(p[k]), np.asarray(s[k]), equal_nan=True), k
        srv.release(t)
    srv.close()


def test_serving_refuses_frames_beyond_the_budget(torch_cuda):
    import paper_2009_07515_gb300 as tpc
    srv = tpc.Tracker(hbm_budget=256 << 20, max_batch_frames=1)
    f = synth.generate("pbpb_2x10000")
    with pytest.raises(tpc.TpcError) as e:
        srv.submit(f.sector, f.row, f.y, f.w)
    assert e.value.code == tpc._lib.TPC_E_BUDGET
    small = synth.generate("pp_500")
    t = srv.submit(small.sector, small.row, small.y, small.w)
    got = []
    for _ in range(1000):
        got += srv.poll(8, 100000)
        if got:
            break
    assert got == [t] and srv.tracks(t)["n_tracks"] > 500
    srv.release(t)
    srv.close()


def test_tracklet_capacity_regrows(torch_cuda):
    import paper_2009_07515_gb300 as tpc
    f = synth.generate("pp_500")
    small = tpc.Tracker(tracklet_capacity=0.0005)
    a = small.run(f.sector, f.row, f.y, f.w)
    small.close()
    b = tpc.Tracker().run(f.sector, f.row, f.y, f.w)
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]), equal_nan=True), k


def test_device_resident_input(tracker, torch_cuda):
    torch = torch_cuda
    f = synth.generate("pp_500")
    host = tracker.run(f.sector, f.row, f.y, f.w)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.sector, f.row, f.y, f.w)]
    stream = torch.cuda.current_stream()
    h = tracker.load(*d)
    tracker.track(h, stream)
    dev = tracker.tracks(h)
    tracker.release(h)
    for k in host:
        assert np.array_equal(np.asarray(host[k]), np.asarray(dev[k]), equal_nan=True), k


@pytest.mark.parametrize("packed", [0, 1], ids=["fp32", "16bit"])
@pytest.mark.parametrize("cfg", ["pp_500", "pbpb_2x10000"])
def test_compression_inputs_match_oracle(torch_cuda, cfg, packed, n_threads):
    """Track-model residuals, predicted-hit counts and the strategy-B keep mask (Sec. 4) of the
    GPU path equal the FP32 oracle's exactly: the same transport of the same fits, integer outputs."""
    import paper_2009_07515_gb300 as tpc
    tr = tpc.Tracker(compress=1, packed=packed)
    try:
        f = synth.generate(cfg)
        h = tr.load(f.sector, f.row, f.y, f.w)
        tr.track(h)
        gpu = tr.tracks(h)
        keep = tr.keep_mask(h, f.n)
        tr.release(h)
    finally:
        tr.close()
    orc = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", packed=bool(packed), n_threads=n_threads)
    gi, oi = compare_tracks(gpu, orc)
    assert np.array_equal(gpu["n_pred"][gi], orc.tr_npred[oi])
    goff, ooff = gpu["hit_offset"], orc.tr_hit_off
    for g, o in zip(gi, oi):
        assert np.array_equal(gpu["residual"][goff[g]:goff[g + 1]], orc.tr_res[ooff[o]:ooff[o + 1]]), (g, o)
    assert np.array_equal(keep, orc.keep)
    assert 0.5 < keep.mean() < 1.0


def test_compression_edge_cases(torch_cuda):
    """Compression inputs on an empty frame, a frame with no tracks, and a context without them."""
    import paper_2009_07515_gb300 as tpc
    tr = tpc.Tracker(compress=1)
    try:
        z8, zf = np.zeros(0, np.uint8), np.zeros(0, np.float32)
        h = tr.load(z8, z8, zf, zf)
        tr.track(h)
        res = tr.tracks(h)
        assert res["n_tracks"] == 0 and res["residual"].shape == (0, 2) and len(res["n_pred"]) == 0
        assert len(tr.keep_mask(h, 0)) == 0
        tr.release(h)
        g = synth.generate("pp_500", seed=9)
        noise = g.truth_track < 0
        h = tr.load(g.sector[noise], g.row[noise], g.y[noise], g.w[noise])
        tr.track(h)
        keep = tr.keep_mask(h, int(noise.sum()))
        orc = oracle.track(g.sector[noise], g.row[noise], g.y[noise], g.w[noise], precision="f32")
        assert np.array_equal(keep, orc.keep)
        tr.release(h)
    finally:
        tr.close()
    plain = tpc.Tracker()
    try:
        f = synth.generate("pp_500", mult_fixed=50)
        h = plain.load(f.sector, f.row, f.y, f.w)
        plain.track(h)
        assert "residual" not in plain.tracks(h)
        with pytest.raises(tpc.TpcError) as e:
            plain.keep_mask(h, f.n)
        assert e.value.code == tpc._lib.TPC_E_STATE
    finally:
        plain.close()
