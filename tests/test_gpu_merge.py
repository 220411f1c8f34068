"""GPU parity of K12, the merging of sector tracks across sector boundaries and the global refit,
with the oracle's step 9 (FP32, the kernels' arithmetic form) on the same frames.

Integer results must be identical: each sector track's outer partner, the chains (head, segments,
hits in order), the sector of the refit result and its hit count. The merge chi2, the refit fits,
covariances and chi2 are compared under the parity bar (1e-4 relative for parameters, 1e-3 for
covariances); they are expected bit for bit, and the count of bit-identical fits is checked too.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import compare_tracks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_07515_gb300 as t
    t.build()
    return t


def _run(tr, f):
    h = tr.load(f.sector, f.row, f.y, f.w)
    tr.track(h)
    res = tr.tracks(h)
    mg = tr.merged(h)
    tr.release(h)
    return res, mg


def compare_merged(mg, M):
    """GPU merged tracks (dict) against the oracle's Merged."""
    assert np.array_equal(mg["track_next"], M.tr_next)
    g_chi, o_chi = mg["track_merge_chi2"].astype(np.float64), M.tr_merge_chi2
    assert np.array_equal(np.isnan(g_chi), np.isnan(o_chi))
    np.testing.assert_allclose(g_chi, o_chi, rtol=1e-4, atol=1e-6, equal_nan=True)
    assert mg["n_merged"] == M.n
    for k, o in (("head", M.head), ("n_seg", M.nseg), ("sector", M.sector), ("ndf", M.ndf), ("n_fit", M.nfit),
                 ("hit_offset", M.hit_off)):
        assert np.array_equal(mg[k], o), k
    assert np.array_equal(mg["hit_index"].astype(np.int64), M.hits.astype(np.int64))
    ok = mg["n_fit"] > 0
    np.testing.assert_allclose(mg["x_ref"][ok], M.xref[ok], rtol=1e-6)
    np.testing.assert_allclose(mg["param"][ok], M.param[ok], rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(mg["cov"][ok], M.cov[ok], rtol=1e-3, atol=1e-9)
    np.testing.assert_allclose(mg["chi2"][ok], M.chi2[ok], rtol=1e-3, atol=1e-5)
    exact = np.all(mg["param"][ok].astype(np.float64) == M.param[ok], axis=1)
    return float(exact.mean()) if ok.any() else 1.0


@pytest.mark.parametrize("packed", [0, 1], ids=["fp32", "16bit"])
@pytest.mark.parametrize("cfg", ["pp_500", "pbpb_2x10000"])
def test_merged_tracks_match_oracle(tpc, cfg, packed, n_threads):
    f = synth.generate(cfg)
    tr = tpc.Tracker(merge=1, packed=packed)
    try:
        res, mg = _run(tr, f)
    finally:
        tr.close()
    orc = oracle.track(f.sector, f.row, f.y, f.w, precision="f32", packed=bool(packed), merge=True,
                       n_threads=n_threads)
    gi, oi = compare_tracks(res, orc)
    assert len(gi) == res["n_tracks"] == orc.n_tracks   # the merge step reads identical sector tracks
    frac = compare_merged(mg, orc.merged)
    assert frac > 0.999, frac
    assert np.sum(mg["n_seg"] >= 2) > (50 if cfg == "pp_500" else 5000)


def test_merging_off_is_refused_and_changes_nothing(tpc):
    f = synth.generate("pp_500")
    plain = tpc.Tracker()
    try:
        h = plain.load(f.sector, f.row, f.y, f.w)
        plain.track(h)
        a = plain.tracks(h)
        with pytest.raises(tpc.TpcError) as e:
            plain.merged(h)
        assert e.value.code == tpc._lib.TPC_E_STATE
        plain.release(h)
    finally:
        plain.close()
    mt = tpc.Tracker(merge=1)
    try:
        b, _ = _run(mt, f)
    finally:
        mt.close()
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]), equal_nan=True), k


def test_merging_of_batched_frames_equals_each_frame_alone(tpc):
    frames = [synth.generate("batch16", frame_id=i) for i in range(4)]
    tr = tpc.Tracker(merge=1)
    try:
        alone = [_run(tr, f)[1] for f in frames]
        hs = [tr.load(f.sector, f.row, f.y, f.w) for f in frames]
        tr.track_batch(hs)
        for h, a in zip(hs, alone):
            b = tr.merged(h)
            for k in a:
                assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]), equal_nan=True), k
            tr.release(h)
    finally:
        tr.close()
