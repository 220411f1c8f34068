"""GPU parity at the full size of the synchronous frame (2.0e8 clusters, 570 collisions over 128
orbits), FP32 and 16-bit cluster storage: the whole frame is tracked on the GPU, and sampled sectors
(one per drift side) are compared with the FP32 oracle run on that sector's clusters alone. Sectors
are independent in the method, so the sector's tracks, hits, fits and beam-line results must agree
under the same bar as the small workloads.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.test_gpu_parity import compare_tracks

pytestmark = pytest.mark.gpu

SECTORS = (7, 25)


@pytest.fixture(scope="module")
def frame():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return synth.generate("full_570", n_threads=0)


def sector_view(res, s, idx):
    """The GPU tracks of sector s, hit indices mapped into the sector's own cluster numbering."""
    sel = np.flatnonzero(res["sector"] == s)
    off = res["hit_offset"]
    hits, new_off = [], [0]
    for i in sel:
        h = res["hit_index"][off[i]:off[i + 1]].astype(np.int64)
        pos = np.searchsorted(idx, h)
        assert np.all(idx[pos] == h), "a track of the sector holds a cluster of another sector"
        hits.append(pos.astype(np.uint32))
        new_off.append(new_off[-1] + len(h))
    return dict(n_tracks=len(sel), sector=res["sector"][sel], x_ref=res["x_ref"][sel], param=res["param"][sel],
                cov=res["cov"][sel], chi2=res["chi2"][sel], ndf=res["ndf"][sel], beam=res["beam"][sel],
                hit_offset=np.array(new_off, np.int64),
                hit_index=np.concatenate(hits) if hits else np.zeros(0, np.uint32))


@pytest.mark.parametrize("packed", [0, 1], ids=["fp32", "16bit"])
def test_full_size_frame_sampled_sectors(frame, packed):
    import paper_2009_07515_gb300 as tpc
    tpc.build()
    f = frame
    assert f.n > 1.5e8
    tr = tpc.Tracker(packed=packed)
    try:
        res = tr.run(f.sector, f.row, f.y, f.w)
    finally:
        tr.close()
    assert res["n_tracks"] > 1_000_000
    for s in SECTORS:
        idx = np.flatnonzero(f.sector == s)
        orc = oracle.track(f.sector[idx], f.row[idx], f.y[idx], f.w[idx], precision="f32",
                           packed=bool(packed), n_threads=1)
        gpu = sector_view(res, s, idx)
        assert orc.n_tracks > 20_000
        gi, oi = compare_tracks(gpu, orc)
        assert len(gi) == orc.n_tracks == gpu["n_tracks"]
