"""Failure detection on the device without a fault: a device wait that can never complete gives
up after its limit, the host receives TPC_E_TIMEOUT, and the GPU and the library stay usable."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_07515_gb300 as tpc
    tpc.build()
    return tpc


def test_bounded_wait_times_out_and_tracking_goes_on(tpc):
    lib = tpc.load()
    t0 = time.perf_counter()
    rc = lib.tpc_check_wait_timeout(20000, None)  # 20 ms limit on a barrier nothing completes
    dt = time.perf_counter() - t0
    assert rc == tpc._lib.TPC_E_TIMEOUT
    assert dt < 10.0
    # the device and a new context work normally afterwards
    f = synth.generate("pp_500")
    tr = tpc.Tracker()
    try:
        res = tr.run(f.sector, f.row, f.y, f.w)
    finally:
        tr.close()
    orc = oracle.track(f.sector, f.row, f.y, f.w, precision="f32")
    assert res["n_tracks"] == orc.n_tracks
    assert np.array_equal(res["hit_index"], orc.tr_hits.astype(np.uint32))
