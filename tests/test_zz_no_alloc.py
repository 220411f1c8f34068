"""The allocation-free entry point tpc_links_static() against the context path.

tpc_links_static() serves callers that cannot allocate device memory when they call (another
allocator owns the device memory, or an allocation-free rule applies): it keeps all of its scratch in
one fixed-size array in the library's device image. Here it must give exactly the cleaned links that
tpc_get_links() returns after tpc_track_sectors() on the same frame, on two calls in a row (the second
call reuses the array the first one left behind), and refuse a frame larger than its fixed maximum.
This file is collected last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_static_links_equal_context_links_on_two_calls(torch_cuda):
    torch = torch_cuda
    import paper_2009_07515_gb300 as tpc
    from paper_2009_07515_gb300 import _lib
    tpc.build()
    lib = _lib.load()
    params = _lib.default_params()
    tr = tpc.Tracker()
    frames = [synth.generate("pp_500"), synth.generate("pp_500", seed=2, mult_fixed=900)]
    assert all(f.n <= _lib.STATIC_MAX_CLUSTERS for f in frames)
    for f in frames:
        h = tr.load(f.sector, f.row, f.y, f.w)
        tr.track(h)
        ref_up, ref_dn = tr.links(h, 2, f.n), tr.links(h, 3, f.n)
        tr.release(h)
        d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.sector, f.row, f.y, f.w)]
        keep = []
        cl = tpc.make_clusters(*d, keep)
        up = torch.full((f.n,), 7, dtype=torch.int32, device="cuda")
        dn = torch.full((f.n,), 7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        rc = lib.tpc_links_static(ctypes.byref(params), ctypes.byref(cl), up.data_ptr(), dn.data_ptr(), None)
        assert rc == _lib.TPC_OK
        assert np.array_equal(up.cpu().numpy(), ref_up)
        assert np.array_equal(dn.cpu().numpy(), ref_dn)
        assert (ref_up >= 0).sum() > 0.5 * f.n
    tr.close()


def test_static_links_refuse_frames_above_the_maximum(torch_cuda):
    torch = torch_cuda
    import paper_2009_07515_gb300 as tpc
    from paper_2009_07515_gb300 import _lib
    lib = _lib.load()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    cl = _lib.tpc_clusters(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                           _lib.STATIC_MAX_CLUSTERS + 1, 1)
    rc = lib.tpc_links_static(None, ctypes.byref(cl), buf.data_ptr(), buf.data_ptr(), None)
    assert rc == _lib.TPC_E_CAPACITY
    host = _lib.tpc_clusters(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 4, 0)
    assert lib.tpc_links_static(None, ctypes.byref(host), buf.data_ptr(), buf.data_ptr(), None) == _lib.TPC_E_INVAL
