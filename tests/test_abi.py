"""The C-ABI library builds, loads without a GPU, and exports every entry point its header declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(tpc_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2009_07515_gb300
    paper_2009_07515_gb300.build()
    from paper_2009_07515_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2009_07515_gb300", "libtpctrack.so")],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tpc_\w+)", out))
    assert set(names) <= exported


def test_binding_covers_header(lib):
    from paper_2009_07515_gb300 import _lib
    bound = {s[0] for s in _lib.SIGNATURES}
    assert bound == set(_declared_functions())


def test_params_struct_layout_and_defaults(lib):
    """Default method parameters equal the oracle's (both state the same method readings)."""
    import oracle
    from paper_2009_07515_gb300 import _lib
    p = _lib.default_params()
    assert p.struct_size == ctypes.sizeof(_lib.tpc_params)
    o = oracle.default_params("f32")
    for k in ("bz", "ky", "kw", "eps", "chi_n_max", "lmin", "sigma_y", "sigma_w", "chi2_hit_max", "n_miss_max",
              "win_nsig", "win_add", "x0_per_row", "max_sin", "y_margin", "nmin", "ext_stop"):
        assert getattr(p, k) == getattr(o, k), k
    assert list(p.cov0) == list(o.cov0)


def test_cluster_finder_defaults_equal_the_oracle(lib):
    """The cluster finder's default parameters are the oracle's (the same reading of the step)."""
    import oracle
    from paper_2009_07515_gb300 import _lib
    p = _lib.cf_default_params()
    o = oracle.cf_default_params("f32")
    for k in ("pad_pitch", "time_bin_w", "q_peak_min", "q_total_min"):
        assert getattr(p, k) == getattr(o, k), k
    assert lib.tpc_find_clusters(None, None, None, 0, None, None) == -1


def test_host_calls_without_gpu(lib):
    """Calls that need no device: version string, error paths on null arguments."""
    assert b"tpctrack" in lib.tpc_version()
    assert lib.tpc_create(None, None) == -1
    assert lib.tpc_load_clusters(None, None, None) == -1
    assert lib.tpc_poll(None, None, 0, 0) == -1
    bad = (ctypes.c_uint8 * 4)()
    assert lib.tpc_last_error(None) == b"null context"
    del bad


def test_launch_shape_parameters_are_validated(lib):
    """Shapes that are not compiled are refused before any device call."""
    from paper_2009_07515_gb300 import _lib
    for bad in (dict(k2_warps=5), dict(k2_tma=3), dict(k5_block=96), dict(k5_regs=32), dict(k5_order=4), dict(sel_lanes=8), dict(k5_blocks_per_sm=-1), dict(k5_ilp=0), dict(k5_ilp=3),
                dict(k5_ilp=2), dict(k5_ilp=2, k5_regs=128, k5_block=256), dict(k5_ilp=2, k5_regs=96, k5_block=128),
                dict(k5_ilp=1, k5_regs=128), dict(wide_votes=2), dict(wide_votes=-1)):
        p = _lib.default_params(**bad)
        ctx = ctypes.c_void_p()
        assert lib.tpc_create(ctypes.byref(p), ctypes.byref(ctx)) == _lib.TPC_E_INVAL, bad
    p = _lib.default_params()
    assert (p.k2_warps, p.k2_tma, p.k5_block, p.k5_regs, p.k5_blocks_per_sm, p.k5_order, p.sel_lanes, p.autotune,
            p.k5_ilp, p.wide_votes) == (8, 1, 128, 80, 0, 1, 32, 0, 1, 0)
    assert lib.tpc_autotune(None, None, 0, 1, None) == _lib.TPC_E_INVAL


def test_wait_diagnostic_validates_its_limit(lib):
    from paper_2009_07515_gb300 import _lib
    assert lib.tpc_check_wait_timeout(0, None) == _lib.TPC_E_INVAL
    assert lib.tpc_check_wait_timeout(2000000, None) == _lib.TPC_E_INVAL
