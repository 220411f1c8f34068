"""Pins of the oracle's cluster finder (cluster finding from digits, Sec. 2 and Table 1 of Sec. 7.2).

The finder takes each digit that wins against its 3x3 neighbours (ties go to the earlier cell in
(time, pad) order), sums the charges of the 3x3 window plus the 5x5 ring cells whose charge does not
rise away from the peak, and reports the charge-weighted mean position and widths. These tests pin it
against closed forms (single cells, two-cell and symmetric clusters), invariances (translation,
input order), charge conservation, an independent dense-array brute force on tiny random maps, the
generator's Gaussian deposits (isolated clusters are found once, at their true position), and the
rejection of malformed input.
"""
import numpy as np
import pytest

import oracle
import synth

PITCH = 0.4
DW = (250.0 / 90.0) * 0.2


def _cf(cells, n_time=64, precision="f64", **kw):
    """cells: list of (sector, row, pad, time, adc)."""
    a = np.array(cells, dtype=np.int64).reshape(-1, 5)
    p = oracle.cf_default_params(precision, **kw)
    return oracle.find_clusters(a[:, 0], a[:, 1], a[:, 2], a[:, 3], a[:, 4], n_time, precision=precision, params=p)


def _y(row, pad_pos):
    return (pad_pos + 0.5 - oracle.n_pads(row) / 2) * PITCH


def test_geometry_matches_the_generator():
    for r in range(152):
        assert oracle.n_pads(r) == synth.n_pads(r)
        assert oracle.n_pads(r) * PITCH / 2 >= (85 + r * 160 / 151) * np.tan(np.pi / 18)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_single_digit_is_a_cluster_at_the_cell_centre(precision):
    c = _cf([(3, 10, 20, 30, 50)], precision=precision)
    assert c["n_clusters"] == 1
    tol = 1e-12 if precision == "f64" else 2e-6
    assert abs(c["y"][0] - _y(10, 20)) < tol * 10
    assert abs(c["w"][0] - 30.5 * DW) < tol * 20
    assert c["sigma_pad"][0] == 0 and c["sigma_time"][0] == 0
    assert c["q_tot"][0] == 50 and c["q_max"][0] == 50 and c["digit"][0] == 0


def test_two_cells_give_the_weighted_mean_and_binomial_width():
    a, b = 40, 25
    c = _cf([(0, 5, 10, 7, a), (0, 5, 11, 7, b)])
    assert c["n_clusters"] == 1 and c["pad"][0] == 10
    m = b / (a + b)
    assert abs(c["y"][0] - _y(5, 10 + m)) < 1e-12
    assert abs(c["sigma_pad"][0] - np.sqrt(a * b) / (a + b)) < 1e-12
    assert abs(c["w"][0] - 7.5 * DW) < 1e-12 and c["sigma_time"][0] == 0


def test_symmetric_cluster_centres_exactly_on_its_peak():
    cells = [(1, 40, 30, 12, 90)]
    for dk, dj, q in ((-1, 0, 30), (1, 0, 30), (0, -1, 20), (0, 1, 20), (-1, -1, 8), (1, 1, 8), (-1, 1, 8),
                      (1, -1, 8), (-2, 0, 3), (2, 0, 3)):
        cells.append((1, 40, 30 + dk, 12 + dj, q))
    for precision in ("f64", "f32"):
        c = _cf(cells, precision=precision)
        assert c["n_clusters"] == 1
        assert c["y"][0] == np.float64(np.float32(_y(40, 30))) if precision == "f32" else abs(c["y"][0] - _y(40, 30)) < 1e-12
        assert c["q_tot"][0] == sum(x[4] for x in cells)
        # second moments: sum q dk^2 / Q
        Q = sum(x[4] for x in cells)
        skk = sum(x[4] * (x[2] - 30) ** 2 for x in cells)
        assert abs(c["sigma_pad"][0] - np.sqrt(skk / Q)) < (1e-12 if precision == "f64" else 1e-6)


def test_plateau_has_one_peak_at_its_first_cell():
    c = _cf([(2, 2, 5, 5, 30), (2, 2, 6, 5, 30)])
    assert c["n_clusters"] == 1 and c["pad"][0] == 5 and c["q_tot"][0] == 60
    c = _cf([(2, 2, 5, 5, 30), (2, 2, 5, 6, 30), (2, 2, 6, 6, 30)])
    assert c["n_clusters"] == 1 and (c["pad"][0], c["time"][0]) == (5, 5)


def test_rising_outer_cell_is_left_to_its_own_cluster():
    # peak A at pad 10 (charge 50), a valley at pad 11 (10), peak B at pad 12 (40): A's ring cell at
    # pad 12 rises from pad 11, so A leaves it out; B keeps A's valley cell, not A's peak.
    c = _cf([(0, 0, 10, 3, 50), (0, 0, 11, 3, 10), (0, 0, 12, 3, 40)])
    assert c["n_clusters"] == 2
    assert list(c["pad"]) == [10, 12]
    assert list(c["q_tot"]) == [60, 50]
    # a falling ring cell is kept
    c = _cf([(0, 0, 10, 3, 50), (0, 0, 11, 3, 20), (0, 0, 12, 3, 5)])
    assert c["n_clusters"] == 1 and c["q_tot"][0] == 75


def test_thresholds():
    assert _cf([(0, 0, 4, 4, 2)])["n_clusters"] == 0                       # peak below q_peak_min = 3
    assert _cf([(0, 0, 4, 4, 9)])["n_clusters"] == 0                       # total below q_total_min = 10
    assert _cf([(0, 0, 4, 4, 9), (0, 0, 5, 4, 1)])["n_clusters"] == 1      # total reaches 10
    assert _cf([(0, 0, 4, 4, 9)], q_total_min=9)["n_clusters"] == 1


def test_row_edges_and_time_edges_read_zero_outside():
    n = oracle.n_pads(151)
    c = _cf([(35, 151, 0, 0, 20), (35, 151, 1, 0, 10), (35, 151, n - 1, 63, 20)], n_time=64)
    assert c["n_clusters"] == 2
    assert abs(c["y"][0] - _y(151, 10 / 30)) < 1e-12
    assert abs(c["y"][1] - _y(151, n - 1)) < 1e-12 and abs(c["w"][1] - 63.5 * DW) < 1e-12


@pytest.mark.parametrize("bad", [
    (36, 0, 0, 0, 5), (0, 152, 0, 0, 5), (0, 0, 76, 0, 5), (0, 0, 0, 64, 5), (0, 0, 0, 0, 0)])
def test_malformed_digits_are_rejected(bad):
    with pytest.raises(ValueError):
        _cf([(0, 0, 3, 3, 9), bad], n_time=64)


def test_two_digits_in_one_cell_are_rejected():
    with pytest.raises(ValueError):
        _cf([(0, 0, 3, 3, 9), (0, 0, 3, 3, 4)])


def _random_map(rng, n_cells, shape=(12, 10)):
    """Tiny random (pad, time) maps in two rows of two sectors, as digit lists."""
    cells = []
    for s, r in ((0, 0), (0, 1), (20, 151)):
        q = np.zeros(shape, np.int64)
        idx = rng.choice(q.size, size=n_cells, replace=False)
        q.flat[idx] = rng.integers(1, 40, size=n_cells)
        for k, j in zip(*np.nonzero(q)):
            cells.append((s, r, int(k), int(j), int(q[k, j])))
    return cells


def _dense_brute_force(cells, n_time):
    """The definition on a dense zero-padded array per row (numpy slicing, no search)."""
    out = []
    by_row = {}
    for i, (s, r, k, j, q) in enumerate(cells):
        by_row.setdefault((s, r), []).append(i)
    grids = {}
    for (s, r), ii in by_row.items():
        g = np.zeros((oracle.n_pads(r) + 4, n_time + 4), np.int64)
        for i in ii:
            g[cells[i][2] + 2, cells[i][3] + 2] = cells[i][4]
        grids[(s, r)] = g
    for i, (s, r, k, j, q) in enumerate(cells):
        g = grids[(s, r)]
        win = g[k + 1:k + 4, j + 1:j + 4]          # win[dk + 1, dj + 1]
        later = np.array([[dj > 0 or (dj == 0 and dk > 0) for dj in (-1, 0, 1)] for dk in (-1, 0, 1)])
        ok = (win < q) | ((win == q) & later)
        ok[1, 1] = True
        if q < 3 or not ok.all():
            continue
        big = g[k:k + 5, j:j + 5].copy()           # big[dk + 2, dj + 2]
        inner_k = np.clip(np.arange(5), 1, 3)
        inner = big[np.ix_(inner_k, inner_k)]
        mask = big <= inner
        mask[1:4, 1:4] = True
        qq = big * mask
        d = np.arange(-2, 3)
        Q = qq.sum()
        if Q < 10:
            continue
        out.append((i, int(Q), int((qq.sum(1) * d).sum()), int((qq.sum(0) * d).sum()),
                    int((qq.sum(1) * d * d).sum()), int((qq.sum(0) * d * d).sum())))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_matches_dense_brute_force_on_tiny_maps(seed):
    rng = np.random.default_rng(seed)
    cells = _random_map(rng, n_cells=50)
    order = rng.permutation(len(cells))
    cells = [cells[i] for i in order]
    n_time = 10
    c = _cf(cells, n_time=n_time)
    want = _dense_brute_force(cells, n_time)
    assert c["n_clusters"] == len(want) > 3
    for o, (i, Q, Sk, Sj, Skk, Sjj) in enumerate(want):
        s, r, k, j, q = cells[i]
        assert c["digit"][o] == i and c["q_tot"][o] == Q and c["q_max"][o] == q
        mk, mj = Sk / Q, Sj / Q
        assert abs(c["y"][o] - _y(r, k + mk)) < 1e-12
        assert abs(c["w"][o] - (j + mj + 0.5) * DW) < 1e-12
        assert abs(c["sigma_pad"][o] - np.sqrt(max(0.0, Skk / Q - mk * mk))) < 1e-12
        assert abs(c["sigma_time"][o] - np.sqrt(max(0.0, Sjj / Q - mj * mj))) < 1e-12


def test_translation_and_input_order_invariance():
    f, d = synth.generate_digits("pp_500", mult_fixed=40)
    c0 = oracle.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time, precision="f64")
    # shift every digit by 7 time bins: same clusters, w moved by 7 dw
    c1 = oracle.find_clusters(d.sector, d.row, d.pad, d.time + 7, d.adc, d.n_time + 7, precision="f64")
    assert c1["n_clusters"] == c0["n_clusters"] > 1000
    assert np.array_equal(c1["digit"], c0["digit"]) and np.array_equal(c1["q_tot"], c0["q_tot"])
    assert np.allclose(c1["w"] - c0["w"], 7 * DW, atol=1e-9) and np.array_equal(c1["y"], c0["y"])
    # a permutation of the digits permutes the clusters
    perm = np.random.default_rng(1).permutation(d.n)
    c2 = oracle.find_clusters(d.sector[perm], d.row[perm], d.pad[perm], d.time[perm], d.adc[perm], d.n_time,
                              precision="f64")
    assert c2["n_clusters"] == c0["n_clusters"]
    k0 = np.lexsort((c0["pad"], c0["time"], c0["row"], c0["sector"]))
    k2 = np.lexsort((c2["pad"], c2["time"], c2["row"], c2["sector"]))
    assert np.array_equal(perm[c2["digit"][k2]], c0["digit"][k0])
    for key in ("y", "w", "q_tot", "sigma_pad", "sigma_time"):
        assert np.array_equal(c2[key][k2], c0[key][k0])
    assert np.all(np.diff(c2["digit"]) > 0)


def test_isolated_gaussian_clusters_are_found_once_at_their_position():
    """Narrow deposits (sigma 0.2 cm) of well separated clusters: every cluster is found once, holds
    all of its charge, and its centroid lies within a small fraction of a pad of the true (y, w)."""
    f = synth.generate("pp_500", mult_fixed=30, noise_frac=0.0, seed=5)
    d = synth.digitize(f, sigma_pad=0.2, sigma_time=0.2)
    c = oracle.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time, precision="f64")
    tc = d.truth_cluster[c["digit"]]
    # clusters whose 5x5 box around their own cell holds no other cluster's digit
    own = np.zeros(f.n, bool)
    own[np.unique(d.truth_cluster)] = True
    u, cnt = np.unique(tc, return_counts=True)
    assert np.all(cnt == 1)
    assert len(u) >= 0.97 * own.sum()
    dy = c["y"] - f.y[tc]
    dwv = c["w"] - f.w[tc]
    assert np.sqrt(np.mean(dy ** 2)) < 0.03 and np.sqrt(np.mean(dwv ** 2)) < 0.04
    # charge conservation: clusters with no shared digits hold every digit of their truth cluster
    qsum = np.bincount(d.truth_cluster, weights=d.adc, minlength=f.n)
    iso = np.abs(c["q_tot"] - qsum[tc]) == 0
    assert iso.mean() > 0.97


def test_digitized_pbpb_row_occupancy_merges_but_keeps_most_clusters():
    f, d = synth.generate_digits("pp_500", n_collisions=1, mult_fixed=3000, seed=7)
    c = oracle.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time, precision="f32", n_threads=4)
    assert 0.85 * f.n < c["n_clusters"] <= f.n
    # f32 and f64 decide every peak identically (integer decisions); positions agree to float rounding
    c64 = oracle.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time, precision="f64", n_threads=4)
    assert np.array_equal(c["digit"], c64["digit"]) and np.array_equal(c["q_tot"], c64["q_tot"])
    assert np.max(np.abs(c["y"] - c64["y"])) < 1e-4 and np.max(np.abs(c["w"] - c64["w"])) < 1e-3


def test_total_charge_threshold_selects_a_subset():
    """Raising q_total_min keeps exactly the clusters whose charge reaches it, unchanged."""
    f, d = synth.generate_digits("pp_500", mult_fixed=200, seed=8)
    lo = oracle.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time, precision="f32")
    p = oracle.cf_default_params("f32", q_total_min=60)
    hi = oracle.find_clusters(d.sector, d.row, d.pad, d.time, d.adc, d.n_time, precision="f32", params=p)
    keep = lo["q_tot"] >= 60
    assert 0 < hi["n_clusters"] == keep.sum() < lo["n_clusters"]
    for k in ("digit", "y", "w", "q_tot", "sigma_pad", "sigma_time"):
        assert np.array_equal(hi[k], lo[k][keep])
