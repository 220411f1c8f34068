"""Throughput benchmark of GB300 TPC sector tracking (clusters tracked per second).

One step = one pass of the whole tracking path (grid, neighbours, cleaning, start hits, tracklet
construction, selection, canonical output, beam line) over one synthetic time frame already resident
in HBM. Default workload: the full-size synchronous frame (570 collisions over 128 LHC orbits,
exponential multiplicity, about 2.0e8 clusters), FP32 cluster storage; the same frame with 16-bit
fixed-point storage is measured beside it. The frame (1.8 GB of clusters, 10 GB and more of working
arrays) is larger than the L2 cache (129 MB), and the L2 is also flushed before each timed step by
writing a 512 MB buffer; each step is timed with CUDA events on the stream the tracking runs on.

Keys beyond the base contract:
  e2e           the same metric through the C-ABI with host buffers: every step submits the frame's
                clusters from pinned host memory and reads its tracks back (pipelined submit/poll;
                the synchronous load/track/read loop is e2e.sync_value)
  roofline      the dominant kernel: algorithmic HBM bytes per launch (bytes per unit of the scope
                table x units of the launch) / its event-timed duration, against the measured HBM
                copy bandwidth; its ALU issue figure beside it (alu), and the whole path's bytes
  storage_16bit the same frame in 16-bit fixed-point storage, same measurements
  extra_workloads  the Pb-Pb-like frame of two 10000-primary collisions, FP32 storage
  serving       frames of U{1..570} collisions arriving as a Poisson stream at several rates: p50/p99
                latency and clusters/s, served (tpc_submit_frame/tpc_poll) against plain
  cpu_baseline  the CPU oracle (FP32) on the machine's host cores, on a bounded sample of the frame
  kernels_ms    per-kernel device time of one step (CUDA events between launches)
  cluster_finding  the upstream step on the Pb-Pb-like frame's digits (digits/s, kernels, roofline,
                end to end, digits -> tracks, FP32 oracle on a sample)
  batched       16 frames of uneven occupancy in one batched graph launch against one at a time
  merging       the step after the sector tracking on the same frame: tracks merged across sector
                boundaries and refit (merge stage device time, merged tracks, segments)
  --impl reference   times the CPU oracle as the reference arm (this method has no other code)
Multi-GPU (torchrun): frames are independent, so every rank tracks its own replica of the
workload on its own GPU with no collective in the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TPC clusters tracked/s"
UNIT = "clusters/s"

# Roofline accounting. Algorithmic (compulsory) HBM bytes per unit of each step of the path, FP32-
# stored / 16-bit stored, counted from the data layout: the grid build reads the input (10 B) and
# writes the sorted coordinates (8 / 4 B) and input index (4 B) per cluster; the neighbour search
# reads the coordinates once with perfect row reuse (8 / 4 B) and writes two links (8 B); cleaning
# reads the links, gathers the partners' and writes them (24 B); start hits read the links (8 B);
# tracklet construction reads, per hit it fits, the coordinates (8 / 4 B) and a link (4 B) and
# writes a hit index (4 B); selection reads each tracklet hit twice (8 B), updates its weight (8 B)
# and writes an output index (4 B); the beam line reads a fit (88 B) and writes 5 values (20 B) per
# track. The unit counts come from the library's device counters (tpc_get_stats).
STEPS = [  # (step, kernels, unit, FP32 bytes per unit, 16-bit bytes per unit)
    ("K1 grid", ("seg_hist", "seg_layout", "scan_seg", "zero_bins", "bin_rank", "scan_bins", "scatter"),
     "clusters", 22.0, 18.0),
    ("K2 neighbours", ("neighbours",), "clusters", 16.0, 12.0),
    ("K3 cleaning", ("clean",), "clusters", 24.0, 24.0),
    ("K4 start hits", ("scan_start", "starts", "start_order"), "clusters", 8.0, 8.0),
    ("K5 tracklets", ("chains", "tracklets"), "tracklet_hits", 16.0, 12.0),
    ("K6/K7 selection", ("zero_w", "votes", "kept", "scan_kept", "write_tracks"), "tracklet_hits", 20.0, 20.0),
    ("K9 beam line", ("beamline",), "tracks", 108.0, 108.0),
]
# The tracklet kernel is also reported against its FP32 issue rate: algorithmic flops = row steps
# (device counter) x FLOPS_PER_STEP, the operations of one helix propagation with scattering noise,
# one chi2 and one Joseph-form update counted from their definition (FMA = 2); peak = SMs x 128 FP32
# lanes x 2 x the maximum SM clock, both read from the device.
FLOPS_PER_STEP = 480.0
E2E_WINDOW = 3  # frames in flight in the end-to-end measurement


def _recorded_traffic(kernel: str, workload: str, method_defaults: dict, units: dict | None = None):
    """DRAM bytes per launch of `kernel` from the committed ncu record (profiles/traffic.json), as
    (bytes, note): None when there is no record, the method defaults differ, or a source the kernel
    is built from has changed since the capture. A record taken on a smaller workload of the same
    kind (`scales_to` names this one) is scaled to this launch by its unit count (`units`: the device
    counter the kernel's traffic grows with), and the note says so."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as fh:
        recs = json.load(fh)
    rec = recs.get(f"{kernel}@{workload}") or recs.get(kernel)
    if not rec or rec.get("method_defaults") != method_defaults:
        return None, None
    scaled = rec.get("workload") != workload
    if scaled and (workload not in rec.get("scales_to", []) or not units):
        return None, None
    h = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec["sources_sha256"]:
        return None, None
    b = float(rec["dram_bytes_per_launch"])
    note = {"capture_workload": rec["workload"], "capture_launch_shape": rec.get("launch_shape")}
    if scaled:
        u = rec["unit"]
        b = b * float(units[u]) / float(rec["units_per_launch"])
        note["scaled_by"] = f"{u}: {units[u]} / {rec['units_per_launch']} of the capture"
    return b, note


def _traffic_fields(kernel: str, workload: str, method_defaults: dict, units: dict | None = None) -> dict:
    traffic, note = _recorded_traffic(kernel, workload, method_defaults, units)
    out = {"traffic": traffic}
    if traffic is not None:
        out["traffic_source"] = note
    return out


def _method_defaults(tpc) -> dict:
    p = tpc.default_params()
    keys = ("bz", "ky", "kw", "eps", "chi_n_max", "lmin", "sigma_y", "sigma_w", "chi2_hit_max", "n_miss_max",
            "win_nsig", "win_add", "x0_per_row", "max_sin", "y_margin", "nmin", "cov0", "packed")
    return {k: (list(getattr(p, k)) if k == "cov0" else getattr(p, k)) for k in keys}


def _cf_defaults(tpc) -> dict:
    p = tpc.cf_default_params()
    return {k: getattr(p, k) for k in ("pad_pitch", "time_bin_w", "q_peak_min", "q_total_min")}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(np.max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _progress(msg: str) -> None:
    """One progress line on stderr with the process's resident and the host's available memory."""
    rss = avail = -1.0
    try:
        with open("/proc/self/status") as fh:
            for ln in fh:
                if ln.startswith("VmRSS:"):
                    rss = int(ln.split()[1]) / 2**20
        with open("/proc/meminfo") as fh:
            for ln in fh:
                if ln.startswith("MemAvailable:"):
                    avail = int(ln.split()[1]) / 2**20
    except OSError:
        pass
    print(f"[bench] {msg} (rss {rss:.1f} GB, host available {avail:.1f} GB)", file=sys.stderr, flush=True)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, steps: int, seconds: float, ws: int) -> float:
    """Replicas: every rank processes its own copy of the workload; the job's throughput is the
    units of all ranks over the slowest rank's time."""
    return units_per_rank * ws * steps / _max_over_ranks(seconds, ws)


def _barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_sample(frame, n_sectors: int, window_clusters: int):
    """A bounded sample of a frame for the CPU oracle: in each of the first `n_sectors` sectors, the
    clusters whose drift coordinate lies in a window around the sector's median w holding about
    `window_clusters` of them (the frame's occupancy and track mix, tracks crossing the window
    edges cut there). Returns the boolean mask."""
    m = np.zeros(frame.n, bool)
    for s in range(n_sectors):
        idx = np.flatnonzero(frame.sector == s)
        if len(idx) <= window_clusters:
            m[idx] = True
            continue
        w = np.sort(frame.w[idx])
        mid = len(w) // 2
        lo, hi = w[mid - window_clusters // 2], w[mid + window_clusters // 2]
        m[idx[(frame.w[idx] >= lo) & (frame.w[idx] < hi)]] = True
    return m


def cpu_baseline(frame, n_threads: int, budget_s: float = 12.0, window: int = 0) -> dict:
    """The FP32 oracle on the host cores over a bounded sample of the frame: whole sectors when a
    sector fits the budget, else one window of each of `n_threads` sectors (sectors are independent and
    run in parallel), sized to about `budget_s` seconds of wall time."""
    import oracle
    per_sector_n = frame.n / 36.0
    if not window:
        # calibrate on a small window of sector 0
        m = cpu_sample(frame, 1, 20000)
        t0 = time.perf_counter()
        oracle.track(frame.sector[m], frame.row[m], frame.y[m], frame.w[m], precision="f32", n_threads=1)
        per_cluster = max(time.perf_counter() - t0, 1e-4) / max(int(m.sum()), 1)
        window = int(min(per_sector_n, max(20000, budget_s / per_cluster)))
    k = int(min(36, max(1, n_threads)))
    m = cpu_sample(frame, k, window)
    t0 = time.perf_counter()
    oracle.track(frame.sector[m], frame.row[m], frame.y[m], frame.w[m], precision="f32", n_threads=n_threads)
    dt = time.perf_counter() - t0
    n = int(m.sum())
    what = (f"sectors 0-{k - 1} whole" if window >= per_sector_n else
            f"sectors 0-{k - 1}, in each the {window} clusters of a drift-coordinate window around its median")
    return {"value": n / dt, "unit": UNIT, "cores": int(n_threads), "kind": "oracle", "window": window,
            "clusters": n, "seconds": dt,
            "sample": f"{what} ({n} clusters of the workload frame), FP32 oracle, {dt:.2f} s"}


def time_ordered_frames(frame):
    """The frame's clusters reordered by the time of the collision they belong to (noise clusters by
    their drift coordinate), and the start of each collision's run: the clusters of collisions
    [a, a + n) in time order are then one contiguous slice, a frame of n collisions with the
    occupancy of the full frame. Returns (sector, row, y, w, offsets[n_collisions + 1])."""
    tc = frame.coll_tc
    order_c = np.argsort(tc, kind="stable")
    rank_c = np.empty_like(order_c)
    rank_c[order_c] = np.arange(len(tc))
    tt = frame.truth_track
    coll = frame.tracks["coll"]
    key = np.empty(frame.n, np.int32)
    sig = tt >= 0
    key[sig] = rank_c[coll[tt[sig]]]
    # a noise cluster belongs to the last collision before the time its w stands for (mid drift)
    t_nom = (frame.w[~sig].astype(np.float64) - 125.0) / (250.0 / 90.0)
    key[~sig] = np.clip(np.searchsorted(np.sort(tc), t_nom, side="right") - 1, 0, len(tc) - 1)
    order = np.argsort(key, kind="stable")
    off = np.zeros(len(tc) + 1, np.int64)
    off[1:] = np.cumsum(np.bincount(key, minlength=len(tc)))
    return (frame.sector[order], frame.row[order], frame.y[order], frame.w[order], off)


def serving_benchmark(tpc, torch, frame, *, max_collisions: int, n_frames: int, loads, seed: int = 5,
                      budget_gb: float = 80.0, params: dict | None = None):
    """Frame p50/p99 latency and throughput, served (continuous batching, tpc_submit_frame/tpc_poll)
    against plain one-frame-at-a-time tracking (load, track, read back), for a Poisson stream of
    frames with collision counts uniform in 1..max_collisions. Each request is n consecutive
    collisions (in time) of the full-size frame, so requests have its occupancy and multiplicity law
    and need no generation: they are views of one page-locked copy of its clusters. Loads are
    arrival rates relative to the plain path's mean service rate, measured on the first frames of
    the stream. Latency = time from a frame's arrival to its tracks being readable on the host.
    Served frames are submitted as borrowed page-locked host input (uploaded at admission); the
    plain path uploads each frame from the same page-locked memory before tracking it."""
    rng = np.random.default_rng(seed)
    sec, row, y, w, off = time_ordered_frames(frame)
    nc = len(off) - 1
    pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (sec, row, y, w)]
    arrs = [p.numpy() for p in pin]
    n_req = rng.integers(1, min(max_collisions, nc) + 1, size=n_frames * len(loads) + 20)
    a_req = np.array([rng.integers(0, nc - k + 1) for k in n_req])
    reqs = [(int(off[a]), int(off[a + k])) for a, k in zip(a_req, n_req)]
    params = params or {}
    plain = tpc.Tracker(**params)

    def view(r):
        return [x[r[0]:r[1]] for x in arrs]

    def plain_run(r):
        # one frame at a time: upload, track, read the tracks back (views of the read-back block)
        h = plain.load(*view(r))
        plain.track(h)
        plain.tracks(h, copy=False)
        plain.release(h)

    for r in reqs[:3]:
        plain_run(r)
    t0 = time.perf_counter()
    for r in reqs[3:20]:
        plain_run(r)
    service = (time.perf_counter() - t0) / 17
    mean_clusters = float(np.mean([b - a for a, b in reqs]))
    out = {"workload": f"Poisson stream of frames of U{{1..{max_collisions}}} consecutive collisions of the "
                       f"full-size frame (mean {mean_clusters:.3g} clusters)",
           "mean_plain_service_ms": service * 1e3, "budget_gb": budget_gb, "frames_per_rate": n_frames,
           "points": []}
    srv = tpc.Tracker(hbm_budget=int(budget_gb * (1 << 30)), **params)
    # warm-up: slot workspaces allocated and their graphs captured before timing (the largest
    # request first, so no workspace grows inside the timed stream)
    warm = sorted(reqs[:20], key=lambda r: r[0] - r[1])[:4]
    tks = [srv.submit(*view(r), borrow=True) for r in warm]
    got = []
    while len(got) < len(tks):
        got += srv.poll(64, 200000)
    for t in got:
        srv.release(t)
    for li, load in enumerate(loads):
        _progress(f"serving load {load}")
        lam = load / service
        arrivals = np.cumsum(rng.exponential(1.0 / lam, n_frames))
        batch = reqs[20 + li * n_frames: 20 + (li + 1) * n_frames]
        clusters = float(sum(b - a for a, b in batch))
        # plain: one frame at a time in arrival order
        lat = []
        t0 = time.perf_counter()
        for a, r in zip(arrivals, batch):
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            plain_run(r)
            lat.append(time.perf_counter() - t0 - a)
        plain_span = (time.perf_counter() - t0) - arrivals[0]
        # served: submit on arrival, poll continuously
        done, sub = {}, {}
        i = 0
        t0 = time.perf_counter()
        while len(done) < n_frames:
            now = time.perf_counter() - t0
            while i < n_frames and arrivals[i] <= now:
                tk = srv.submit(*view(batch[i]), borrow=True)
                sub[tk] = arrivals[i]
                i += 1
            wait_us = int(max(0.0, (arrivals[i] - now) * 1e6)) if i < n_frames else 200000
            for tk in srv.poll(64, min(wait_us, 200000)):
                srv.tracks(tk, copy=False)
                done[tk] = time.perf_counter() - t0
                srv.release(tk)
        srv_lat = [done[t] - sub[t] for t in done]
        served_span = max(done.values()) - arrivals[0]
        pt = {"load": load, "rate_per_s": lam, "frames": n_frames, "clusters": clusters,
              "plain": {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                        "clusters_per_s": clusters / plain_span},
              "served": {"p50_ms": float(np.percentile(srv_lat, 50) * 1e3),
                         "p99_ms": float(np.percentile(srv_lat, 99) * 1e3), "clusters_per_s": clusters / served_span}}
        out["points"].append(pt)
    plain.close()
    srv.close()
    return out


def merging_benchmark(tpc, torch, frame, tuned_params: dict, flush, stream, reps: int = 3) -> dict:
    """K12 on a frame: its sector tracks merged across sector boundaries and refit (Sec. 6; Table 1
    of Sec. 7.2 "Track Fit"), measured apart from the tracking step: the device time of the merge
    stage (CUDA events between stages, L2 flushed before each run), the merged tracks and their
    segments."""
    dev = torch.device("cuda", torch.cuda.current_device())
    tr = tpc.Tracker(merge=1, **tuned_params)
    try:
        d_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (frame.sector, frame.row, frame.y, frame.w)]
        h = tr.load(*d_in)
        tr.track(h, stream)
        tr.tracks(h, copy=False)
        tr.set_timing(True)
        times, total = [], []
        for _ in range(reps):
            flush.zero_()
            tr.track(h, stream)
            tr.tracks(h, copy=False)
            kt = tr.kernel_times()
            times.append(kt["merge"])
            total.append(sum(kt.values()))
        tr.set_timing(False)
        res = tr.tracks(h, copy=False)
        mg = tr.merged(h)
        nseg = mg["n_seg"]
        out = {"merge_ms": float(np.median(times)), "tracking_plus_merge_ms": float(np.median(total)),
               "sector_tracks": int(res["n_tracks"]), "merged_tracks": int(mg["n_merged"]),
               "chains_by_segments": {int(k): int(v) for k, v in zip(*np.unique(nseg, return_counts=True))},
               "refit_failed": int(np.sum(mg["n_fit"] < np.diff(mg["hit_offset"]))),
               "tracks_per_s": float(res["n_tracks"] / (np.median(times) * 1e-3))}
        tr.release(h)
    finally:
        tr.close()
    return out


def compression_benchmark(tpc, torch, d_in, tuned_params: dict, storage: dict, n: int, reps: int = 5) -> dict:
    """The compression inputs of the bench frame (Sec. 4), measured apart from the tracking step:
    the device time of the residual / keep-mask stage, the fraction of clusters strategy B keeps,
    and the empirical entropy (bits per hit) of the stored residuals against the absolute
    positions of the same hits, both in 2^-9 cm steps."""
    tr = tpc.Tracker(compress=1, **tuned_params, **storage)
    try:
        h = tr.load(*d_in)
        tr.set_timing(True)
        times = []
        for _ in range(reps):
            tr.track(h)
            tr.tracks(h, copy=False)
            times.append(tr.kernel_times()["compress"])
        tr.set_timing(False)
        res = tr.tracks(h)
        keep = tr.keep_mask(h, n)
    finally:
        tr.close()
    off, npred = res["hit_offset"], res["n_pred"]
    pred = np.concatenate([np.arange(off[i], off[i] + npred[i]) for i in range(len(npred))]) if len(npred) else \
        np.zeros(0, np.int64)

    def bits(v):
        _, c = np.unique(v, return_counts=True)
        p = c / c.sum()
        return float(-(p * np.log2(p)).sum())

    hits = res["hit_index"][pred].astype(np.int64)
    y = d_in[2].cpu().numpy()[hits].astype(np.float64)
    w = d_in[3].cpu().numpy()[hits].astype(np.float64)
    r = res["residual"][pred]
    return {"kernel_ms": float(np.median(times)), "kept_fraction": float(keep.mean()),
            "hits_predicted": int(len(pred)),
            "bits_per_hit": {"residual_y": bits(r[:, 0]), "residual_w": bits(r[:, 1]),
                             "absolute_y": bits(np.rint(y * 512)), "absolute_w": bits(np.rint(w * 512))}}


# Algorithmic bytes of the cluster-finder kernels: (per digit, per cluster). A digit is 8 bytes
# (sector, row, pad, time, adc); its map cell 2; a cluster 28 (sector, row, y, w, q_tot, q_max,
# sigma_pad, sigma_time, digit index), written compacted per warp by the peak kernel and copied to
# its slot; a count (and its offset) per 32 digits.
CF_BYTES = {"cf_fill": (8 + 2, 0), "cf_peaks": (8 + 2 + 4.0 / 32, 28), "cf_copy": (8.0 / 32, 28 + 28),
            "cf_clear": (6 + 2, 0), "cf_scan": (8.0 / 32, 0)}


def cluster_finding_benchmark(tpc, synth, torch, workload: str, steps: int = 10, warmup: int = 3,
                              cpu: bool = True) -> dict:
    """Cluster finding from the digits of the workload frame (its clusters digitized by the generator):
    device time of the kernel sequence with digits resident and L2 flushed before each call (CUDA
    events on the call's stream), the roofline of its dominant kernel, end to end from page-locked
    host digits to host clusters, digits -> tracks through the device cluster list, and the FP32
    oracle on a bounded sample of sectors."""
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    f, d = synth.generate_digits(workload)
    nd = d.n
    host = [torch.from_numpy(a.astype(np.int32)) for a in (d.sector, d.row, d.pad, d.time, d.adc)]
    host = [host[0].to(torch.uint8), host[1].to(torch.uint8)] + [x.to(torch.uint16) for x in host[2:]]
    pinned = [x.pin_memory() for x in host]
    dv = [x.to(dev) for x in host]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    tr = tpc.Tracker()
    try:
        for _ in range(warmup):
            cl = tr.find_clusters(*dv, d.n_time, to_host=False, stream=stream)
        nc = int(cl.n_clusters)
        tr.set_timing(True)
        per = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            tr.find_clusters(*dv, d.n_time, to_host=False, stream=stream)
            per.append(tr.cf_kernel_times())
        tr.set_timing(False)
        kern = {k: float(np.median([p[k] for p in per])) for k in per[0]}
        dev_ms = float(np.median([sum(p.values()) for p in per]))
        top = max(kern, key=kern.get)
        bpd, bpc = CF_BYTES[top]
        alg = bpd * nd + bpc * nc
        peak, src = _peaks()
        achieved = alg / (kern[top] * 1e-3) / 1e9
        # end to end: page-locked host digits in, host cluster copies out
        for _ in range(2):
            tr.find_clusters(*pinned, d.n_time, stream=stream)
        t0 = time.perf_counter()
        for _ in range(steps):
            out = tr.find_clusters(*pinned, d.n_time, stream=stream, copy=False)
        e2e_s = (time.perf_counter() - t0) / steps
        assert out["n_clusters"] == nc
        # digits -> tracks: device clusters loaded as a frame and tracked
        def chain():
            c = tr.find_clusters(*pinned, d.n_time, to_host=False, stream=stream)
            h = tr.load_cluster_list(c)
            tr.track(h)
            r = tr.tracks(h)
            tr.release(h)
            return r
        chain()
        t0 = time.perf_counter()
        for _ in range(3):
            r = chain()
        chain_s = (time.perf_counter() - t0) / 3
    finally:
        tr.close()
    line = {"metric": "TPC digits clustered per second", "unit": "digits/s", "value": nd / (dev_ms * 1e-3),
            "ms": dev_ms, "digits": nd, "clusters": nc, "time_bins": d.n_time,
            "data": f"synthetic: the {workload} clusters digitized (0.4 cm pads, 0.2 us bins, 0.3 cm spread), "
                    "in readout order (grouped by sector and row, time-major)",
            "l2": "flushed (512 MB write) before each call", "kernels_ms": kern,
            "roofline": {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": src, "algorithmic_bytes": alg,
                         "bytes_per_digit": bpd, "bytes_per_cluster": bpc,
                         **_traffic_fields(top, workload, _cf_defaults(tpc))},
            "e2e": {"value": nd / e2e_s, "unit": "digits/s", "ms": e2e_s * 1e3, "h2d_bytes_per_step": 8 * nd,
                    "d2h_bytes_per_step": 28 * nc},
            "digits_to_tracks": {"ms": chain_s * 1e3, "tracks": int(r["n_tracks"]),
                                 "value": nd / chain_s, "unit": "digits/s"},
            "gpu_launches": 7 * steps}
    if not cpu:
        return line
    # FP32 oracle on whole sectors (about 10 s on one core)
    m0 = d.sector == 0
    t0 = time.perf_counter()
    oracle.find_clusters(d.sector[m0], d.row[m0], d.pad[m0], d.time[m0], d.adc[m0], d.n_time, precision="f32",
                         n_threads=1)
    per_sector = max(time.perf_counter() - t0, 1e-3)
    k = int(min(36, max(1, 10.0 / per_sector)))
    m = d.sector < k
    t0 = time.perf_counter()
    oracle.find_clusters(d.sector[m], d.row[m], d.pad[m], d.time[m], d.adc[m], d.n_time, precision="f32", n_threads=1)
    cpu_s = time.perf_counter() - t0
    line["cpu_baseline"] = {"value": int(m.sum()) / cpu_s, "unit": "digits/s", "cores": 1, "kind": "oracle",
                            "sample": f"sectors 0-{k - 1} ({int(m.sum())} digits), FP32 oracle, {cpu_s:.2f} s"}
    return line


def batched_benchmark(tpc, synth, torch, *, n_frames: int = 16, steps: int = 5, packed: bool = True) -> dict:
    """The batched path: n_frames frames of uneven occupancy (Poisson(5) collisions, exponential
    multiplicity) tracked by one batched graph launch (tpc_track_batch) with launch shapes autotuned
    on the batch, against the same frames tracked one at a time; inputs resident, L2 flushed before
    each step, device time by CUDA events on the tracking stream."""
    dev = torch.device("cuda", torch.cuda.current_device())
    frames = [synth.generate("batch16", frame_id=i) for i in range(n_frames)]
    total = int(sum(f.n for f in frames))
    tr = tpc.Tracker(packed=1 if packed else 0)
    d_in = [[torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (f.sector, f.row, f.y, f.w)] for f in frames]
    hs = [tr.load(*d) for d in d_in]
    rep = tr.autotune(hs, reps=2)
    shape = {k: v for k, v in rep["best"].items() if k not in ("ms", "total_ms", "stage")}
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(run) -> float:
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            run()
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        return ms / steps

    batch_ms = timed(lambda: tr.track_batch(hs, stream))
    batch_tracks = int(sum(tr.tracks(h, copy=False)["n_tracks"] for h in hs))

    def one_by_one():
        for h in hs:
            tr.track(h, stream)

    single_ms = timed(one_by_one)
    single_tracks = int(sum(tr.tracks(h, copy=False)["n_tracks"] for h in hs))
    tr.close()
    return {"workload": f"{n_frames} frames of batch16 (Poisson(5) collisions, Exp(2500) multiplicity capped at 12000)",
            "clusters": total, "frame_clusters_min": int(min(f.n for f in frames)),
            "frame_clusters_max": int(max(f.n for f in frames)), "storage": "16-bit" if packed else "fp32",
            "launch_shape": shape, "batched_ms": batch_ms, "batched_clusters_per_s": total / (batch_ms / 1e3),
            "one_at_a_time_ms": single_ms, "one_at_a_time_clusters_per_s": total / (single_ms / 1e3),
            "tracks": batch_tracks, "tracks_equal": batch_tracks == single_tracks}


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle, timed on the host cores, on bounded samples of the workload."""
    if rank != 0:
        return
    import synth
    frame = synth.generate(args.workload)
    cores = os.cpu_count() or 1
    budget = max(1.0, 60.0 / max(1, args.steps))
    first = cpu_baseline(frame, cores, budget_s=budget)
    for _ in range(max(0, args.warmup - 1)):
        cpu_baseline(frame, cores, window=first["window"])
    times = [cpu_baseline(frame, cores, window=first["window"]) for _ in range(args.steps)]
    value = float(np.mean([t["value"] for t in times]))
    # a step is one bounded sample of the workload (its clusters and wall time are in the line)
    ms_per_step = float(np.mean([t["seconds"] for t in times]) * 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "parallelism": "host threads over sectors"},
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": times[0]["sample"], "value": value,
                             "clusters_per_step": times[0]["clusters"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _alu_peak_tflops(torch, sm_max_mhz) -> tuple[float, str]:
    """FP32 issue peak of the device: SMs x 128 lanes x 2 (FMA) x the maximum SM clock."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_max_mhz or 2070.0
    src = "sampled clocks.max.sm" if sm_max_mhz else "nominal maximum SM clock (no clock sample)"
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz ({src})"


def step_rooflines(kernels: dict, stats: dict, packed: bool, hbm_peak: float) -> dict:
    """Per step of the path: algorithmic bytes (bytes per unit x device unit count), device time and
    the fraction of the HBM copy bandwidth."""
    out = {}
    for name, ks, unit, b32, b16 in STEPS:
        ms = sum(kernels.get(k, 0.0) for k in ks)
        units = stats.get(unit, 0)
        alg = (b16 if packed else b32) * units
        gbs = alg / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        out[name] = {"kernels": list(ks), "ms": ms, "unit": unit, "units": units,
                     "bytes_per_unit": b16 if packed else b32, "alg_bytes": alg, "achieved_gbs": gbs,
                     "frac": gbs / hbm_peak}
    return out


def measure_tracking(tpc, torch, frame, *, workload: str, storage: dict, shape: dict, steps: int, warmup: int,
                     ws: int, autotune: bool, stream, flush, e2e_window: int, tune_reps: int = 2) -> dict:
    """Device throughput of the tracking step on one resident frame (autotuned launch shape, L2 flushed
    before each step, CUDA events on the tracking stream), per-kernel times, the roofline of the
    dominant kernel and of every step, and the end-to-end rate through the C-ABI from pinned host
    memory (pipelined submit/poll, and the synchronous load/track/read loop)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    n = frame.n
    packed = bool(storage.get("packed"))
    tr = tpc.Tracker(**shape, **storage)
    d_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (frame.sector, frame.row, frame.y, frame.w)]
    h = tr.load(*d_in)
    _progress(f"{workload} {'16-bit' if packed else 'fp32'}: loaded")
    tuned = None
    tuned_params = dict(shape)
    if autotune and not shape:
        # the library's autotuner picks the launch shapes on this frame (results do not depend on them)
        rep = tr.autotune([h], reps=tune_reps)
        tuned = {k: v for k, v in rep["best"].items() if k not in ("ms", "total_ms", "stage")}
        tuned_params = dict(tuned)
        tuned["configs_timed"] = len(rep["entries"])
        for e in rep["entries"]:  # the tuner's log goes to stderr; stdout keeps the one result line
            print("tune", workload, json.dumps(e), file=sys.stderr)
    for _ in range(warmup):
        tr.track(h, stream)
    res = tr.tracks(h)
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident, L2 flushed before each step)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    _barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            tr.track(h, stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    _barrier(ws)
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    value = whole_job_value(n, steps, dev_ms / 1e3, ws)
    dev_ms = _max_over_ranks(dev_ms, ws)
    ms_per_step = dev_ms / steps
    res = tr.tracks(h)
    clocks = clk.summary()

    # ---- per-kernel times (eager launches with events between kernels)
    tr.set_timing(True)
    kt_runs = []
    for _ in range(5):
        flush.zero_()
        tr.track(h, stream)
        tr.tracks(h)
        kt_runs.append(tr.kernel_times())
    tr.set_timing(False)
    kernels = {k: float(np.median([r[k] for r in kt_runs])) for k in kt_runs[0]}
    launches_per_step = int(sum(tr.kernel_times(launches=True).values()))
    stats = tr.stats(h)
    stats["tracks"] = int(res["n_tracks"])
    dominant = max(kernels, key=kernels.get)
    hbm_peak, peak_src = _peaks()
    steps_rl = step_rooflines(kernels, stats, packed, hbm_peak)
    step_of = {k: st for st, ks, *_ in STEPS for k in ks}
    st = steps_rl[step_of[dominant]]
    alg = st["bytes_per_unit"] * st["units"]
    achieved = alg / (kernels[dominant] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_src == "measured" else peak_src,
                "alg_bytes_per_launch": alg, "bytes_per_unit": st["bytes_per_unit"], "unit_counted": st["unit"],
                "units_per_launch": st["units"], "kernel_ms": kernels[dominant],
                **_traffic_fields(dominant, workload, {**_method_defaults(tpc), "packed": int(packed)}, stats)}
    whole_alg = sum(v["alg_bytes"] for v in steps_rl.values())
    roofline["whole_path"] = {"alg_bytes": whole_alg, "ms": ms_per_step,
                              "achieved_gbs": whole_alg / (ms_per_step * 1e-3) / 1e9,
                              "frac": whole_alg / (ms_per_step * 1e-3) / 1e9 / hbm_peak}
    if dominant == "tracklets":
        peak_t, psrc = _alu_peak_tflops(torch, clocks.get("sm_max_mhz"))
        flops = stats["steps"] * FLOPS_PER_STEP
        roofline["alu"] = {"achieved": flops / (kernels[dominant] * 1e-3) / 1e12, "peak": peak_t,
                           "unit": "TFLOP/s", "frac": flops / (kernels[dominant] * 1e-3) / 1e12 / peak_t,
                           "peak_source": psrc, "alg_flops_per_launch": flops, "row_steps": stats["steps"],
                           "flops_per_row_step": FLOPS_PER_STEP}

    # ---- end to end through the C-ABI with host buffers (pinned), copies inside the timed region.
    # Pipelined, as a production loop drives the serving calls: every step submits the frame from
    # pinned host memory (borrowed: uploaded on the slot's stream when the frame is admitted) and
    # every finished frame's tracks are read back to the host and released;
    # up to e2e_window frames are in flight, so the upload and read-back of one frame overlap the
    # tracking of another. The synchronous loop (load, track, read back) is e2e.sync_value.
    tr.release(h)
    del d_in
    _progress(f"{workload} {'16-bit' if packed else 'fp32'}: device steps done, end to end next")
    pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (frame.sector, frame.row, frame.y, frame.w)]
    pin_np = [p.numpy() for p in pin]
    h2d = int(sum(p.numel() * p.element_size() for p in pin))
    e2e_tr = tpc.Tracker(**tuned_params, **storage)

    def pipelined(k: int) -> int:
        done = sub = inflight = d2h = 0
        while done < k:
            while sub < k and inflight < e2e_window:
                e2e_tr.submit(*pin_np, borrow=True)  # page-locked input, uploaded at admission
                sub += 1
                inflight += 1
            for t in e2e_tr.poll(64, 200000):
                out = e2e_tr.tracks(t, copy=False)  # views of the read-back tracks, until release
                d2h = int(sum(np.asarray(v).nbytes for kk, v in out.items() if kk != "n_tracks"))
                e2e_tr.release(t)
                done += 1
                inflight -= 1
        return d2h

    e2e_steps = max(3, min(steps, 10))
    pipelined(2 * e2e_window)  # warm-up: slot workspaces and their graphs
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    d2h = pipelined(e2e_steps)
    e2e_s = _max_over_ranks(time.perf_counter() - t0, ws)
    e2e_tr.close()
    for _ in range(2):
        tr.run(*pin_np)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        tr.run(*pin_np)
    sync_s = _max_over_ranks(time.perf_counter() - t0, ws)
    tr.close()
    del pin, pin_np
    _progress(f"{workload} {'16-bit' if packed else 'fp32'}: end to end done")
    e2e = {"value": n * ws * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps,
           "mode": f"pipelined submit/poll, {e2e_window} frames in flight",
           "sync_value": n * ws * e2e_steps / sync_s}
    return {"value": value, "ms_per_step": ms_per_step, "clusters_per_frame": n,
            "tracks_per_frame": int(res["n_tracks"]), "stats": stats, "kernels_ms": kernels, "roofline": roofline,
            "steps_roofline": steps_rl, "clocks": clocks, "e2e": e2e, "gpu_launches": launches_per_step * steps,
            "launch_shape": tuned if tuned is not None else (shape or "default"), "autotuned": tuned is not None,
            "tuned_params": tuned_params}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="full_570")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-collisions", type=int, default=570,
                    help="serving stream: collisions per frame uniform in 1..N (570 = full-size frames)")
    ap.add_argument("--serve-loads", default="0.7,0.9,1.1",
                    help="comma-separated arrival rates / plain service rate")
    ap.add_argument("--serve-frames", type=int, default=300, help="frames per arrival rate")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-16bit", action="store_true", help="skip the 16-bit storage measurement of the workload")
    ap.add_argument("--no-extra", action="store_true", help="skip the Pb-Pb-like frame measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 16-frame batched-path measurement")
    ap.add_argument("--no-compression", action="store_true", help="skip the compression-inputs measurement")
    ap.add_argument("--no-merging", action="store_true", help="skip the merging and refit measurement")
    ap.add_argument("--no-cluster-finding", action="store_true", help="skip the cluster-finding measurement")
    ap.add_argument("--cf-only", action="store_true", help="run only the cluster-finding measurement")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "packed"],
                    help="cluster storage of the headline: FP32 or 16-bit fixed point")
    ap.add_argument("--no-autotune", action="store_true", help="run the default launch shape, untuned")
    ap.add_argument("--e2e-window", type=int, default=E2E_WINDOW, help="frames in flight in the end-to-end measurement")
    ap.add_argument("--shape", default="",
                    help='launch shape as JSON tpc_params overrides, e.g. \'{"k5_block": 64}\' (no autotuning)')
    ap.add_argument("--profile-only", action="store_true",
                    help="only track the workload warmup + steps times (eager launches), for ncu captures")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__
    __graft_entry__.build()
    import synth
    import paper_2009_07515_gb300 as tpc

    if args.cf_only:
        # the cluster-finding measurement alone (for profiling its kernels)
        print(json.dumps(cluster_finding_benchmark(tpc, synth, torch, args.workload, steps=args.steps,
                                                   warmup=args.warmup, cpu=not args.no_cpu_baseline)), flush=True)
        return

    frame = synth.generate(args.workload)
    n = frame.n
    _progress(f"{args.workload} generated ({n} clusters)")
    shape = json.loads(args.shape) if args.shape else {}
    storage = {"packed": 1} if args.storage == "packed" else {}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    # a dedicated (non-default) stream: the tracking kernels are launched on it, and the step
    # events are recorded on it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    if args.profile_only:
        tr = tpc.Tracker(**shape, **storage)
        d_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (frame.sector, frame.row, frame.y, frame.w)]
        h = tr.load(*d_in)
        tr.set_timing(True)  # eager launches, one kernel per launch for the profiler
        for _ in range(args.warmup + args.steps):
            tr.track(h, stream)
            tr.tracks(h)
        st = tr.stats(h)
        print(json.dumps({"profile_only": True, "workload": args.workload, "clusters": n,
                          "runs": args.warmup + args.steps, "stats": st}), flush=True)
        tr.close()
        return

    common = dict(steps=args.steps, warmup=args.warmup, ws=ws, autotune=not args.no_autotune, stream=stream,
                  flush=flush, e2e_window=args.e2e_window)
    head = measure_tracking(tpc, torch, frame, workload=args.workload, storage=storage, shape=shape, **common)
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "clusters_per_frame": n, "tracks_per_frame": head["tracks_per_frame"],
                       "tracklets_per_frame": int(head["stats"].get("tracklets", 0)),
                       "storage": "16-bit fixed point" if storage else "fp32",
                       "l2": "inputs larger than L2 (1.8 GB of clusters), and flushed (512 MB write) before each step",
                       "parallelism": f"replicas x{ws}", "launch_shape": head["launch_shape"],
                       "autotuned": head["autotuned"]},
            "e2e": head["e2e"], "roofline": head["roofline"], "clocks": head["clocks"],
            "gpu_launches": head["gpu_launches"], "kernels_ms": head["kernels_ms"],
            "steps_roofline": head["steps_roofline"], "counters": head["stats"]}
    if not args.no_16bit and not storage:
        o = measure_tracking(tpc, torch, frame, workload=args.workload, storage={"packed": 1}, shape=shape, **common)
        line["storage_16bit"] = {k: o[k] for k in ("value", "ms_per_step", "tracks_per_frame", "kernels_ms", "roofline",
                                                    "steps_roofline", "e2e", "clocks", "launch_shape")}
        line["storage_16bit"]["vs_fp32"] = o["value"] / head["value"]
    if not args.no_merging:
        _progress("merging")
        line["merging"] = merging_benchmark(tpc, torch, frame, head["tuned_params"], flush, stream)
        line["merging"]["workload"] = args.workload
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        _progress("cpu baseline")
        line["cpu_baseline"] = cpu_baseline(frame, os.cpu_count() or 1)
    if not args.no_serving:
        _progress("serving")
        line["serving"] = serving_benchmark(
            tpc, torch, frame, max_collisions=args.serve_collisions, n_frames=args.serve_frames,
            loads=[float(x) for x in args.serve_loads.split(",")], seed=5 + rank, params=head["tuned_params"])
    del frame
    _progress("extra workloads")
    extra_name = "pbpb_2x10000"
    if not args.no_extra or not args.no_compression:
        ef = synth.generate(extra_name)
        o = measure_tracking(tpc, torch, ef, workload=extra_name, storage={}, shape=shape, **common)
        if not args.no_extra:
            line["extra_workloads"] = {extra_name: {k: o[k] for k in ("value", "ms_per_step", "clusters_per_frame",
                                                                      "tracks_per_frame", "kernels_ms", "roofline",
                                                                      "e2e", "launch_shape")}}
        if not args.no_compression:
            d_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (ef.sector, ef.row, ef.y, ef.w)]
            line["compression"] = compression_benchmark(tpc, torch, d_in, o["tuned_params"], {}, ef.n)
            line["compression"]["workload"] = extra_name
    if not args.no_cluster_finding:
        _progress("cluster finding")
        line["cluster_finding"] = cluster_finding_benchmark(
            tpc, synth, torch, extra_name, cpu=rank == 0 and ws == 1 and not args.no_cpu_baseline)
    if not args.no_batched:
        _progress("batched")
        line["batched"] = batched_benchmark(tpc, synth, torch)
    _progress("done")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
