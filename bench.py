"""Throughput benchmark of GB300 TPC sector tracking (clusters tracked per second).

One step = one pass of the whole tracking path (grid, neighbours, cleaning, start hits, tracklet
construction, selection, canonical output) over one synthetic time frame already resident in HBM.
Default workload: the overlapping Pb-Pb-like frame of two central-like collisions of 10000
primaries each (about 3 M clusters, FP32 storage). The L2 cache (129 MB) is flushed before each
timed step by writing a 512 MB buffer; each step is timed with CUDA events on the stream the
tracking runs on, and the flush lies outside the timed interval.

Keys beyond the base contract:
  e2e           the same metric through the C-ABI with host buffers: every step copies the frame's
                clusters from pinned host memory, tracks, and reads the tracks back
  roofline      the dominant kernel, algorithmic bytes per launch / its event-timed duration against
                the measured HBM copy bandwidth
  cpu_baseline  the CPU oracle (FP32) on the machine's host cores, on a bounded sample
  kernels_ms    per-kernel device time of one step (CUDA events between launches)
  cluster_finding  the upstream step on the same frame: its clusters digitized by the generator, the
                clusters found again from the digits on the GPU (digits/s, kernels, roofline, end to
                end, digits -> tracks, and the FP32 oracle on a sample)
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

# Roofline accounting:
#  - memory-bound kernels: algorithmic bytes per cluster counted from the data layout, e.g. the
#    neighbour search reads its row's (y, w) and the two adjacent rows once (3 x 8 B) and writes
#    the links (8 B);
#  - the tracklet kernel is bound by FP32 issue: algorithmic flops = row steps (device counter) x
#    FLOPS_PER_STEP, the add/sub/mul/div/sqrt operations of one helix propagation with scattering
#    noise, one chi2 and one Joseph-form update, counted from their definition; peak = 152 SMs x
#    128 FP32 lanes x 2 flops (FMA) x the maximum SM clock.
ALG_BYTES_PER_CLUSTER = {"neighbours": 32.0, "clean": 24.0, "seg_hist": 10.0, "bin_rank": 10.0,
                         "scatter": 30.0, "starts": 12.0}
FLOPS_PER_STEP = 480.0
E2E_WINDOW = 3  # frames in flight in the end-to-end measurement


def _recorded_traffic(kernel: str, workload: str, shape: dict, method_defaults: dict):
    """(DRAM bytes per launch of `kernel`, launch shape of the capture) from the committed ncu record
    (profiles/traffic.json), or (None, None) when there is none for this workload, the method
    defaults differ, or a source the kernel is built from has changed since the capture. The launch
    shape changes no source: the caller reports the capture's shape beside the figure when it
    differs from the timed one."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as fh:
        rec = json.load(fh).get(kernel)
    if not rec or rec.get("workload") != workload or rec.get("method_defaults") != method_defaults:
        return None, None
    h = hashlib.sha256()
    for src in rec["sources"]:
        with open(os.path.join(ROOT, src), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec["sources_sha256"]:
        return None, None
    return float(rec["dram_bytes_per_launch"]), rec.get("launch_shape")


def _traffic_fields(kernel: str, workload: str, shape: dict, method_defaults: dict) -> dict:
    traffic, cap_shape = _recorded_traffic(kernel, workload, shape, method_defaults)
    out = {"traffic": traffic}
    if traffic is not None and cap_shape != shape:
        out["traffic_launch_shape"] = cap_shape  # the capture's shape; the timed one is config.launch_shape
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


def cpu_baseline(frame, n_threads: int, budget_s: float = 20.0) -> dict:
    """The FP32 oracle on the host cores over whole sectors of the frame (sectors are independent),
    as many sectors as fit about `budget_s` seconds on `n_threads` threads."""
    import oracle
    sec = frame.sector
    m1 = sec == 0
    t0 = time.perf_counter()
    oracle.track(sec[m1], frame.row[m1], frame.y[m1], frame.w[m1], precision="f32", n_threads=1)
    per_sector = max(time.perf_counter() - t0, 1e-3)
    k = int(min(36, max(1, budget_s * n_threads / per_sector)))
    m = sec < k
    t0 = time.perf_counter()
    oracle.track(sec[m], frame.row[m], frame.y[m], frame.w[m], precision="f32", n_threads=n_threads)
    dt = time.perf_counter() - t0
    n = int(m.sum())
    return {"value": n / dt, "unit": UNIT, "cores": int(n_threads), "kind": "oracle",
            "sample": f"sectors 0-{k - 1} of the workload frame ({n} clusters), FP32 oracle, {dt:.2f} s"}


def serving_benchmark(tpc, synth, *, max_collisions: int, pool_size: int, n_frames: int, loads, seed: int = 5,
                      budget_gb: float = 80.0, params: dict | None = None):
    """Frame p50/p99 latency and throughput, served (continuous batching, tpc_submit_frame/tpc_poll)
    against plain one-frame-at-a-time tracking (load, track, read back), for a Poisson stream of
    frames with collision counts uniform in 1..max_collisions (drawn from a pool of generated frames).
    Loads are arrival rates relative to the plain path's mean service rate. Latency = time from a
    frame's arrival to its tracks being readable on the host."""
    import torch
    rng = np.random.default_rng(seed)
    colls = rng.integers(1, max_collisions + 1, pool_size)
    pool = [synth.generate("serve", n_collisions=int(c), frame_id=i) for i, c in enumerate(colls)]
    # requests arrive in pinned host memory (both arms read the same buffers)
    for f in pool:
        for k in ("sector", "row", "y", "w"):
            setattr(f, k, torch.from_numpy(np.ascontiguousarray(getattr(f, k))).pin_memory().numpy())
    params = params or {}
    plain = tpc.Tracker(**params)

    def plain_run(f):
        # one frame at a time: upload, track, read the tracks back (views of the read-back block)
        h = plain.load(f.sector, f.row, f.y, f.w)
        plain.track(h)
        plain.tracks(h, copy=False)
        plain.release(h)

    for f in pool[:2]:
        plain_run(f)
    t0 = time.perf_counter()
    for f in pool:
        plain_run(f)
    service = (time.perf_counter() - t0) / pool_size
    out = {"workload": f"Poisson stream, frames of U{{1..{max_collisions}}} collisions (pool of {pool_size})",
           "mean_plain_service_ms": service * 1e3, "budget_gb": budget_gb, "points": []}
    srv = tpc.Tracker(hbm_budget=int(budget_gb * (1 << 30)), **params)
    # warm-up: slot workspaces allocated and their graphs captured before timing
    warm = [srv.submit(f.sector, f.row, f.y, f.w) for f in pool[:6]]
    got = []
    while len(got) < len(warm):
        got += srv.poll(64, 100000)
    for t in got:
        srv.release(t)
    for load in loads:
        lam = load / service
        arrivals = np.cumsum(rng.exponential(1.0 / lam, n_frames))
        pick = rng.integers(0, pool_size, n_frames)
        clusters = float(sum(pool[k].n for k in pick))
        # plain: one frame at a time in arrival order
        lat = []
        t0 = time.perf_counter()
        for a, k in zip(arrivals, pick):
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            plain_run(pool[k])
            lat.append(time.perf_counter() - t0 - a)
        plain_span = (time.perf_counter() - t0) - arrivals[0]
        # served: submit on arrival, poll continuously
        done, sub = {}, {}
        i = 0
        t0 = time.perf_counter()
        while len(done) < n_frames:
            now = time.perf_counter() - t0
            while i < n_frames and arrivals[i] <= now:
                f = pool[pick[i]]
                tk = srv.submit(f.sector, f.row, f.y, f.w)
                sub[tk] = arrivals[i]
                i += 1
            wait_us = int(max(0.0, (arrivals[i] - now) * 1e6)) if i < n_frames else 200000
            for tk in srv.poll(64, min(wait_us, 200000)):
                srv.tracks(tk, copy=False)
                done[tk] = time.perf_counter() - t0
                srv.release(tk)
        srv_lat = [done[t] - sub[t] for t in done]
        served_span = max(done.values()) - arrivals[0]
        pt = {"load": load, "rate_per_s": lam, "frames": n_frames,
              "plain": {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                        "clusters_per_s": clusters / plain_span},
              "served": {"p50_ms": float(np.percentile(srv_lat, 50) * 1e3),
                         "p99_ms": float(np.percentile(srv_lat, 99) * 1e3), "clusters_per_s": clusters / served_span}}
        out["points"].append(pt)
    plain.close()
    srv.close()
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
    if workload == "full_570":
        return {"skipped": "digitizing the full-size frame (about 1.5e9 digits) is beyond the host generator"}
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
                         **_traffic_fields(top, workload, {}, _cf_defaults(tpc))},
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
    for _ in range(args.warmup):
        cpu_baseline(frame, cores, budget_s=budget / 4)
    times = []
    for _ in range(args.steps):
        times.append(cpu_baseline(frame, cores, budget_s=budget))
    vals = [t["value"] for t in times]
    value = float(np.mean(vals))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "parallelism": "host threads over sectors"},
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": times[0]["sample"], "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="pbpb_2x10000")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-collisions", type=int, default=40,
                    help="serving stream: collisions per frame uniform in 1..N (570 = full-size frames)")
    ap.add_argument("--serve-loads", default="0.9", help="comma-separated arrival rates / plain service rate")
    ap.add_argument("--serve-frames", type=int, default=80)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 16-frame batched-path measurement")
    ap.add_argument("--no-compression", action="store_true", help="skip the compression-inputs measurement")
    ap.add_argument("--no-cluster-finding", action="store_true", help="skip the cluster-finding measurement")
    ap.add_argument("--cf-only", action="store_true", help="run only the cluster-finding measurement")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "packed"],
                    help="cluster storage of the main workload: FP32 or 16-bit fixed point")
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
    shape = json.loads(args.shape) if args.shape else {}
    storage = {"packed": 1} if args.storage == "packed" else {}
    tr = tpc.Tracker(**shape, **storage)
    # inputs resident in HBM
    d_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (frame.sector, frame.row, frame.y, frame.w)]
    h = tr.load(*d_in)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    # a dedicated (non-default) stream: the tracking kernels are launched on it, and the step
    # events are recorded on it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    if args.profile_only:
        tr.set_timing(True)  # eager launches, one kernel per launch for the profiler
        for _ in range(args.warmup + args.steps):
            tr.track(h, stream)
            tr.tracks(h)
        print(json.dumps({"profile_only": True, "workload": args.workload, "clusters": n,
                          "runs": args.warmup + args.steps}), flush=True)
        tr.close()
        return
    tuned = None
    tuned_params = dict(shape)
    if not shape and not args.no_autotune:
        # the library's autotuner picks the launch shapes on this workload (results do not depend
        # on them); the chosen shape is reported in config.launch_shape
        rep = tr.autotune([h], reps=3)
        tuned = {k: v for k, v in rep["best"].items() if k not in ("ms", "total_ms", "stage")}
        tuned_params = dict(tuned)
        tuned["configs_timed"] = len(rep["entries"])
        for e in rep["entries"]:  # the tuner's log goes to stderr; stdout keeps the one result line
            print("tune", json.dumps(e), file=sys.stderr)
    for _ in range(args.warmup):
        tr.track(h, stream)
    res = tr.tracks(h)
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident, L2 flushed before each step)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    _barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            tr.track(h, stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    _barrier(ws)
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    value = whole_job_value(n, args.steps, dev_ms / 1e3, ws)
    dev_ms = _max_over_ranks(dev_ms, ws)
    ms_per_step = dev_ms / args.steps
    res = tr.tracks(h)

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
    dominant = max(kernels, key=kernels.get)
    hbm_peak, peak_src = _peaks()
    if dominant == "tracklets":
        flops = stats["steps"] * FLOPS_PER_STEP
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        achieved = flops / (kernels[dominant] / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, **_traffic_fields(dominant, args.workload, tuned_params,
                                                               _method_defaults(tpc)),
                    "peak_source": "derived (FP32 lanes x 2 x max SM clock)",
                    "alg_flops_per_launch": flops, "row_steps": stats["steps"]}
    else:
        alg = ALG_BYTES_PER_CLUSTER.get(dominant, 32.0) * n
        achieved = alg / (kernels[dominant] / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, **_traffic_fields(dominant, args.workload, tuned_params,
                                                                   _method_defaults(tpc)),
                    "peak_source": peak_src,
                    "alg_bytes_per_launch": alg}

    # ---- end to end through the C-ABI with host buffers (pinned), copies inside the timed region.
    # Pipelined, as a production loop drives the serving calls: every step submits the frame from
    # pinned host memory (uploaded at submit) and every finished frame's tracks are read back to
    # the host and released; up to E2E_WINDOW frames are in flight, so the upload and read-back of
    # one frame overlap the tracking of another. The synchronous path (load, track, read back, one
    # frame at a time) is reported beside it as e2e.sync_value.
    pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (frame.sector, frame.row, frame.y, frame.w)]
    pin_np = [p.numpy() for p in pin]
    h2d = int(sum(p.numel() * p.element_size() for p in pin))
    e2e_tr = tpc.Tracker(**tuned_params, **storage)

    def pipelined(k: int) -> int:
        done = sub = inflight = d2h = 0
        while done < k:
            while sub < k and inflight < args.e2e_window:
                e2e_tr.submit(*pin_np)
                sub += 1
                inflight += 1
            for t in e2e_tr.poll(64, 200000):
                out = e2e_tr.tracks(t, copy=False)  # views of the read-back tracks, until release
                d2h = int(sum(np.asarray(v).nbytes for kk, v in out.items() if kk != "n_tracks"))
                e2e_tr.release(t)
                done += 1
                inflight -= 1
        return d2h

    pipelined(2 * args.e2e_window)  # warm-up: slot workspaces and their graphs
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    d2h = pipelined(args.steps)
    e2e_s = _max_over_ranks(time.perf_counter() - t0, ws)
    e2e_tr.close()
    for _ in range(2):
        tr.run(*pin_np)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tr.run(*pin_np)
    sync_s = _max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": n * ws * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "mode": f"pipelined submit/poll, {args.e2e_window} frames in flight",
           "sync_value": n * ws * args.steps / sync_s}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "clusters_per_frame": n, "tracks_per_frame": int(res["n_tracks"]),
                       "tracklets_per_frame": int(stats.get("tracklets", 0)),
                       "storage": "16-bit fixed point" if storage else "fp32", "l2": "flushed (512 MB write) before each step",
                       "parallelism": f"replicas x{ws}",
                       "launch_shape": tuned if tuned is not None else (shape or "default"),
                       "autotuned": tuned is not None},
            "e2e": e2e, "roofline": roofline, "clocks": clk.summary(), "gpu_launches": launches_per_step * args.steps,
            "kernels_ms": kernels}
    tr.release(h)
    if not args.no_compression:
        line["compression"] = compression_benchmark(tpc, torch, d_in, tuned_params, storage, n)
    if not args.no_cluster_finding:
        line["cluster_finding"] = cluster_finding_benchmark(
            tpc, synth, torch, args.workload, cpu=rank == 0 and ws == 1 and not args.no_cpu_baseline)
    if not args.no_batched:
        line["batched"] = batched_benchmark(tpc, synth, torch)
    if not args.no_serving:
        line["serving"] = serving_benchmark(
            tpc, synth, max_collisions=args.serve_collisions, pool_size=12, n_frames=args.serve_frames,
            loads=[float(x) for x in args.serve_loads.split(",")], seed=5 + rank, params=tuned_params)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(frame, os.cpu_count() or 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    tr.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
