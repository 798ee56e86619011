"""Benchmark of the world-cache / screen-probe hot path on the 1080p workload.

One step = one frame of the whole path on one batch of synthetic input:
probe spawn, cache update (key, insert, fixed-point accumulation), resolve
(blend + decay), query + probe irradiance, per-pixel interpolation.  The
headline metric is hit records per second over the update + resolve + query
window, with the full frame time reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

--impl reference times the CPU oracle (float64 numpy) on a bounded sample
of each frame, on the host cores.  With N > 1 (torchrun) every rank runs an
independent replica on its own frames (the path has no exchange step).
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIG = 2  # the 1080p workload; --config 5 selects the 4K stress workload
METRIC = "M hit records/s and ms/frame (update+resolve+query), % HBM roofline"
UNIT = "M records/s"
N_FRAMES_DEFAULT = 16
L2_FLUSH_BYTES = 256 << 20
L2_NOTE = ("flushed between timed steps outside the events: a 256 MB buffer written, then another 256 MB "
           "buffer read, so the L2 holds only clean lines of neither the path's inputs nor its table; then the "
           "GPU idles ~1 ms (outside the events) while the host enqueues the whole step, so no pass interval "
           "contains a wait for the host")
HOST_AHEAD_CYCLES = 2_000_000  # ~1 ms at 2 GHz


class L2Flush:
    """Between timed steps: write a buffer larger than the L2 (nothing of the previous step stays),
    then read a second one, so the L2 is left clean and the write-back of the first buffer's dirty
    lines is not billed to the first timed kernel."""

    def __init__(self, torch):
        self.torch = torch
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def zero_(self):
        self.w.zero_()
        self.r.sum()
        # the GPU waits here while the host enqueues the step: the step's events then bracket GPU
        # work only, even where a pass is shorter than the host's time to launch it
        self.torch.cuda._sleep(HOST_AHEAD_CYCLES)
REFERENCE_BUDGET_S = 90.0

# DRAM traffic per launch of the dominant kernel from an ncu capture, keyed by
# "configuration:kernel" and by the source it was taken on; null when that source has changed
# since.  A source is a file of csrc/, or (file, first line, line after the last) for one section.
UPDATE_SECTION = ("gi_cache.cu", "// ---------------------------------------------------------------- update",
                  "// ---------------------------------------------------------------- resolve")
# the shared header up to the update's argument block: constants, accumulator, counters, key
# parameters and hashing, UpdateArgs
UPDATE_HEADER = ("gi_internal.cuh", "namespace gi {", "struct ResolveArgs {")
NRC_ADAM_SECTION = ("gi_nrc.cu", "// ---------------------------------------------------------------- gradient scatter and Adam",
                    "// ---------------------------------------------------------------- query selection")
NCU_TRAFFIC = {
    # k_update, boxes-1080p (5th launch): 156.84 MB read + 31.24 MB written
    "2:update": {"bytes_per_launch": 188079872, "sources": (UPDATE_SECTION, "gi_cache_dev.cuh", UPDATE_HEADER),
                 "source_sha": "1af4e79846bba09c"},
    # k_nrc_adam_table, Cornell 1080p: 3.22 TB/s x 40.16 us
    "4:adam_table": {"bytes_per_launch": 129501000, "sources": (NRC_ADAM_SECTION,), "source_sha": "a33b80b7d73defb0"},
}


def ncu_traffic(key):
    tr = NCU_TRAFFIC.get(key)
    if not tr:
        return None
    return tr["bytes_per_launch"] if _source_sha(tr["sources"]) == tr["source_sha"] else None


def _source_sha(sources):
    """Hash of the code of the sources, comments and layout left out (a comment edit keeps it)."""
    h = hashlib.sha256()
    for src in sources:
        name = src if isinstance(src, str) else src[0]
        text = open(os.path.join(ROOT, "paper_2310_19855_gb300", "csrc", name), encoding="utf-8").read()
        if not isinstance(src, str):
            a = text.index(src[1])
            text = text[a:text.index(src[2], a)]
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a moment to deliver its first sample: the timed region starts after it
            t_end = time.time() + 3.0
            while not self.lines and time.time() < t_end:
                time.sleep(0.02)
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0=None, t1=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)  # one more sample after the timed region (a region can be shorter than 200 ms)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for (tr, ln) in self.lines:
            # keep the samples taken while the timed region ran (200 ms cadence), by nvidia-smi's own
            # timestamp (the pipe may deliver lines late), with one cadence of slack after the region
            # so that a region shorter than the cadence still has its next sample
            try:
                tr = datetime.datetime.strptime(ln.split(",")[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                pass
            if t0 is not None and not (t0 - 0.05 <= tr <= t1 + 0.25):
                continue
            f = [x.strip() for x in ln.split(",")[1:]]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


E2E_NOTE = ("pipelined through the public calls: each step uploads its own inputs from pinned host memory "
            "(copy stream, double-buffered device inputs) while the previous step computes, then reads its "
            "irradiance back (download stream); ms per step = first upload to last download / steps; no L2 "
            "flush inside this timeline (every step's inputs arrive fresh from host memory)")


def e2e_pipelined(torch, n_steps, upload, compute, download):
    """Steady-state time per step of a two-deep pipeline.  upload(j, b) enqueues step j's
    host-to-device copies into buffer set b, compute(j, b) the step's passes reading set b and
    writing output set b, download(j, b) the device-to-host read of output set b; each is called
    with its stream current.  A set is reused only after the step two back has finished with it."""
    cs, ds = torch.cuda.Stream(), torch.cuda.Stream()
    st = torch.cuda.current_stream()
    up = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    down = [torch.cuda.Event(), torch.cuda.Event()]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(cs)
    for j in range(n_steps):
        b = j & 1
        with torch.cuda.stream(cs):
            if j >= 2:
                cs.wait_event(done[b])
            upload(j, b)
            up[b].record(cs)
        st.wait_event(up[b])
        if j >= 2:
            st.wait_event(down[b])
        compute(j, b)
        done[b].record(st)
        with torch.cuda.stream(ds):
            ds.wait_event(done[b])
            download(j, b)
            down[b].record(ds)
    t1.record(ds)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / n_steps


def host_link(torch, pairs_up, pairs_down, reps=5):
    """The host link alone: the step's copies (pinned host -> device, device -> pinned host), each
    direction on its own with nothing else running, best of reps; returns the e2e block's `link`."""
    st = torch.cuda.current_stream()
    out = {}
    for name, pairs in (("h2d", pairs_up), ("d2h", pairs_down)):
        nbytes = sum(src.numel() * src.element_size() for _, src in pairs)
        best = None
        for _ in range(reps):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0.record(st)
            for dst, src in pairs:
                dst.copy_(src, non_blocking=True)
            t1.record(st)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1)
            best = ms if best is None else min(best, ms)
        out[name + "_ms_per_step"] = best
        out[name + "_gbs"] = nbytes / (best * 1e-3) / 1e9
    out["note"] = ("the same copies alone (one direction at a time, one stream, best of 5): the link's "
                   "copy rate for these buffers, against which the pipelined e2e step is bounded")
    return out


# ------------------------------------------------------------------ workload
def make_frames(n_frames: int, rank: int):
    import workload as wl
    from paper_2310_19855_gb300.replicas import frame_indices
    scene = wl.make_scene(CONFIG)
    return [wl.make_frame(CONFIG, f, scene) for f in frame_indices(rank, n_frames, wl.CONFIGS[CONFIG]["frames"])]


def distinct_cells(frames, log2_slots, resolved_format=0):
    """Cells touched per frame (U), counted by the library between update and resolve."""
    import torch
    import paper_2310_19855_gb300 as gi
    from paper_2310_19855_gb300.pipeline import view_of
    h = gi.gi_cache_create(log2_slots, resolved_format=resolved_format)
    R = frames[0].n_records
    slots = torch.empty(R, dtype=torch.int32, device="cuda")
    out = []
    try:
        for i, fr in enumerate(frames):
            rec = torch.from_numpy(fr.records).cuda()
            gi.gi_cache_update(h, gi.hits_from_planes(rec, R), view_of(fr.camera, fr.frame), slots)
            out.append(gi.gi_cache_stats(h)["touched"])
            gi.gi_cache_resolve(h, i)
    finally:
        gi.gi_cache_destroy(h)
    return out


# ------------------------------------------------------------------ reference arm (CPU oracle)
def oracle_window(frames, steps, warmup, sample_frac):
    """Times the oracle's update + resolve + query + probe integration on the first
    `sample_frac` of each frame's probes (whole probes, records in order)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.cache import OracleCache
    from oracle import probes as OP
    from oracle.frame import ray_radiance
    import workload as wl
    cfg = wl.CONFIGS[CONFIG]
    oc = OracleCache(cfg["log2_slots"])
    fr0 = frames[0]
    P = fr0.tiles_x * fr0.tiles_y
    Ps = max(1, int(P * sample_frac))
    rpp = fr0.rays_per_probe
    Rs = Ps * rpp
    times = []
    for i in range(warmup + steps):
        fr = frames[i % len(frames)]
        cam = fr.camera
        sp = OP.spawn(fr.gbuffer, cam, fr.frame)
        rec = np.ascontiguousarray(fr.records[:, :Rs])
        t0 = time.perf_counter()
        ident = oc.update(rec, i, cam.pos, cam.fov_y, cam.width, cam.height)
        oc.resolve(i)
        rad, has = ray_radiance(oc, rec, ident)
        OP.integrate(sp["valid"][:Ps], sp["nrm"][:Ps], rad.reshape(Ps, rpp, 3), has.reshape(Ps, rpp))
        t1 = time.perf_counter()
        if i >= warmup:
            times.append(t1 - t0)
    return Rs, times


def host_cores() -> int:
    """Cores this process may run on (what `nproc` prints)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_share(job):
    """One worker of the all-cores oracle: the window (update, resolve, query, probe irradiance)
    over its own share of the sampled probes of every frame, with its own cache table; returns the
    seconds of each timed step."""
    log2_slots, shares, steps, warmup = job
    from oracle.cache import OracleCache
    from oracle import probes as OP
    from oracle.frame import ray_radiance
    oc = OracleCache(log2_slots)
    times = []
    for i in range(warmup + steps):
        rec, cam, valid, nrm, rpp = shares[i % len(shares)]
        t0 = time.perf_counter()
        ident = oc.update(rec, i, cam[0], cam[1], cam[2], cam[3])
        oc.resolve(i)
        rad, has = ray_radiance(oc, rec, ident)
        n = valid.size
        OP.integrate(valid, nrm, rad.reshape(n, rpp, 3), has.reshape(n, rpp))
        if i >= warmup:
            times.append(time.perf_counter() - t0)
    return times


def oracle_window_all_cores(frames, steps, warmup, sample_frac, workers):
    """The oracle's window on `workers` processes (spawned, one thread each): the sampled probes of
    each frame are split into `workers` contiguous shares, each share's records go through the
    oracle in its own process with its own cache table (a cell hit from several shares is kept
    once per share).  Returns (records per step, the slowest worker's seconds per step)."""
    import multiprocessing as mp
    os.environ["OMP_NUM_THREADS"] = "1"
    import workload as wl
    from oracle import probes as OP
    cfg = wl.CONFIGS[CONFIG]
    fr0 = frames[0]
    P = fr0.tiles_x * fr0.tiles_y
    Ps = max(workers, int(P * sample_frac))
    rpp = fr0.rays_per_probe
    bounds = [Ps * w // workers for w in range(workers + 1)]
    jobs = [[] for _ in range(workers)]
    for fr in frames[:warmup + steps]:
        cam = fr.camera
        sp = OP.spawn(fr.gbuffer, cam, fr.frame)
        camt = (np.asarray(cam.pos, np.float64), cam.fov_y, cam.width, cam.height)
        for w in range(workers):
            p0, p1 = bounds[w], bounds[w + 1]
            jobs[w].append((np.ascontiguousarray(fr.records[:, p0 * rpp:p1 * rpp]), camt, sp["valid"][p0:p1],
                            sp["nrm"][p0:p1], rpp))
    with mp.get_context("spawn").Pool(workers) as pool:
        per_worker = pool.map(_oracle_share, [(cfg["log2_slots"], jobs[w], steps, warmup) for w in range(workers)])
    slowest = np.max(np.array(per_worker), axis=0)
    return Ps * rpp, list(slowest)


def cpu_baselines(frames, sample_frac, steps=3):
    """The oracle on the same bounded sample, on one core and on all the host's cores."""
    Rs, ct = oracle_window(frames, steps=steps, warmup=1, sample_frac=sample_frac)
    cores = host_cores()
    Rp, pt = oracle_window_all_cores(frames, steps, 1, sample_frac, cores)
    what = (f"{steps} frames (after one untimed) x first {sample_frac:.3f} of the probes ({Rs} records each): "
            "update + resolve + query + probe irradiance, numpy float64")
    return {"value": Rs * len(ct) / sum(ct) / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": what + ", one thread",
            "all_cores": {"value": Rp * len(pt) / sum(pt) / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                          "sample": what + f", split into {cores} shares of whole probes on {cores} spawned "
                                           "processes (one thread each, own cache table each); time of the "
                                           "slowest share per frame (host cores from the process's CPU affinity, "
                                           "as nproc)"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    frames = make_frames(min(args.frames, args.steps + args.warmup), 0)
    cores = host_cores()
    # keep the whole run within about REFERENCE_BUDGET_S: size the per-step sample from one
    # calibration step (at most every probe of the frame)
    _, t_cal = oracle_window_all_cores(frames, 1, 0, args.sample, cores)
    per_step = REFERENCE_BUDGET_S / (args.steps + args.warmup)
    sample = min(1.0, args.sample * per_step / max(t_cal[0], 1e-6))
    sample = max(sample, 64.0 * cores / (frames[0].tiles_x * frames[0].tiles_y))
    args.sample = sample
    Rs, times = oracle_window_all_cores(frames, args.steps, args.warmup, sample, cores)
    total = sum(times)
    value = Rs * len(times) / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config_dict(frames[0], "oracle sample"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {args.sample:.4f} of the probes of each 1080p frame ({Rs} records): "
                                   f"update + resolve + query + probe irradiance, numpy float64, split into {cores} "
                                   f"shares of whole probes on {cores} spawned processes (one thread and one cache "
                                   "table each); time of the slowest share per frame"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config_dict(fr, note):
    import workload as wl
    cfg = wl.CONFIGS[CONFIG]
    return {"workload": f"{cfg['name']}: {cfg['width']}x{cfg['height']} G-buffer, {fr.tiles_x * fr.tiles_y} probes x "
                        f"{fr.rays_per_probe} rays = {fr.n_records} hit records/frame, {cfg['n_boxes']} boxes, "
                        f"2^{cfg['log2_slots']} slots, 4 LODs, alpha 0.1, evict 8",
            "records_per_step": fr.n_records, "pixels_per_step": cfg["width"] * cfg["height"],
            "l2": L2_NOTE, "note": note}


# ------------------------------------------------------------------ native arm
def run_native(args, rank, world, local_rank):
    import torch
    import paper_2310_19855_gb300 as gi
    from paper_2310_19855_gb300.build import build
    from paper_2310_19855_gb300.pipeline import Pipeline, view_of
    from paper_2310_19855_gb300.replicas import aggregate_rate, barrier, max_over_ranks
    import workload as wl
    import workload.scene as wscene

    build()
    wscene.build_tracer()
    torch.cuda.set_device(local_rank)
    cfg = wl.CONFIGS[CONFIG]
    n_frames = min(args.frames, args.steps + args.warmup)
    # (frames are cycled: frame k of the path is replayed every n_frames steps)
    frames = make_frames(n_frames, rank)
    fr0 = frames[0]
    W, H, R = fr0.camera.width, fr0.camera.height, fr0.n_records
    U = distinct_cells(frames, cfg["log2_slots"], cfg["resolved_format"])

    pl = Pipeline(W, H, fr0.rays_per_probe, cfg["log2_slots"], resolved_format=cfg["resolved_format"])
    dev_rec = [torch.from_numpy(np.ascontiguousarray(f.records[:10])).cuda() for f in frames]
    dev_gb = [torch.from_numpy(f.gbuffer).cuda() for f in frames]
    views = [view_of(f.camera, f.frame) for f in frames]
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()

    names = ["spawn", "update", "resolve", "integrate", "interpolate"]

    def step(i, ev=None):
        k = i % n_frames
        gb, rec, v = dev_gb[k], dev_rec[k], views[k]
        if ev is not None:
            ev[0].record(stream)
        pl.spawn(gb, v, stream)
        if ev is not None:
            ev[1].record(stream)
        gi.gi_cache_update(pl.cache, gi.hits_from_planes(rec, R), v, pl.slot_ids, stream)
        if ev is not None:
            ev[2].record(stream)
        pl.resolve(i, stream)
        if ev is not None:
            ev[3].record(stream)
        pl.integrate((0.0, 0.0, 0.0), stream)
        if ev is not None:
            ev[4].record(stream)
        pl.interpolate(gb, v, stream)
        if ev is not None:
            ev[5].record(stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    rebuilds0 = gi.gi_cache_stats(pl.cache)["rebuilds"]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.5)  # let nvidia-smi start sampling before the timed region
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    t_start_wall = time.time()
    for j in range(args.steps):
        flush.zero_()
        step(args.warmup + j, evs[j])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_start
    clk = clocks.stop(t_start_wall, time.time())
    barrier(world)
    st = gi.gi_cache_stats(pl.cache)
    rebuilds = st["rebuilds"] - rebuilds0
    per = np.array([[evs[j][k].elapsed_time(evs[j][k + 1]) for k in range(5)] for j in range(args.steps)])
    frame_ms = per.sum(axis=1)
    window_ms = per[:, 1:4].sum(axis=1)

    # ---- end to end through host buffers: pinned host input -> device, frame, irradiance -> host
    h_rec = [torch.from_numpy(np.ascontiguousarray(f.records[:10])).pin_memory() for f in frames[:2]]
    h_gb = [torch.from_numpy(f.gbuffer).pin_memory() for f in frames[:2]]
    h_out = [torch.empty((H, W, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
    d_rec = [torch.empty_like(dev_rec[0]) for _ in range(2)]
    d_gb = [torch.empty_like(dev_gb[0]) for _ in range(2)]
    d_g = [gi.make_gbuffer(g, W, H) for g in d_gb]
    d_irr = [torch.empty((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    e_steps = max(3, min(args.steps, 100))  # steady state: the pipeline fill and drain spread over 100 steps
    base = args.warmup + args.steps

    def e_up(j, b):
        d_rec[b].copy_(h_rec[j % 2], non_blocking=True)
        d_gb[b].copy_(h_gb[j % 2], non_blocking=True)

    def e_frame(j, b):
        v = views[j % 2]
        pl.spawn(d_gb[b], v, stream)
        gi.gi_cache_update(pl.cache, gi.hits_from_planes(d_rec[b], R), v, pl.slot_ids, stream)
        pl.resolve(base + j, stream)
        pl.integrate((0.0, 0.0, 0.0), stream)
        gi.gi_probes_interpolate(d_g[b], v, pl.probes.struct, d_irr[b], stream)

    def e_down(j, b):
        h_out[b].copy_(d_irr[b], non_blocking=True)

    e2e_ms = np.full(e_steps, e2e_pipelined(torch, e_steps, e_up, e_frame, e_down))
    h2d = h_rec[0].numel() * 4 + h_gb[0].numel() * 4
    d2h = h_out[0].numel() * 4
    link = host_link(torch, [(d_rec[0], h_rec[0]), (d_gb[0], h_gb[0])], [(h_out[0], d_irr[0])])

    # ---- the filtered probe chain (Algorithm 5): gather, filter x, filter y, project, per pass
    # (left out of a compact run: the default configuration's line carries it)
    P = fr0.tiles_x * fr0.tiles_y
    atlas = torch.empty((P, 64, 4), dtype=torch.float32, device="cuda")
    atlas_tmp = torch.empty_like(atlas)
    f_steps = 0 if args.sub else max(3, min(args.steps, 50))
    f_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(f_steps)]
    for j in range(f_steps):
        k = j % n_frames
        flush.zero_()
        f_ev[j][0].record(stream)
        gi.gi_probes_gather(pl.cache, pl.probes.struct, pl.slot_ids, dev_rec[k][9], fr0.rays_per_probe, atlas,
                            stream=stream)
        f_ev[j][1].record(stream)
        gi.gi_probes_filter(pl.probes.struct, views[k], atlas, atlas_tmp, 0, stream)
        f_ev[j][2].record(stream)
        gi.gi_probes_filter(pl.probes.struct, views[k], atlas_tmp, atlas, 1, stream)
        f_ev[j][3].record(stream)
        gi.gi_probes_project(pl.probes.struct, atlas, stream)
        f_ev[j][4].record(stream)
    torch.cuda.synchronize()
    f_ms = (np.array([[f_ev[j][i].elapsed_time(f_ev[j][i + 1]) for i in range(4)] for j in range(f_steps)]).mean(axis=0)
            if f_steps else None)

    # ---- the update's accumulation floor: its L2 atomics alone, on a frame's slot ids
    floor_ms, floor_first = update_atomic_floor(gi, torch, pl.slot_ids, R, cfg["log2_slots"], flush, stream,
                                                args.steps)

    # ---- the two-level cache (Section 2.2.3): the same frames through a tile cache
    tiles = None if args.sub else run_tiles(args, gi, Pipeline, frames, dev_rec, dev_gb, views, flush, stream, cfg, R)

    # ---- max over ranks
    tot = np.array(max_over_ranks([window_ms.sum(), frame_ms.sum(), t_wall, e2e_ms.sum()], world, "cuda"))
    if rank != 0:
        return
    value = aggregate_rate(R, world, args.steps, tot[0] / 1e3) / 1e6
    frame_rate = aggregate_rate(R, world, args.steps, tot[1] / 1e3) / 1e6
    e2e_value = aggregate_rate(R, world, e_steps, tot[3] / 1e3) / 1e6

    # ---- roofline of the dominant kernel (algorithmic bytes / event-timed duration)
    peak, peak_src = _peaks()
    pass_ms = per.mean(axis=0)
    dominant = names[int(np.argmax(pass_ms))]
    U_mean = float(np.mean(U))
    res_b = 8 if cfg["resolved_format"] == 1 else 16
    P = fr0.tiles_x * fr0.tiles_y
    X = W * H
    alg = {
        # records 40 B in + slot id 4 B out; per touched cell a 32 B tag sector read, the 32 B
        # accumulator read and written, and a 4 B touch-list entry
        "update": R * 44 + U_mean * (32 + 64 + 4),
        # per touched cell: touch entry 4, accumulator 32 read + 32 written, resolved read + written
        "resolve": U_mean * (4 + 64 + 2 * res_b),
        # per ray a 4 B slot id and a resolved gather; per probe the normal 16 B and 112 B of SH out
        "integrate": R * (4 + res_b) + P * (16 + 112),
        # per pixel 16 B G-buffer in, 16 B out; per probe 16 + 16 + 112 B read
        "interpolate": X * 32 + P * 144,
        # per probe 16 B G-buffer read, mask 4 B + pos 16 B + nrm 16 B written
        "spawn": P * 52,
    }
    d_ms = pass_ms[names.index(dominant)]
    achieved = alg[dominant] / (d_ms * 1e-3) / 1e9
    traffic = ncu_traffic(f"{CONFIG}:{dominant}")

    # ---- oracle on the host cores, bounded sample (rank 0, N = 1 only)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(frames, args.sample)

    # k_filter: each atlas entry (16 B) read once and written once per pass, plus the probe's and its
    # neighbours' position and normal (32 B per probe); the neighbours' same cell are L2 re-reads
    filt_bytes = P * 64 * 32 + P * 32
    probe_filter = None
    if f_ms is not None:
        filt_ms = float(min(f_ms[1], f_ms[2]))
        probe_filter = {
            "pass_ms": {"gather": float(f_ms[0]), "filter_x": float(f_ms[1]), "filter_y": float(f_ms[2]),
                        "project": float(f_ms[3])},
            "note": "gi_probes_gather + 2 x gi_probes_filter + gi_probes_project in place of "
                    "gi_probes_integrate (Algorithm 5), L2 flushed before each chain",
            "roofline": {"bound": "hbm", "kernel": "k_filter", "algorithmic_bytes_per_launch": filt_bytes,
                         "achieved": filt_bytes / (filt_ms * 1e-3) / 1e9, "peak": peak,
                         "frac": filt_bytes / (filt_ms * 1e-3) / 1e9 / peak, "unit": "GB/s"}}
    launches_per_step = 6  # k_spawn, k_mip_tail, k_update, k_resolve_bitmap, k_integrate, k_interpolate
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(tot[1] / args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config_dict(fr0, "value over update+resolve+query(+probe irradiance); ms_per_step is the "
                                    "whole frame (spawn ... interpolation)"),
        "window_ms_per_step": float(tot[0] / args.steps),
        "full_frame_records_per_s": frame_rate,
        "pass_ms": {n: float(m) for n, m in zip(names, pass_ms)},
        "touched_cells_per_frame": U_mean,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": dominant,
                     "algorithmic_bytes_per_launch": alg[dominant], "peak_source": peak_src},
        "update_atomic_floor": {
            "kernel": "k_diag_atomics (gi_diag_update_atomics)", "ms": floor_ms, "update_ms": float(pass_ms[1]),
            "update_over_floor": float(pass_ms[1]) / floor_ms, "touched_slots": floor_first,
            "note": "the update's accumulation alone (bitmap form: one 32-byte bulk reduction of the sums and count "
                    "plus a bitmap bit per hit) on a frame's own slot ids, nothing else, L2 flushed before each "
                    "launch: the floor of k_update's accumulation"},
        "roofline_window": {"achieved": sum(alg[n] for n in ("update", "resolve", "integrate")) /
                                        (pass_ms[1:4].sum() * 1e-3) / 1e9, "peak": peak, "unit": "GB/s"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": float(tot[3] / e_steps), "steps": e_steps, "note": E2E_NOTE, "link": link},
        "gpu_launches": int(args.steps * launches_per_step + rebuilds),
        "dropped_hits": int(st["dropped"]),
        "table": {"slots": int(st["slots"]), "occupied": int(st["occupied"]), "live": int(st["live"]),
                  "max_probe_seen": int(st["max_probe_seen"]), "rebuilds_total": int(st["rebuilds"])},
        "rebuilds_in_timed_region": int(rebuilds),
        "probe_filter": probe_filter,
        "tiles": tiles,
        "clocks": clk,
        "wall_s_timed": float(tot[2]),
    }
    if tiles is not None:
        for k in ("update", "resolve"):
            r = tiles["roofline"][k]
            r["peak"] = peak
            r["frac"] = r["achieved"] / peak
    pl.close()
    return line




def update_atomic_floor(gi, torch, slot_ids, R, log2_slots, flush, stream, steps):
    """gi_diag_update_atomics on one frame's slot ids (the update's accumulation in the form the
    cache uses by default, the bitmap form, and nothing else) into a zeroed table of the cache's
    size, L2 flushed before each launch: mean event-timed ms over the launches after 3 warm-up
    ones, and the slots touched (bits set)."""
    slots = 1 << log2_slots
    scratch = torch.zeros(slots * 8 + slots // 32, dtype=torch.int32, device="cuda")
    n = max(3, min(steps, 50))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n + 3)]
    for j in range(n + 3):
        scratch.zero_()
        flush.zero_()
        ev[j][0].record(stream)
        gi.gi_diag_update_atomics(slot_ids, R, log2_slots, scratch, first_touch=gi.GI_FIRST_TOUCH_BITMAP,
                                  stream=stream)
        ev[j][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev[3:]]))
    bits = scratch[slots * 8:].cpu().numpy().view(np.uint32)
    touched = int(np.unpackbits(bits.view(np.uint8)).sum())
    del scratch
    return ms, touched


def tile_bytes(R, touched_tiles, touched_cells, live_in_touched, res_b, tile_slots):
    """Algorithmic bytes of the tile cache's update (k_tile_key + k_tile_compact +
    k_tile_accumulate) and resolve (k_tile_resolve) for one frame."""
    # update: records 40 B in and the slot id 4 B out, then slot id + radiance 16 B in again; per
    # touched tile a 32 B tag sector, its 8 B mask set, its block index and list entry 8 B written;
    # per touched cell the 32 B accumulator read and written; the compaction scans 12 B (mask +
    # block index) per slot
    upd = R * (44 + 16) + touched_tiles * (32 + 8 + 8) + touched_cells * 64 + tile_slots * 12
    # resolve: per touched tile the list entry 4 B, masks 8 + 8 B read and 8 + 8 B + 4 B index
    # written, 256 B of stamps, 336 B of MIP values written; per touched cell the accumulator read +
    # cleared, state and stamp written; per live cell of a touched tile its state read and its
    # answer written
    res = touched_tiles * (4 + 16 + 20 + 256 + 336) + touched_cells * (64 + 20) + live_in_touched * (16 + res_b)
    return upd, res
TILE_MIN_SAMPLES = 16


def run_tiles(args, gi, Pipeline, frames, dev_rec, dev_gb, views, flush, stream, cfg, R):
    """Update + resolve + probe irradiance through a tile cache (8 x 8 cells with MIP levels),
    per pass, L2 flushed before each frame; the resolve's algorithmic bytes from one frame's
    touched tiles, touched cells and live cells in the touched tiles."""
    import torch

    fr0 = frames[0]
    W, H = fr0.camera.width, fr0.camera.height
    n_frames = len(frames)
    log2_tiles = cfg["log2_tiles"]  # 2^18 tile slots of 64 cells at 1080p, 2^20 at 4K
    pt = Pipeline(W, H, fr0.rays_per_probe, log2_tiles, resolved_format=cfg["resolved_format"], tiles=True,
                  min_samples=TILE_MIN_SAMPLES)
    try:
        def frame(i, ev=None):
            k = i % n_frames
            pt.spawn(dev_gb[k], views[k], stream)
            if ev is not None:
                ev[0].record(stream)
            gi.gi_cache_update(pt.cache, gi.hits_from_planes(dev_rec[k], R), views[k], pt.slot_ids, stream)
            if ev is not None:
                ev[1].record(stream)
            pt.resolve(i, stream)
            if ev is not None:
                ev[2].record(stream)
            pt.integrate((0.0, 0.0, 0.0), stream)
            if ev is not None:
                ev[3].record(stream)

        for i in range(args.warmup):
            frame(i)
        steps = max(3, args.steps)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        torch.cuda.synchronize()
        for j in range(steps):
            flush.zero_()
            frame(args.warmup + j, evs[j])
        torch.cuda.synchronize()
        ms = np.array([[evs[j][i].elapsed_time(evs[j][i + 1]) for i in range(3)] for j in range(steps)]).mean(axis=0)
        # one more frame, counted: touched tiles and cells, live cells of the touched tiles
        i = args.warmup + steps
        k = i % n_frames
        gi.gi_cache_update(pt.cache, gi.hits_from_planes(dev_rec[k], R), views[k], pt.slot_ids, stream)
        st = gi.gi_cache_stats(pt.cache, stream)
        ids = pt.slot_ids.cpu().numpy().view(np.uint32)
        cells_total = (1 << log2_tiles) * 64
        ids = ids[ids < cells_total]
        touched_tiles = np.unique(ids >> 6)
        touched_cells = int(np.unique(ids).size)
        pt.resolve(i, stream)
        ex = gi.gi_cache_export(pt.cache)
        live_in_touched = int(np.isin(ex["slot"] >> 6, touched_tiles).sum())
        res_b = 8 if cfg["resolved_format"] == 1 else 16
        Tt = float(touched_tiles.size)
        upd_b, res_bytes = tile_bytes(R, Tt, touched_cells, live_in_touched, res_b, float(1 << log2_tiles))
        return {
            "note": "gi_cache_create(tiles=1): 2^%d tile slots of 8 x 8 cells, min_samples %d; spawn untimed, "
                    "update + resolve + probe irradiance per pass, L2 flushed per frame" % (log2_tiles, TILE_MIN_SAMPLES),
            "pass_ms": {"update": float(ms[0]), "resolve": float(ms[1]), "integrate": float(ms[2])},
            "window_records_per_s_M": R / (ms.sum() * 1e-3) / 1e6,
            "touched_tiles": int(Tt), "touched_cells": touched_cells, "live_cells_in_touched_tiles": live_in_touched,
            "table": {"slots": int(st["slots"]), "occupied": int(st["occupied"]), "rebuilds": int(st["rebuilds"]),
                      "dropped": int(st["dropped"])},
            "roofline": {
                "update": {"kernel": "k_tile_key + k_tile_compact + k_tile_accumulate", "bound": "hbm",
                           "algorithmic_bytes_per_launch": upd_b,
                           "achieved": upd_b / (ms[0] * 1e-3) / 1e9, "unit": "GB/s"},
                "resolve": {"kernel": "k_tile_resolve", "bound": "hbm", "algorithmic_bytes_per_launch": res_bytes,
                            "achieved": res_bytes / (ms[1] * 1e-3) / 1e9, "unit": "GB/s"}},
        }
    finally:
        pt.close()


# ------------------------------------------------------------------ temporal arm (configuration 6)
def oracle_temporal_window(frames, steps):
    """Times the oracle's frame of the temporal path: reprojection, upscaled spawn, cache update +
    resolve on the spawn tiles' rays, the frame atlas (Algorithm 4) and SH projection."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.cache import OracleCache
    from oracle import probes as OP
    from oracle import temporal as OT
    from oracle.frame import ray_radiance
    import workload as wl
    cfg = wl.CONFIGS[CONFIG]
    oc = OracleCache(cfg["log2_slots"])
    fr0 = frames[0]
    st = OT.empty_state(fr0.tiles_x, fr0.tiles_y)
    atlas = np.zeros((st["pos"].shape[0], 64, 4))
    times = []
    for i in range(steps):
        fr = frames[i % len(frames)]
        cam = fr.camera
        t0 = time.perf_counter()
        st = OT.reproject(st, fr.gbuffer, cam, fr.motion)
        ft = OT.spawn_fresh(st, fr.gbuffer, cam, fr.frame, fr.upscale)
        ident = oc.update(fr.records, i, cam.pos, cam.fov_y, cam.width, cam.height)
        oc.resolve(i)
        rad, has = ray_radiance(oc, fr.records, ident)
        S = ft.size
        atlas = OT.temporal_atlas(st, atlas, ft, rad.reshape(S, fr.rays_per_probe, 3),
                                  has.reshape(S, fr.rays_per_probe), fr.records[9])
        OP.project(OT.probe_valid(st), st["nrm"][:, 0:3].astype(np.float64), atlas)
        times.append(time.perf_counter() - t0)
    return fr0.n_records, times


def run_temporal(args, rank, world, local_rank):
    """Configuration 6: the 1080p boxes workload at 2x2 temporal upscale.  Per frame: reprojection
    (Algorithm 1), upscaled spawn, cache update + resolve on the spawn tiles' rays (a quarter of
    the probes trace), the frame atlas (fresh probes blended with their history by Algorithm 4,
    reprojected probes carried), SH projection, per-pixel interpolation."""
    import torch
    import paper_2310_19855_gb300 as gi
    from paper_2310_19855_gb300.build import build
    from paper_2310_19855_gb300.pipeline import TemporalPipeline, view_of
    from paper_2310_19855_gb300.replicas import aggregate_rate, barrier, max_over_ranks
    import workload as wl
    import workload.scene as wscene

    build()
    wscene.build_tracer()
    torch.cuda.set_device(local_rank)
    cfg = wl.CONFIGS[CONFIG]
    n_frames = min(args.frames, args.steps + args.warmup)
    frames = make_frames(n_frames, rank)
    fr0 = frames[0]
    W, H, R = fr0.camera.width, fr0.camera.height, fr0.n_records
    u = fr0.upscale
    tiles = bool(cfg.get("tiles", False))
    filtered = bool(cfg.get("filtered", False))
    log2 = cfg["log2_tiles"] if tiles else cfg["log2_slots"]
    cache_kw = dict(resolved_format=cfg["resolved_format"])
    if tiles:
        cache_kw.update(tiles=True, min_samples=cfg["min_samples"])
    tp = TemporalPipeline(W, H, fr0.rays_per_probe, log2, upscale=u, filtered=filtered, **cache_kw)
    dev_rec = [torch.from_numpy(np.ascontiguousarray(f.records[:10])).cuda() for f in frames]
    dev_gb = [torch.from_numpy(f.gbuffer).cuda() for f in frames]
    dev_mv = [torch.from_numpy(f.motion).cuda() for f in frames]
    views = [view_of(f.camera, f.frame) for f in frames]
    gbs = [gi.make_gbuffer(g, W, H) for g in dev_gb]
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()
    names = ["reproject", "spawn", "update", "resolve", "gather_temporal"]
    names += ["filter_x", "filter_y"] if filtered else []
    names += ["project", "interpolate"]
    n_ev = len(names) + 1

    def step(i, ev=None, rec=None, gb=None, mv=None):
        k = i % n_frames
        rec = dev_rec[k] if rec is None else rec
        g = gbs[k] if gb is None else gb
        mv = dev_mv[k] if mv is None else mv
        v = views[k]
        cur, prev = tp.bufs[tp.k], tp.bufs[tp.k ^ 1]

        def mark(j):
            if ev is not None:
                ev[j].record(stream)
        mark(0)
        gi.gi_probes_reproject(g, v, mv, prev.struct, cur.struct, tp.src, stream)
        mark(1)
        gi.gi_probes_spawn_upscaled(g, v, u, True, cur.struct, stream)
        mark(2)
        gi.gi_cache_update(tp.cache, gi.hits_from_planes(rec, R), v, tp.slot_ids, stream)
        mark(3)
        gi.gi_cache_resolve(tp.cache, i, stream)
        mark(4)
        gi.gi_probes_gather_temporal(tp.cache, g, v, u, cur.struct, tp.slot_ids, rec[9], tp.rpp, tp.src,
                                     tp.atlases[tp.k ^ 1], tp.atlases[tp.k], stream=stream)
        mark(5)
        shown, j = tp.atlases[tp.k], 6
        if filtered:
            gi.gi_probes_filter(cur.struct, v, shown, tp.filt[0], 0, stream)
            mark(6)
            gi.gi_probes_filter(cur.struct, v, tp.filt[0], tp.filt[1], 1, stream)
            mark(7)
            shown, j = tp.filt[1], 8
        gi.gi_probes_project(cur.struct, shown, stream)
        mark(j)
        gi.gi_probes_interpolate(g, v, cur.struct, tp.irr, stream)
        mark(j + 1)
        tp.k ^= 1

    U = distinct_cells(frames, cfg["log2_slots"], cfg["resolved_format"])
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    rebuilds0 = gi.gi_cache_stats(tp.cache)["rebuilds"]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.5)
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    t_start_wall = time.time()
    for j in range(args.steps):
        flush.zero_()
        step(args.warmup + j, evs[j])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_start
    clk = clocks.stop(t_start_wall, time.time())
    barrier(world)
    per = np.array([[evs[j][k].elapsed_time(evs[j][k + 1]) for k in range(len(names))] for j in range(args.steps)])
    frame_ms = per.sum(axis=1)
    # update, resolve, temporal gather (+ filter), projection
    window_ms = per[:, names.index("update"):names.index("project") + 1].sum(axis=1)
    st = gi.gi_cache_stats(tp.cache)
    rebuilds = st["rebuilds"] - rebuilds0
    valid = int((tp.probes.mask[:tp.probes.layout.num_probes] != -1).sum().item())
    reproj = int((tp.src != -1).sum().item())

    # ---- end to end: records, G-buffer and motion vectors from pinned host memory, irradiance back
    h_rec = [torch.from_numpy(np.ascontiguousarray(f.records[:10])).pin_memory() for f in frames[:2]]
    h_gb = [torch.from_numpy(f.gbuffer).pin_memory() for f in frames[:2]]
    h_mv = [torch.from_numpy(f.motion).pin_memory() for f in frames[:2]]
    h_out = [torch.empty((H, W, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
    d_rec = [torch.empty_like(dev_rec[0]) for _ in range(2)]
    d_gb = [torch.empty_like(dev_gb[0]) for _ in range(2)]
    d_mv = [torch.empty_like(dev_mv[0]) for _ in range(2)]
    d_g = [gi.make_gbuffer(g, W, H) for g in d_gb]
    d_irr = [torch.empty((H, W, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    e_steps = max(3, min(args.steps, 100))  # steady state: the pipeline fill and drain spread over 100 steps
    base = args.warmup + args.steps

    def e_up(j, b):
        d_rec[b].copy_(h_rec[j % 2], non_blocking=True)
        d_gb[b].copy_(h_gb[j % 2], non_blocking=True)
        d_mv[b].copy_(h_mv[j % 2], non_blocking=True)

    def e_frame(j, b):
        irr = tp.irr
        tp.irr = d_irr[b]
        step(base + j, None, d_rec[b], d_g[b], d_mv[b])
        tp.irr = irr

    def e_down(j, b):
        h_out[b].copy_(d_irr[b], non_blocking=True)

    e2e_ms = np.full(e_steps, e2e_pipelined(torch, e_steps, e_up, e_frame, e_down))
    h2d = h_rec[0].numel() * 4 + h_gb[0].numel() * 4 + h_mv[0].numel() * 4
    d2h = h_out[0].numel() * 4
    link = host_link(torch, [(d_rec[0], h_rec[0]), (d_gb[0], h_gb[0]), (d_mv[0], h_mv[0])], [(h_out[0], d_irr[0])])

    tot = np.array(max_over_ranks([window_ms.sum(), frame_ms.sum(), t_wall, e2e_ms.sum()], world, "cuda"))
    if rank != 0:
        tp.close()
        return
    value = aggregate_rate(R, world, args.steps, tot[0] / 1e3) / 1e6
    e2e_value = aggregate_rate(R, world, e_steps, tot[3] / 1e3) / 1e6
    pass_ms = per.mean(axis=0)
    peak, peak_src = _peaks()
    P = fr0.tiles_x * fr0.tiles_y
    X = W * H
    S = fr0.spawn_x * fr0.spawn_y
    alg = {
        # per pixel the 16 B G-buffer and 8 B motion vector; per tile the previous probe (mask 4 B,
        # position 16 B, normal 16 B) and the new one (36 B + 4 B source)
        "reproject": X * 24 + P * (36 + 40),
        # per tile the 16 B G-buffer texel of a fresh probe and 36 B written, the mask chain
        "spawn": P * 52,
        # as configuration 2, with the measured touched-cell count U of these frames
        "update": R * 44 + float(np.mean(U)) * (32 + 64 + 4),
        "resolve": float(np.mean(U)) * (4 + 64 + 2 * (8 if cfg["resolved_format"] == 1 else 16)),
        # per spawn-tile ray its slot id 4 B, ray length 4 B and a 16 B resolved gather; per tile the
        # previous atlas 1 KB read and the new one 1 KB written
        "gather_temporal": R * 24 + P * 2048,
        "project": P * (1024 + 16 + 112),
        "interpolate": X * 32 + P * 144,
    }
    if filtered:
        # per probe and cell the 16 B atlas entry read and written, 32 B of probe data per probe
        alg["filter_x"] = alg["filter_y"] = P * 64 * 32 + P * 32
    if tiles:
        # one more frame, counted: touched tiles and cells, live cells of the touched tiles
        i = args.warmup + args.steps + e_steps
        k = i % n_frames
        cur, prev = tp.bufs[tp.k], tp.bufs[tp.k ^ 1]
        gi.gi_probes_reproject(gbs[k], views[k], dev_mv[k], prev.struct, cur.struct, tp.src, stream)
        gi.gi_probes_spawn_upscaled(gbs[k], views[k], u, True, cur.struct, stream)
        gi.gi_cache_update(tp.cache, gi.hits_from_planes(dev_rec[k], R), views[k], tp.slot_ids, stream)
        ids = tp.slot_ids.cpu().numpy().view(np.uint32)
        ids = ids[ids < (1 << log2) * 64]
        touched_tiles = np.unique(ids >> 6)
        gi.gi_cache_resolve(tp.cache, i, stream)
        ex = gi.gi_cache_export(tp.cache)
        live_in = int(np.isin(ex["slot"] >> 6, touched_tiles).sum())
        ub, rb = tile_bytes(R, float(touched_tiles.size), int(np.unique(ids).size), live_in,
                            8 if cfg["resolved_format"] == 1 else 16, float(1 << log2))
        alg["update"], alg["resolve"] = ub, rb
    dominant = max((n for n in names if alg[n] > 0), key=lambda n: pass_ms[names.index(n)])
    d_ms = pass_ms[names.index(dominant)]
    achieved = alg[dominant] / (d_ms * 1e-3) / 1e9
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        Rs, ct = oracle_temporal_window(frames[:4], 3)
        cpu = {"value": Rs * len(ct) / sum(ct) / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"3 whole frames ({Rs} records each): reprojection, upscaled spawn, update + resolve, "
                         "frame atlas with Algorithm 4, SH projection; numpy float64 (float32 where the "
                         "reprojection's decisions need it), one thread"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(tot[1] / args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{cfg['name']}: {W}x{H} G-buffer, 2x2 temporal upscale: {S} spawn tiles x "
                               f"{fr0.rays_per_probe} rays = {R} hit records/frame for {P} probe tiles, "
                               f"{cfg['n_boxes']} boxes, "
                               + (f"two-level cache of 2^{log2} tiles (min_samples {cfg['min_samples']}), "
                                  if tiles else f"2^{log2} slots, ")
                               + ("probe filter (Algorithm 5), " if filtered else "")
                               + f"motion vectors from the analytic camera ({n_frames} frames cycled)",
                   "records_per_step": R, "pixels_per_step": X,
                   "l2": L2_NOTE,
                   "note": "value over update + resolve + temporal gather (+ filter) + SH projection; "
                           "ms_per_step is the whole frame (reprojection ... interpolation)"},
        "window_ms_per_step": float(tot[0] / args.steps),
        "pass_ms": {n: float(m) for n, m in zip(names, pass_ms)},
        "probes_valid_last_frame": valid, "probes_reprojected_last_frame": reproj, "probe_tiles": P,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": dominant, "algorithmic_bytes_per_launch": alg[dominant],
                     "peak_source": peak_src},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": float(tot[3] / e_steps), "steps": e_steps, "note": E2E_NOTE, "link": link},
        # k_reproject, k_spawn, k_mip_tail, the update (1 kernel, or 3 for tiles), the resolve,
        # k_gather_temporal, (2 x k_filter,) k_project, k_interpolate
        "gpu_launches": int(args.steps * (8 + (2 if tiles else 0) + (2 if filtered else 0)) + rebuilds),
        "rebuilds_in_timed_region": int(rebuilds),
        "dropped_hits": int(st["dropped"]),
        "clocks": clk,
        "wall_s_timed": float(tot[2]),
    }
    tp.close()
    return line


# ------------------------------------------------------------------ batched arm (many views)
def run_batched(args, rank, world, local_rank):
    """16 views of uneven resolution per frame: batched passes replayed from a CUDA graph (launch
    shapes from the autotuner), against the same views run one after another through the
    single-view calls."""
    import torch
    import paper_2310_19855_gb300 as gi
    from paper_2310_19855_gb300 import autotune
    from paper_2310_19855_gb300.build import build
    from paper_2310_19855_gb300.pipeline import BatchPipeline, Pipeline, view_of
    from paper_2310_19855_gb300.replicas import aggregate_rate, barrier, frame_indices, max_over_ranks
    import workload as wl
    import workload.scene as wscene

    build()
    wscene.build_tracer()
    torch.cuda.set_device(local_rank)
    specs = wl.batched_views(wl.CONFIGS[3]["n_views"])
    F = max(1, min(args.frames, 2))
    frames = []
    for cfg, seed in specs:
        scene = wl.make_scene(cfg, seed)
        frames.append([wl.make_frame(cfg, g, scene, seed_base=seed) for g in frame_indices(rank, F, cfg["frames"])])
    V = len(specs)
    recs = [[torch.from_numpy(np.ascontiguousarray(frames[v][k].records[:10])).cuda() for v in range(V)]
            for k in range(F)]
    gbufs = [[torch.from_numpy(frames[v][k].gbuffer).cuda() for v in range(V)] for k in range(F)]
    gviews = [[view_of(frames[v][k].camera, frames[v][k].frame) for v in range(V)] for k in range(F)]
    R_total = sum(frames[v][0].n_records for v in range(V))
    X_total = sum(cfg["width"] * cfg["height"] for cfg, _ in specs)
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()

    bp = BatchPipeline([(cfg["width"], cfg["height"], cfg["log2_slots"]) for cfg, _ in specs], 64)
    counter = [0]

    def batched_frame(use_graph=True):
        k = counter[0]
        bp.frame(gbufs[k % F], recs[k % F], gviews[k % F], use_graph=use_graph, stream=stream, resolve_frame=k)
        counter[0] += 1

    tuning, timings = autotune.tune(bp, batched_frame, frames=3)

    def timed(fn, steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for j in range(steps):
            flush.zero_()
            evs[j][0].record(stream)
            fn()
            evs[j][1].record(stream)
        torch.cuda.synchronize()
        return np.array([a.elapsed_time(b) for a, b in evs])

    for _ in range(args.warmup):
        batched_frame(True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    barrier(world)
    clocks.start()
    time.sleep(0.5)
    torch.cuda.synchronize()
    t0 = time.time()
    ms_graph = timed(lambda: batched_frame(True), args.steps)
    clk = clocks.stop(t0, time.time())
    barrier(world)
    ms_nograph = timed(lambda: batched_frame(False), max(3, min(args.steps, 50)))

    # the same views one after another through the single-view calls (own caches)
    singles = [Pipeline(cfg["width"], cfg["height"], 64, cfg["log2_slots"]) for cfg, _ in specs]
    scount = [0]

    def sequential_frame():
        k = scount[0]
        for v in range(V):
            sp = singles[v]
            sp.spawn(gbufs[k % F][v], gviews[k % F][v], stream)
            gi.gi_cache_update(sp.cache, gi.hits_from_planes(recs[k % F][v], sp.n_records), gviews[k % F][v],
                               sp.slot_ids, stream)
            sp.resolve(k, stream)
            sp.integrate((0.0, 0.0, 0.0), stream)
            sp.interpolate(gbufs[k % F][v], gviews[k % F][v], stream)
        scount[0] += 1

    for _ in range(args.warmup):
        sequential_frame()
    ms_seq = timed(sequential_frame, max(3, min(args.steps, 50)))
    for sp in singles:
        sp.close()
    surr = batched_surrogate(args, gi, torch, BatchPipeline, specs, frames, recs, gbufs, gviews, bp, counter, F, V,
                             timed, stream)
    tot = np.array(max_over_ranks([ms_graph.sum(), ms_nograph.mean(), ms_seq.mean()], world, "cuda"))
    bp.close()
    if rank != 0:
        return
    value = aggregate_rate(R_total, world, args.steps, tot[0] / 1e3) / 1e6
    frame_ms = tot[0] / args.steps
    peak, peak_src = _peaks()
    # whole-frame algorithmic bytes (same per-unit figures as the single-view bench, U not measured
    # here: 0.4 touched cells per record, the 1080p workload's ratio)
    U = 0.4 * R_total
    P = R_total / 64
    alg = (R_total * 44 + U * 100) + U * 100 + (R_total * 20 + P * 128) + (X_total * 32 + P * 144) + P * 52
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(frame_ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: {V} views ("
                               + ", ".join(f"{c['width']}x{c['height']}" for c, _ in specs)
                               + f"), {R_total} records and {X_total} pixels per frame, one launch per pass "
                                 "over all views, CUDA-graph replay",
                   "records_per_step": R_total, "pixels_per_step": X_total,
                   "l2": L2_NOTE,
                   "tuning": {"update_records_per_block": tuning.update_records_per_block,
                              "resolve_blocks_per_sm": tuning.resolve_blocks_per_sm,
                              "integrate_threads": tuning.integrate_threads},
                   "note": "value and ms_per_step over the whole frame of all views (spawn ... interpolation)"},
        "frames_per_s": {"batched_graph": 1e3 / frame_ms, "batched_no_graph": 1e3 / tot[1],
                         "sequential_single_view_calls": 1e3 / tot[2]},
        "ms_per_frame": {"batched_graph": float(frame_ms), "batched_no_graph": float(tot[1]),
                         "sequential_single_view_calls": float(tot[2])},
        "autotune_ms": timings,
        "roofline": {"bound": "hbm", "achieved": alg / (frame_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / (frame_ms * 1e-3) / 1e9 / peak, "traffic": None,
                     "kernel": "whole batched frame (six launches)", "algorithmic_bytes_per_launch": alg,
                     "peak_source": peak_src},
        "surrogate_batched": surr,
        "cpu_baseline": None,
        "gpu_launches": int(args.steps * 7),
        "clocks": clk,
    }
    return line


def lr_step(gi, nrcs, lr0, i, total):
    """Adam's step size of the online training at step i of `total`: lr0 over the first half, a
    quarter of it over the third quarter, a sixteenth over the last (gi_nrc_set_learning_rate).
    Used by the blocks that train for 2048 steps (configuration 3's per-view networks, 4-far: 0.9 %
    and 4.1 % error on the routed hits against 2.9 % and 6.7 % at a constant step size); the
    Cornell block's 128 setup frames keep the configuration's step size (6.3 % with this schedule
    against 4.3 % without)."""
    if total >= 4 and i in (total // 2, (3 * total) // 4):
        lr = lr0 / (4.0 if i == total // 2 else 16.0)
        for nrc in nrcs:
            if nrc is not None:
                gi.gi_nrc_set_learning_rate(nrc, lr)


def batched_surrogate(args, gi, torch, BatchPipeline, specs, frames, recs, gbufs, gviews, bp, counter, F, V, timed,
                      stream):
    """The surrogate-plus-batched form on the same 16 views: each view its own network (configuration
    4's size, over the box of the view's hits; the views are distinct scenes in the same world box,
    which one network cannot fit), trained online on the plain batch's cache of its view over
    `rounds` rounds of one plain batched frame and one training call per view (after 64 rounds,
    only the views that route hits keep their network); then a second batch
    whose caches route hits of LOD >= 2 to their view's network (trust set to 1 so that the routing
    takes place) and whose probe pass takes its answers (gi_batch_set_view_surrogates: the query
    frame and the probe pass per view), timed against the plain batch with and without the graph;
    one round of training calls timed on its own.  The networks' error on the routed hits of every
    view, against the plain batch's cells of the same records, is reported."""
    import workload as wl
    cfg4 = wl.CONFIGS[4]
    rounds = 2048 if args.setup_frames is None else max(1, args.setup_frames)
    nets = []
    try:
        for v in range(V):
            pv = np.concatenate([frames[v][k].records[0:3, np.isfinite(frames[v][k].records[9])] for k in range(F)],
                                axis=1)
            lo, hi = tuple(pv.min(axis=1) - 0.5), tuple(pv.max(axis=1) + 0.5)
            n_v = frames[v][0].n_records
            ncfg = gi.make_nrc_config(lo, hi, log2_table=cfg4["nrc_log2_table"], resolutions=cfg4["nrc_resolutions"],
                                      lr=cfg4["nrc_lr"], batch=cfg4["nrc_batch"], train_steps=cfg4["nrc_train_steps"],
                                      max_records=n_v, max_queries=min(n_v, gi.GI_NRC_MAX_BATCH), trust=1.0,
                                      query_lod=4, seed=1 + v)
            nets.append(gi.gi_nrc_create(ncfg))
        return _batched_surrogate_run(args, gi, torch, BatchPipeline, specs, frames, recs, gbufs, gviews, bp,
                                      counter, F, V, timed, stream, nets, rounds)
    finally:
        for nrc in nets:
            gi.gi_nrc_destroy(nrc)


def _batched_surrogate_run(args, gi, torch, BatchPipeline, specs, frames, recs, gbufs, gviews, bp, counter, F, V,
                           timed, stream, nets, rounds):
    import workload as wl
    bs = BatchPipeline([(cfg["width"], cfg["height"], cfg["log2_slots"]) for cfg, _ in specs], 64)
    scount = [0]
    tcount = [0]

    def plain_frame():
        k = counter[0]
        bp.frame(gbufs[k % F], recs[k % F], gviews[k % F], use_graph=True, stream=stream, resolve_frame=k)
        counter[0] += 1

    def train_round():
        # one training call per view that keeps a network, on the plain batch's latest frame (its
        # records and slot ids)
        k = counter[0] - 1
        for v in range(V):
            if active[v] is None:
                continue
            st = bp.views[v]
            gi.gi_nrc_train_frame(active[v], st["cache"], gi.hits_from_planes(recs[k % F][v], st["n_records"]),
                                  st["slot_ids"], tcount[0], stream)
        tcount[0] += 1

    def surrogate_frame():
        k = scount[0]
        bs.frame(gbufs[k % F], recs[k % F], gviews[k % F], stream=stream, resolve_frame=k)
        scount[0] += 1

    active = list(nets)
    try:
        # every view's network first; then only those of the views that route hits to them
        t0 = time.time()
        first = min(rounds, 64)
        for _ in range(first):
            plain_frame()
            train_round()
        bs.set_view_surrogates(nets, far_lod=2)
        surrogate_frame()
        torch.cuda.synchronize()
        active = [nets[v] if np.any(st["slot_ids"].cpu().numpy().view(np.uint32) == gi.GI_SLOT_FAR) else None
                  for v, st in enumerate(bs.views)]
        bs.set_view_surrogates(active, far_lod=2)
        for r in range(first, rounds):
            lr_step(gi, active, float(wl.CONFIGS[4]["nrc_lr"]), r, rounds)
            plain_frame()
            train_round()
        torch.cuda.synchronize()
        setup_s = time.time() - t0
        steps = max(3, min(args.steps, 20))
        for _ in range(args.warmup):
            surrogate_frame()
        ms_surr = timed(surrogate_frame, steps)
        # the routed hits of every view's last frame; the plain batch on the same inputs
        k = scount[0] - 1
        bp.frame(gbufs[k % F], recs[k % F], gviews[k % F], use_graph=True, stream=stream, resolve_frame=counter[0])
        counter[0] += 1
        torch.cuda.synchronize()
        far_v = [st["slot_ids"].cpu().numpy().view(np.uint32) == gi.GI_SLOT_FAR for st in bs.views]
        routed = sum(int(f.sum()) for f in far_v)
        # what a viewer sees: the interpolated irradiance of the two batches on the same frame
        i_num = i_den = 0.0
        for v in range(V):
            a_s = bs.views[v]["irr"][..., :3].double()
            a_p = bp.views[v]["irr"][..., :3].double()
            i_num += float((a_s - a_p).abs().sum())
            i_den += float(a_p.abs().sum())
        hits = sum(int(np.count_nonzero(np.isfinite(frames[v][k % F].records[9]))) for v in range(V))
        # every view's query frame again (untimed): its network's answers against the plain batch's
        # cells of the same records
        num = den = 0.0
        per_view = []
        for v in range(V):
            sv, pv = bs.views[v], bp.views[v]
            R = pv["n_records"]
            if active[v] is None or not far_v[v].any():
                continue
            gi.gi_nrc_query_frame(nets[v], sv["cache"], gi.hits_from_planes(recs[k % F][v], R), sv["slot_ids"],
                                  gviews[k % F][v], stream)
            cnt = gi.gi_nrc_answers(nets[v], stream=stream)
            rec_ids = torch.empty(max(cnt, 1), dtype=torch.int32, device="cuda")
            rads = torch.empty((max(cnt, 1), 4), dtype=torch.float32, device="cuda")
            gi.gi_nrc_answers(nets[v], rec_ids, rads, cnt, stream=stream)
            ids = rec_ids.cpu().numpy().view(np.uint32)[:cnt]
            ans = rads.cpu().numpy()[:cnt, :3]
            cache_val = torch.empty((R, 4), dtype=torch.float32, device="cuda")
            gi.gi_cache_query(pv["cache"], cache_val, R, slot_ids=pv["slot_ids"])
            ref_all = cache_val.cpu().numpy()
            sel = far_v[v][ids] & (ref_all[ids, 3] == 1.0)
            ref = ref_all[ids[sel], :3]
            e_num, e_den = float(np.abs(ans[sel] - ref).sum()), float(np.abs(ref).sum())
            num, den = num + e_num, den + e_den
            per_view.append({"view": v, "routed": int(far_v[v].sum()), "compared": int(sel.sum()),
                             "rel_l1": e_num / e_den if e_den > 0 else None})
        judged = [float(gi.gi_nrc_stats(nrc, stream)["judged_error"]) for nrc in active if nrc is not None]
        ms_train = timed(train_round, steps)
    finally:
        bs.set_view_surrogates(None)
        bs.close()
    s_ms, t_ms = float(ms_surr.mean()), float(ms_train.mean())
    return {
        "note": f"gi_batch_set_view_surrogates on the same {V} views: one network per view (each view is its own "
                "scene), hits of LOD >= 2 routed to it (trust set to 1), the probe pass per view through its "
                "answers (query frame + probe pass), the other passes one launch over all views, no graph; each "
                f"network trained online on its view of the plain batch, {rounds} rounds of one plain frame and "
                f"one training call per view (after the first {first} rounds only the views that route hits keep "
                "their network; the others take the plain probe pass); one round of training calls timed on its "
                "own",
        "views_with_a_network": [v for v in range(V) if active[v] is not None],
        "ms_per_frame": {"surrogate_batched": s_ms, "training_round_views_with_a_network": t_ms},
        "frames_per_s": {"surrogate_batched_without_training": 1e3 / s_ms,
                         "surrogate_batched_with_one_training_round": 1e3 / (s_ms + t_ms)},
        "routed_hits_per_frame": routed, "hits_per_frame": hits,
        "network_rel_l1_error_on_routed_hits_vs_plain_cache": num / den if den > 0 else None,
        "per_view_error": per_view,
        "irradiance_rel_l1_vs_plain_batch": i_num / i_den if i_den > 0 else None,
        "judged_error_max_over_views": max(judged),
        "training_rounds": rounds, "setup_s": setup_s,
        # six batched passes, and per view with a network its query frame (selection, encoding,
        # network) and its probe pass with answers
        "gpu_launches_per_frame": 6 + 4 * sum(nrc is not None for nrc in active),
    }


# ------------------------------------------------------------------ surrogate arm (configuration 4)
def run_surrogate(args, rank, world, local_rank):
    """The Cornell box at 1080p with the learned surrogate: per frame spawn, update, resolve, one
    training call (65,536 resolved cells in 4 minibatches, each with its Adam step), the query
    frame (cold cells, dropped inserts, LOD >= 2 answered by the network while it is trusted),
    probe irradiance with those answers, interpolation -- against the plain frame on its own
    cache.  The network is first trained over the configuration's 128 frames (untimed setup)."""
    import torch
    import paper_2310_19855_gb300 as gi
    from paper_2310_19855_gb300.build import build
    from paper_2310_19855_gb300.pipeline import Pipeline, view_of
    from paper_2310_19855_gb300.replicas import aggregate_rate, barrier, max_over_ranks
    import workload as wl
    import workload.scene as wscene

    build()
    wscene.build_tracer()
    torch.cuda.set_device(local_rank)
    cfg = wl.CONFIGS[4]
    n_frames = min(args.frames, args.steps + args.warmup)
    frames = make_frames(n_frames, rank)
    fr0 = frames[0]
    W, H, R, rpp = fr0.camera.width, fr0.camera.height, fr0.n_records, fr0.rays_per_probe
    lo, hi = wl.surrogate_inputs.CORNELL_AABB
    ncfg = gi.make_nrc_config(lo, hi, log2_table=cfg["nrc_log2_table"], resolutions=cfg["nrc_resolutions"],
                              lr=cfg["nrc_lr"], batch=cfg["nrc_batch"], train_steps=cfg["nrc_train_steps"],
                              max_records=R, max_queries=min(R, gi.GI_NRC_MAX_BATCH), trust=cfg["nrc_trust"],
                              query_lod=cfg["nrc_query_lod"],
                              seed=1)
    nrc = gi.gi_nrc_create(ncfg)
    ps = Pipeline(W, H, rpp, cfg["log2_slots"])  # surrogate form
    pp = Pipeline(W, H, rpp, cfg["log2_slots"])  # plain form
    dev_rec = [torch.from_numpy(np.ascontiguousarray(f.records[:10])).cuda() for f in frames]
    dev_gb = [torch.from_numpy(f.gbuffer).cuda() for f in frames]
    views = [view_of(f.camera, f.frame) for f in frames]
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()
    s_names = ["spawn", "update", "resolve", "train", "query", "integrate", "interpolate"]
    p_names = ["spawn", "update", "resolve", "integrate", "interpolate"]

    def surr_step(i, ev=None):
        k = i % n_frames
        gb, rec, v = dev_gb[k], dev_rec[k], views[k]
        hits = gi.hits_from_planes(rec, R)
        mark = (lambda j: ev[j].record(stream)) if ev is not None else (lambda j: None)
        mark(0)
        ps.spawn(gb, v, stream)
        mark(1)
        gi.gi_cache_update(ps.cache, hits, v, ps.slot_ids, stream)
        mark(2)
        ps.resolve(i, stream)
        mark(3)
        gi.gi_nrc_train_frame(nrc, ps.cache, hits, ps.slot_ids, i, stream)
        mark(4)
        gi.gi_nrc_query_frame(nrc, ps.cache, hits, ps.slot_ids, v, stream)
        mark(5)
        gi.gi_probes_integrate_nrc(ps.cache, nrc, ps.probes.struct, ps.slot_ids, rpp, (0.0, 0.0, 0.0), stream)
        mark(6)
        ps.interpolate(gb, v, stream)
        mark(7)

    def plain_step(i, ev=None):
        k = i % n_frames
        gb, rec, v = dev_gb[k], dev_rec[k], views[k]
        mark = (lambda j: ev[j].record(stream)) if ev is not None else (lambda j: None)
        mark(0)
        pp.spawn(gb, v, stream)
        mark(1)
        gi.gi_cache_update(pp.cache, gi.hits_from_planes(rec, R), v, pp.slot_ids, stream)
        mark(2)
        pp.resolve(i, stream)
        mark(3)
        pp.integrate((0.0, 0.0, 0.0), stream)
        mark(4)
        pp.interpolate(gb, v, stream)
        mark(5)

    # setup: the configuration's frames of online training (both caches see the same frames)
    setup = cfg["frames"] if args.setup_frames is None else args.setup_frames
    judged = []
    for i in range(setup):
        surr_step(i)
        plain_step(i)
        if i % 16 == 15:
            judged.append(round(gi.gi_nrc_stats(nrc, stream)["judged_error"], 4))
    for i in range(setup, setup + args.warmup):
        surr_step(i)
        plain_step(i)
    torch.cuda.synchronize()

    def timed(fn, names, start):
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(args.steps)]
        for j in range(args.steps):
            flush.zero_()
            fn(start + j, evs[j])
        torch.cuda.synchronize()
        return np.array([[evs[j][k].elapsed_time(evs[j][k + 1]) for k in range(len(names))]
                         for j in range(args.steps)])

    clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    barrier(world)
    clocks.start()
    time.sleep(0.5)
    torch.cuda.synchronize()
    t0 = time.time()
    base = setup + args.warmup
    s_per = timed(surr_step, s_names, base)
    clk = clocks.stop(t0, time.time())
    p_per = timed(plain_step, p_names, base)
    # both caches now hold the same frames: the last frame of each form, compared
    last = base + args.steps - 1
    st = gi.gi_nrc_stats(nrc, stream)
    answered = gi.gi_nrc_answers(nrc)
    irr_s, irr_p = ps.irr.cpu().numpy(), pp.irr.cpu().numpy()
    surf = irr_p[..., 3] < 3
    form_err = float(np.abs(irr_s[surf, :3] - irr_p[surf, :3]).sum() / max(np.abs(irr_p[surf, :3]).sum(), 1e-30))
    # the network against the cache at every hit of the last frame
    fl = frames[last % n_frames]
    hit = np.isfinite(fl.records[9]) & (fl.records[9] >= 0)
    cache_val = torch.empty((R, 4), dtype=torch.float32, device="cuda")
    gi.gi_cache_query(ps.cache, cache_val, R, slot_ids=ps.slot_ids)
    Pd = torch.from_numpy(np.ascontiguousarray(fl.records[0:3, hit])).cuda()
    Nd = torch.from_numpy(np.ascontiguousarray(fl.records[3:6, hit])).cuda()
    nh = int(hit.sum())
    net = torch.empty((nh, 4), dtype=torch.float32, device="cuda")
    gi.gi_nrc_infer(nrc, gi.make_points(Pd, Nd, nh), net)
    ref = cache_val.cpu().numpy()[hit, :3]
    net_err = float(np.abs(net.cpu().numpy()[:, :3] - ref).sum() / np.abs(ref).sum())

    # ---- the table's Adam step alone (the surrogate's HBM-bound kernel), after a backward pass
    mb = cfg["nrc_batch"] // cfg["nrc_train_steps"]
    sel = np.flatnonzero(hit)[:mb]
    Pb = torch.from_numpy(np.ascontiguousarray(fl.records[0:3, sel])).cuda()
    Nb = torch.from_numpy(np.ascontiguousarray(fl.records[3:6, sel])).cuda()
    Tb = cache_val[torch.from_numpy(sel).cuda(), :3].T.contiguous()
    pts = gi.make_points(Pb, Nb, sel.size)
    gi.gi_nrc_backward(nrc, pts, [Tb[0], Tb[1], Tb[2]])
    gtab = gi.gi_nrc_get_gradients(nrc, cfg["nrc_log2_table"])[0]
    touched = np.any(gtab != 0, axis=2).reshape(-1)
    n_touched = int(touched.sum())
    n_groups = int(touched.reshape(-1, 4).any(axis=1).sum())
    gi.gi_nrc_adam(nrc, stream)
    a_ev = []
    for _ in range(20):
        gi.gi_nrc_backward(nrc, pts, [Tb[0], Tb[1], Tb[2]], None, 0, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        gi.gi_nrc_adam(nrc, stream)
        e1.record(stream)
        a_ev.append((e0, e1))
    torch.cuda.synchronize()
    adam_ms = float(np.mean([a.elapsed_time(b) for a, b in a_ev]))
    entries = 16 << cfg["nrc_log2_table"]
    # gradient scan 8 B per entry; per touched entry its 32 B record read and written and the 4 B
    # float16 copy; 32 B of cleared gradients per touched group of 4 entries
    adam_bytes = 8 * entries + n_touched * 68 + n_groups * 32
    gi.gi_nrc_destroy(nrc)
    ps.close()
    pp.close()

    s_ms, p_ms = s_per.sum(axis=1), p_per.sum(axis=1)
    tot = np.array(max_over_ranks([s_ms.sum(), p_ms.sum()], world, "cuda"))
    if rank != 0:
        return
    value = aggregate_rate(R, world, args.steps, tot[0] / 1e3) / 1e6
    peak, peak_src = _peaks()
    achieved = adam_bytes / (adam_ms * 1e-3) / 1e9
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(frames, args.sample)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(tot[0] / args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 cache, bf16 network (f32 accumulate)",
        "data": "synthetic",
        "config": {"workload": f"{cfg['name']}: {W}x{H} G-buffer of the Cornell box, {fr0.tiles_x * fr0.tiles_y} "
                               f"probes x {rpp} rays = {R} records/frame, 2^{cfg['log2_slots']} slots; surrogate "
                               f"16 levels x 2^{cfg['nrc_log2_table']} entries x 2 fp16 features, 32-64-64-3 "
                               f"bf16 network, {cfg['nrc_batch']} training cells/frame in "
                               f"{cfg['nrc_train_steps']} Adam steps, queried for cold cells, dropped inserts "
                               f"and LOD >= {cfg['nrc_query_lod']} while its judged error <= {cfg['nrc_trust']}",
                   "records_per_step": R, "pixels_per_step": W * H,
                   "l2": L2_NOTE,
                   "setup": f"{setup} frames of online training before the warm-up (untimed)",
                   "note": "value and ms_per_step: whole surrogate-form frame; frames_per_s compares the forms"},
        "frames_per_s": {"surrogate_form": 1e3 * args.steps / tot[0], "plain_form": 1e3 * args.steps / tot[1]},
        "pass_ms": {"surrogate_form": {n: float(m) for n, m in zip(s_names, s_per.mean(axis=0))},
                    "plain_form": {n: float(m) for n, m in zip(p_names, p_per.mean(axis=0))}},
        "surrogate": {"network_rel_l1_error_vs_cache": net_err, "judged_error": float(st["judged_error"]),
                      "trusted": int(st["trusted"]), "records_answered_last_frame": int(answered),
                      "irradiance_rel_l1_vs_plain_form": form_err, "judged_error_every_16_setup_frames": judged,
                      "adam_steps": int(st["steps"]),
                      "note": "errors against the float32 cache, which matches the float64 oracle cache to 1e-4 "
                              "(parity tests); the float64-oracle comparison of the network is in the tests"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic("4:adam_table"), "kernel": "k_nrc_adam_table (sparse Adam on the hash table)",
                     "algorithmic_bytes_per_launch": adam_bytes, "touched_entries": n_touched,
                     "launch_ms": adam_ms, "peak_source": peak_src},
        "cpu_baseline": cpu,
        # per surrogate-form frame: spawn 2, update, resolve, 5 per training minibatch (encode, network,
        # scatter, two Adam kernels), query 3 (select, encode, network), integrate, interpolate;
        # per plain frame 6
        "gpu_launches": int(args.steps * ((9 + 5 * cfg["nrc_train_steps"]) + 6)),
        "clocks": clk,
    }
    return line


FAR_SETUP_FRAMES = 2048  # online training of the far-hit network before the timed frames


def run_far_routing(args, rank, world, local_rank):
    """Far hits to the surrogate on the boxes at 1080p (15 % of the hits have LOD >= 2): a network
    trained online on a plain cache (the configuration's level schedule over the room) for
    FAR_SETUP_FRAMES frames (4 cycled frames: ~1.2 s), then per
    frame the plain form (update, resolve, probe irradiance) against the routed form (update with
    LOD >= 2 hits left out of the table, resolve, query frame answering them, probe irradiance with
    the answers), each on its own cache over the same frames; the training call timed on its own.
    The trust threshold is set to 1 so that the routing takes place whatever the network's error;
    that error, on the routed hits against the plain cache's values of their cells, is reported."""
    import torch
    import paper_2310_19855_gb300 as gi
    from paper_2310_19855_gb300.pipeline import Pipeline, view_of
    import workload as wl

    global CONFIG
    CONFIG = 2
    cfg2, cfg4 = wl.CONFIGS[2], wl.CONFIGS[4]
    n_frames = min(args.frames, args.steps + args.warmup)
    frames = make_frames(n_frames, rank)
    fr0 = frames[0]
    W, H, R, rpp = fr0.camera.width, fr0.camera.height, fr0.n_records, fr0.rays_per_probe
    # the box the network normalises positions into: every hit point of the frames, 0.5 m margin
    allp = np.concatenate([f.records[0:3, np.isfinite(f.records[9])] for f in frames], axis=1)
    lo, hi = tuple(allp.min(axis=1) - 0.5), tuple(allp.max(axis=1) + 0.5)
    ncfg = gi.make_nrc_config(lo, hi, log2_table=cfg4["nrc_log2_table"], resolutions=cfg4["nrc_resolutions"],
                              lr=cfg4["nrc_lr"], batch=cfg4["nrc_batch"], train_steps=cfg4["nrc_train_steps"],
                              max_records=R, max_queries=min(R, gi.GI_NRC_MAX_BATCH), trust=1.0, query_lod=4,
                              seed=1)
    nrc = gi.gi_nrc_create(ncfg)
    pp = Pipeline(W, H, rpp, cfg2["log2_slots"])   # plain form
    pr = Pipeline(W, H, rpp, cfg2["log2_slots"])   # routed form
    dev_rec = [torch.from_numpy(np.ascontiguousarray(f.records[:10])).cuda() for f in frames]
    dev_gb = [torch.from_numpy(f.gbuffer).cuda() for f in frames]
    views = [view_of(f.camera, f.frame) for f in frames]
    flush = L2Flush(torch)
    stream = torch.cuda.current_stream()
    try:
        def plain(i, ev=None):
            k = i % n_frames
            mark = (lambda j: ev[j].record(stream)) if ev is not None else (lambda j: None)
            pp.spawn(dev_gb[k], views[k], stream)
            mark(0)
            gi.gi_cache_update(pp.cache, gi.hits_from_planes(dev_rec[k], R), views[k], pp.slot_ids, stream)
            mark(1)
            pp.resolve(i, stream)
            mark(2)
            pp.integrate((0.0, 0.0, 0.0), stream)
            mark(3)

        def routed(i, ev=None):
            k = i % n_frames
            hits = gi.hits_from_planes(dev_rec[k], R)
            mark = (lambda j: ev[j].record(stream)) if ev is not None else (lambda j: None)
            pr.spawn(dev_gb[k], views[k], stream)
            mark(0)
            gi.gi_cache_update(pr.cache, hits, views[k], pr.slot_ids, stream)
            mark(1)
            pr.resolve(i, stream)
            mark(2)
            gi.gi_nrc_query_frame(nrc, pr.cache, hits, pr.slot_ids, views[k], stream)
            mark(3)
            gi.gi_probes_integrate_nrc(pr.cache, nrc, pr.probes.struct, pr.slot_ids, rpp, (0.0, 0.0, 0.0), stream)
            mark(4)

        def train(i, ev=None):
            k = i % n_frames
            if ev is not None:
                ev[0].record(stream)
            gi.gi_nrc_train_frame(nrc, pp.cache, gi.hits_from_planes(dev_rec[k], R), pp.slot_ids, i, stream)
            if ev is not None:
                ev[1].record(stream)

        setup = FAR_SETUP_FRAMES if args.setup_frames is None else max(1, args.setup_frames)
        for i in range(setup):
            lr_step(gi, [nrc], float(cfg4["nrc_lr"]), i, setup)
            plain(i)
            train(i)
        gi.gi_cache_route_far(pr.cache, nrc, 2)
        for i in range(setup, setup + args.warmup):
            plain(i)
            routed(i)
            train(i)
        torch.cuda.synchronize()
        steps = args.steps
        ev_p = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        ev_r = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        ev_t = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
        clocks = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
        clocks.start()
        time.sleep(0.5)
        torch.cuda.synchronize()
        t0 = time.time()
        base = setup + args.warmup
        for j in range(steps):
            flush.zero_()
            plain(base + j, ev_p[j])
            flush.zero_()
            routed(base + j, ev_r[j])
            flush.zero_()
            train(base + j, ev_t[j])
        torch.cuda.synchronize()
        clk = clocks.stop(t0, time.time())
        pm = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(3)] for e in ev_p]).mean(axis=0)
        rm = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(4)] for e in ev_r]).mean(axis=0)
        tm = float(np.mean([e[0].elapsed_time(e[1]) for e in ev_t]))
        # the routed hits of the last frame: the network's answers against the plain cache's cells
        ids_r = pr.slot_ids.cpu().numpy().view(np.uint32)
        far = ids_r == gi.GI_SLOT_FAR
        cnt = gi.gi_nrc_answers(nrc)
        recs = torch.empty(max(cnt, 1), dtype=torch.int32, device="cuda")
        rads = torch.empty((max(cnt, 1), 4), dtype=torch.float32, device="cuda")
        gi.gi_nrc_answers(nrc, recs, rads, cnt)
        rec_ids = recs.cpu().numpy().view(np.uint32)[:cnt]
        ans = rads.cpu().numpy()[:cnt, :3]
        cache_val = torch.empty((R, 4), dtype=torch.float32, device="cuda")
        gi.gi_cache_query(pp.cache, cache_val, R, slot_ids=pp.slot_ids)
        ref_all = cache_val.cpu().numpy()
        sel = far[rec_ids] & (ref_all[rec_ids, 3] == 1.0)
        ref = ref_all[rec_ids[sel], :3]
        net_err = float(np.abs(ans[sel] - ref).sum() / max(np.abs(ref).sum(), 1e-30))
        st = gi.gi_nrc_stats(nrc, stream)
    finally:
        gi.gi_cache_route_far(pr.cache, None, 4)
        pp.close()
        pr.close()
        gi.gi_nrc_destroy(nrc)
    if rank != 0:
        return None
    plain_ms, routed_ms = float(pm.sum()), float(rm.sum())
    return {
        "metric": "update + resolve + probe irradiance with far hits routed to the surrogate, against the plain form",
        "value": R / (routed_ms * 1e-3) / 1e6, "unit": UNIT, "steps": steps, "ms_per_step": routed_ms,
        "dtype": "f32 cache, bf16 network (f32 accumulate)",
        "config": {"workload": f"boxes-1080p: {W}x{H}, {R} records/frame, 2^{cfg2['log2_slots']} slots; network "
                               f"16 levels x 2^{cfg4['nrc_log2_table']} entries over the hits' box, trained online for "
                               f"{setup} frames on the plain cache; hits with LOD >= 2 routed (trust set to 1)",
                   "records_per_step": R, "l2": L2_NOTE},
        "pass_ms": {"plain_form": {"update": float(pm[0]), "resolve": float(pm[1]), "integrate": float(pm[2])},
                    "routed_form": {"update": float(rm[0]), "resolve": float(rm[1]), "query": float(rm[2]),
                                    "integrate_with_answers": float(rm[3])},
                    "training_call": tm},
        "frames_per_s": {"plain_form": 1e3 / plain_ms, "routed_form_without_training": 1e3 / routed_ms,
                         "routed_form_with_training": 1e3 / (routed_ms + tm)},
        "routed_hits_last_frame": int(far.sum()), "answered_last_frame": int(cnt),
        "network_rel_l1_error_on_routed_hits_vs_plain_cache": net_err,
        "judged_error": float(st["judged_error"]),
        "gpu_launches": int(steps * (4 + 7 + 5 * cfg4["nrc_train_steps"])),
        "clocks": clk,
    }


def run_config(config, args, rank, world, local_rank):
    """One configuration's run; its JSON line (rank 0) or None."""
    global CONFIG
    CONFIG = config
    if config == 3:
        return run_batched(args, rank, world, local_rank)
    if config == 4:
        return run_surrogate(args, rank, world, local_rank)
    if config in (6, 7):
        return run_temporal(args, rank, world, local_rank)
    return run_native(args, rank, world, local_rank)


# keys of a configuration's line that its compact block in the default line leaves out
SUB_DROP = ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data", "cpu_baseline", "warmup",
            "probe_filter", "tiles")
SUB_STEPS, SUB_WARMUP, SUB_FRAMES = 20, 5, 4


def other_configs(args, rank, world, local_rank):
    """Compact runs of configurations 5 (4K), 6 (temporal upscale), 7 (the whole chain), 3 (16
    batched views) and 4 (the learned surrogate) after the default configuration, each with its own
    events, roofline and clock record: at most SUB_STEPS timed steps over SUB_FRAMES cycled frames,
    no CPU baseline and no end-to-end arm (the default line carries those)."""
    import argparse as _ap
    import torch
    out = {}
    for c in (5, 6, 7, 3, 4, "4-far"):
        sub = _ap.Namespace(**vars(args))
        sub.steps, sub.warmup = min(args.steps, SUB_STEPS), min(max(args.warmup, 3), SUB_WARMUP)
        sub.frames, sub.no_cpu_baseline, sub.sub = SUB_FRAMES, True, True
        t0 = time.perf_counter()
        if c == "4-far":
            line = run_far_routing(sub, rank, world, local_rank)
        else:
            line = run_config(c, sub, rank, world, local_rank)
        torch.cuda.empty_cache()
        if line is None:
            continue
        block = {k: v for k, v in line.items() if k not in SUB_DROP}
        block["metric"] = line["metric"] if c != 3 else "frames/s of 16 batched views"
        block["wall_s"] = time.perf_counter() - t0
        out[str(c)] = block
    global CONFIG
    CONFIG = 2
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--frames", type=int, default=N_FRAMES_DEFAULT, help="distinct pre-generated frames to cycle")
    ap.add_argument("--sample", type=float, default=0.125, help="fraction of probes in the oracle's sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--setup-frames", type=int, default=None,
                    help="configuration 4: frames of online training before the warm-up (default: the "
                         "configuration's 128); configuration 3: training rounds of the per-view networks "
                         "(default 2048); block 4-far: frames of online training (default 2048)")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="configuration 2: skip the compact runs of configurations 3-7 added to its line")
    ap.add_argument("--config", type=int, default=2, choices=[2, 3, 4, 5, 6, 7],
                    help="2: boxes at 1080p (default); 3: 16 batched views; 4: Cornell box at 1080p with the "
                         "learned surrogate; 5: boxes at 4K, 2^24 slots, FP16 resolved radiance; 6: boxes at "
                         "1080p with 2x2 temporal upscale, probe reprojection and hysteresis; 7: as 6 with the "
                         "two-level tile cache and the probe filter (the paper's whole chain)")
    args = ap.parse_args()
    args.sub = False
    global CONFIG
    CONFIG = args.config
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        line = run_config(CONFIG, args, rank, world, local_rank)
        if line is not None and CONFIG == 2 and world == 1 and not args.no_other_configs:
            line["configs"] = other_configs(args, rank, world, local_rank)
        if line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
