"""Autotuner of the batched pass chain's launch shapes (gi_batch_tuning).

It times every candidate shape on the caller's own frames with CUDA events, keeps the fastest,
and remembers the choice in a JSON file keyed by the GPU name and the batch's view signature
(view sizes, records per view), so a later run with the same views reuses it without sweeping."""
from __future__ import annotations

import json
import os

import torch

from . import gi_batch_set_tuning, gi_batch_tuning
from .build import BUILD_DIR

DEFAULT_CACHE = os.path.join(BUILD_DIR, "autotune.json")
CANDIDATES = [(r, b, t) for r in (1024, 2048) for b in (1, 2, 4) for t in (64, 128)]


def signature(views) -> str:
    """Key of a batch: GPU name and per-view (width, height, records)."""
    name = torch.cuda.get_device_name()
    return name + "|" + ";".join(f"{v['width']}x{v['height']}:{v['n_records']}" for v in views)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(pipeline, run_frame, frames: int = 3, warmup: int = 1, cache_path: str = DEFAULT_CACHE,
         force: bool = False):
    """Choose and apply the fastest launch shapes for `pipeline` (a BatchPipeline).

    run_frame() must run the next frame of the batch on the current stream (frame numbers keep
    increasing).  Returns (tuning, per-candidate mean ms)."""
    key = signature(pipeline.views)
    db = _load(cache_path)
    if not force and key in db:
        t = gi_batch_tuning(*db[key]["tuning"])
        gi_batch_set_tuning(pipeline.batch, t)
        return t, db[key].get("timings", {})
    timings = {}
    best = None
    for cand in CANDIDATES:
        t = gi_batch_tuning(*cand)
        gi_batch_set_tuning(pipeline.batch, t)
        for _ in range(warmup):
            run_frame()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(frames):
            run_frame()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / frames
        timings["%d/%d/%d" % cand] = ms
        if best is None or ms < best[1]:
            best = (cand, ms)
    t = gi_batch_tuning(*best[0])
    gi_batch_set_tuning(pipeline.batch, t)
    db[key] = {"tuning": list(best[0]), "timings": timings}
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return t, timings
