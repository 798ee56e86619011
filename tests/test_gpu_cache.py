"""GPU parity of the world cache (Section 2.2) against the oracle, through the
C ABI: keys/occupancy/fixed-point sums bit-exact, resolved radiance within
1e-4 relative (float32 path vs float64 oracle)."""
import math

import numpy as np
import pytest
import torch

import paper_2310_19855_gb300 as gi
import workload as wl
from oracle.cache import OracleCache
from oracle.key import KEY_DIR_RAY

from _gpu_util import check_export_matches, check_slot_ids, close, dev, require_gpu, u32, view_of

pytestmark = pytest.mark.gpu

FOV = math.radians(60.0)


class _Cam:
    def __init__(self, pos=(0.0, 0.0, 0.0), W=64, H=64):
        self.pos = np.asarray(pos, np.float32)
        self.fwd = np.array([0, 0, -1], np.float32)
        self.right = np.array([1, 0, 0], np.float32)
        self.up = np.array([0, 1, 0], np.float32)
        self.fov_y, self.width, self.height = FOV, W, H


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _run_update(h, rec_np, view, n_slots):
    n = rec_np.shape[1]
    rec = dev(rec_np)
    slots = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    gi.gi_cache_update(h, gi.hits_from_planes(rec, n), view, slots)
    torch.cuda.synchronize()
    return u32(slots)[:n]


# both records of the slots touched since the last resolve (results must not depend on it)
FIRST_TOUCH = pytest.mark.parametrize("first_touch", [gi.GI_FIRST_TOUCH_LIST, gi.GI_FIRST_TOUCH_BITMAP],
                                      ids=["touch-list", "bitmap"])
# the update with and without the warp merge of same-cell hits: identical results
MERGE = pytest.mark.parametrize("merge", [gi.GI_MERGE_NONE, gi.GI_MERGE_WARP], ids=["no-merge", "warp-merge"])


def _frames_parity(config, frames, key_dir=0, log2_slots=None, resolved_format=0, value_rel=1e-4, first_touch=0):
    cfg = wl.CONFIGS[config]
    ls = log2_slots or cfg["log2_slots"]
    oc = OracleCache(ls, key_dir=key_dir)
    h = gi.gi_cache_create(ls, key_dir=key_dir, resolved_format=resolved_format, first_touch=first_touch)
    try:
        for fr in frames:
            cam = fr.camera
            view = view_of(cam, fr.frame)
            slots = _run_update(h, fr.records, view, 1 << ls)
            ident = oc.update(fr.records, fr.frame, cam.pos, cam.fov_y, cam.width, cam.height)
            ex = gi.gi_cache_export(h)
            check_export_matches(ex, oc, resolved=False)
            check_slot_ids(slots, ex, fr.records, ident, 1 << ls)
            assert gi.gi_cache_stats(h)["touched"] == int(np.count_nonzero(oc.count))
            gi.gi_cache_resolve(h, fr.frame)
            oc.resolve(fr.frame)
            check_export_matches(gi.gi_cache_export(h), oc, resolved=True, value_rel=value_rel)
        st = gi.gi_cache_stats(h)
        assert st["dropped"] == 0 and st["error_word"] == 0
        assert st["live"] == oc.live_count()
        assert st["clamped"] == oc.clamped
    finally:
        gi.gi_cache_destroy(h)


@FIRST_TOUCH
def test_cornell_frames_bit_exact(first_touch):
    _frames_parity(1, wl.make_frames(1), first_touch=first_touch)


def test_cornell_frames_ray_direction_descriptor():
    _frames_parity(1, wl.make_frames(1, frames=2), key_dir=KEY_DIR_RAY)


def test_cornell_frames_fp16_resolved():
    # FP16-packed resolved radiance: FP32 blend, one rounding to half (relative 2^-11) per resolve;
    # the blend carries (1 - alpha) of the previous rounding into the next frame, so after k frames
    # the error is at most 2^-11 * sum_{j<k} (1 - alpha)^j relative, plus the float32 path's 1e-4.
    frames = wl.make_frames(1)
    bound = 2.0 ** -11 * sum(0.9 ** j for j in range(len(frames))) + 1e-4
    _frames_parity(1, frames, resolved_format=gi.GI_RESOLVED_F16, value_rel=bound)


@FIRST_TOUCH
def test_full_size_1080p_two_frames(first_touch):
    # the 1080p workload at full size, in the launch configuration the bench uses
    scene = wl.make_scene(2)
    _frames_parity(2, [wl.make_frame(2, f, scene) for f in (0, 1)], first_touch=first_touch)


@MERGE
@FIRST_TOUCH
@pytest.mark.parametrize("n", [0, 1, 31, 33, 257, 10007])
def test_ragged_batches_and_split_updates(n, first_touch, merge):
    cam = _Cam((0.3, -0.2, 0.1))
    ls = 16
    oc = OracleCache(ls)
    h = gi.gi_cache_create(ls, first_touch=first_touch, merge=merge)
    try:
        for f in range(3):
            rec = wl.records_random(n, seed=100 + f, extent=1.5, cam=cam.pos)
            view = view_of(cam, f)
            # two updates per frame: the halves must add up to one batch
            k = n // 2
            s1 = _run_update(h, np.ascontiguousarray(rec[:, :k]), view, 1 << ls)
            s2 = _run_update(h, np.ascontiguousarray(rec[:, k:]), view, 1 << ls)
            ident = oc.update(rec, f, cam.pos, FOV, 64, 64)
            ex = gi.gi_cache_export(h)
            check_export_matches(ex, oc, resolved=False)
            check_slot_ids(np.concatenate([s1, s2]), ex, rec, ident, 1 << ls)
            gi.gi_cache_resolve(h, f)
            oc.resolve(f)
            check_export_matches(gi.gi_cache_export(h), oc, resolved=True)
    finally:
        gi.gi_cache_destroy(h)


@MERGE
@FIRST_TOUCH
def test_all_records_in_one_cell(first_touch, merge):
    # every lane of every warp names the same cell: the warp merge (or one reduction per record) and
    # the atomics must add up exactly
    n = 50000
    rec = np.zeros((13, n), np.float32)
    rec[0:3] = np.float32(0.31)
    rec[5] = 1.0
    rng = np.random.default_rng(5)
    rec[6:9] = rng.uniform(0, 3, (3, n)).astype(np.float32)
    rec[9] = 1.0
    cam = _Cam()
    oc = OracleCache(10)
    h = gi.gi_cache_create(10, first_touch=first_touch, merge=merge)
    try:
        view = view_of(cam, 0)
        _run_update(h, rec, view, 1 << 10)
        oc.update(rec, 0, cam.pos, FOV, 64, 64)
        ex = gi.gi_cache_export(h)
        assert ex.size == 1 and ex["count"][0] == n
        check_export_matches(ex, oc, resolved=False)
    finally:
        gi.gi_cache_destroy(h)


@MERGE
@FIRST_TOUCH
def test_every_key_retrievable_in_a_crowded_table(first_touch, merge):
    # 2^10 slots at ~60 % load: long probing runs, no drop, no duplicate, every record finds its cell
    cam = _Cam(W=1920, H=1080)  # every cell at LOD 0 within 12 m
    rng = np.random.default_rng(9)
    cells = rng.integers(-40, 40, (3, 620)).astype(np.float32) * np.float32(0.05) + np.float32(0.025)
    idx = rng.integers(0, 620, 6000)
    rec = np.zeros((13, idx.size), np.float32)
    rec[0:3] = cells[:, idx]
    rec[4] = 1.0
    rec[6:9] = rng.uniform(0, 1, (3, idx.size)).astype(np.float32)
    rec[9] = 1.0
    ls = 10
    oc = OracleCache(ls)
    h = gi.gi_cache_create(ls, max_probe=255, first_touch=first_touch, merge=merge)
    try:
        view = view_of(cam, 0)
        slots = _run_update(h, rec, view, 1 << ls)
        ident = oc.update(rec, 0, cam.pos, FOV, cam.width, cam.height)
        ex = gi.gi_cache_export(h)
        assert np.unique(ex["identity"]).size == ex.size == oc.ids.size
        assert np.unique(ex["slot"]).size == ex.size
        check_slot_ids(slots, ex, rec, ident, 1 << ls)
        gi.gi_cache_resolve(h, 0)
        oc.resolve(0)
        # lookups without insertion find every record's cell with its resolved value
        out = torch.empty((rec.shape[1], 4), dtype=torch.float32, device="cuda")
        gi.gi_cache_query(h, out, rec.shape[1], points=gi.hits_from_planes(dev(rec), rec.shape[1]), view=view)
        o = out.cpu().numpy()
        want, found = oc.query_records(rec, cam.pos, FOV, cam.width, cam.height)
        assert np.all(found) and np.all(o[:, 3] == 1.0)
        assert close(o[:, :3], want).all()
        st = gi.gi_cache_stats(h)
        assert st["dropped"] == 0 and st["max_probe_seen"] > 4
    finally:
        gi.gi_cache_destroy(h)


@FIRST_TOUCH
def test_eviction_at_eighth_untouched_resolve_and_fresh_restart(first_touch):
    cam = _Cam()
    a = np.zeros((13, 64), np.float32)
    a[0:3] = np.float32(0.11)
    a[5] = 1.0
    a[6:9] = 2.0
    a[9] = 1.0
    b = a.copy()
    b[0:3] = np.float32(0.61)
    oc = OracleCache(12)
    h = gi.gi_cache_create(12, first_touch=first_touch)
    try:
        for f in range(0, 20):
            rec = np.concatenate([a, b], axis=1) if f == 0 else b
            if f == 12:
                rec = np.concatenate([a * np.array([1] * 6 + [2.5] * 3 + [1] * 4, np.float32)[:, None], b], axis=1)
            view = view_of(cam, f)
            _run_update(h, np.ascontiguousarray(rec), view, 1 << 12)
            oc.update(rec, f, cam.pos, FOV, 64, 64)
            gi.gi_cache_resolve(h, f)
            oc.resolve(f)
            ex = gi.gi_cache_export(h)
            check_export_matches(ex, oc, resolved=True)
            assert ex.size == (2 if (f < 8 or f >= 12) else 1), f
        # the revived cell restarted from its new mean (5.0), it did not blend with the old 2.0
        v = np.sort(gi.gi_cache_export(h)["value"][:, 0])
        assert 5.0 in v
    finally:
        gi.gi_cache_destroy(h)


@FIRST_TOUCH
def test_compaction_keeps_the_live_set(first_touch):
    # a small table that fills with stale cells and is compacted several times
    cam = _Cam()
    ls = 14
    oc = OracleCache(ls, evict_frames=2)
    h = gi.gi_cache_create(ls, evict_frames=2, rebuild_load=0.3, first_touch=first_touch)
    try:
        for f in range(16):
            rec = wl.records_random(1500, seed=500 + f, extent=1.0)
            view = view_of(cam, f)
            slots = _run_update(h, rec, view, 1 << ls)
            ident = oc.update(rec, f, cam.pos, FOV, 64, 64)
            ex = gi.gi_cache_export(h)
            check_export_matches(ex, oc, resolved=False)
            check_slot_ids(slots, ex, rec, ident, 1 << ls)
            gi.gi_cache_resolve(h, f)
            oc.resolve(f)
            torch.cuda.synchronize()
            check_export_matches(gi.gi_cache_export(h), oc, resolved=True)
        st = gi.gi_cache_stats(h)
        assert st["rebuilds"] >= 2, st
        assert st["dropped"] == 0
    finally:
        gi.gi_cache_destroy(h)


def test_query_by_slot_matches_export():
    fr = wl.make_frame(1, 0)
    cam = fr.camera
    h = gi.gi_cache_create(16)
    try:
        view = view_of(cam, 0)
        rec = dev(fr.records)
        R = fr.n_records
        slots = torch.empty(R, dtype=torch.int32, device="cuda")
        gi.gi_cache_update(h, gi.hits_from_planes(rec, R), view, slots)
        gi.gi_cache_resolve(h, 0)
        out = torch.empty((R, 4), dtype=torch.float32, device="cuda")
        gi.gi_cache_query(h, out, R, slot_ids=slots, env=(0.5, 0.25, 0.125))
        o = out.cpu().numpy()
        s = u32(slots)
        ex = gi.gi_cache_export(h)
        table = {int(k): v for k, v in zip(ex["slot"], ex["value"])}
        real = s < (1 << 16)
        assert np.array_equal(o[real, :3], np.array([table[int(k)] for k in s[real]]))
        assert np.all(o[s == gi.GI_SLOT_MISS] == np.array([0.5, 0.25, 0.125, 1.0], np.float32))
        assert np.all(o[s == gi.GI_SLOT_NONE] == 0)
    finally:
        gi.gi_cache_destroy(h)


def test_clamped_and_invalid_records_are_counted():
    cam = _Cam()
    rec = wl.records_random(4000, seed=77, extent=1.0)
    rec[6, :50] = -1.0
    rec[7, 50:100] = np.nan
    rec[8, 100:150] = 1e6
    rec[9, 150:200] = np.nan     # no sample
    rec[0, 200:250] = np.inf     # not a hit
    oc = OracleCache(14)
    h = gi.gi_cache_create(14)
    try:
        view = view_of(cam, 0)
        slots = _run_update(h, rec, view, 1 << 14)
        ident = oc.update(rec, 0, cam.pos, FOV, 64, 64)
        ex = gi.gi_cache_export(h)
        check_export_matches(ex, oc, resolved=False)
        check_slot_ids(slots, ex, rec, ident, 1 << 14)
        st = gi.gi_cache_stats(h)
        assert st["clamped"] == oc.clamped > 0
    finally:
        gi.gi_cache_destroy(h)


@pytest.mark.parametrize("form", [gi.GI_FIRST_TOUCH_LIST, gi.GI_FIRST_TOUCH_BITMAP])
def test_diag_update_atomics_counts_every_record(form):
    """The diagnostic accumulation pass (not a step of the path), in either form: per slot, the
    counts and sums add up to the slot's records (one reduction each); the first touches (list) or
    the bits (bitmap) mark exactly the distinct slots; records without a slot skipped."""
    rng = np.random.default_rng(5)
    log2 = 12
    n = 50_000
    ids = rng.integers(0, 1 << log2, n).astype(np.uint32)
    ids[rng.random(n) < 0.1] = 0xFFFFFFFE  # misses
    ids[:64] = 7  # two warps on one slot: still one reduction per record
    slots = 1 << log2
    scratch = torch.zeros(slots * 8 + slots // 32, dtype=torch.int32, device="cuda")
    first = torch.zeros(1, dtype=torch.int32, device="cuda")
    gi.gi_diag_update_atomics(dev(ids.view(np.int32)), n, log2, scratch, first, first_touch=form)
    raw = scratch.cpu().numpy().view(np.uint32)
    acc = raw[: slots * 8].reshape(-1, 8)
    valid = ids[ids < slots]
    want = np.bincount(valid, minlength=slots)
    assert np.array_equal(acc[:, 6], want)
    assert np.all(acc[:, 7] == 0)  # the stamp word is never touched
    if form == gi.GI_FIRST_TOUCH_LIST:
        assert int(first.item()) == int((want > 0).sum())
    else:
        bits = np.unpackbits(raw[slots * 8:].view(np.uint8), bitorder="little").astype(bool)
        assert np.array_equal(bits, want > 0)
    # sums: 1, 2, 3 per record (the update's default form merges nothing)
    s0 = acc[:, 0].astype(np.uint64) | (acc[:, 1].astype(np.uint64) << 32)
    s1 = acc[:, 2].astype(np.uint64) | (acc[:, 3].astype(np.uint64) << 32)
    s2 = acc[:, 4].astype(np.uint64) | (acc[:, 5].astype(np.uint64) << 32)
    assert np.array_equal(s0, want.astype(np.uint64))
    assert np.all(s1 == 2 * s0) and np.all(s2 == 3 * s0)
