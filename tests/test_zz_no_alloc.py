"""The allocation-free entry point gi_cell_means_noalloc, for callers that cannot call
cudaMalloc (for example a renderer plugin whose host engine owns the whole GPU memory
budget, or a thread that must never block in the allocator), must give the same per-record
cell means as the allocating path: a fresh cache of 2^GI_NOALLOC_LOG2_SLOTS slots,
gi_cache_update, gi_cache_resolve and gi_cache_query by slot.  It computes the same cell
descriptor, the same fixed-point sums and the same float32 mean, so the two agree bit for bit.
Two calls in a row check that each call starts from a clean scratch table; both direction
sources of the descriptor are covered, and the means are also checked against the oracle.

This file is collected last on purpose: the entry point shares one device array between all
calls, and a failure here should come after every other test has run."""
import numpy as np
import pytest
import torch

import paper_2310_19855_gb300 as gi
import workload as wl
from oracle.cache import OracleCache
from oracle.key import KEY_DIR_NORMAL, KEY_DIR_RAY

from _gpu_util import ABS, REL, dev, require_gpu, view_of

pytestmark = pytest.mark.gpu

ENV = (0.25, 0.5, 0.125)


def _allocating_path(rec_dev, n, view, key_dir):
    h = gi.gi_cache_create(gi.GI_NOALLOC_LOG2_SLOTS, cell_size=0.05, num_lods=4, max_probe=255, key_dir=key_dir)
    try:
        slots = torch.empty(n, dtype=torch.int32, device="cuda")
        gi.gi_cache_update(h, gi.hits_from_planes(rec_dev, n), view, slots)
        gi.gi_cache_resolve(h, 0)
        out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        gi.gi_cache_query(h, out, n, slot_ids=slots, env=ENV)
        torch.cuda.synchronize()
        st = gi.gi_cache_stats(h)
        assert st["dropped"] == 0
        return out.cpu().numpy(), int(st["clamped"])
    finally:
        gi.gi_cache_destroy(h)


def _oracle_means(rec, cam, key_dir):
    oc = OracleCache(gi.GI_NOALLOC_LOG2_SLOTS, cell_size=0.05, num_lods=4, key_dir=key_dir)
    ident = oc.update(rec, 0, cam.pos, cam.fov_y, cam.width, cam.height)
    oc.resolve(0)
    rad, found = oc.radiance(ident)
    miss = np.isposinf(rec[9])
    rad[miss] = ENV
    return rad, (found & (ident != 0)) | miss


@pytest.mark.parametrize("key_dir", [gi.GI_KEY_DIR_NORMAL, gi.GI_KEY_DIR_RAY])
def test_noalloc_matches_allocating_path_on_two_calls(key_dir):
    require_gpu()
    fr = wl.make_frame(1, 0)
    view = view_of(fr.camera, 0)
    first = fr.records
    # same hit points, other radiance (one channel pushed past the clamp) and fewer records: a
    # table or counters left dirty by the first call would change these means and counts
    second = first[:, : first.shape[1] - 1000].copy()
    second[6:9] = np.float32(3.0) - second[6:9]
    second[6, ::97] = np.float32(40000.0)
    stats = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    for rec in (first, second):
        n = rec.shape[1]
        rec_dev = dev(rec)
        out = torch.full((n, 4), -7.0, dtype=torch.float32, device="cuda")
        gi.gi_cell_means_noalloc(gi.hits_from_planes(rec_dev, n), view, out, cell_size=0.05, num_lods=4,
                                 key_dir=key_dir, env=ENV, stats_out=stats)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want, clamped = _allocating_path(rec_dev, n, view, key_dir)
        # same descriptor, fixed-point sums and reciprocal-times-sum mean: bit for bit
        assert np.array_equal(got, want)
        dropped_got, clamped_got = (int(x) for x in stats.cpu().numpy())
        assert dropped_got == 0 and clamped_got == clamped
        assert np.count_nonzero(got[:, 3] == 1.0) > n // 2
        # and against the float64 oracle cache (fresh table, one resolve, no history)
        rad, has = _oracle_means(rec, fr.camera, KEY_DIR_NORMAL if key_dir == gi.GI_KEY_DIR_NORMAL else KEY_DIR_RAY)
        assert np.array_equal(got[:, 3] == 1.0, has)
        assert np.all(got[~has] == 0.0)
        assert np.all(np.abs(got[has, :3] - rad[has]) <= REL * np.abs(rad[has]) + ABS)
    assert clamped_got > 0


def test_noalloc_rejects_batches_above_its_maximum():
    require_gpu()
    n = gi.GI_NOALLOC_MAX_RECORDS + 1
    rec = torch.zeros((13, n), dtype=torch.float32, device="cuda")
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    view = view_of(wl.make_frame(1, 0).camera, 0)
    with pytest.raises(gi.GiError) as e:
        gi.gi_cell_means_noalloc(gi.hits_from_planes(rec, n), view, out)
    assert e.value.status == gi.GI_ERR_INVALID_ARG
