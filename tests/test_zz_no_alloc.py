"""The allocation-free entry point gi_cell_means_noalloc, for callers that cannot call
cudaMalloc (for example a renderer plugin whose host engine owns the whole GPU memory
budget), must give the same per-record cell means as the allocating path: a fresh cache of
2^GI_NOALLOC_LOG2_SLOTS slots, gi_cache_update, gi_cache_resolve and gi_cache_query by slot.
Two calls in a row check that each call starts from a clean scratch table."""
import math

import numpy as np
import pytest
import torch

import paper_2310_19855_gb300 as gi
import workload as wl

from _gpu_util import ABS, REL, dev, require_gpu, view_of

pytestmark = pytest.mark.gpu

ENV = (0.25, 0.5, 0.125)


def _allocating_path(rec_dev, n, view):
    h = gi.gi_cache_create(gi.GI_NOALLOC_LOG2_SLOTS, cell_size=0.05, num_lods=4, max_probe=255)
    try:
        slots = torch.empty(n, dtype=torch.int32, device="cuda")
        gi.gi_cache_update(h, gi.hits_from_planes(rec_dev, n), view, slots)
        gi.gi_cache_resolve(h, 0)
        out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        gi.gi_cache_query(h, out, n, slot_ids=slots, env=ENV)
        torch.cuda.synchronize()
        assert gi.gi_cache_stats(h)["dropped"] == 0
        return out.cpu().numpy()
    finally:
        gi.gi_cache_destroy(h)


def test_noalloc_matches_allocating_path_on_two_calls():
    require_gpu()
    fr = wl.make_frame(1, 0)
    view = view_of(fr.camera, 0)
    first = fr.records
    # same hit points, other radiance and fewer records: a table left dirty by the first call
    # would change these means
    second = first[:, : first.shape[1] - 1000].copy()
    second[6:9] = np.float32(3.0) - second[6:9]
    for rec in (first, second):
        n = rec.shape[1]
        rec_dev = dev(rec)
        out = torch.full((n, 4), -1.0, dtype=torch.float32, device="cuda")
        gi.gi_cell_means_noalloc(gi.hits_from_planes(rec_dev, n), view, out, cell_size=0.05, num_lods=4,
                                 env=ENV)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = _allocating_path(rec_dev, n, view)
        assert np.all(np.abs(got - want) <= REL * np.abs(want) + ABS)
        assert np.count_nonzero(got[:, 3] == 1.0) > n // 2


def test_noalloc_rejects_batches_above_its_maximum():
    require_gpu()
    n = gi.GI_NOALLOC_MAX_RECORDS + 1
    rec = torch.zeros((13, n), dtype=torch.float32, device="cuda")
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    view = view_of(wl.make_frame(1, 0).camera, 0)
    with pytest.raises(gi.GiError) as e:
        gi.gi_cell_means_noalloc(gi.hits_from_planes(rec, n), view, out)
    assert e.value.status == gi.GI_ERR_INVALID_ARG
