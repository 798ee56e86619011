"""Many views per frame (gi_batch_frame): one launch per pass over all views, with and without
CUDA-graph replay, must give bit for bit what the single-view calls give, and a batched view
matches the oracle like a single view does."""
import numpy as np
import pytest
import torch

import paper_2310_19855_gb300 as gi
import workload as wl
from oracle.cache import OracleCache
from oracle.frame import run_frame
from paper_2310_19855_gb300.pipeline import BatchPipeline, Pipeline, view_of

from _gpu_util import compare_frame, dev, require_gpu, u32

pytestmark = pytest.mark.gpu

SIZES = ((160, 96), (320, 180), (96, 64), (256, 144), (200, 120))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _views_and_frames(n_frames):
    specs = wl.batched_views(len(SIZES), sizes=SIZES)
    out = []
    for cfg, seed in specs:
        cfg = dict(cfg, log2_slots=16)
        scene = wl.make_scene(cfg, seed)
        out.append((cfg, [wl.make_frame(cfg, f, scene, seed_base=seed) for f in range(n_frames)]))
    return out


def _export_by_identity(cache):
    ex = gi.gi_cache_export(cache)
    return ex[["identity", "sum", "count", "stamp", "value"]]


# (the ray-direction descriptor splits a surface into more cells: 2^17 slots keep its tables below
# the load where a full probing run drops hits, which would make the cell set order-dependent)
@pytest.mark.parametrize("use_graph,key_dir,log2", [(False, gi.GI_KEY_DIR_NORMAL, 16), (True, gi.GI_KEY_DIR_NORMAL, 16),
                                                   (True, gi.GI_KEY_DIR_RAY, 17)])
def test_batched_equals_single_view_calls(use_graph, key_dir, log2):
    data = _views_and_frames(3)
    bp = BatchPipeline([(c["width"], c["height"], log2) for c, _ in data], 64, cache_kw=dict(key_dir=key_dir))
    singles = [Pipeline(c["width"], c["height"], 64, log2, key_dir=key_dir) for c, _ in data]
    try:
        for f in range(3):
            gbufs = [dev(frs[f].gbuffer) for _, frs in data]
            recs = [dev(frs[f].records) for _, frs in data]
            views = [view_of(frs[f].camera, f) for _, frs in data]
            bp.frame(gbufs, recs, views, use_graph=use_graph)
            for v, sp in enumerate(singles):
                sp.frame(gbufs[v], recs[v], views[v])
            torch.cuda.synchronize()
            for v, sp in enumerate(singles):
                st = bp.views[v]
                assert np.array_equal(_export_by_identity(st["cache"]), _export_by_identity(sp.cache))
                assert np.array_equal(st["probes"].mask.cpu().numpy(), sp.probes.mask.cpu().numpy())
                assert torch.equal(st["probes"].pos, sp.probes.pos)
                assert torch.equal(st["probes"].sh, sp.probes.sh)
                assert torch.equal(st["irr"], sp.irr)
                # slot ids name the same cells (slot numbers may differ with insertion order)
                a, b = u32(st["slot_ids"]), u32(sp.slot_ids)
                assert np.array_equal(a >= (1 << log2), b >= (1 << log2))
                assert gi.gi_cache_stats(sp.cache)["dropped"] == 0
    finally:
        bp.close()
        for sp in singles:
            sp.close()


def test_batched_view_matches_oracle():
    data = _views_and_frames(2)
    bp = BatchPipeline([(c["width"], c["height"], 16) for c, _ in data], 64)
    ocs = [OracleCache(16) for _ in data]
    try:
        for f in range(2):
            bp.frame([dev(frs[f].gbuffer) for _, frs in data], [dev(frs[f].records) for _, frs in data],
                     [view_of(frs[f].camera, f) for _, frs in data], use_graph=True)
            torch.cuda.synchronize()
            for v, (cfg, frs) in enumerate(data):
                out = run_frame(ocs[v], frs[f], f)
                st = bp.views[v]

                class _PL:  # the comparison helper reads pipeline-shaped buffers
                    probes = st["probes"]
                    irr = st["irr"]
                compare_frame(_PL, frs[f], out)
                ex = gi.gi_cache_export(st["cache"])
                assert np.array_equal(ex["identity"], ocs[v].ids)
    finally:
        bp.close()


def test_batched_full_size_views_match_oracle():
    # the batched workload's own view sizes at full resolution: a 1920x1080 box room and a 2560x1440
    # Cornell box (2^21 slots each), with a small view between them, one launch per pass over all
    specs = wl.batched_views(16)
    pick = [specs[3], specs[0], specs[2]]  # 2560x1440 boxes, 640x360 Cornell, 1920x1080 Cornell
    sizes = [(c["width"], c["height"]) for c, _ in pick]
    assert (2560, 1440) in sizes and (1920, 1080) in sizes
    data = []
    for cfg, seed in pick:
        scene = wl.make_scene(cfg, seed)
        data.append((cfg, [wl.make_frame(cfg, 0, scene, seed_base=seed)]))
    bp = BatchPipeline([(c["width"], c["height"], c["log2_slots"]) for c, _ in data], 64)
    try:
        bp.frame([dev(frs[0].gbuffer) for _, frs in data], [dev(frs[0].records) for _, frs in data],
                 [view_of(frs[0].camera, 0) for _, frs in data], use_graph=True)
        torch.cuda.synchronize()
        for v, (cfg, frs) in enumerate(data):
            oc = OracleCache(cfg["log2_slots"])
            out = run_frame(oc, frs[0], 0)
            st = bp.views[v]

            class _PL:
                probes = st["probes"]
                irr = st["irr"]
            compare_frame(_PL, frs[0], out)
            ex = gi.gi_cache_export(st["cache"])
            assert np.array_equal(ex["identity"], oc.ids)
    finally:
        bp.close()


def test_batch_rejects_inconsistent_views():
    data = _views_and_frames(1)
    bp = BatchPipeline([(c["width"], c["height"], 16) for c, _ in data], 64)
    try:
        recs = [dev(frs[0].records) for _, frs in data]
        views = [view_of(frs[0].camera, 0) for _, frs in data]
        views[1].width += 8  # the G-buffer and probe layout no longer match this view
        with pytest.raises(gi.GiError) as e:
            bp.frame([dev(frs[0].gbuffer) for _, frs in data], recs, views)
        assert e.value.status == gi.GI_ERR_INVALID_ARG
    finally:
        bp.close()


@pytest.mark.parametrize("per_view", [False, True])
def test_surrogate_batch_equals_single_view_calls(per_view):
    """gi_batch_set_surrogate: far hits of every view routed to one trusted network, the probe pass
    per view through the network's answers; gi_batch_set_view_surrogates: two networks and two
    views without one (their plain probe pass).  Bit for bit what the single-view calls give
    (update with routing, resolve, gi_nrc_query_frame, gi_probes_integrate_nrc or
    gi_probes_integrate, interpolation)."""
    from test_gpu_surrogate import _nrc, _spec, _trust_as_is

    data = _views_and_frames(2)
    allrec = np.concatenate([frs[f].records for _, frs in data for f in range(2)], axis=1)
    hitpos = allrec[0:3, np.isfinite(allrec[9])]
    spec = _spec(aabb=(tuple(hitpos.min(axis=1) - 1.0), tuple(hitpos.max(axis=1) + 1.0)))
    n_max = max(frs[0].n_records for _, frs in data)
    nets = [_nrc(spec, batch=1024, max_records=n_max, max_queries=n_max, trust=1e30, query_lod=2)
            for _ in range(2 if per_view else 1)]
    nrcs = [nets[0], None, nets[1], None, nets[1]] if per_view else [nets[0]] * len(data)
    bp = BatchPipeline([(c["width"], c["height"], 16) for c, _ in data], 64)
    singles = [Pipeline(c["width"], c["height"], 64, 16) for c, _ in data]
    try:
        for j, nrc in enumerate(nets):
            gi.gi_nrc_set_params(nrc, *wl.surrogate_inputs.params(11 + j, spec.log2_table))
            _trust_as_is(nrc, spec)
        if per_view:
            bp.set_view_surrogates(nrcs, far_lod=2)
        else:
            bp.set_surrogate(nets[0], far_lod=2)
        for sp, nrc in zip(singles, nrcs):
            gi.gi_cache_route_far(sp.cache, nrc, 2 if nrc else 4)
        routed = 0
        for f in range(2):
            gbufs = [dev(frs[f].gbuffer) for _, frs in data]
            recs = [dev(frs[f].records) for _, frs in data]
            views = [view_of(frs[f].camera, f) for _, frs in data]
            bp.frame(gbufs, recs, views, use_graph=True)
            for v, sp in enumerate(singles):
                sp.spawn(gbufs[v], views[v])
                sp.update(recs[v], views[v])
                sp.resolve(f)
                if nrcs[v] is None:
                    sp.integrate()
                else:
                    gi.gi_nrc_query_frame(nrcs[v], sp.cache, gi.hits_from_planes(recs[v], sp.n_records), sp.slot_ids,
                                          views[v])
                    gi.gi_probes_integrate_nrc(sp.cache, nrcs[v], sp.probes.struct, sp.slot_ids, 64)
                sp.interpolate(gbufs[v], views[v])
            torch.cuda.synchronize()
            for v, sp in enumerate(singles):
                st = bp.views[v]
                a, b = u32(st["slot_ids"]), u32(sp.slot_ids)
                assert np.array_equal(a == gi.GI_SLOT_FAR, b == gi.GI_SLOT_FAR)
                assert np.array_equal(a >= (1 << 16), b >= (1 << 16))
                routed += int(np.count_nonzero(a == gi.GI_SLOT_FAR))
                assert np.array_equal(_export_by_identity(st["cache"]), _export_by_identity(sp.cache))
                assert torch.equal(st["probes"].sh, sp.probes.sh)
                assert torch.equal(st["irr"], sp.irr)
        assert routed > 0
    finally:
        bp.set_surrogate(None)
        for sp in singles:
            gi.gi_cache_route_far(sp.cache, None, 4)
        bp.close()
        for sp in singles:
            sp.close()
        for nrc in nets:
            gi.gi_nrc_destroy(nrc)
