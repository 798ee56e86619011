"""Per-view frame chain on the GPU: spawn -> cache update -> resolve ->
probe irradiance -> per-pixel interpolation (the paper's pass order,
Sections 2.1.1, 2.2, 2.1.4, 2.4).  PyTorch only allocates device memory;
every step is a call into libgi.so."""
from __future__ import annotations

import torch

from . import (GI_RESOLVED_F32, GI_SH_STRIDE, gi_batch_create, gi_batch_destroy, gi_batch_frame,
               gi_batch_set_surrogate, gi_batch_set_view_surrogates, gi_batch_view, gi_cache_create,
               gi_cache_destroy, gi_cache_route_far, gi_cache_resolve, gi_cache_update, gi_probes_filter, gi_probes_gather,
               gi_probes_gather_temporal, gi_probes_integrate, gi_probes_interpolate, gi_probes_layout,
               gi_probes_project, gi_probes_reproject, gi_probes_spawn, gi_probes_spawn_upscaled, hits_from_planes,
               make_gbuffer, make_probes, make_view)


def view_of(camera, frame: int):
    """gi_view from an object with pos, fwd, right, up, fov_y, width, height."""
    return make_view(frame, camera.width, camera.height, camera.pos, camera.fwd, camera.right, camera.up,
                     camera.fov_y)


class ProbeBuffers:
    """Device buffers of the screen probes of one view size."""

    def __init__(self, width: int, height: int, device="cuda"):
        self.layout = gi_probes_layout(width, height)
        P = self.layout.num_probes
        self.mask = torch.empty(self.layout.mask_words, dtype=torch.int32, device=device)
        self.pos = torch.empty((P, 4), dtype=torch.float32, device=device)
        self.nrm = torch.empty((P, 4), dtype=torch.float32, device=device)
        self.sh = torch.empty((P, GI_SH_STRIDE), dtype=torch.float32, device=device)
        self.struct = make_probes(self.layout, self.mask, self.pos, self.nrm, self.sh)

    def mask_levels(self):
        """Host copies of the MIP levels of the probe mask (uint32)."""
        m = self.mask.cpu().numpy().view("uint32")
        lv = []
        for k in range(self.layout.mip_count):
            w, h, off = self.layout.mip_w[k], self.layout.mip_h[k], self.layout.mip_offset[k]
            lv.append(m[off:off + w * h].reshape(h, w))
        return lv


class Pipeline:
    def __init__(self, width: int, height: int, rays_per_probe: int, log2_slots: int, cell_size=0.05,
                 num_lods=4, alpha=0.1, evict_frames=8, max_probe=128, key_dir=0,
                 resolved_format=GI_RESOLVED_F32, rebuild_load=0.8, first_touch=0, tiles=False, min_samples=16,
                 device="cuda"):
        self.width, self.height, self.rpp = width, height, rays_per_probe
        self.probes = ProbeBuffers(width, height, device)
        self.n_records = self.probes.layout.num_probes * rays_per_probe
        self.slot_ids = torch.empty(self.n_records, dtype=torch.int32, device=device)
        self.irr = torch.empty((height, width, 4), dtype=torch.float32, device=device)
        self.cache = gi_cache_create(log2_slots, cell_size, num_lods, alpha, evict_frames, max_probe, key_dir,
                                     resolved_format, rebuild_load, first_touch, tiles, min_samples)
        self.atlas = self.atlas_tmp = None

    def spawn(self, gbuf, view, stream=None):
        gi_probes_spawn(make_gbuffer(gbuf, self.width, self.height), view, self.probes.struct, stream)

    def update(self, records, view, stream=None):
        gi_cache_update(self.cache, hits_from_planes(records, self.n_records), view, self.slot_ids, stream)

    def resolve(self, frame: int, stream=None):
        gi_cache_resolve(self.cache, frame, stream)

    def integrate(self, env=(0.0, 0.0, 0.0), stream=None):
        gi_probes_integrate(self.cache, self.probes.struct, self.slot_ids, self.rpp, env, stream)

    def integrate_filtered(self, records, view, env=(0.0, 0.0, 0.0), stream=None):
        """Probe irradiance through the probe atlas with the separable filter (x pass, then y).
        records: the (planes, R) record tensor of the frame (its ray-length plane is read)."""
        if self.atlas is None:
            P = self.probes.layout.num_probes
            self.atlas = torch.empty((P, 64, 4), dtype=torch.float32, device=self.irr.device)
            self.atlas_tmp = torch.empty_like(self.atlas)
        ray_len = records[9]
        gi_probes_gather(self.cache, self.probes.struct, self.slot_ids, ray_len, self.rpp, self.atlas, env, stream)
        gi_probes_filter(self.probes.struct, view, self.atlas, self.atlas_tmp, 0, stream)
        gi_probes_filter(self.probes.struct, view, self.atlas_tmp, self.atlas, 1, stream)
        gi_probes_project(self.probes.struct, self.atlas, stream)

    def interpolate(self, gbuf, view, stream=None):
        gi_probes_interpolate(make_gbuffer(gbuf, self.width, self.height), view, self.probes.struct, self.irr,
                              stream)

    def frame(self, gbuf, records, view, env=(0.0, 0.0, 0.0), stream=None):
        """One frame of the whole path; gbuf (H, W, 4) and records (13, R) float32 on the device."""
        self.spawn(gbuf, view, stream)
        self.update(records, view, stream)
        self.resolve(view.frame, stream)
        self.integrate(env, stream)
        self.interpolate(gbuf, view, stream)

    def close(self):
        if self.cache:
            gi_cache_destroy(self.cache)
            self.cache = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPipeline:
    """Many views per frame through one batch (one launch per pass over all views).

    views: list of (width, height, log2_slots) per view; every view uses rays_per_probe rays per
    probe.  Each view owns a cache and its probe / slot-id / irradiance buffers."""

    def __init__(self, views, rays_per_probe: int = 64, tuning=None, cache_kw=None, device="cuda"):
        cache_kw = cache_kw or {}
        self.rpp = rays_per_probe
        self.views = []
        for (w, h, log2_slots) in views:
            pb = ProbeBuffers(w, h, device)
            n = pb.layout.num_probes * rays_per_probe
            self.views.append(dict(
                width=w, height=h, probes=pb, n_records=n,
                slot_ids=torch.empty(n, dtype=torch.int32, device=device),
                irr=torch.empty((h, w, 4), dtype=torch.float32, device=device),
                cache=gi_cache_create(log2_slots, **cache_kw)))
        self.batch = gi_batch_create(len(self.views), rays_per_probe, tuning)
        self._desc = (gi_batch_view * len(self.views))()

    def frame(self, gbufs, records, gviews, env=(0.0, 0.0, 0.0), use_graph=False, stream=None,
              resolve_frame: int | None = None):
        """One frame of every view: gbufs[v] (H, W, 4), records[v] (planes, R) on the device, gviews[v]
        the view (camera, size, frame index of the spawn jitter); the caches resolve at
        resolve_frame (default: each view's frame index)."""
        for v, st in enumerate(self.views):
            d = self._desc[v]
            d.cache = st["cache"]
            d.view = gviews[v]
            d.resolve_frame = gviews[v].frame if resolve_frame is None else int(resolve_frame)
            d.hits = hits_from_planes(records[v], st["n_records"])
            d.gbuf = make_gbuffer(gbufs[v], st["width"], st["height"])
            d.probes = st["probes"].struct
            d.slot_ids = st["slot_ids"].data_ptr()
            d.irradiance = st["irr"].data_ptr()
            for k in range(3):
                d.env[k] = float(env[k])
        gi_batch_frame(self.batch, self._desc, use_graph, stream)

    def set_surrogate(self, nrc, far_lod: int = 4):
        """The batch's probe pass through the surrogate nrc (None: the plain form); far_lod < 4 also
        routes every view's hits of that LOD and above to it (gi_cache_route_far)."""
        for st in self.views:
            gi_cache_route_far(st["cache"], nrc if far_lod < 4 else None, far_lod)
        gi_batch_set_surrogate(self.batch, nrc)

    def set_view_surrogates(self, nrcs, far_lod: int = 4):
        """View v's probe pass through the surrogate nrcs[v] (None: that view's plain probe pass;
        nrcs None: the plain form); far_lod < 4 also routes view v's hits of that LOD and above to
        nrcs[v] (gi_cache_route_far)."""
        if nrcs is not None and len(nrcs) != len(self.views):
            raise ValueError(f"set_view_surrogates: {len(nrcs)} networks for {len(self.views)} views")
        for v, st in enumerate(self.views):
            nrc = None if nrcs is None else nrcs[v]
            gi_cache_route_far(st["cache"], nrc if far_lod < 4 else None, far_lod)
        gi_batch_set_view_surrogates(self.batch, nrcs)

    def close(self):
        if self.batch:
            gi_batch_destroy(self.batch)
            self.batch = None
        for st in self.views:
            if st.get("cache"):
                gi_cache_destroy(st["cache"])
                st["cache"] = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TemporalPipeline:
    """The screen-probe temporal path of one view (Sections 2.1.1-2.1.4): per frame, reprojection of
    the previous probes (Algorithm 1), spawn with temporal upscale u, cache update + resolve on the
    spawn tiles' rays, the frame atlas (fresh probes blended with their reprojected history by
    Algorithm 4, reprojected probes carried), SH projection and per-pixel interpolation.  Probe
    buffers and atlases alternate between frames."""

    def __init__(self, width: int, height: int, rays_per_probe: int, log2_slots: int, upscale: int = 2,
                 filtered: bool = False, device="cuda", **cache_kw):
        """filtered: the frame atlas goes through the probe filter (Algorithm 5, an x then a y pass)
        before the SH projection; the unfiltered atlas stays the next frame's history.  cache_kw
        go to gi_cache_create (tiles=True gives the two-level cache, log2_slots then counts tiles)."""
        self.width, self.height, self.rpp, self.upscale = width, height, rays_per_probe, upscale
        self.filtered = filtered
        self.bufs = [ProbeBuffers(width, height, device), ProbeBuffers(width, height, device)]
        for b in self.bufs:
            b.mask.fill_(-1)
            b.pos.zero_()
            b.nrm.zero_()
        P = self.bufs[0].layout.num_probes
        self.atlases = [torch.zeros((P, 64, 4), dtype=torch.float32, device=device) for _ in range(2)]
        self.filt = [torch.zeros((P, 64, 4), dtype=torch.float32, device=device) for _ in range(2)] if filtered else None
        self.src = torch.empty(P, dtype=torch.int32, device=device)
        su = 8 * upscale
        self.spawn_tiles = ((width + su - 1) // su) * ((height + su - 1) // su)
        self.n_records = self.spawn_tiles * rays_per_probe
        self.slot_ids = torch.empty(self.n_records, dtype=torch.int32, device=device)
        self.irr = torch.empty((height, width, 4), dtype=torch.float32, device=device)
        self.cache = gi_cache_create(log2_slots, **cache_kw)
        self.k = 0

    @property
    def probes(self):
        """The probe buffers of the latest frame."""
        return self.bufs[self.k ^ 1]

    @property
    def atlas(self):
        return self.atlases[self.k ^ 1]

    def frame(self, gbuf, records, motion, view, env=(0.0, 0.0, 0.0), stream=None):
        cur, prev = self.bufs[self.k], self.bufs[self.k ^ 1]
        g = make_gbuffer(gbuf, self.width, self.height)
        gi_probes_reproject(g, view, motion, prev.struct, cur.struct, self.src, stream)
        gi_probes_spawn_upscaled(g, view, self.upscale, True, cur.struct, stream)
        gi_cache_update(self.cache, hits_from_planes(records, self.n_records), view, self.slot_ids, stream)
        gi_cache_resolve(self.cache, view.frame, stream)
        gi_probes_gather_temporal(self.cache, g, view, self.upscale, cur.struct, self.slot_ids, records[9], self.rpp,
                                  self.src, self.atlases[self.k ^ 1], self.atlases[self.k], env, stream)
        shown = self.atlases[self.k]
        if self.filtered:
            gi_probes_filter(cur.struct, view, shown, self.filt[0], 0, stream)
            gi_probes_filter(cur.struct, view, self.filt[0], self.filt[1], 1, stream)
            shown = self.filt[1]
        gi_probes_project(cur.struct, shown, stream)
        gi_probes_interpolate(g, view, cur.struct, self.irr, stream)
        self.k ^= 1

    def close(self):
        if self.cache:
            gi_cache_destroy(self.cache)
            self.cache = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
