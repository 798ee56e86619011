"""GPU parity of the screen-probe stage (Sections 2.1.1, 2.1.5, 2.4) against the
oracle, through the C ABI: probe mask and MIP chain bit-exact, probe
positions to float32 rounding, SH irradiance and interpolated irradiance
within 1e-4 relative on every pixel whose flag agrees (flag flips bounded)."""
import math

import numpy as np
import pytest
import torch

import paper_2310_19855_gb300 as gi
import workload as wl
from oracle import probes as OP
from oracle import sh as OSH
from oracle.cache import OracleCache
from oracle.frame import run_frame

from _gpu_util import Pipeline, check_export_matches, close, dev, require_gpu, u32, view_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


from _gpu_util import compare_frame as _compare_frame, run_frames as _run_frames, sh_gpu as _sh_gpu


def test_cornell_chain():
    _run_frames(1, wl.make_frames(1))


def test_1080p_chain_full_size():
    scene = wl.make_scene(2)
    _run_frames(2, [wl.make_frame(2, f, scene) for f in (0, 1)])


def test_1080p_ten_frames_cross_an_eviction_and_a_compaction():
    # ten frames of the 1080p workload, every second frame of its camera path (faster motion): cells
    # seen only early are evicted at their 8th untouched resolve, and a low rebuild_load makes the
    # table compact itself at full size; after every resolve the cell set, stamps and values match
    # the oracle, and the last frame's probes and pixels match too
    scene = wl.make_scene(2)
    frames = [wl.make_frame(2, f, scene) for f in range(0, 20, 2)]
    cfg = wl.CONFIGS[2]
    pl = Pipeline(1920, 1080, 64, cfg["log2_slots"], rebuild_load=0.25)
    oc = OracleCache(cfg["log2_slots"])
    evicted = 0
    try:
        for i, fr in enumerate(frames):
            view = view_of(fr.camera, i)
            pl.frame(dev(fr.gbuffer), dev(fr.records), view)
            torch.cuda.synchronize()
            cam = fr.camera
            if i < len(frames) - 1:
                before = oc.live_count()
                oc.update(fr.records, i, cam.pos, cam.fov_y, cam.width, cam.height)
                grown = oc.live_count()
                oc.resolve(i)
                evicted += grown - oc.live_count()
            else:
                out = run_frame(oc, fr, i)
                _compare_frame(pl, fr, out)
            check_export_matches(gi.gi_cache_export(pl.cache), oc, resolved=True)
        st = gi.gi_cache_stats(pl.cache)
        assert evicted > 0 and st["rebuilds"] >= 1 and st["dropped"] == 0, (evicted, st["rebuilds"])
    finally:
        pl.close()


def test_uniform_radiance_gives_pi_L_on_gpu():
    # every probe ray returns the same radiance L (hits resolve to L exactly, misses see env = L)
    fr = wl.make_frame(1, 0)
    L = np.array([0.75, 1.5, 0.25], np.float32)
    rec = fr.records.copy()
    rec[6:9] = L[:, None]
    pl = Pipeline(64, 64, fr.rays_per_probe, 16)
    try:
        view = view_of(fr.camera, 0)
        pl.frame(dev(fr.gbuffer), dev(rec), view, env=L)
        torch.cuda.synchronize()
        v = pl.probes.nrm.cpu().numpy()
        valid = v[:, 3] == 1.0
        E = OSH.irradiance(_sh_gpu(pl)[valid], v[valid, :3])
        assert np.abs(E - math.pi * L).max() < 2e-6 * math.pi * L.max()
        # and every pixel interpolates pi L
        irr = pl.irr.cpu().numpy()
        px = irr[..., 3] == gi.GI_INTERP_OK  # neighbours weighted in share the pixel's normal
        assert np.abs(irr[px][:, :3] - math.pi * L).max() < 4e-6 * math.pi * L.max()
    finally:
        pl.close()


def test_integrate_rejects_misaligned_slot_ids():
    # the probe pass reads a probe's slot ids 16 bytes at a time: a buffer that does not start on a
    # 16-byte boundary is refused on the host, before any launch
    pl = Pipeline(64, 64, 64, 12)
    try:
        ids = torch.zeros(pl.n_records + 4, dtype=torch.int32, device="cuda")
        pl.probes.nrm.zero_()  # no probe: the accepted call below only writes zeros
        with pytest.raises(gi.GiError) as e:
            gi.gi_probes_integrate(pl.cache, pl.probes.struct, ids.data_ptr() + 4, 64)
        assert e.value.status == gi.GI_ERR_INVALID_ARG
        gi.gi_probes_integrate(pl.cache, pl.probes.struct, ids.data_ptr(), 64)  # aligned: accepted
        torch.cuda.synchronize()
    finally:
        pl.close()


def test_spawn_jitter_sequence_and_sky_tiles():
    fr = wl.make_frame(1, 0)
    gb = fr.gbuffer.copy()
    gb[:24, :, 3] = np.inf  # the top three tile rows see the sky
    pl = Pipeline(64, 64, 256, 16)
    try:
        for f in range(6):
            view = view_of(fr.camera, f)
            pl.spawn(dev(gb), view)
            torch.cuda.synchronize()
            sp = OP.spawn(gb, fr.camera, f)
            mg = pl.probes.mask_levels()
            assert np.array_equal(mg[0], sp["mask"])
            for a, b in zip(OP.build_mips(sp["mask"]), mg):
                assert np.array_equal(a, b)
            assert np.all(mg[0][:3] == gi.GI_PROBE_NONE)
    finally:
        pl.close()


def test_odd_view_sizes():
    # views whose size is not a multiple of 8 (partial tiles, clamped probe pixels)
    for (W, H) in ((61, 37), (200, 9), (8, 8)):
        cam = wl.scene._camera(wl.make_scene(1), dict(wl.CONFIGS[1], width=W, height=H), 0)
        gb, _ = wl.scene.render_gbuffer(wl.make_scene(1), cam)
        pl = Pipeline(W, H, 64, 14)
        try:
            for f in (0, 3):
                pl.spawn(dev(gb), view_of(cam, f))
                torch.cuda.synchronize()
                sp = OP.spawn(gb, cam, f)
                for a, b in zip(OP.build_mips(sp["mask"]), pl.probes.mask_levels()):
                    assert np.array_equal(a, b)
        finally:
            pl.close()
