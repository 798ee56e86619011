"""GPU parity of the screen-probe stage (Sections 2.1.1, 2.1.5, 2.4) against the
oracle, through the C ABI: probe mask and MIP chain bit-exact, probe
positions to float32 rounding, SH irradiance and interpolated irradiance
within 1e-4 relative, flags identical outside decision-sensitive pixels."""
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

from _gpu_util import Pipeline, close, dev, require_gpu, u32, view_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _sh_gpu(pl):
    return pl.probes.sh.cpu().numpy()[:, :27].reshape(-1, 9, 3).astype(np.float64)


def _compare_frame(pl, fr, out, allow_sensitive_frac):
    P = pl.probes.layout.num_probes
    # spawn: mask levels bit-exact, probe positions to float32 rounding
    mips_o = OP.build_mips(out["spawn"]["mask"])
    mips_g = pl.probes.mask_levels()
    assert len(mips_o) == len(mips_g)
    for a, b in zip(mips_o, mips_g):
        assert np.array_equal(a, b)
    pos_g = pl.probes.pos.cpu().numpy()
    nrm_g = pl.probes.nrm.cpu().numpy()
    v = out["spawn"]["valid"]
    assert np.array_equal(nrm_g[:, 3] == 1.0, v)
    scale = 1.0 + np.abs(fr.camera.pos).max() + np.abs(out["spawn"]["dist"]).max()
    assert np.abs(pos_g[v, :3] - out["spawn"]["pos"][v]).max() < 4e-7 * scale
    assert np.array_equal(nrm_g[v, :3], out["spawn"]["nrm"][v])
    # probe SH: relative to the probe's band-0 magnitude (individual coefficients can cancel)
    sg, so = _sh_gpu(pl), out["sh"]
    mag = np.abs(so[:, 0:1, :]).max(axis=2, keepdims=True) + 1e-6
    err = np.abs(sg - so) / mag
    assert err.max() < 1e-4, err.max()
    # irradiance at each probe normal
    Eg = OSH.irradiance(sg[v], out["spawn"]["nrm"][v])
    Eo = OSH.irradiance(so[v], out["spawn"]["nrm"][v])
    assert close(Eg, Eo, atol=1e-6).all()
    # interpolation
    irr = pl.irr.cpu().numpy()
    flag_g = irr[..., 3].astype(np.int64)
    flag_o = out["flag"]
    wsum, margin = out["diag"]["wsum"], out["diag"]["margin"]
    # decision-sensitive pixels: a neighbour's plane test within 1e-3 of its cut, or a weight
    # sum so small that float32 weight rounding moves the weighted mean by more than 1e-4
    sensitive = (margin < 1e-3) | ((wsum > 0) & (wsum < 1e-2))
    agree = ~sensitive
    assert np.array_equal(flag_g[agree], flag_o[agree]), np.count_nonzero(flag_g[agree] != flag_o[agree])
    # float32 evaluation of sum_k A_l Y_k(n) c_k cancels in dark pixels: bound the absolute error by the
    # magnitude of the summed terms (emag) as well as 1e-4 of the value
    emag = out["diag"]["emag"][..., None]
    ok = (np.abs(irr[..., :3] - out["irr"]) <= 1e-4 * np.abs(out["irr"]) + 1e-5 * emag + 1e-7).all(axis=-1)
    bad = agree & ~ok
    assert np.count_nonzero(bad) == 0, (np.count_nonzero(bad), np.abs(irr[..., :3] - out["irr"])[bad].max())
    X = flag_o.size
    assert np.count_nonzero(sensitive) <= allow_sensitive_frac * X, np.count_nonzero(sensitive) / X
    return np.count_nonzero(sensitive), np.count_nonzero(flag_g != flag_o)


def _run_frames(config, frames, allow_sensitive_frac=0.02):
    cfg = wl.CONFIGS[config]
    fr0 = frames[0]
    pl = Pipeline(fr0.camera.width, fr0.camera.height, fr0.rays_per_probe, cfg["log2_slots"])
    oc = OracleCache(cfg["log2_slots"])
    stats = []
    try:
        for fr in frames:
            view = view_of(fr.camera, fr.frame)
            gb = dev(fr.gbuffer)
            rec = dev(fr.records)
            pl.frame(gb, rec, view)
            torch.cuda.synchronize()
            out = run_frame(oc, fr)
            stats.append(_compare_frame(pl, fr, out, allow_sensitive_frac))
    finally:
        pl.close()
    return stats


def test_cornell_chain():
    _run_frames(1, wl.make_frames(1))


def test_1080p_chain_full_size():
    scene = wl.make_scene(2)
    _run_frames(2, [wl.make_frame(2, f, scene) for f in (0, 1)])


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
