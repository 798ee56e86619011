"""GPU parity of the probe atlas path (Sections 2.1.4, 2.3, 2.4.2; Algorithm 5) against the oracle:
gather (cell radiance + hit distance), gather + project against the fused integrate, one filter
pass on the same input atlas, and the whole gather -> filter x -> filter y -> project chain.

The filter's accept/reject tests compare float32 quantities (plane distance vs cell_size, normal
dot, angle cosine vs cos(pi/50)); cells whose oracle margin to any of these cuts is below 1e-4 can
legitimately decide the other way in float32, so the strict comparison covers the others, and
over all cells the mismatches must stay rare.  Many margins are exactly 0 -- the diagonal cells'
directions have an exactly zero component, so against an axis-aligned neighbour normal the dot
is +-0 on both sides and decides alike -- which is why the bound is on mismatches, not margins."""
import numpy as np
import pytest
import torch

import paper_2310_19855_gb300 as gi
import workload as wl
from oracle import probes as OP
from oracle.cache import OracleCache
from oracle.frame import ray_radiance
from paper_2310_19855_gb300.pipeline import Pipeline, view_of

from _gpu_util import dev, require_gpu

pytestmark = pytest.mark.gpu
MARGIN = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _frame(kind):
    if kind == "cornell":
        return wl.make_frame(1, 1), wl.CONFIGS[1]["log2_slots"]
    cfg = dict(wl.CONFIGS[2], width=320, height=184, n_boxes=512, room=(24.0, 8.0, 24.0), frames=8)
    seed = wl.scene.SEED_BASE + 4200
    return wl.make_frame(cfg, 3, wl.make_scene(cfg, seed), seed_base=seed), 18


def _gpu_frame(fr, log2_slots):
    cam = fr.camera
    pl = Pipeline(cam.width, cam.height, fr.rays_per_probe, log2_slots)
    view = view_of(cam, fr.frame)
    R = dev(fr.records)
    gb = dev(fr.gbuffer)
    pl.spawn(gb, view)
    pl.update(R, view)
    pl.resolve(fr.frame)
    return pl, view, R


def _oracle_frame(fr, log2_slots):
    cam = fr.camera
    oc = OracleCache(log2_slots)
    sp = OP.spawn(fr.gbuffer, cam, fr.frame)
    ident = oc.update(fr.records, fr.frame, cam.pos, cam.fov_y, cam.width, cam.height)
    oc.resolve(fr.frame)
    rad, has = ray_radiance(oc, fr.records, ident)
    P = sp["valid"].size
    rpp = fr.rays_per_probe
    atlas = OP.gather(sp["valid"], rad.reshape(P, rpp, 3), has.reshape(P, rpp), fr.records[9])
    return sp, atlas


def _close_mask(got, want, rel, atol):
    g, w = np.asarray(got, np.float64), np.asarray(want, np.float64)
    both_inf = np.isinf(g) & np.isinf(w) & (np.sign(g) == np.sign(w))
    with np.errstate(invalid="ignore"):
        return both_inf | (np.abs(g - w) <= rel * np.abs(w) + atol)


def _atlas_close(got, want, rel=1e-4, atol=1e-7):
    ok = _close_mask(got, want, rel, atol)
    assert ok.all(), (np.count_nonzero(~ok), ok.size)


@pytest.mark.parametrize("kind", ["cornell", "boxes"])
def test_gather_matches_oracle(kind):
    fr, ls = _frame(kind)
    pl, view, R = _gpu_frame(fr, ls)
    try:
        atlas = torch.empty((pl.probes.layout.num_probes, 64, 4), dtype=torch.float32, device="cuda")
        gi.gi_probes_gather(pl.cache, pl.probes.struct, pl.slot_ids, R[9], fr.rays_per_probe, atlas)
        got = atlas.cpu().numpy()
    finally:
        pl.close()
    _, want = _oracle_frame(fr, ls)
    _atlas_close(got, want)


def test_gather_then_project_agrees_with_integrate():
    # the two-pass form (atlas in between, a warp per probe) and the fused pass (a thread per probe)
    # sum the cells in other orders: float32 agreement relative to the probe's band-0 magnitude
    fr, ls = _frame("boxes")
    pl, view, R = _gpu_frame(fr, ls)
    try:
        pl.integrate()
        fused = pl.probes.sh.cpu().numpy()[:, :27].reshape(-1, 9, 3).astype(np.float64)
        atlas = torch.empty((pl.probes.layout.num_probes, 64, 4), dtype=torch.float32, device="cuda")
        gi.gi_probes_gather(pl.cache, pl.probes.struct, pl.slot_ids, R[9], fr.rays_per_probe, atlas)
        pl.probes.sh.fill_(-1.0)
        gi.gi_probes_project(pl.probes.struct, atlas)
        two = pl.probes.sh.cpu().numpy()[:, :27].reshape(-1, 9, 3).astype(np.float64)
        mag = np.abs(two[:, 0:1, :]).max(axis=2, keepdims=True) + 1e-6
        assert (np.abs(fused - two) / mag).max() < 1e-5
    finally:
        pl.close()


def _filter_both(fr, ls, axis):
    """One filter pass on the oracle's own atlas (rounded to float32) on both sides."""
    sp, atlas = _oracle_frame(fr, ls)
    a32 = atlas.astype(np.float32)
    pl, view, R = _gpu_frame(fr, ls)
    try:
        src = dev(a32)
        dst = torch.empty_like(src)
        gi.gi_probes_filter(pl.probes.struct, view, src, dst, axis)
        got = dst.cpu().numpy()
    finally:
        pl.close()
    want, margin = OP.filter_pass(a32.astype(np.float64), sp, fr.camera, axis)
    return got, want, margin, sp


@pytest.mark.parametrize("kind", ["cornell", "boxes"])
@pytest.mark.parametrize("axis", [0, 1])
def test_filter_pass_matches_oracle(kind, axis):
    fr, ls = _frame(kind)
    got, want, margin, sp = _filter_both(fr, ls, axis)
    robust = margin > MARGIN
    _atlas_close(got[robust], want[robust], rel=2e-6, atol=1e-7)
    cell_ok = _close_mask(got, want, 2e-6, 1e-7).all(axis=-1)
    valid = sp["valid"][:, None].repeat(64, axis=1)
    assert np.count_nonzero(~cell_ok & valid) <= 0.005 * np.count_nonzero(valid)
    # the filter changed something: some accepted neighbours
    assert np.abs(want[..., :3] - _oracle_frame(fr, ls)[1][..., :3]).max() > 0.0


def test_filtered_chain_matches_oracle():
    fr, ls = _frame("boxes")
    sp, atlas = _oracle_frame(fr, ls)
    a1, m1 = OP.filter_pass(atlas, sp, fr.camera, 0)
    a2, m2 = OP.filter_pass(a1, sp, fr.camera, 1)
    want = OP.project(sp["valid"], sp["nrm"], a2)
    pl, view, R = _gpu_frame(fr, ls)
    try:
        pl.integrate_filtered(R, view)
        got = pl.probes.sh.cpu().numpy()[:, :27].reshape(-1, 9, 3)
    finally:
        pl.close()
    # SH within 1e-4 of the probe's largest band-0 coefficient; a probe may differ only through a
    # near-tie decision (its own or a first-pass neighbour's), which must stay rare
    scale = np.abs(want[:, 0, :]).max(axis=1)[:, None, None]
    err = (np.abs(got - want) / np.maximum(scale, 1e-12)).max(axis=(1, 2))
    valid = sp["valid"]
    bad = valid & (err > 1e-4)
    assert np.count_nonzero(bad) <= 0.01 * np.count_nonzero(valid), (np.count_nonzero(bad), err[valid].max())


def test_full_size_1080p_filter_pass():
    # one filter pass of the 1080p workload at full size (32,400 probes) on the oracle's atlas
    fr = wl.make_frame(2, 0)
    ls = wl.CONFIGS[2]["log2_slots"]
    sp, atlas = _oracle_frame(fr, ls)
    a32 = atlas.astype(np.float32)
    pl, view, R = _gpu_frame(fr, ls)
    try:
        src = dev(a32)
        dst = torch.empty_like(src)
        gi.gi_probes_filter(pl.probes.struct, view, src, dst, 0)
        got = dst.cpu().numpy()
    finally:
        pl.close()
    want, margin = OP.filter_pass(a32.astype(np.float64), sp, fr.camera, 0)
    robust = margin > MARGIN
    _atlas_close(got[robust], want[robust], rel=2e-6, atol=1e-7)
    cell_ok = _close_mask(got, want, 2e-6, 1e-7).all(axis=-1)
    valid = sp["valid"][:, None].repeat(64, axis=1)
    assert np.count_nonzero(~cell_ok & valid) <= 0.005 * np.count_nonzero(valid)
