"""Pins for the probe-atlas path of oracle/probes.py (Algorithm 5, Section 2.3): gather + project
equals the pinned probe integration; the gathered hit distance; and the filter pass against cases
worked by hand: identical probes stay unchanged, an isolated probe stays unchanged, a pair of
coplanar probes averages with the stated depth weight, and each rejection test (plane distance,
normal check, angle error) removes exactly the neighbours it should."""
import math

import numpy as np

from oracle import probes
from oracle.key import distance_scale
import workload as wl

S = probes.SENTINEL


class _Cam:
    def __init__(self, W, H, fov=math.radians(60.0)):
        self.width, self.height, self.fov_y = W, H, fov
        self.pos = np.zeros(3)


def _grid(pos, nrm, dist, tiles_x, tiles_y, valid=None):
    """Spawn dict of a tiles_x x tiles_y probe grid, probe pixel = tile corner."""
    P = tiles_x * tiles_y
    valid = np.ones(P, bool) if valid is None else np.asarray(valid, bool)
    p = np.arange(P)
    px, py = 8 * (p % tiles_x), 8 * (p // tiles_x)
    mask = np.where(valid, (py << 16) | px, S).astype(np.uint32).reshape(tiles_y, tiles_x)
    return dict(mask=mask, pos=np.asarray(pos, np.float64), nrm=np.asarray(nrm, np.float64),
                dist=np.asarray(dist, np.float64), valid=valid, tiles_x=tiles_x, tiles_y=tiles_y)


def _wall(tiles_x, tiles_y, spacing=0.05, depth=2.0):
    """Probes on the plane z = -depth facing +z (towards a camera at the origin)."""
    P = tiles_x * tiles_y
    p = np.arange(P)
    pos = np.stack([(p % tiles_x) * spacing, (p // tiles_x) * spacing, np.full(P, -depth)], axis=1)
    nrm = np.tile([0.0, 0.0, 1.0], (P, 1))
    return pos, nrm, np.linalg.norm(pos, axis=1)


def test_gather_then_project_equals_integrate():
    fr = wl.make_frame(1, 1)
    sp = probes.spawn(fr.gbuffer, fr.camera, 1)
    rng = np.random.default_rng(3)
    P, rpp = sp["valid"].size, fr.rays_per_probe
    rad = rng.uniform(0, 2, (P, rpp, 3))
    has = rng.uniform(size=(P, rpp)) > 0.3
    ln = rng.uniform(0.1, 3.0, P * rpp)
    atlas = probes.gather(sp["valid"], rad, has, ln)
    a = probes.project(sp["valid"], sp["nrm"], atlas)
    b = probes.integrate(sp["valid"], sp["nrm"], rad, has)
    assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())


def test_gather_hit_distance_means_hits_only():
    rpp = 128  # two rays per cell
    rad = np.ones((2, rpp, 3))
    has = np.ones((2, rpp), bool)
    ln = np.full((2, rpp), 2.0)
    ln[0, 0], ln[0, 64] = 1.0, 3.0           # cell 0: mean of 1 and 3
    ln[0, 1], ln[0, 65] = np.inf, 5.0        # cell 1: one miss, one hit at 5
    ln[0, 2], ln[0, 66] = np.inf, np.inf     # cell 2: misses only
    has[0, 3] = has[0, 67] = False           # cell 3: no sample at all
    atlas = probes.gather(np.array([True, False]), rad, has, ln.reshape(-1))
    assert atlas[0, 0, 3] == 2.0 and atlas[0, 1, 3] == 5.0
    assert np.isinf(atlas[0, 2, 3]) and np.isinf(atlas[0, 3, 3])
    assert np.all(atlas[1] == 0.0)           # no probe: zeros


def test_filter_leaves_identical_probes_unchanged():
    pos, nrm, dist = _wall(5, 4)
    sp = _grid(pos, nrm, dist, 5, 4)
    atlas = np.tile(np.concatenate([np.linspace(0.1, 2.0, 64)[:, None].repeat(3, 1), np.full((64, 1), 1.5)], 1),
                    (20, 1, 1))
    cam = _Cam(40, 32)
    for axis in (0, 1):
        out, _ = probes.filter_pass(atlas, sp, cam, axis)
        np.testing.assert_allclose(out, atlas, rtol=1e-13)


def test_filter_isolated_probe_unchanged():
    pos, nrm, dist = _wall(3, 3)
    valid = np.zeros(9, bool)
    valid[4] = True
    sp = _grid(pos, nrm, dist, 3, 3, valid)
    atlas = np.random.default_rng(1).uniform(0, 1, (9, 64, 4))
    out, _ = probes.filter_pass(atlas, sp, _Cam(24, 24), 0)
    np.testing.assert_array_equal(out[4], atlas[4])


def _pair(offset_q, nrm_q=(0.0, 0.0, 1.0), depth_q=None):
    """Two probes in a 2x1 grid: p at tile 0 on the wall at depth 2, q at tile 1."""
    pos = np.array([[0.0, 0.0, -2.0], list(offset_q)], np.float64)
    nrm = np.array([[0.0, 0.0, 1.0], list(nrm_q)], np.float64)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    dist = np.linalg.norm(pos, axis=1) if depth_q is None else np.array([2.0, depth_q])
    return _grid(pos, nrm, dist, 2, 1)


HD = (1920, 1080)  # cell_size(2 m) = 2 tan(8 fov / 1080) ~ 3.1 cm


def test_filter_pair_closed_form():
    # q beside p on the same plane, slightly farther from the camera: weight 1 / (1 + |dd| / cs)
    cam = _Cam(*HD)
    sp = _pair((0.03, 0.0, -2.0))
    rng = np.random.default_rng(2)
    atlas = np.concatenate([rng.uniform(0, 1, (2, 64, 3)), np.full((2, 64, 1), 10.0)], axis=-1)
    out, _ = probes.filter_pass(atlas, sp, cam, 0)
    cs = distance_scale(cam.fov_y, *HD) * 2.0
    w = 1.0 / (1.0 + abs(2.0 - math.sqrt(0.03 ** 2 + 4.0)) / cs)
    # only step +1 finds q: steps -1..-3 and +2, +3 leave the 2x1 grid (and its 1x1 MIP level)
    expect = (atlas[0, :, :3] + w * atlas[1, :, :3]) / (1.0 + w)
    np.testing.assert_allclose(out[0, :, :3], expect, rtol=1e-12)
    np.testing.assert_allclose(out[0, :, 3], 10.0, rtol=1e-12)


def test_filter_rejects_neighbour_off_the_plane():
    cam = _Cam(*HD)
    cs = distance_scale(cam.fov_y, *HD) * 2.0
    atlas = np.concatenate([np.zeros((2, 64, 3)), np.full((2, 64, 1), 10.0)], axis=-1)
    atlas[1, :, :3] = 1.0
    near = _pair((0.03, 0.0, -2.0 + 0.5 * cs))
    far = _pair((0.03, 0.0, -2.0 + 1.5 * cs))
    o_near, _ = probes.filter_pass(atlas, near, cam, 0)
    o_far, _ = probes.filter_pass(atlas, far, cam, 0)
    assert np.all(o_near[0, :, :3] > 0.0)
    assert np.all(o_far[0, :, :3] == 0.0)


def test_filter_normal_check_rejects_cells_behind_the_neighbour():
    # q tilted 80 degrees about y: cells whose direction has a negative dot with n_q are skipped
    cam = _Cam(*HD)
    th = math.radians(80.0)
    sp = _pair((0.03, 0.0, -2.0), nrm_q=(math.sin(th), 0.0, math.cos(th)))
    atlas = np.concatenate([np.zeros((2, 64, 3)), np.full((2, 64, 1), np.inf)], axis=-1)
    atlas[1, :, :3] = 1.0
    out, _ = probes.filter_pass(atlas, sp, cam, 0)
    d = probes.cell_dirs_world(sp["nrm"])[0]
    behind = d @ sp["nrm"][1] < 0.0
    assert behind.any() and (~behind).any()
    assert np.all(out[0, behind, :3] == 0.0) and np.all(out[0, ~behind, :3] > 0.0)


def test_filter_angle_test_rejects_close_hits_seen_from_afar():
    # q 0.3 m to the side; a short hit distance makes the hit point seen from p far off the cell
    # direction (rejected), a long one keeps it within pi/50 (accepted)
    cam = _Cam(*HD)
    sp = _pair((0.3, 0.0, -2.0), depth_q=2.0)
    sp["dist"] = np.array([2.0, 2.0])
    atlas = np.zeros((2, 64, 4))
    atlas[1, :, :3] = 1.0
    c = 27  # a cell near the normal direction
    d = probes.cell_dirs_world(sp["nrm"])[0, c]
    for hdist, accepted in ((0.5, False), (1000.0, True)):
        atlas[:, :, 3] = hdist
        out, _ = probes.filter_pass(atlas, sp, cam, 0)  # coplanar: only the angle test decides
        hp = sp["pos"][1] + d * hdist
        ang = d @ ((hp - sp["pos"][0]) / np.linalg.norm(hp - sp["pos"][0]))
        assert (ang >= probes.FILTER_COS) == accepted
        assert (out[0, c, 0] > 0.0) == accepted
