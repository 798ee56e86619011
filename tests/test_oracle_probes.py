"""Pins for oracle/probes.py: Halton jitter (golden values from the
sequence's definition), spawn against the tracer's own hit points, the
probe-mask MIP chain against a brute-force Morton-order search, Algorithm 3
properties, the radiance-backup rule, and interpolation special cases."""
import json
import math
import os

import numpy as np

from oracle import probes, sh
from oracle.key import distance_scale
import workload as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sequences.json")))
S = probes.SENTINEL


def test_halton_jitter_golden():
    for i in range(16):
        assert probes.halton_jitter(i) == (GOLDEN["halton2_times8"][i], GOLDEN["halton3_times8"][i])


def test_spawn_positions_match_tracer_hit_points():
    fr = wl.make_frame(1, 2)
    sp = probes.spawn(fr.gbuffer, fr.camera, 2)
    assert sp["jitter"] == probes.halton_jitter(2)
    jx, jy = sp["jitter"]
    m = sp["mask"]
    valid = m != S
    assert np.array_equal(valid.reshape(-1), fr.probe_valid)
    px, py = m & 0xFFFF, m >> 16
    ty, tx = np.nonzero(valid)
    assert np.all(px[valid] == np.minimum(8 * tx + jx, 63)) and np.all(py[valid] == np.minimum(8 * ty + jy, 63))
    # the tracer's own float32 hit point of the same pixel
    _, hit = wl.scene.render_gbuffer(wl.make_scene(1), fr.camera)
    ref = hit[py[valid], px[valid]].astype(np.float64)
    got = sp["pos"][valid.reshape(-1)]
    assert np.abs(got - ref).max() < 2e-6 * (1 + np.abs(ref).max())


def _morton_first_valid(m0, level, X, Y):
    """First valid entry of the level-`level` block (X, Y) of m0 in recursive (x, y) scan order."""
    n = 1 << level
    best, best_code = S, None
    for dy in range(n):
        for dx in range(n):
            x, y = X * n + dx, Y * n + dy
            if y >= m0.shape[0] or x >= m0.shape[1] or m0[y, x] == S:
                continue
            code = 0
            for bit in range(level):
                code |= ((dx >> bit) & 1) << (2 * bit) | ((dy >> bit) & 1) << (2 * bit + 1)
            if best_code is None or code < best_code:
                best, best_code = m0[y, x], code
    return best


def test_mip_chain_matches_morton_bruteforce():
    rng = np.random.default_rng(0)
    for (h, w) in ((13, 21), (8, 8), (1, 5), (9, 1)):
        m0 = np.where(rng.uniform(size=(h, w)) < 0.3, rng.integers(0, 1 << 20, (h, w)), S).astype(np.uint32)
        mips = probes.build_mips(m0)
        assert mips[-1].shape == (1, 1)
        for lev, m in enumerate(mips):
            for Y in range(m.shape[0]):
                for X in range(m.shape[1]):
                    assert m[Y, X] == _morton_first_valid(m0, lev, X, Y)


def test_find_closest_probe_properties():
    rng = np.random.default_rng(1)
    m0 = np.where(rng.uniform(size=(17, 30)) < 0.1, np.arange(17 * 30).reshape(17, 30), S).astype(np.uint32)
    mips = probes.build_mips(m0)
    ty, tx = np.meshgrid(np.arange(-1, 18), np.arange(-1, 31), indexing="ij")
    for (ox, oy) in probes.NEIGHBOUR_OFFSETS:
        q = probes.find_closest_probe(mips, tx, ty, ox, oy)
        x0, y0 = tx + ox, ty + oy
        inb = (x0 >= 0) & (x0 < 30) & (y0 >= 0) & (y0 < 17)
        # outside the grid at level 0: nothing
        assert np.all(q[~inb] == S)
        # a valid level-0 neighbour is returned as is
        direct = np.zeros_like(inb)
        direct[inb] = m0[y0[inb], x0[inb]] != S
        assert np.all(q[direct] == m0[y0[direct], x0[direct]])
        # otherwise the probe returned lies in the block of the level where it was found
        for idx in zip(*np.nonzero(inb & ~direct & (q != S))):
            val = int(q[idx])
            qy, qx = divmod(val, 30)
            X, Y = int(tx[idx]), int(ty[idx])
            for lev in range(len(mips)):
                bx, by = X + ox, Y + oy
                if not (0 <= bx < mips[lev].shape[1] and 0 <= by < mips[lev].shape[0]):
                    break
                if mips[lev][by, bx] != S:
                    assert mips[lev][by, bx] == val
                    assert bx << lev <= qx < (bx + 1) << lev and by << lev <= qy < (by + 1) << lev
                    break
                X >>= 1
                Y >>= 1


def test_radiance_backup_fills_empty_cells():
    rad = np.zeros((1, 64, 3))
    has = np.zeros((1, 64), bool)
    rad[0, :10] = 2.0
    has[0, :10] = True
    a = probes.integrate(np.ones(1, bool), np.array([[0.0, 0.0, 1.0]]), rad, has)
    full = probes.integrate(np.ones(1, bool), np.array([[0.0, 0.0, 1.0]]), np.full((1, 64, 3), 2.0),
                            np.ones((1, 64), bool))
    assert np.allclose(a, full, atol=1e-13)
    none = probes.integrate(np.ones(1, bool), np.array([[0.0, 0.0, 1.0]]), rad, np.zeros((1, 64), bool))
    assert np.all(none == 0)


class _Cam:
    def __init__(self, W, H):
        self.pos = np.array([0.0, 0.0, 0.0], np.float32)
        self.fwd = np.array([0.0, 0.0, -1.0], np.float32)
        self.right = np.array([1.0, 0.0, 0.0], np.float32)
        self.up = np.array([0.0, 1.0, 0.0], np.float32)
        self.fov_y = math.radians(60.0)
        self.width, self.height = W, H


def _plane_gbuffer(W, H, depth_plane=3.0):
    """A camera facing the plane z = -depth_plane: G-buffer normal +z, distance along each ray."""
    cam = _Cam(W, H)
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    d = probes.pixel_dirs(cam.pos, cam.fwd, cam.right, cam.up, cam.fov_y, W, H, xs, ys)
    t = depth_plane / -d[..., 2]
    gb = np.zeros((H, W, 4), np.float32)
    gb[..., 2] = 1.0
    gb[..., 3] = t
    return gb, cam


def test_interpolation_of_identical_probes_is_exact():
    gb, cam = _plane_gbuffer(40, 24)
    sp = probes.spawn(gb, cam, 0)
    P = sp["valid"].size
    rng = np.random.default_rng(5)
    c = rng.normal(size=(9, 3))
    coeffs = np.broadcast_to(c, (P, 9, 3)).copy()
    irr, flag, _ = probes.interpolate(gb, cam, sp, coeffs)
    want = sh.irradiance(c[None], np.array([[0.0, 0.0, 1.0]]))[0]
    assert np.all(flag == 0)
    assert np.abs(irr - want).max() < 1e-12 * np.abs(want).max()


def test_interpolation_relaxed_none_and_sky_flags():
    gb, cam = _plane_gbuffer(32, 32)
    gb[0:8, 0:8, 3] = np.inf  # sky pixels in the first tile
    sp = probes.spawn(gb, cam, 0)
    P = sp["valid"].size
    coeffs = np.zeros((P, 9, 3))
    coeffs[:, 0, :] = 1.0
    # move every probe far off the pixel plane: all weights vanish, interpolation relaxes
    sp_far = dict(sp)
    sp_far["pos"] = sp["pos"] + np.array([0.0, 0.0, 10.0])
    irr, flag, _ = probes.interpolate(gb, cam, sp_far, coeffs)
    sky = ~np.isfinite(gb[..., 3])
    assert np.all(flag[sky] == probes.FLAG_SKY) and np.all(irr[sky] == 0)
    assert np.all(flag[~sky] == probes.FLAG_RELAXED)
    assert np.allclose(irr[~sky], math.pi * sh.C0)
    # no probe anywhere: flag 2 and zero
    sp_none = dict(sp)
    sp_none["mask"] = np.full_like(sp["mask"], S)
    irr, flag, _ = probes.interpolate(gb, cam, sp_none, coeffs)
    assert np.all(flag[~sky] == probes.FLAG_NONE) and np.all(irr == 0)


def test_interpolation_weights_plane_cut_and_bilinear():
    # two probe values: where a neighbour is beyond cell_size from the plane its weight is 0
    gb, cam = _plane_gbuffer(16, 16)
    sp = probes.spawn(gb, cam, 0)
    P = sp["valid"].size
    coeffs = np.zeros((P, 9, 3))
    coeffs[:, 0, 0] = np.arange(P)
    irr, flag, diag = probes.interpolate(gb, cam, sp, coeffs)
    # pixel (7, 7): base tile (0, 0); neighbours are the four probes, all on the plane (pd ~ 0)
    y, x = 7, 7
    fx = fy = (x + 0.5 - 4.0) / 8.0
    wts = np.array([(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy])
    pts = sp["pos"]
    dist = gb[y, x, 3]
    d = probes.pixel_dirs(cam.pos, cam.fwd, cam.right, cam.up, cam.fov_y, 16, 16, np.array(x), np.array(y))
    Pp = d * dist
    cs = distance_scale(cam.fov_y, 16, 16) * dist
    wd = np.maximum(0, 1 - np.abs((pts - Pp) @ np.array([0, 0, 1.0])) / cs)
    vals = math.pi * sh.C0 * np.arange(P)  # A_0 * L_00 * Y_00
    want = (wts * wd * vals).sum() / (wts * wd).sum()
    assert flag[y, x] == 0
    assert abs(irr[y, x, 0] - want) < 1e-12 * max(1.0, abs(want))
