"""Pins for oracle/temporal.py (temporal upscale, Algorithm 1, Algorithm 4): the hysteresis against
closed forms worked by hand; the upscaled spawn against the plain spawn (u = 1) and hand-computed
Halton jitters; the float32 pixel positions against the float64 camera rays; reprojection under a
static camera (every probe stays), under a pan of exactly one tile (every probe moves one tile),
its rejections and its tie rule; persistence of probes across frames; the atlas rules."""
import math

import numpy as np

from oracle import probes as OP
from oracle import temporal as T
from oracle.key import distance_scale


class _Cam:
    def __init__(self, pos=(0.0, 0.0, 0.0), W=64, H=48, fov=math.radians(60.0)):
        self.pos = np.asarray(pos, np.float32)
        self.fwd = np.array([0, 0, -1], np.float32)
        self.right = np.array([1, 0, 0], np.float32)
        self.up = np.array([0, 1, 0], np.float32)
        self.fov_y, self.width, self.height = fov, W, H


def _wall_gbuffer(cam, depth=3.0):
    """G-buffer of the plane z = cam_z - depth facing +z, every pixel a hit."""
    W, H = cam.width, cam.height
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    d = OP.pixel_dirs(cam.pos, cam.fwd, cam.right, cam.up, cam.fov_y, W, H, xs, ys)
    g = np.zeros((H, W, 4), np.float32)
    g[..., 2] = 1.0
    g[..., 3] = (depth / -d[..., 2]).astype(np.float32)
    return g


# ------------------------------------------------------------------ Algorithm 4
def test_hysteresis_closed_forms():
    c = np.array([[0.2, 0.3, 0.4]])
    # new radiance darker than or as bright as the history: taken as is (alpha = 0)
    assert np.array_equal(T.hysteresis(c, 2 * c), c)
    assert np.array_equal(T.hysteresis(c, c), c)
    # l1 = 4 l2: alpha = ((4 - 1 - 1) / 4)^2 = 1/4
    p = np.array([[0.1, 0.1, 0.1]])
    n = np.array([[0.4, 0.4, 0.4]])
    np.testing.assert_allclose(T.hysteresis(n, p), n + 0.25 * (p - n), rtol=1e-15)
    # l1 = 2 l2: the numerator vanishes (continuous at the kink)
    np.testing.assert_allclose(T.hysteresis(2 * p, p), 2 * p, rtol=1e-15)
    # black history, bright new: alpha = clamp(1, 0, 0.95)^2 = 0.9025
    np.testing.assert_allclose(T.hysteresis(n, 0 * n), n * (1 - 0.9025), rtol=1e-15)
    # both black: 0 / 1e-4
    assert np.array_equal(T.hysteresis(0 * n, 0 * n), 0 * n)


# ------------------------------------------------------------------ spawn with upscale
def test_upscale_one_is_the_plain_spawn():
    cam = _Cam(W=61, H=35)
    for f in range(5):
        px, py, sx, sy = T.spawn_pixels(61, 35, f, 1)
        jx, jy = OP.halton_jitter(f)
        ty, tx = np.meshgrid(np.arange(sy), np.arange(sx), indexing="ij")
        assert np.array_equal(px, np.minimum(8 * tx + jx, 60).reshape(-1))
        assert np.array_equal(py, np.minimum(8 * ty + jy, 34).reshape(-1))
    assert (sx, sy) == (8, 5)


def test_upscale_two_jitter_by_hand():
    # Halton bases 2 and 3, points 1..4, scaled by 16: (8, 5), (4, 10), (12, 1), (2, 7)
    want = [(8, 5), (4, 10), (12, 1), (2, 7)]
    assert [T.upscale_jitter(f, 2) for f in range(4)] == want
    px, py, sx, sy = T.spawn_pixels(64, 48, 0, 2)
    assert (sx, sy) == (4, 3) and px.size == 12
    # one probe per 16 x 16 spawn tile, inside it
    assert np.array_equal(px // 16, np.tile(np.arange(4), 3)) and np.array_equal(py // 16, np.repeat(np.arange(3), 4))


def test_float32_pixel_positions_follow_the_camera_rays():
    cam = _Cam((0.5, -0.25, 2.0), W=80, H=45)
    rng = np.random.default_rng(1)
    xs, ys = rng.integers(0, 80, 200), rng.integers(0, 45, 200)
    d = rng.uniform(0.1, 50.0, 200).astype(np.float32)
    w32 = T.pixel_world_f32(T.cam_consts(cam), xs, ys, d)
    w64 = cam.pos.astype(np.float64) + OP.pixel_dirs(cam.pos, cam.fwd, cam.right, cam.up, cam.fov_y, 80, 45, xs, ys) * d[:, None]
    assert np.abs(w32 - w64).max() <= 2e-6 * (np.abs(cam.pos).max() + d.max())


# ------------------------------------------------------------------ Algorithm 1
def _spawned_state(gbuf, cam, f, upscale=1):
    st = T.empty_state((cam.width + 7) // 8, (cam.height + 7) // 8)
    T.spawn_fresh(st, gbuf, cam, f, upscale)
    return st


def test_static_camera_keeps_every_probe_in_place():
    cam = _Cam()
    g = _wall_gbuffer(cam)
    prev = _spawned_state(g, cam, 3)
    cur = T.reproject(prev, g, cam, np.zeros(g.shape[:2] + (2,), np.float32))
    assert np.array_equal(cur["mask"], prev["mask"])
    assert np.array_equal(cur["src"], np.arange(prev["mask"].size, dtype=np.uint32))
    assert np.array_equal(cur["pos"], prev["pos"])


def test_pan_by_one_tile_moves_every_probe_one_tile():
    # camera moved +x by 8 pixel widths at the wall's depth: the image content moves 8 pixels left,
    # so pixel p was at p + 8 in the previous frame (motion vector (+8, 0))
    cam0 = _Cam()
    depth = 3.0
    pitch = 2 * depth * math.tan(0.5 * cam0.fov_y) / cam0.height
    cam1 = _Cam((8 * pitch, 0.0, 0.0))
    g0, g1 = _wall_gbuffer(cam0, depth), _wall_gbuffer(cam1, depth)
    prev = _spawned_state(g0, cam0, 2)
    mv = np.zeros(g1.shape[:2] + (2,), np.float32)
    mv[..., 0] = 8.0
    cur = T.reproject(prev, g1, cam1, mv)
    tx_n = prev["tiles_x"]
    pm = prev["mask"]
    for ty in range(prev["tiles_y"]):
        for tx in range(tx_n):
            if tx == tx_n - 1:
                assert cur["mask"][ty, tx] == T.SENTINEL  # every q falls outside the image
                continue
            src = pm[ty, tx + 1]
            assert cur["src"][ty * tx_n + tx] == ty * tx_n + tx + 1
            assert cur["mask"][ty, tx] == src - 8  # same row, 8 pixels to the left
    # the reprojected probe sits on the surface point the source probe had
    t = np.flatnonzero(cur["src"] != T.SENTINEL)
    assert np.abs(cur["pos"][t, :3] - prev["pos"][cur["src"][t].astype(np.int64), :3]).max() < 1e-5


def test_reprojection_rejects_off_plane_and_turned_probes():
    cam = _Cam(W=16, H=16)
    g = _wall_gbuffer(cam)
    prev = _spawned_state(g, cam, 0)
    zero = np.zeros((16, 16, 2), np.float32)
    cs = distance_scale(cam.fov_y, 16, 16) * 3.0
    # every previous probe moved off the plane by more than cell_size: nothing reprojects
    far = {k: v.copy() if isinstance(v, np.ndarray) else v for k, v in prev.items()}
    far["pos"][:, 2] += np.float32(1.5 * cs)
    assert (T.reproject(far, g, cam, zero)["mask"] == T.SENTINEL).all()
    # ... by less than cell_size: all reproject
    near = {k: v.copy() if isinstance(v, np.ndarray) else v for k, v in prev.items()}
    near["pos"][:, 2] += np.float32(0.5 * cs)
    assert (T.reproject(near, g, cam, zero)["mask"] != T.SENTINEL).all()
    # normals turned by 20 degrees (cos = 0.94 <= 0.95): nothing; by 15 degrees (0.966): all
    for deg, kept in ((20.0, False), (15.0, True)):
        turned = {k: v.copy() if isinstance(v, np.ndarray) else v for k, v in prev.items()}
        a = math.radians(deg)
        turned["nrm"][:, 0:3] = np.array([math.sin(a), 0.0, math.cos(a)], np.float32)
        m = T.reproject(turned, g, cam, zero)["mask"]
        assert ((m != T.SENTINEL).all() if kept else (m == T.SENTINEL).all())


def test_equal_half_distances_go_to_the_lower_lane():
    # the probe's own pixel (0, 0) is sky in the new frame; pixels (1, 0) and (0, 1), one pitch away,
    # round to the same half-float distance: lane 1 beats lane 8
    cam = _Cam(W=8, H=8)
    g = _wall_gbuffer(cam, 3.0)
    st = T.empty_state(1, 1)
    st["mask"][0, 0] = 0  # pixel (0, 0)
    st["pos"][0, 0:3] = T.pixel_world_f32(T.cam_consts(cam), [0], [0], [g[0, 0, 3]])[0]
    st["nrm"][0] = (0.0, 0.0, 1.0, 1.0)
    g2 = g.copy()
    g2[0, 0, 3] = np.inf
    c = T.cam_consts(cam)
    w = T.pixel_world_f32(c, [1, 0], [0, 1], [g2[0, 1, 3], g2[1, 0, 3]])
    d = np.sqrt(((w - st["pos"][0, 0:3]) ** 2).sum(axis=1)).astype(np.float32)
    assert d.astype(np.float16)[0] == d.astype(np.float16)[1]
    out = T.reproject(st, g2, cam, np.zeros((8, 8, 2), np.float32))
    assert out["mask"][0, 0] == 1  # (y 0 << 16) | x 1


def test_static_camera_probes_persist_under_upscale():
    # u = 2, static camera: each frame adds its fresh tiles, none is lost
    cam = _Cam()
    g = _wall_gbuffer(cam)
    zero = np.zeros(g.shape[:2] + (2,), np.float32)
    st = T.empty_state(8, 6)
    seen = set()
    for f in range(8):
        st = T.reproject(st, g, cam, zero)
        ft = T.spawn_fresh(st, g, cam, f, 2)
        assert np.unique(ft).size == ft.size == 12  # one fresh tile per spawn tile
        seen |= set(int(t) for t in ft)
        assert set(np.flatnonzero(T.probe_valid(st))) == seen


def test_atlas_rules():
    rng = np.random.default_rng(4)
    cam = _Cam(W=32, H=32)
    g = _wall_gbuffer(cam)
    P = 16
    # plain frame (u = 1, no history): the gather of every probe
    st = T.empty_state(4, 4)
    ft = T.spawn_fresh(st, g, cam, 0, 1)
    rad = rng.uniform(0, 2, (P, 64, 3))
    has = rng.uniform(size=(P, 64)) > 0.2
    ln = rng.uniform(0.5, 5.0, P * 64)
    a = T.temporal_atlas(st, np.zeros((P, 64, 4)), ft, rad, has, ln)
    np.testing.assert_array_equal(a, OP.gather(np.ones(P, bool), rad, has, ln)[ft])
    # a fresh probe with history blends by Algorithm 4; a reprojected-only probe carries its source
    prev_atlas = rng.uniform(0, 2, (P, 64, 4))
    st2 = T.reproject(st, g, cam, np.zeros((32, 32, 2), np.float32))
    ft2 = T.spawn_fresh(st2, g, cam, 1, 2)  # 4 fresh tiles out of 16
    S = ft2.size
    a2 = T.temporal_atlas(st2, prev_atlas, ft2, rad[:S], has[:S], ln[:S * 64])
    g2 = OP.gather(np.ones(S, bool), rad[:S], has[:S], ln[:S * 64])
    for s, t in enumerate(ft2):
        np.testing.assert_allclose(a2[t, :, :3], T.hysteresis(g2[s, :, :3], prev_atlas[st2["src"][t], :, :3]))
        np.testing.assert_array_equal(a2[t, :, 3], g2[s, :, 3])
    others = np.setdiff1d(np.arange(P), ft2)
    np.testing.assert_array_equal(a2[others], prev_atlas[st2["src"][others].astype(np.int64)])
