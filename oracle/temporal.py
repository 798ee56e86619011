"""Screen-probe temporal path: temporal upscale of the probe spawn (Section 2.1.1, "Temporal
Upscale"), screen-probe reprojection (Algorithm 1), the biased temporal hysteresis (Algorithm 4)
and the probe atlas each frame carries to the next.

Test infrastructure only: nothing in the product imports this module.

Readings taken here (the paper leaves them open):

* Spawn with upscale u: spawn tiles of 8u x 8u pixels; the frame's jitter is
  (floor(8u H_2(f+1)), floor(8u H_3(f+1))), the Halton point f+1 with bases 2 and 3, shared by
  every spawn tile; the probe pixel of spawn tile S is min(8u S + jitter, (W-1, H-1)) and the 8x8
  tile containing it receives the frame's fresh probe, unless the pixel is sky.  u = 1 is the
  plain spawn.  (With bases 2 and 3 the first four frames of u = 2 cover three of the four 8x8
  tiles of a spawn tile; the rest fills in later frames and through reprojection.)
* Motion vectors (an input, as a renderer supplies them): per pixel, the offset in pixels from
  the pixel centre to where its surface point was in the previous frame; the previous pixel is
  q = (floor(x + 0.5 + mv_x), floor(y + 0.5 + mv_y)).
* "probe_q": the previous frame's level-0 probe mask at q's 8x8 tile (no MIP search).
* World position of a pixel, of a fresh probe and of a reprojected one: the camera ray through
  the pixel centre times the G-buffer distance, every operation in float32 round-to-nearest in a
  fixed order (no fused multiply-add): sx = (2 (x + 0.5) inv_w - 1) sx_scale,
  sy = (1 - 2 (y + 0.5) inv_h) sy_scale, dir = (fwd + sx right) + sy up,
  len = sqrt((dx^2 + dy^2) + dz^2), world = pos + dir (d / len), with sy_scale = tan(fov/2),
  sx_scale = tan(fov/2) W/H, inv_w = 1/W, inv_h = 1/H each rounded once from float64.  The
  reprojection's decisions (plane distance, normal check, half-float distance, argmin) are then
  taken from identical float32 values on both sides.
* cell_size = distance_scale (Algorithm 6, float64 rounded once to float32) x the pixel's
  distance, in float32.
* Score = half(dist) << 16 | lane, lane = 8 ly + lx inside the tile; the smallest score wins
  (ties to the lower lane); the initial score half(65504) << 16 | 0xFFFF marks "no candidate".
* The reprojected probe sits at the winning pixel (its current position and normal) and carries
  the radiance atlas of the previous probe the winner found.
* Hysteresis: curr = the fresh probe's gathered cell radiance, prev = the same cell of the tile's
  reprojected probe (the paper's reconstruction with parallax correction belongs to ray
  guiding, which is out of scope); the result keeps the fresh cell's hit distance.  A tile with
  a reprojected probe and no fresh one carries the source atlas unchanged; a tile with neither
  has no probe.
"""
from __future__ import annotations

import math

import numpy as np

from . import probes as OP
from .key import distance_scale

F32 = np.float32
SENTINEL = OP.SENTINEL
SCORE_NONE = (0x7BFF << 16) | 0xFFFF  # half(65504) << 16 | 0xFFFF


# ------------------------------------------------------------------ spawn with temporal upscale
def radical_inverse_scaled(i: int, base: int, scale: int) -> int:
    """floor(scale * radical_inverse_base(i)), exact (digits of i reversed behind the radix point)."""
    num, den = 0, 1
    while i:
        num = num * base + i % base
        den *= base
        i //= base
    return (scale * num) // den


def upscale_jitter(frame: int, upscale: int):
    return (radical_inverse_scaled(frame + 1, 2, 8 * upscale), radical_inverse_scaled(frame + 1, 3, 8 * upscale))


def spawn_pixels(width: int, height: int, frame: int, upscale: int):
    """Probe pixel (px, py) of every spawn tile, spawn-tile major (row by row), and the grid size."""
    s = 8 * upscale
    sx_n, sy_n = (width + s - 1) // s, (height + s - 1) // s
    jx, jy = upscale_jitter(frame, upscale)
    sy, sx = np.meshgrid(np.arange(sy_n), np.arange(sx_n), indexing="ij")
    px = np.minimum(s * sx + jx, width - 1).reshape(-1)
    py = np.minimum(s * sy + jy, height - 1).reshape(-1)
    return px, py, sx_n, sy_n


# ------------------------------------------------------------------ exact float32 pixel positions
def cam_consts(cam):
    th = math.tan(0.5 * float(cam.fov_y))
    return dict(pos=np.asarray(cam.pos, F32), fwd=np.asarray(cam.fwd, F32), right=np.asarray(cam.right, F32),
                up=np.asarray(cam.up, F32), sy_scale=F32(th), sx_scale=F32(th * cam.width / cam.height),
                inv_w=F32(1.0 / cam.width), inv_h=F32(1.0 / cam.height))


def pixel_world_f32(c, x, y, d):
    """World position (n, 3) float32 of pixels (x, y) at distance d, operation by operation."""
    x = np.asarray(x).astype(F32)
    y = np.asarray(y).astype(F32)
    d = np.asarray(d, F32)
    sx = ((F32(2.0) * (x + F32(0.5))) * c["inv_w"] - F32(1.0)) * c["sx_scale"]
    sy = (F32(1.0) - (F32(2.0) * (y + F32(0.5))) * c["inv_h"]) * c["sy_scale"]
    dx = (c["fwd"][0] + sx * c["right"][0]) + sy * c["up"][0]
    dy = (c["fwd"][1] + sx * c["right"][1]) + sy * c["up"][1]
    dz = (c["fwd"][2] + sx * c["right"][2]) + sy * c["up"][2]
    ln = np.sqrt((dx * dx + dy * dy) + dz * dz)
    s = d / ln
    return np.stack([c["pos"][0] + dx * s, c["pos"][1] + dy * s, c["pos"][2] + dz * s], axis=-1).astype(F32)


# ------------------------------------------------------------------ probe state of a frame
def empty_state(tiles_x: int, tiles_y: int):
    P = tiles_x * tiles_y
    return dict(mask=np.full((tiles_y, tiles_x), SENTINEL, np.uint32), pos=np.zeros((P, 4), F32),
                nrm=np.zeros((P, 4), F32), atlas=np.zeros((P, 64, 4)), src=np.full(P, SENTINEL, np.uint32),
                fresh=np.zeros(P, bool), tiles_x=tiles_x, tiles_y=tiles_y)


def spawn_fresh(state, gbuf, cam, frame: int, upscale: int):
    """Fresh probes of the frame written over `state` (positions exact float32).  Returns the
    8x8 tile of each spawn tile's fresh probe (-1 where the pixel is sky)."""
    H, W = gbuf.shape[:2]
    px, py, _, _ = spawn_pixels(W, H, frame, upscale)
    d = gbuf[py, px, 3]
    ok = np.isfinite(d) & (d >= 0)
    tile = (py // 8) * state["tiles_x"] + (px // 8)
    c = cam_consts(cam)
    wp = pixel_world_f32(c, px[ok], py[ok], d[ok])
    t_ok = tile[ok]
    state["mask"].reshape(-1)[t_ok] = ((py[ok].astype(np.uint64) << np.uint64(16)) | px[ok].astype(np.uint64)).astype(np.uint32)
    state["pos"][t_ok, 0:3] = wp
    state["pos"][t_ok, 3] = d[ok]
    state["nrm"][t_ok, 0:3] = gbuf[py[ok], px[ok], 0:3]
    state["nrm"][t_ok, 3] = F32(1.0)
    state["fresh"][t_ok] = True
    return np.where(ok, tile, -1)


# ------------------------------------------------------------------ Algorithm 1
def reproject(prev, gbuf, cam, mv):
    """Screen-probe reprojection into a new state: per 8x8 tile the best previous probe found by
    its 64 pixels, placed at the winning pixel; src = the previous probe's index."""
    H, W = gbuf.shape[:2]
    tx_n, ty_n = prev["tiles_x"], prev["tiles_y"]
    out = empty_state(tx_n, ty_n)
    c = cam_consts(cam)
    dscale = F32(distance_scale(float(cam.fov_y), W, H))
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    d = gbuf[..., 3]
    ok = np.isfinite(d) & (d >= 0)
    qx = np.floor((xs.astype(F32) + F32(0.5)) + mv[..., 0].astype(F32)).astype(np.int64)
    qy = np.floor((ys.astype(F32) + F32(0.5)) + mv[..., 1].astype(F32)).astype(np.int64)
    ok &= (qx >= 0) & (qx < W) & (qy >= 0) & (qy < H)
    qt = np.where(ok, (np.clip(qy, 0, H - 1) // 8) * tx_n + np.clip(qx, 0, W - 1) // 8, 0)
    probe_q = prev["mask"].reshape(-1)[qt]
    ok &= probe_q != SENTINEL
    wp = pixel_world_f32(c, xs, ys, np.where(ok, d, F32(0.0)))
    npix = gbuf[..., 0:3].astype(F32)
    ppos = prev["pos"][qt, 0:3]
    pn = prev["nrm"][qt, 0:3]
    vx, vy, vz = ppos[..., 0] - wp[..., 0], ppos[..., 1] - wp[..., 1], ppos[..., 2] - wp[..., 2]
    plane = np.abs((vx * npix[..., 0] + vy * npix[..., 1]) + vz * npix[..., 2])
    ncheck = (pn[..., 0] * npix[..., 0] + pn[..., 1] * npix[..., 1]) + pn[..., 2] * npix[..., 2]
    cell = dscale * d.astype(F32)
    ok &= (plane < cell) & (ncheck > F32(0.95))
    dist = np.sqrt((vx * vx + vy * vy) + vz * vz)
    half = np.where(ok, dist, F32(0.0)).astype(np.float16).view(np.uint16).astype(np.uint64)
    lane = ((ys % 8) * 8 + (xs % 8)).astype(np.uint64)
    score = np.where(ok, (half << np.uint64(16)) | lane, np.uint64(SCORE_NONE))
    tile = (ys // 8) * tx_n + xs // 8
    flat = tile.reshape(-1)
    best = np.full(tx_n * ty_n, np.uint64(SCORE_NONE), np.uint64)
    np.minimum.at(best, flat, score.reshape(-1))
    won = best != np.uint64(SCORE_NONE)
    # the winning pixel of each tile: its lane
    wl = (best & np.uint64(0xFFFF)).astype(np.int64)
    t_idx = np.flatnonzero(won)
    wx = (t_idx % tx_n) * 8 + wl[t_idx] % 8
    wy = (t_idx // tx_n) * 8 + wl[t_idx] // 8
    out["mask"].reshape(-1)[t_idx] = ((wy.astype(np.uint64) << np.uint64(16)) | wx.astype(np.uint64)).astype(np.uint32)
    out["pos"][t_idx, 0:3] = wp[wy, wx]
    out["pos"][t_idx, 3] = d[wy, wx]
    out["nrm"][t_idx, 0:3] = npix[wy, wx]
    out["nrm"][t_idx, 3] = F32(1.0)
    out["src"][t_idx] = qt[wy, wx].astype(np.uint32)
    return out


# ------------------------------------------------------------------ Algorithm 4
def hysteresis(curr, prev):
    """Biased temporal hysteresis of Algorithm 4 on (..., 3) radiance arrays (float64)."""
    curr = np.asarray(curr, np.float64)
    prev = np.asarray(prev, np.float64)
    l1 = curr.sum(axis=-1) / 3.0
    l2 = prev.sum(axis=-1) / 3.0
    a = np.maximum(l1 - l2 - np.minimum(l1, l2), 0.0) / np.maximum(np.maximum(l1, l2), 1e-4)
    a = np.clip(a, 0.0, 0.95) ** 2
    return curr + a[..., None] * (prev - curr)


# ------------------------------------------------------------------ the frame's probe atlas
def temporal_atlas(state, prev_atlas, fresh_tile, ray_rad, ray_has, ray_len):
    """Atlas (P, 64, 4) of the frame: fresh probes gather their spawn tile's rays (ray_rad
    (S, rpp, 3), ray_has (S, rpp), ray_len (S * rpp,)), blended by Algorithm 4 with their tile's
    reprojected probe when there is one; reprojected-only probes carry their source atlas."""
    S, rpp = ray_has.shape
    valid_s = fresh_tile >= 0
    gathered = OP.gather(valid_s, ray_rad, ray_has, ray_len)
    P = state["pos"].shape[0]
    atlas = np.zeros((P, 64, 4))
    src = state["src"]
    has_src = src != SENTINEL
    carry = has_src & ~state["fresh"]
    atlas[carry] = prev_atlas[src[carry].astype(np.int64)]
    for s in np.flatnonzero(valid_s):
        t = int(fresh_tile[s])
        cur = gathered[s]
        if has_src[t]:
            prev = prev_atlas[int(src[t])]
            blended = hysteresis(cur[:, 0:3], prev[:, 0:3])
            atlas[t, :, 0:3] = blended
            atlas[t, :, 3] = cur[:, 3]
        else:
            atlas[t] = cur
    return atlas


def probe_valid(state):
    return state["mask"].reshape(-1) != SENTINEL
