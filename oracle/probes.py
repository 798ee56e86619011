"""Screen probes: spawn, probe mask + MIP chain, directional search, probe
irradiance and per-pixel interpolation.

* Spawn (Section 2.1.1): one probe per 8x8 tile, placed on the pixel picked
  by a Halton (bases 2 and 3) jitter shared by every tile of the frame
  (upscale 1x1); position rebuilt from the G-buffer distance and the camera,
  normal read from the G-buffer (Section 2.1.1, G-buffer paragraph).
* Probe mask (Section 2.1.5): the probe pixel packed as y << 16 | x in 32
  bits, 0xFFFFFFFF for a tile without probe (sky under the picked pixel);
  MIP level k+1 keeps the first valid probe of each 2x2 block of level k
  (scan order (0,0), (1,0), (0,1), (1,1)).
* Directional search: Algorithm 3 (find_closest_probe), with the division by
  two taken as a floor.
* Probe irradiance (Sections 2.1.4, 2.4.2): per-cell mean of the rays'
  radiance; cells with no sample get the mean of the populated cells
  (radiance backup); projection to three SH bands through the cells'
  direction moments.
* Probe filtering (Section 2.3, Algorithm 5): the probe's 8x8 cell radiance (and
  the mean hit distance of each cell's rays, in the 4th channel) blurred with the
  same cell of the probes found by Algorithm 3 at steps -1, +1, -2, +2, -3, +3
  along one probe-grid axis per pass (x, then y: a separable 7x7 sparse blur);
  a neighbour is skipped when it lies farther than cell_size from the probe's
  plane, when the cell direction points behind its normal, or when the hit point
  seen from it (at the smaller of the two hit distances) is more than pi/50 off
  the cell direction from the probe.  Readings: the depth weight, which the paper
  leaves unspecified, is 1 / (1 + |d_p - d_q| / cell_size(d_p)); a cell whose rays
  all missed has hit distance +inf, and a hit point at infinity is exactly along
  the cell direction (angle test passes); the cell direction is the world
  direction of the cell's centre (u, v) in the probe frame.
* Interpolation (Section 2.4.1): four neighbours found with Algorithm 3 at
  offsets (0,0), (1,0), (0,1), (1,1) from the tile below-left of the pixel
  (pixel - (4,4) in probe space); weight = bilinear * max(0, n_p.n_q)^8 *
  max(0, 1 - plane_dist / cell_size(d_p)); all weights zero -> equal weights
  over the neighbours found ("relaxed", flag 1); no neighbour -> 0 (flag 2);
  sky pixel -> 0 (flag 3).
"""
from __future__ import annotations

import math

import numpy as np

from . import hemioct, sh
from .key import distance_scale

SENTINEL = 0xFFFFFFFF
NEIGHBOUR_OFFSETS = ((0, 0), (1, 0), (0, 1), (1, 1))
NORMAL_POWER = 8
FLAG_OK, FLAG_RELAXED, FLAG_NONE, FLAG_SKY = 0, 1, 2, 3


def radical_inverse_times8(i: int, base: int) -> int:
    """floor(8 * radical_inverse_base(i)), exact: digits of i reversed behind the radix point."""
    num, den = 0, 1
    while i:
        num = num * base + i % base
        den *= base
        i //= base
    return (8 * num) // den


def halton_jitter(frame: int):
    """Jitter of frame f inside the 8x8 spawn tile: Halton point number f+1, bases 2 and 3."""
    return radical_inverse_times8(frame + 1, 2), radical_inverse_times8(frame + 1, 3)


def pixel_dirs(cam_pos, fwd, right, up, fov_y, width, height, xs, ys):
    """Unit camera-ray directions through pixel centres (x + 0.5, y + 0.5), row 0 on top."""
    th = math.tan(0.5 * fov_y)
    sx = (2.0 * (np.asarray(xs, np.float64) + 0.5) / width - 1.0) * th * (width / height)
    sy = (1.0 - 2.0 * (np.asarray(ys, np.float64) + 0.5) / height) * th
    d = (np.asarray(fwd, np.float64) + sx[..., None] * np.asarray(right, np.float64)
         + sy[..., None] * np.asarray(up, np.float64))
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def spawn(gbuf, cam, frame: int):
    """Probe per 8x8 tile.  gbuf (H, W, 4) = normal, distance (inf = sky)."""
    H, W = gbuf.shape[:2]
    tx_n, ty_n = (W + 7) // 8, (H + 7) // 8
    jx, jy = halton_jitter(frame)
    ty, tx = np.meshgrid(np.arange(ty_n), np.arange(tx_n), indexing="ij")
    px = np.minimum(8 * tx + jx, W - 1)
    py = np.minimum(8 * ty + jy, H - 1)
    dist = gbuf[py, px, 3].astype(np.float64)
    valid = np.isfinite(dist) & (dist >= 0)
    mask = np.where(valid, (py.astype(np.uint64) << np.uint64(16)) | px.astype(np.uint64),
                    np.uint64(SENTINEL)).astype(np.uint32)
    d = pixel_dirs(cam.pos, cam.fwd, cam.right, cam.up, cam.fov_y, W, H, px, py)
    pos = np.asarray(cam.pos, np.float64) + d * np.where(valid, dist, 0.0)[..., None]
    nrm = gbuf[py, px, 0:3].astype(np.float64)
    return dict(mask=mask, pos=pos.reshape(-1, 3), nrm=nrm.reshape(-1, 3), dist=np.where(valid, dist, 0.0).reshape(-1),
                valid=valid.reshape(-1), tiles_x=tx_n, tiles_y=ty_n, jitter=(jx, jy))


def build_mips(mask0):
    """Probe-mask MIP chain down to 1x1; level k+1 keeps the first valid of each 2x2 block."""
    mips = [np.asarray(mask0, np.uint32)]
    while max(mips[-1].shape) > 1:
        m = mips[-1]
        h, w = m.shape
        nh, nw = (h + 1) // 2, (w + 1) // 2
        pad = np.full((2 * nh, 2 * nw), SENTINEL, np.uint32)
        pad[:h, :w] = m
        out = np.full((nh, nw), SENTINEL, np.uint32)
        for (dx, dy) in ((0, 0), (1, 0), (0, 1), (1, 1)):  # scan order: first valid wins
            cand = pad[dy::2, dx::2]
            take = (out == SENTINEL) & (cand != SENTINEL)
            out = np.where(take, cand, out)
        mips.append(out)
    return mips


def find_closest_probe(mips, tx, ty, ox: int, oy: int):
    """Algorithm 3, vectorised: probe-space position (tx, ty) (already divided by 8),
    offset (ox, oy); ascend the MIP chain until a probe is found or the position leaves
    the level."""
    tx = np.asarray(tx, np.int64).copy()
    ty = np.asarray(ty, np.int64).copy()
    out = np.full(tx.shape, SENTINEL, np.uint32)
    active = np.ones(tx.shape, bool)
    for m in mips:
        h, w = m.shape
        x = tx + ox
        y = ty + oy
        inb = (x >= 0) & (x < w) & (y >= 0) & (y < h)
        active &= inb
        val = np.full(tx.shape, SENTINEL, np.uint32)
        val[active] = m[y[active], x[active]]
        hit = active & (val != SENTINEL)
        out[hit] = val[hit]
        active &= ~hit
        tx >>= 1  # floor division by two
        ty >>= 1
    return out


def integrate(valid, nrm, ray_rad, ray_has, moments=None):
    """Probe SH coefficients (P, 9, 3).

    ray_rad (P, RPP, 3): radiance returned for ray k of probe p (cache value at
    the hit, environment on a miss); ray_has (P, RPP): the ray produced a sample.
    Ray k samples cell k mod 64."""
    if moments is None:
        moments = hemioct.moments()
    omega, m1, m2 = moments
    P, rpp = ray_has.shape
    cell = np.arange(rpp) & 63
    onehot = (cell[:, None] == np.arange(64)[None, :]).astype(np.float64)  # (RPP, 64)
    w = ray_has.astype(np.float64)
    csum = np.einsum("pk,kc,pkx->pcx", w, onehot, np.asarray(ray_rad, np.float64))
    cnt = np.einsum("pk,kc->pc", w, onehot)
    pop = cnt > 0
    L = np.where(pop[..., None], csum / np.maximum(cnt, 1.0)[..., None], 0.0)
    npop = pop.sum(axis=1)
    backup = np.where((npop > 0)[:, None], L.sum(axis=1) / np.maximum(npop, 1)[:, None], 0.0)
    L = np.where(pop[..., None], L, backup[:, None, :])
    S0 = np.einsum("c,pcx->px", omega, L)
    S1 = np.einsum("ca,pcx->pax", m1, L)
    S2 = np.einsum("cab,pcx->pabx", m2, L)
    t, b = hemioct.onb(nrm)
    R = np.stack([t, b, np.asarray(nrm, np.float64)], axis=-1)  # R[p, i, a]: world i of local axis a
    S1w = np.einsum("pia,pax->pix", R, S1)
    S2w = np.einsum("pia,pjb,pabx->pijx", R, R, S2)
    coeffs = sh.project_moments(S0, S1w, S2w)
    return np.where(np.asarray(valid)[:, None, None], coeffs, 0.0)


def gather(valid, ray_rad, ray_has, ray_len):
    """Probe atlas (P, 64, 4): per hemi-octahedral cell the mean radiance of its rays that produced
    a sample, the radiance backup (mean of the populated cells) where none did (Section 2.1.4), and
    in the 4th channel the mean ray length of its rays that hit a surface (+inf when none did).
    Probes that do not exist get zeros."""
    ray_has = np.asarray(ray_has, bool)
    P, rpp = ray_has.shape
    cell = np.arange(rpp) & 63
    onehot = (cell[:, None] == np.arange(64)[None, :]).astype(np.float64)  # (RPP, 64)
    w = ray_has.astype(np.float64)
    csum = np.einsum("pk,kc,pkx->pcx", w, onehot, np.asarray(ray_rad, np.float64))
    cnt = np.einsum("pk,kc->pc", w, onehot)
    pop = cnt > 0
    L = np.where(pop[..., None], csum / np.maximum(cnt, 1.0)[..., None], 0.0)
    npop = pop.sum(axis=1)
    backup = np.where((npop > 0)[:, None], L.sum(axis=1) / np.maximum(npop, 1)[:, None], 0.0)
    L = np.where(pop[..., None], L, backup[:, None, :])
    ln = np.asarray(ray_len, np.float64).reshape(P, rpp)
    hit = ray_has & np.isfinite(ln) & (ln >= 0)
    hsum = np.einsum("pk,kc->pc", np.where(hit, ln, 0.0), onehot)
    hcnt = np.einsum("pk,kc->pc", hit.astype(np.float64), onehot)
    with np.errstate(divide="ignore", invalid="ignore"):
        hd = np.where(hcnt > 0, hsum / np.maximum(hcnt, 1.0), np.inf)
    atlas = np.concatenate([L, hd[..., None]], axis=-1)
    return np.where(np.asarray(valid)[:, None, None], atlas, 0.0)


def project(valid, nrm, atlas, moments=None):
    """SH coefficients (P, 9, 3) of the cell radiance atlas[..., :3] through the cells' direction
    moments (Section 2.4.2), in the probe frame rotated to world space."""
    if moments is None:
        moments = hemioct.moments()
    omega, m1, m2 = moments
    L = np.asarray(atlas, np.float64)[..., :3]
    S0 = np.einsum("c,pcx->px", omega, L)
    S1 = np.einsum("ca,pcx->pax", m1, L)
    S2 = np.einsum("cab,pcx->pabx", m2, L)
    t, b = hemioct.onb(nrm)
    R = np.stack([t, b, np.asarray(nrm, np.float64)], axis=-1)
    S1w = np.einsum("pia,pax->pix", R, S1)
    S2w = np.einsum("pia,pjb,pabx->pijx", R, R, S2)
    coeffs = sh.project_moments(S0, S1w, S2w)
    return np.where(np.asarray(valid)[:, None, None], coeffs, 0.0)


def cell_dirs_world(nrm):
    """World direction (P, 64, 3) of each cell centre: cell 8 j + i at u = -1 + (i + 0.5)/4,
    v = -1 + (j + 0.5)/4 in the probe frame (t, b, n)."""
    c = np.arange(64)
    local = hemioct.uv_to_dir(-1.0 + ((c & 7) + 0.5) * 0.25, -1.0 + ((c >> 3) + 0.5) * 0.25)  # (64, 3)
    n = np.asarray(nrm, np.float64)
    t, b = hemioct.onb(n)
    return (local[None, :, 0:1] * t[:, None, :] + local[None, :, 1:2] * b[:, None, :]
            + local[None, :, 2:3] * n[:, None, :])


FILTER_COS = math.cos(math.pi / 50.0)


def filter_pass(atlas, sp, cam, axis: int):
    """One pass of Algorithm 5 along probe-grid axis 0 (x) or 1 (y).  atlas (P, 64, 4) as from
    gather; sp the spawn dict (mask, pos, nrm, dist, valid, tiles_x, tiles_y).  Returns the
    filtered atlas and, per probe and cell, the smallest margin of its accept/reject decisions
    (|plane - cs| / cs, |n_q . dir|, |angle - cos(pi/50)|), for comparisons in other precisions."""
    atlas = np.asarray(atlas, np.float64)
    P = atlas.shape[0]
    mips = build_mips(sp["mask"])
    txn = sp["tiles_x"]
    pidx = np.arange(P)
    tx, ty = pidx % txn, pidx // txn
    valid = np.asarray(sp["valid"], bool)
    pos, nrm, dist = sp["pos"], sp["nrm"], sp["dist"]
    cs = distance_scale(cam.fov_y, cam.width, cam.height) * dist  # (P,)
    dirs = cell_dirs_world(nrm)  # (P, 64, 3)
    rad = atlas[..., :3].copy()
    acc_a = atlas[..., 3].copy()
    weight = np.ones((P, 64))
    hd = atlas[..., 3].copy()
    margin = np.full((P, 64), np.inf)
    for i in range(6):
        step = (((i & 1) << 1) - 1) * ((i >> 1) + 1)
        ox, oy = (step, 0) if axis == 0 else (0, step)
        q = find_closest_probe(mips, tx, ty, ox, oy)
        found = (q != SENTINEL) & valid
        qx = (q & 0xFFFF).astype(np.int64)
        qy = (q >> 16).astype(np.int64)
        qi = np.where(found, (qy >> 3) * txn + (qx >> 3), 0)
        plane = np.abs(((pos[qi] - pos) * nrm).sum(axis=-1))  # (P,)
        with np.errstate(divide="ignore", invalid="ignore"):
            pm = np.where(cs > 0, np.abs(plane - cs) / cs, np.inf)
        ncheck = (dirs * nrm[qi][:, None, :]).sum(axis=-1)  # (P, 64)
        hdc = np.minimum(atlas[qi, :, 3], hd)
        fin = np.isfinite(hdc)
        hp = pos[qi][:, None, :] + dirs * np.where(fin, hdc, 0.0)[..., None]
        v = hp - pos[:, None, :]
        vn = np.linalg.norm(v, axis=-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            ang = np.where(fin, (dirs * v).sum(axis=-1) / vn, 1.0)
        ang = np.where(fin & (vn == 0), 1.0, ang)
        ok = found[:, None] & (plane <= cs)[:, None] & (ncheck >= 0.0) & (ang >= FILTER_COS)
        with np.errstate(divide="ignore", invalid="ignore"):
            w = 1.0 / (1.0 + np.abs(dist - dist[qi]) / cs)
        w = np.where(ok, w[:, None], 0.0)
        rad += w[..., None] * atlas[qi, :, :3]
        with np.errstate(invalid="ignore"):  # 0 * inf in rejected entries, discarded by the where
            acc_a += np.where(ok, w * hdc, 0.0)
        weight += w
        with np.errstate(invalid="ignore"):
            hd = np.where(ok, acc_a / weight, hd)
        m = np.minimum(np.minimum(np.where(found, pm, np.inf)[:, None], np.abs(ncheck)),
                       np.where(fin, np.abs(ang - FILTER_COS), np.inf))
        margin = np.where(found[:, None], np.minimum(margin, m), margin)
    out = np.concatenate([rad / weight[..., None], (acc_a / weight)[..., None]], axis=-1)
    return np.where(valid[:, None, None], out, atlas), margin


def interpolate(gbuf, cam, sp, coeffs):
    """Per-pixel irradiance (H, W, 3), flag (H, W), and diagnostics (weight sum, smallest
    distance of a neighbour's plane test to its cut)."""
    H, W = gbuf.shape[:2]
    mips = build_mips(sp["mask"])
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    dist = gbuf[..., 3].astype(np.float64)
    sky = ~(np.isfinite(dist) & (dist >= 0))
    d = pixel_dirs(cam.pos, cam.fwd, cam.right, cam.up, cam.fov_y, W, H, xs, ys)
    Pp = np.asarray(cam.pos, np.float64) + d * np.where(sky, 0.0, dist)[..., None]
    n_p = gbuf[..., 0:3].astype(np.float64)
    cs = distance_scale(cam.fov_y, W, H) * np.where(sky, 0.0, dist)
    tx = (xs - 4) >> 3
    ty = (ys - 4) >> 3
    fx = (xs + 0.5 - 4.0) / 8.0 - tx
    fy = (ys + 0.5 - 4.0) / 8.0 - ty
    wsum = np.zeros((H, W))
    esum = np.zeros((H, W, 3))
    nfound = np.zeros((H, W), np.int64)
    erel = np.zeros((H, W, 3))
    emag = np.zeros((H, W))
    margin = np.full((H, W), np.inf)
    for (ox, oy) in NEIGHBOUR_OFFSETS:
        q = find_closest_probe(mips, tx, ty, ox, oy)
        ok = (q != SENTINEL) & ~sky
        qx = (q & 0xFFFF).astype(np.int64)
        qy = (q >> 16).astype(np.int64)
        pi = np.where(ok, (qy >> 3) * sp["tiles_x"] + (qx >> 3), 0)
        Pq = sp["pos"][pi]
        nq = sp["nrm"][pi]
        bil = (fx if ox else 1.0 - fx) * (fy if oy else 1.0 - fy)
        ndot = np.maximum((n_p * nq).sum(axis=-1), 0.0)
        pd = np.abs(((Pq - Pp) * n_p).sum(axis=-1))
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(cs > 0, pd / cs, np.inf)
        wd = np.maximum(1.0 - ratio, 0.0)
        w = np.where(ok, bil * ndot ** NORMAL_POWER * wd, 0.0)
        Eq = sh.irradiance(coeffs[pi], n_p)
        Eq = np.where(ok[..., None], Eq, 0.0)
        # size of the terms summed into Eq (diagnostic for rounding bounds, not part of the result)
        terms = np.abs(sh.basis(n_p) * np.array([sh.A_HAT[b] for b in sh.BAND]))[..., :, None] * np.abs(coeffs[pi])
        emag = np.maximum(emag, np.where(ok, terms.sum(axis=(-2, -1)), 0.0))
        wsum += w
        esum += w[..., None] * Eq
        erel += Eq
        nfound += ok
        margin = np.where(ok, np.minimum(margin, np.abs(1.0 - ratio)), margin)
    irr = np.zeros((H, W, 3))
    flag = np.full((H, W), FLAG_OK, np.int64)
    good = wsum > 0
    irr[good] = esum[good] / wsum[good][:, None]
    relaxed = ~good & (nfound > 0)
    irr[relaxed] = erel[relaxed] / nfound[relaxed][:, None]
    flag[relaxed] = FLAG_RELAXED
    flag[nfound == 0] = FLAG_NONE
    irr[sky] = 0.0
    flag[sky] = FLAG_SKY
    return irr, flag, dict(wsum=wsum, margin=margin, nfound=nfound, emag=emag)
