"""Cell descriptor of a hit record (Sections 2.2.1, 2.2.2; Algorithm 6).

The descriptor is the quantised world position and quantised direction of
the secondary vertex (Section 2.2.1), the quantisation level, which grows
with distance so that cells keep a roughly constant sample count (ibid.),
and the light-leak bit ray_length < cell_size (Section 2.2.2).

Readings taken where the paper leaves the details open:

* LOD l uses the cell side s_l = s0 * 2^l.  The screen-space cell size of
  Algorithm 6, cell_size(d) = distance_scale * d with distance_scale =
  tan(fov_y * proj_size * max(1/H, H/W^2)) and proj_size = 8, picks the
  level: l = floor(log2(cell_size(d) / s0)) clamped to [0, num_lods - 1],
  evaluated without logarithms as l = #{k < num_lods-1 : d^2 >= T_k},
  T_k = (2^(k+1) * s0 / distance_scale)^2.
* Direction: the dominant axis of the direction (ties go to x, then y) and
  the sign bit of that component, 6 codes.  The direction is the surface
  normal by default, or the outgoing direction (minus the probe ray) when
  the paper's ray-direction descriptor is asked for.
* Positions quantise to floor(p * (1/s_l)) in float32, wrapped to 19-bit
  two's complement per axis.
* Packing: lod (2 bits) | leak (1) | direction (3) | qx, qy, qz (19 each).

The key is an integer function of float32 inputs, so this module computes it
with explicit float32 operations (numpy float32 arithmetic rounds each
operation to nearest and never fuses), in this order:
  d = p - cam;  d2 = (dx*dx + dy*dy) + dz*dz;  q = floor(p * inv_s[lod]).
Everything derived from the view (thresholds, inverse sides) is computed in
float64 on the host and rounded to float32 once.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

F32 = np.float32
PROJ_SIZE = 8.0
Q_BITS = 19
Q_MASK = (1 << Q_BITS) - 1
KEY_DIR_NORMAL = 0
KEY_DIR_RAY = 1


def distance_scale(fov_y: float, width: int, height: int) -> float:
    """Algorithm 6: cell_size(d) = distance_scale * d."""
    return math.tan(fov_y * PROJ_SIZE * max(1.0 / height, height / (float(width) * float(width))))


@dataclass
class LodParams:
    thresholds: np.ndarray  # (3,) float32 squared distances
    side: np.ndarray        # (4,) float32 s_l
    inv_side: np.ndarray    # (4,) float32 1/s_l
    num_lods: int


def lod_params(cell_size: float, num_lods: int, fov_y: float, width: int, height: int) -> LodParams:
    s0 = float(F32(cell_size))
    ds = distance_scale(fov_y, width, height)
    d0 = s0 / ds
    thr = np.array([(d0 * 2.0 ** (k + 1)) * (d0 * 2.0 ** (k + 1)) for k in range(3)], np.float64).astype(F32)
    side = np.array([s0 * 2.0 ** k for k in range(4)], np.float64).astype(F32)
    inv0 = F32(1.0 / s0)
    inv = np.array([float(inv0) * 2.0 ** (-k) for k in range(4)], np.float64).astype(F32)
    return LodParams(thr, side, inv, int(num_lods))


def record_is_hit(rec: np.ndarray) -> np.ndarray:
    """A record updates the cache when its ray length is finite and >= 0 and its position is finite."""
    ln = rec[9]
    ok = np.isfinite(ln) & (ln >= 0)
    for a in range(3):
        ok &= np.isfinite(rec[a])
    return ok


def _floor_to_i32(x: np.ndarray) -> np.ndarray:
    """floor() of float32 to int32 with saturation; NaN -> 0 (float-to-int conversion semantics)."""
    f = np.floor(x.astype(F32)).astype(np.float64)
    f = np.where(np.isnan(f), 0.0, f)
    f = np.clip(f, -2.0 ** 31, 2.0 ** 31 - 1)
    return f.astype(np.int64)


def cell_key(rec: np.ndarray, cam_pos, lp: LodParams, key_dir: int = KEY_DIR_NORMAL):
    """64-bit descriptor and LOD of every record (13, n); meaningful where record_is_hit."""
    p = rec[0:3].astype(F32)
    c = np.asarray(cam_pos, F32)
    dx = p[0] - c[0]
    dy = p[1] - c[1]
    dz = p[2] - c[2]
    d2 = (dx * dx + dy * dy) + dz * dz
    lod = np.zeros(p.shape[1], np.int64)
    for k in range(lp.num_lods - 1):
        lod += (d2 >= lp.thresholds[k]).astype(np.int64)
    inv = lp.inv_side[lod]
    q = [(_floor_to_i32(p[a] * inv) & Q_MASK).astype(np.uint64) for a in range(3)]
    leak = (rec[9].astype(F32) < lp.side[lod]).astype(np.uint64)
    if key_dir == KEY_DIR_NORMAL:
        src = rec[3:6].astype(F32)
    else:
        src = -rec[10:13].astype(F32)
    ax = np.abs(src)
    axis = np.where((ax[0] >= ax[1]) & (ax[0] >= ax[2]), 0, np.where(ax[1] >= ax[2], 1, 2))
    comp = np.choose(axis, src)
    code = (2 * axis + np.signbit(comp).astype(np.int64)).astype(np.uint64)
    key = ((lod.astype(np.uint64) << np.uint64(61)) | (leak << np.uint64(60)) | (code << np.uint64(57))
           | (q[0] << np.uint64(38)) | (q[1] << np.uint64(19)) | q[2])
    return key, lod


# --------------------------------------------------------------------------- fixed point
FIX_SHIFT = 24
RAD_MAX = 32768.0


def quantize_radiance(rad: np.ndarray):
    """Per-channel fixed point q = round_half_even(clamp(r, 0, RAD_MAX) * 2^24) of float32
    radiance (3, n); NaN counts as 0.  Returns (q int64 (3, n), clamped (n,) bool)."""
    r = rad.astype(F32)
    bad = ~((r >= 0) & (r <= F32(RAD_MAX)))
    rc = np.where(np.isnan(r), F32(0.0), np.clip(r, F32(0.0), F32(RAD_MAX))).astype(F32)
    q = np.rint(rc.astype(np.float64) * float(1 << FIX_SHIFT)).astype(np.int64)
    return q, bad.any(axis=0)
