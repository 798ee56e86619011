"""Two-level world cache: cells grouped into 8x8 tiles with MIP levels (Section 2.2.3, "Prefiltering
Radiance").

The paper indexes tiles, not cells, with the spatial hash; a tile is an 8x8 region of cells laid
out linearly with its MIP chain, built on the plane obtained by dropping the main axis (the largest
component of the direction), so that surfaces fill tiles densely; MIP levels above the first are
box-filtered from the level below after the temporal blend; a query takes the finest level that
has accumulated enough samples.

Readings taken here:

* Tile descriptor: the cell descriptor of key.py (LOD, leak bit, direction code, float32
  quantised position q at the LOD's cell side) with the two in-plane coordinates -- the axes
  other than the direction code's axis, in increasing axis order (u, v) -- replaced by
  floor(q / 8) (16 bits each after the 19-bit wrap), the main-axis coordinate kept (19 bits):
  lod (2) | leak (1) | dir (3) | tile_u (16) | tile_v (16) | q_w (19).  The cell inside the tile
  is (q_u mod 8) + 8 (q_v mod 8).  The tile hashes like a cell (hashing.py) into the tile table.
* Per cell: fixed-point sums and count per frame as in cache.py; the resolve blends (first
  resolve takes the mean, then the EMA) and keeps a sample count n: the samples blended since
  the cell last started without history.  Decay and eviction per cell as in cache.py.
* MIP levels of a tile touched this frame, after its cells are blended: level k + 1 cell (i, j) =
  mean of the values of its four level-k children that hold one (a live level-0 cell, or a MIP
  cell with at least one live descendant), n = the sum of the children's n; levels 4x4, 2x2, 1x1.
* Query: the value at the finest level (0..3) whose n >= min_samples; when none reaches it, the
  1x1 level.
"""
from __future__ import annotations

import numpy as np

from .cache import OracleCache
from .hashing import cell_identity, identity_u64
from .key import F32, KEY_DIR_NORMAL, Q_MASK, _floor_to_i32, lod_params, record_is_hit

LEVELS = 4
MIP_OFFSET = (0, 64, 80, 84)
MIP_SIDE = (8, 4, 2, 1)
TILE_CELLS = 85


def tile_key(rec: np.ndarray, cam_pos, lp, key_dir: int = KEY_DIR_NORMAL):
    """(64-bit tile descriptor, cell index in the tile, LOD) of every record (13, n)."""
    p = rec[0:3].astype(F32)
    c = np.asarray(cam_pos, F32)
    dx, dy, dz = p[0] - c[0], p[1] - c[1], p[2] - c[2]
    d2 = (dx * dx + dy * dy) + dz * dz
    lod = np.zeros(p.shape[1], np.int64)
    for k in range(lp.num_lods - 1):
        lod += (d2 >= lp.thresholds[k]).astype(np.int64)
    inv = lp.inv_side[lod]
    q = np.stack([_floor_to_i32(p[a] * inv) for a in range(3)])  # signed int64
    leak = (rec[9].astype(F32) < lp.side[lod]).astype(np.uint64)
    src = rec[3:6].astype(F32) if key_dir == KEY_DIR_NORMAL else -rec[10:13].astype(F32)
    ax = np.abs(src)
    axis = np.where((ax[0] >= ax[1]) & (ax[0] >= ax[2]), 0, np.where(ax[1] >= ax[2], 1, 2))
    comp = np.choose(axis, src)
    code = (2 * axis + np.signbit(comp).astype(np.int64)).astype(np.uint64)
    u_ax = np.where(axis == 0, 1, 0)
    v_ax = np.where(axis == 2, 1, 2)
    qu = np.choose(u_ax, q)
    qv = np.choose(v_ax, q)
    qw = np.choose(axis, q)
    tu = ((qu >> 3) & 0xFFFF).astype(np.uint64)
    tv = ((qv >> 3) & 0xFFFF).astype(np.uint64)
    w = (qw & Q_MASK).astype(np.uint64)
    cell = ((qu & 7) + 8 * (qv & 7)).astype(np.int64)
    key = ((lod.astype(np.uint64) << np.uint64(61)) | (leak << np.uint64(60)) | (code << np.uint64(57))
           | (tu << np.uint64(35)) | (tv << np.uint64(19)) | w)
    return key, cell, lod


def mip_index(cell, level: int):
    """Index in the tile's 85-value layout of the level-`level` ancestor of level-0 cell `cell`."""
    i, j = np.asarray(cell) & 7, np.asarray(cell) >> 3
    s = 1 << level
    return MIP_OFFSET[level] + (i // s) + MIP_SIDE[level] * (j // s)


class OracleTileCache:
    """Per (tile identity, cell): the plain cache's accumulate / resolve / decay (cache.py);
    per touched tile: its MIP levels after every resolve."""

    def __init__(self, log2_tiles: int, cell_size: float = 0.05, num_lods: int = 4, alpha: float = 0.1,
                 evict_frames: int = 8, key_dir: int = KEY_DIR_NORMAL, min_samples: int = 16):
        self.log2_tiles = int(log2_tiles)
        self.cells = OracleCache(0, cell_size, num_lods, alpha, evict_frames, key_dir)
        self.min_samples = int(min_samples)
        self.n = {}      # cell id -> samples blended since the cell last started without history
        self.mips = {}   # tile identity -> (85, 3) values, (85,) n, (85,) has-value
        self._touched_tiles = set()

    def identities(self, rec, cam_pos, fov_y, width, height):
        """(cell id = tile identity << 6 | cell, tile identity, cell index, hit) of every record."""
        lp = lod_params(self.cells.cell_size, self.cells.num_lods, fov_y, width, height)
        hit = record_is_hit(rec)
        key, cell, _ = tile_key(rec, cam_pos, lp, self.cells.key_dir)
        home, fp = cell_identity(key, self.log2_tiles)
        tid = identity_u64(home, fp)
        return (tid << np.uint64(6)) | cell.astype(np.uint64), tid, cell, hit

    def update(self, rec, frame: int, cam_pos, fov_y, width, height):
        cid, tid, cell, hit = self.identities(rec, cam_pos, fov_y, width, height)
        self._touched_tiles |= set(int(t) for t in np.unique(tid[hit]))
        return self.cells.accumulate(rec, cid, hit, frame)

    def resolve(self, frame: int):
        c = self.cells
        t = c.count > 0
        ids = c.ids[t]
        fresh = ~c.has_hist[t]
        for k, f, cnt in zip(ids.tolist(), fresh.tolist(), c.count[t].tolist()):
            self.n[k] = cnt if f else self.n.get(k, 0) + cnt
        c.resolve(frame)
        live = set(int(x) for x in c.ids)
        self.n = {k: v for k, v in self.n.items() if k in live}
        for tile in self._touched_tiles:
            self.mips[tile] = self._build_mips(tile)
        self._touched_tiles = set()

    def _build_mips(self, tile: int):
        vals = np.zeros((TILE_CELLS, 3))
        n = np.zeros(TILE_CELLS, np.int64)
        has = np.zeros(TILE_CELLS, bool)
        base = np.uint64(tile) << np.uint64(6)
        row = self.cells.find(base + np.arange(64, dtype=np.uint64))
        ok = row >= 0
        vals[:64][ok] = self.cells.value[row[ok]]
        has[:64] = ok
        for cell in np.flatnonzero(ok):
            n[cell] = self.n[int(base) + int(cell)]
        for lv in range(1, LEVELS):
            side = MIP_SIDE[lv]
            for j in range(side):
                for i in range(side):
                    dst = MIP_OFFSET[lv] + i + side * j
                    kids = [MIP_OFFSET[lv - 1] + (2 * i + di) + MIP_SIDE[lv - 1] * (2 * j + dj)
                            for dj in (0, 1) for di in (0, 1)]
                    kh = [k for k in kids if has[k]]
                    if kh:
                        vals[dst] = np.mean([vals[k] for k in kh], axis=0)
                        n[dst] = sum(n[k] for k in kh)
                        has[dst] = True
        return vals, n, has

    def radiance(self, cell_ids):
        """Query value (n, 3), level used, found flag of each cell id (0 = no cell)."""
        cell_ids = np.asarray(cell_ids, np.uint64)
        out = np.zeros((cell_ids.size, 3))
        level = np.full(cell_ids.size, -1, np.int64)
        found = np.zeros(cell_ids.size, bool)
        row = self.cells.find(cell_ids)
        for r, cid in enumerate(cell_ids.tolist()):
            if row[r] < 0 or not self.cells.has_hist[row[r]]:
                continue
            tile, cell = cid >> 6, cid & 63
            vals, n, has = self.mips[tile]
            for lv in range(LEVELS):
                k = int(mip_index(cell, lv))
                if (has[k] and n[k] >= self.min_samples) or lv == LEVELS - 1:
                    out[r] = vals[k]
                    level[r] = lv
                    found[r] = True
                    break
        return out, level, found
