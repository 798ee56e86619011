"""World cache: insert/accumulate, resolve, decay/eviction and lookup.

Follows Section 2.2.1 (descriptor hashed to a bucket, fingerprint to find
the cell; one lookup per vertex whose cell index is cached), Section 2.2.3
(samples accumulated each frame, then blended into the cell with an
exponential moving average) and the decay rule of Section 2.2.1 (a cell's
decay is reset when it is accessed and the cell is freed once it has
decayed away).

The oracle keeps no slot array: a cell is its identity (home, fingerprint)
(see hashing.py), held in a table sorted by identity.  Readings:

* accumulation is per channel in 64-bit fixed point, sum of
  round(r * 2^24) (key.quantize_radiance), plus a sample count;
* resolve: mean m = sum / (count * 2^24); a cell without history takes
  v = m, otherwise v <- v + alpha (m - v); cells with no sample this frame
  keep v; the accumulators are then cleared;
* decay: stamp = last frame with a sample; at the resolve of frame f a cell
  with f - stamp >= E (E = evict_frames) is removed, i.e. it survives E-1
  untouched resolves and goes at the E-th; a removed cell that is hit again
  starts over without history.
"""
from __future__ import annotations

import numpy as np

from .hashing import cell_identity, identity_u64
from .key import FIX_SHIFT, KEY_DIR_NORMAL, cell_key, lod_params, quantize_radiance, record_is_hit

NO_CELL = np.int64(-1)


class OracleCache:
    def __init__(self, log2_slots: int, cell_size: float = 0.05, num_lods: int = 4, alpha: float = 0.1,
                 evict_frames: int = 8, key_dir: int = KEY_DIR_NORMAL):
        self.log2_slots = int(log2_slots)
        self.cell_size = float(np.float32(cell_size))
        self.num_lods = int(num_lods)
        # the blend weight is a float32 parameter of the method
        self.alpha = float(np.float32(alpha))
        self.evict_frames = int(evict_frames)
        self.key_dir = int(key_dir)
        self.ids = np.zeros(0, np.uint64)          # sorted identities
        self.sums = np.zeros((0, 3), np.int64)
        self.count = np.zeros(0, np.int64)
        self.stamp = np.zeros(0, np.int64)         # last frame with a sample
        self.value = np.zeros((0, 3), np.float64)  # resolved radiance
        self.has_hist = np.zeros(0, bool)
        self.last_resolved = None
        self.clamped = 0

    # ------------------------------------------------------------------ keys
    def identities(self, rec, cam_pos, fov_y, width, height):
        """Identity (uint64, home<<24|fp) of every hit record and the hit mask."""
        lp = lod_params(self.cell_size, self.num_lods, fov_y, width, height)
        hit = record_is_hit(rec)
        key, _ = cell_key(rec, cam_pos, lp, self.key_dir)
        home, fp = cell_identity(key, self.log2_slots)
        return identity_u64(home, fp), hit

    # ------------------------------------------------------------------ update
    def update(self, rec, frame: int, cam_pos, fov_y, width, height):
        """Accumulate one batch of records; returns the identity per record (0 where no hit)."""
        ident, hit = self.identities(rec, cam_pos, fov_y, width, height)
        return self.accumulate(rec, ident, hit, frame)

    def accumulate(self, rec, ident, hit, frame: int):
        """Add the radiance of the hit records to the cells named by their identities."""
        q, bad = quantize_radiance(rec[6:9])
        self.clamped += int((bad & hit).sum())
        ids = ident[hit]
        qh = q[:, hit]
        uniq, inv = np.unique(ids, return_inverse=True)
        order = np.argsort(inv, kind="stable")
        starts = np.searchsorted(inv[order], np.arange(uniq.size))
        if uniq.size:
            add = np.stack([np.add.reduceat(qh[c][order], starts) for c in range(3)], axis=1).astype(np.int64)
        else:
            add = np.zeros((0, 3), np.int64)
        cnt = np.bincount(inv, minlength=uniq.size).astype(np.int64)
        # merge into the table
        pos = np.searchsorted(self.ids, uniq)
        present = (pos < self.ids.size) & (self.ids[np.minimum(pos, max(self.ids.size - 1, 0))] == uniq) \
            if self.ids.size else np.zeros(uniq.size, bool)
        pi = pos[present]
        self.sums[pi] += add[present]
        self.count[pi] += cnt[present]
        self.stamp[pi] = frame
        new = ~present
        if new.any():
            self.ids = np.concatenate([self.ids, uniq[new]])
            self.sums = np.concatenate([self.sums, add[new]])
            self.count = np.concatenate([self.count, cnt[new]])
            self.stamp = np.concatenate([self.stamp, np.full(int(new.sum()), frame, np.int64)])
            self.value = np.concatenate([self.value, np.zeros((int(new.sum()), 3))])
            self.has_hist = np.concatenate([self.has_hist, np.zeros(int(new.sum()), bool)])
            o = np.argsort(self.ids, kind="stable")
            self.ids, self.sums, self.count = self.ids[o], self.sums[o], self.count[o]
            self.stamp, self.value, self.has_hist = self.stamp[o], self.value[o], self.has_hist[o]
        out = np.zeros(rec.shape[1], np.uint64)
        out[hit] = ids
        return out

    # ------------------------------------------------------------------ resolve
    def resolve(self, frame: int):
        t = self.count > 0
        m = self.sums[t].astype(np.float64) / (self.count[t, None].astype(np.float64) * float(1 << FIX_SHIFT))
        v = self.value[t]
        h = self.has_hist[t]
        self.value[t] = np.where(h[:, None], v + self.alpha * (m - v), m)
        self.has_hist[t] = True
        self.sums[t] = 0
        self.count[t] = 0
        keep = (frame - self.stamp) < self.evict_frames
        self.ids, self.sums, self.count = self.ids[keep], self.sums[keep], self.count[keep]
        self.stamp, self.value, self.has_hist = self.stamp[keep], self.value[keep], self.has_hist[keep]
        self.last_resolved = frame

    # ------------------------------------------------------------------ lookup
    def find(self, ident):
        """Row of each identity in the table, or -1."""
        ident = np.asarray(ident, np.uint64)
        if self.ids.size == 0:
            return np.full(ident.shape, NO_CELL, np.int64)
        pos = np.searchsorted(self.ids, ident)
        pc = np.minimum(pos, self.ids.size - 1)
        return np.where(self.ids[pc] == ident, pc, NO_CELL).astype(np.int64)

    def radiance(self, ident):
        """Resolved radiance (n, 3) of each identity; zeros and found=False where absent."""
        row = self.find(ident)
        found = row >= 0
        # a cell answers queries once it has been resolved
        found[found] = self.has_hist[row[found]]
        out = np.zeros((row.size, 3))
        out[found] = self.value[row[found]]
        return out, found

    def query_records(self, rec, cam_pos, fov_y, width, height):
        """Lookup without insertion (the cache query of Section 2.1.3 for hit points)."""
        ident, hit = self.identities(rec, cam_pos, fov_y, width, height)
        out, found = self.radiance(ident)
        found &= hit
        out[~found] = 0.0
        return out, found

    def live_count(self) -> int:
        return int(self.ids.size)
