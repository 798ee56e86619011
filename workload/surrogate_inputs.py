"""Seeded inputs of the learned-surrogate tests: parameter sets, sample points and targets.

Random numbers only (uniform draws in the stated ranges, axis-aligned unit normals); nothing of the
surrogate's arithmetic.  Both the CUDA path (through gi_nrc_set_params / device buffers) and the
oracle read these arrays unchanged."""
from __future__ import annotations

import numpy as np

LEVELS = 16
HIDDEN = 64
OUTPUTS = 3

# a level mix for small tables (2^14 entries): levels 0-5 dense, 6-15 hashed
SMALL_RESOLUTIONS = (2, 3, 4, 6, 8, 11, 15, 20, 28, 38, 52, 70, 96, 130, 180, 250)
# the Cornell box of configuration 1 (walls included)
CORNELL_AABB = ((-1.05, -0.05, -1.05), (1.05, 2.05, 1.05))


def params(seed: int, log2_table: int, table_scale: float = 0.5):
    """(table (16, 2^log2_table, 2), w1 (64, 32), w2 (64, 64), w3 (3, 64)) float32: table uniform in
    +-table_scale, weights uniform in +-sqrt(6 / (fan_in + fan_out))."""
    rng = np.random.default_rng(seed)
    table = rng.uniform(-table_scale, table_scale, (LEVELS, 1 << log2_table, 2)).astype(np.float32)
    w1 = (rng.uniform(-1, 1, (HIDDEN, 2 * LEVELS)) * np.sqrt(6.0 / (2 * LEVELS + HIDDEN))).astype(np.float32)
    w2 = (rng.uniform(-1, 1, (HIDDEN, HIDDEN)) * np.sqrt(6.0 / (2 * HIDDEN))).astype(np.float32)
    w3 = (rng.uniform(-1, 1, (OUTPUTS, HIDDEN)) * np.sqrt(6.0 / (HIDDEN + OUTPUTS))).astype(np.float32)
    return table, w1, w2, w3


def points(seed: int, n: int, aabb=CORNELL_AABB, margin: float = 0.02):
    """pos (3, n) uniform inside the box (shrunk by `margin` of its extent), nrm (3, n) axis-aligned
    unit vectors of random axis and sign, both float32."""
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(aabb[0], np.float64), np.asarray(aabb[1], np.float64)
    pos = (lo[:, None] + (hi - lo)[:, None] * rng.uniform(margin, 1 - margin, (3, n))).astype(np.float32)
    nrm = np.zeros((3, n), np.float32)
    nrm[rng.integers(0, 3, n), np.arange(n)] = rng.choice([-1.0, 1.0], n)
    return pos, nrm


def targets(seed: int, n: int, hi: float = 2.0, mask_frac: float = 0.15):
    """target (3, n) uniform in [0, hi) float32 and a 0/1 float32 mask with about mask_frac zeros."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, hi, (3, n)).astype(np.float32)
    m = (rng.uniform(size=n) >= mask_frac).astype(np.float32)
    return t, m


def gradients(seed: int, log2_table: int, scale: float = 1e-3):
    """Gradient arrays shaped like params(): normal draws times scale, about half the table zero."""
    rng = np.random.default_rng(seed)
    table = (rng.normal(size=(LEVELS, 1 << log2_table, 2)) * scale).astype(np.float32)
    table[rng.uniform(size=table.shape[:2]) < 0.5] = 0.0
    w1 = (rng.normal(size=(HIDDEN, 2 * LEVELS)) * scale).astype(np.float32)
    w2 = (rng.normal(size=(HIDDEN, HIDDEN)) * scale).astype(np.float32)
    w3 = (rng.normal(size=(OUTPUTS, HIDDEN)) * scale).astype(np.float32)
    return table, w1, w2, w3
