"""Online-trained radiance surrogate: multiresolution hash encoding of position and normal, a
two-hidden-layer ReLU network with three outputs, relative L2 loss, back-propagation and Adam.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Float64 throughout, except where a float32
operation decides an integer (the grid cell of a position), which is computed with explicit
float32 operations like the cell key.

The paper caches radiance in hash cells only and defines no learned part, so this module follows
the published methods the surrogate is built from:

* multiresolution hash encoding (Mueller, Evans, Schied, Keller 2022, "Instant neural graphics
  primitives", Section 3): L levels of grids of increasing resolution; at each level the point's
  feature vector is the trilinear interpolation of the F-wide feature vectors stored at the 8
  vertices of its grid cell; a vertex is addressed densely when the level's grid fits the
  level's table of T entries, else by the spatial hash (XOR over axes of coordinate * pi_axis)
  mod T with pi = (1, 2654435761, 805459861); the levels' outputs are concatenated;
* the relative L2 loss (Lehtinen et al. 2018, used for radiance by Mueller et al. 2021,
  "Real-time neural radiance caching"): (y - t)^2 / (sg(y)^2 + eps), sg = no gradient through
  the denominator;
* Adam (Kingma and Ba 2015) with both bias corrections; on the hash table in its sparse form
  (PyTorch's SparseAdam): an entry whose gradient is exactly zero in a step -- no sample of the
  step touched it -- keeps its value and both moments, the others step with the global step
  count's bias correction.

Readings taken for this surrogate:

* Input: the hit position, normalised into the unit cube of a given box (x = (p - lo) * inv_ext,
  float32, clamped to [0, 1]), and the normal's direction code (dominant axis and sign, 6 codes,
  the same quantisation as the cell key's direction).  The code is folded into the vertex address
  (a 4th coordinate: dense index ((d (R+1) + z)(R+1) + y)(R+1) + x, or the hash term d * pi_4
  with pi_4 = 2246822519), so every facing direction owns its own features, as every cell key
  does; interpolation stays trilinear in position.
* Level l has an integer resolution R_l (cells per axis, given by the caller); the point's cell
  is i = min(floor(x * R_l), R_l - 1) per axis (float32 product), its fraction x R_l - i.  A level
  is dense when 6 (R_l + 1)^3 <= T.
* Network: 2L encoded features -> 64 -> ReLU -> 64 -> ReLU -> 3, no bias terms.  Radiance
  returned by a query is max(y, 0).
* Precision of the tensor-core path, emulated when asked: stored features rounded to float16,
  weights, encoded features and hidden activations rounded to bfloat16 (nearest even), the
  output gradient rounded to bfloat16, every sum in float64 (float32 on the GPU).
* Loss over a batch of B samples with 0/1 masks m: (1/B) sum_s m_s sum_c (y - t)^2 / (y^2 + eps).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

F32 = np.float32
PRIMES = (1, 2654435761, 805459861, 2246822519)
HIDDEN = 64
OUTPUTS = 3
N_DIRS = 6


@dataclass
class Spec:
    resolutions: tuple          # R_l per level
    log2_table: int             # T = 2^log2_table entries per level
    aabb_lo: tuple
    aabb_hi: tuple
    loss_eps: float = 0.01
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.99
    adam_eps: float = 1e-15
    features: int = field(default=2, init=False)

    @property
    def levels(self) -> int:
        return len(self.resolutions)

    @property
    def table_size(self) -> int:
        return 1 << self.log2_table

    def inv_extent(self) -> np.ndarray:
        """1 / (hi - lo) per axis, computed in float64 and rounded to float32 once."""
        lo = np.asarray(self.aabb_lo, np.float64)
        hi = np.asarray(self.aabb_hi, np.float64)
        return (1.0 / (hi - lo)).astype(F32)


def is_dense(res: int, table_size: int) -> bool:
    return N_DIRS * (res + 1) ** 3 <= table_size


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) of the float32 value, returned as float64."""
    f = np.asarray(x, np.float64).astype(F32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (rounded & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(F32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


def fp16_round(x) -> np.ndarray:
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


def direction_code(nrm: np.ndarray) -> np.ndarray:
    """Dominant axis of the normal (ties to x, then y) and the sign bit of that component: 2 axis + sign."""
    n = np.asarray(nrm, F32)
    a = np.abs(n)
    axis = np.where((a[0] >= a[1]) & (a[0] >= a[2]), 0, np.where(a[1] >= a[2], 1, 2))
    comp = np.choose(axis, n)
    return (2 * axis + np.signbit(comp).astype(np.int64)).astype(np.int64)


def normalise(spec: Spec, pos: np.ndarray) -> np.ndarray:
    """x = clamp((p - lo) * inv_ext, 0, 1) per axis in float32; NaN -> 0."""
    p = np.asarray(pos, F32)
    lo = np.asarray(spec.aabb_lo, np.float64).astype(F32)
    inv = spec.inv_extent()
    x = (p - lo[:, None]) * inv[:, None]
    x = np.where(np.isnan(x), F32(0.0), x)
    return np.clip(x, F32(0.0), F32(1.0)).astype(F32)


def corners(spec: Spec, pos: np.ndarray, nrm: np.ndarray):
    """Table indices (n, L, 8) and trilinear weights (n, L, 8) of every sample and level.

    Corner c has offsets (c & 1, (c >> 1) & 1, (c >> 2) & 1) along (x, y, z)."""
    x = normalise(spec, pos)
    d = direction_code(nrm)
    n = x.shape[1]
    T = spec.table_size
    idx = np.zeros((n, spec.levels, 8), np.int64)
    w = np.zeros((n, spec.levels, 8), np.float64)
    for l, R in enumerate(spec.resolutions):
        s = x * F32(R)                                   # float32 product
        i = np.minimum(np.floor(s).astype(np.int64), R - 1)
        frac = s.astype(np.float64) - i                  # exact: s and i share the binade or i = 0
        dense = is_dense(R, T)
        for c in range(8):
            off = np.array([(c >> a) & 1 for a in range(3)])
            v = i + off[:, None]
            if dense:
                V = R + 1
                idx[:, l, c] = ((d * V + v[2]) * V + v[1]) * V + v[0]
            else:
                h = np.zeros(n, np.uint64)
                for a in range(3):
                    h ^= (v[a].astype(np.uint64) * np.uint64(PRIMES[a])) & np.uint64(0xFFFFFFFF)
                h ^= (d.astype(np.uint64) * np.uint64(PRIMES[3])) & np.uint64(0xFFFFFFFF)
                idx[:, l, c] = (h & np.uint64(T - 1)).astype(np.int64)
            wc = np.ones(n)
            for a in range(3):
                wc = wc * (frac[a] if off[a] else 1.0 - frac[a])
            w[:, l, c] = wc
    return idx, w


def encode(spec: Spec, table: np.ndarray, pos, nrm, emulate: bool = True) -> np.ndarray:
    """Encoded features (n, 2L): level l occupies columns 2l, 2l + 1.  table: (L, T, 2)."""
    tab = fp16_round(table) if emulate else np.asarray(table, np.float64)
    idx, w = corners(spec, pos, nrm)
    n = idx.shape[0]
    e = np.zeros((n, 2 * spec.levels))
    for l in range(spec.levels):
        f = tab[l][idx[:, l, :]]                         # (n, 8, 2)
        e[:, 2 * l:2 * l + 2] = np.einsum("nc,ncf->nf", w[:, l, :], f)
    return e


@dataclass
class Params:
    table: np.ndarray   # (L, T, 2)
    w1: np.ndarray      # (64, 2L)
    w2: np.ndarray      # (64, 64)
    w3: np.ndarray      # (3, 64)

    def copy(self) -> "Params":
        return Params(self.table.copy(), self.w1.copy(), self.w2.copy(), self.w3.copy())


def forward(spec: Spec, prm: Params, pos, nrm, emulate: bool = True) -> dict:
    """Network evaluation; returns every intermediate (e, z1, h1, z2, h2, y), y of shape (n, 3)."""
    rnd = bf16_round if emulate else (lambda a: np.asarray(a, np.float64))
    e = rnd(encode(spec, prm.table, pos, nrm, emulate))
    w1, w2, w3 = rnd(prm.w1), rnd(prm.w2), rnd(prm.w3)
    z1 = e @ w1.T
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ w2.T
    h2 = rnd(np.maximum(z2, 0.0))
    y = h2 @ w3.T
    return dict(e=e, z1=z1, h1=h1, z2=z2, h2=h2, y=y, w1=w1, w2=w2, w3=w3)


def query(spec: Spec, prm: Params, pos, nrm, emulate: bool = True) -> np.ndarray:
    """Radiance (n, 3) = max(y, 0)."""
    return np.maximum(forward(spec, prm, pos, nrm, emulate)["y"], 0.0)


def loss(spec: Spec, y: np.ndarray, target: np.ndarray, mask: np.ndarray, batch: int, y_denominator=None) -> float:
    """(1/B) sum_s m_s sum_c (y - t)^2 / (yd^2 + eps), yd = y unless given (the no-gradient copy)."""
    yd = y if y_denominator is None else y_denominator
    r = (y - target) ** 2 / (yd * yd + spec.loss_eps)
    return float((mask[:, None] * r).sum() / batch)


def backward(spec: Spec, prm: Params, pos, nrm, target, mask=None, batch: int | None = None,
             emulate: bool = True):
    """Loss and gradients of every parameter (relative L2, no gradient through the denominator).

    target: (n, 3); mask: (n,) 0/1 (default all 1); batch: B of the loss normalisation (default n).
    Returns (loss, judge, grads) where grads is a Params of gradients (table gradient dense) and
    judge = (sum m |y - t|, sum m |t|) over channels, the surrogate's L1 error and scale."""
    fw = forward(spec, prm, pos, nrm, emulate)
    y = fw["y"]
    n = y.shape[0]
    target = np.asarray(target, np.float64)
    mask = np.ones(n) if mask is None else np.asarray(mask, np.float64)
    B = n if batch is None else batch
    rnd = bf16_round if emulate else (lambda a: np.asarray(a, np.float64))
    L = loss(spec, y, target, mask, B)
    judge = (float((mask[:, None] * np.abs(y - target)).sum()), float((mask[:, None] * np.abs(target)).sum()))
    dy = rnd(mask[:, None] * 2.0 * (y - target) / (y * y + spec.loss_eps) / B)
    gw3 = dy.T @ fw["h2"]
    dz2 = rnd((dy @ fw["w3"]) * (fw["z2"] > 0))
    gw2 = dz2.T @ fw["h1"]
    dz1 = rnd((dz2 @ fw["w2"]) * (fw["z1"] > 0))
    gw1 = dz1.T @ fw["e"]
    de = dz1 @ fw["w1"]                                  # (n, 2L)
    idx, w = corners(spec, pos, nrm)
    gt = np.zeros((spec.levels, spec.table_size, 2))
    for l in range(spec.levels):
        for f in range(2):
            np.add.at(gt[l, :, f], idx[:, l, :].reshape(-1), (w[:, l, :] * de[:, 2 * l + f, None]).reshape(-1))
    return L, judge, Params(gt, gw1, gw2, gw3)


@dataclass
class AdamState:
    m: Params
    v: Params
    step: int = 0


def adam_init(prm: Params) -> AdamState:
    z = lambda a: np.zeros_like(a, np.float64)
    return AdamState(Params(z(prm.table), z(prm.w1), z(prm.w2), z(prm.w3)),
                     Params(z(prm.table), z(prm.w1), z(prm.w2), z(prm.w3)), 0)


def adam_step(spec: Spec, prm: Params, grads: Params, st: AdamState, sparse_table: bool = True) -> Params:
    """One Adam step: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), t the global step count.  With
    sparse_table, table entries whose gradient (both features) is exactly 0 are left as they are,
    moments included.  Updates st in place."""
    st.step += 1
    t = st.step
    c1 = 1.0 - spec.beta1 ** t
    c2 = 1.0 - spec.beta2 ** t
    out = {}
    for name in ("table", "w1", "w2", "w3"):
        g = np.asarray(getattr(grads, name), np.float64)
        m0, v0 = getattr(st.m, name), getattr(st.v, name)
        p0 = np.asarray(getattr(prm, name), np.float64)
        m = spec.beta1 * m0 + (1.0 - spec.beta1) * g
        v = spec.beta2 * v0 + (1.0 - spec.beta2) * g * g
        p = p0 - spec.lr * (m / c1) / (np.sqrt(v / c2) + spec.adam_eps)
        if name == "table" and sparse_table:
            keep = np.all(g == 0.0, axis=-1, keepdims=True)
            m, v, p = np.where(keep, m0, m), np.where(keep, v0, v), np.where(keep, p0, p)
        setattr(st.m, name, m)
        setattr(st.v, name, v)
        out[name] = p
    return Params(out["table"], out["w1"], out["w2"], out["w3"])


def training_indices(frame: int, batch: int, n_records: int) -> np.ndarray:
    """Record index of training sample k of a frame: pcg(k ^ pcg(frame + 1)) mod n (PCG hash,
    see hashing.py), a counter-based draw that both sides compute from its definition."""
    from .hashing import pcg_hash
    seed = pcg_hash(np.uint32(frame + 1))[0]
    k = np.arange(batch, dtype=np.uint32)
    return (pcg_hash(k ^ seed).astype(np.uint64) % np.uint64(n_records)).astype(np.int64)
