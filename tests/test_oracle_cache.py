"""Pins for oracle/cache.py: closed forms of the exponential moving average
(Section 2.2.3), the exact frame of eviction (decay rule, Section 2.2.1), the
mean of a noisy constant field, and brute-force grouping of tiny inputs."""
import math

import numpy as np

from oracle import hashing
from oracle import key as K
from oracle.cache import OracleCache

FOV, W, H = math.radians(60.0), 64, 64
CAM = np.zeros(3, np.float32)


def _cell_records(n, rad, base=(0.30, 0.30, 0.30), jitter=0.0, seed=0, nrm=(0, 0, 1)):
    """n records inside one LOD-0 cell around `base` (cell side 0.05 near the camera)."""
    rng = np.random.default_rng(seed)
    rec = np.zeros((13, n), np.float32)
    rec[0:3] = (np.asarray(base)[:, None] + rng.uniform(0.001, 0.049, (3, n)) * (jitter > 0)).astype(np.float32)
    if jitter == 0:
        rec[0:3] = np.asarray(base, np.float32)[:, None] + np.float32(0.01)
    rec[3:6] = np.asarray(nrm, np.float32)[:, None]
    rec[6:9] = np.asarray(rad, np.float32).reshape(3, -1)
    rec[9] = 1.0
    return rec


def _cache(**kw):
    return OracleCache(12, cell_size=0.05, num_lods=4, alpha=0.1, evict_frames=8, **kw)


def test_constant_field_resolves_exactly():
    c = _cache()
    rad = np.array([0.75, 2.5, 1.0 / 1024], np.float32)
    for f in range(5):
        c.update(_cell_records(37, np.repeat(rad[:, None], 37, axis=1), jitter=1, seed=f), f, CAM, FOV, W, H)
        c.resolve(f)
        assert c.live_count() == 1
        assert np.array_equal(c.value[0], rad.astype(np.float64))


def test_step_response_closed_form():
    # v_{j+k} = c1 + (c0 - c1) (1 - alpha)^(k+1) after the field steps from c0 to c1 at frame j
    c = _cache()
    c0, c1, j = 2.0, 0.5, 3
    alpha = float(np.float32(0.1))
    for f in range(12):
        v = c0 if f < j else c1
        c.update(_cell_records(8, np.full((3, 8), v, np.float32)), f, CAM, FOV, W, H)
        c.resolve(f)
        if f >= j:
            want = c1 + (c0 - c1) * (1.0 - alpha) ** (f - j + 1)
            assert abs(c.value[0, 0] - want) <= 1e-12 * want


def test_eviction_at_the_eighth_untouched_resolve():
    c = _cache()
    c.update(_cell_records(4, np.ones((3, 4), np.float32)), 10, CAM, FOV, W, H)
    c.resolve(10)
    for f in range(11, 18):
        c.resolve(f)
        assert c.live_count() == 1, f
    c.resolve(18)
    assert c.live_count() == 0
    # a cell hit again after its eviction starts over without history
    c.update(_cell_records(4, np.full((3, 4), 3.0, np.float32)), 19, CAM, FOV, W, H)
    c.resolve(19)
    assert c.value[0, 0] == 3.0


def test_untouched_cell_keeps_value():
    c = _cache()
    a = _cell_records(4, np.ones((3, 4), np.float32), base=(0.3, 0.3, 0.3))
    b = _cell_records(4, np.full((3, 4), 5.0, np.float32), base=(0.6, 0.6, 0.6))
    c.update(np.concatenate([a, b], axis=1), 0, CAM, FOV, W, H)
    c.resolve(0)
    c.update(a, 1, CAM, FOV, W, H)
    c.resolve(1)
    vals = sorted(c.value[:, 0])
    assert vals == [1.0, 5.0]


def test_noisy_field_mean_converges():
    # c + U[0, 0.05]: the EMA of per-frame means settles at c + 0.025 within a CLT bound
    c = _cache()
    rng = np.random.default_rng(7)
    n = 64
    for f in range(200):
        rad = (1.0 + rng.uniform(0, 0.05, (3, n))).astype(np.float32)
        c.update(_cell_records(n, rad), f, CAM, FOV, W, H)
        c.resolve(f)
    alpha = 0.1
    # stationary variance of the EMA of means of n uniforms: alpha/(2-alpha) * (0.05^2/12)/n
    sd = math.sqrt(alpha / (2 - alpha) * (0.05 ** 2 / 12) / n)
    assert np.all(np.abs(c.value[0] - 1.025) < 6 * sd)


def test_bruteforce_grouping_tiny():
    # group records one at a time with a dict keyed by (home, fingerprint) and compare sums
    rng = np.random.default_rng(11)
    n = 3000
    rec = np.zeros((13, n), np.float32)
    rec[0:3] = rng.uniform(-0.4, 0.4, (3, n)).astype(np.float32)
    nv = rng.normal(size=(3, n))
    rec[3:6] = (nv / np.linalg.norm(nv, axis=0)).astype(np.float32)
    rec[6:9] = rng.uniform(0, 4, (3, n)).astype(np.float32)
    rec[9] = rng.uniform(0, 0.2, n).astype(np.float32)
    rec[9, ::17] = np.inf
    c = _cache()
    ident = c.update(rec, 0, CAM, FOV, W, H)
    lp = K.lod_params(0.05, 4, FOV, W, H)
    table = {}
    for r in range(n):
        one = rec[:, r:r + 1]
        if not K.record_is_hit(one)[0]:
            assert ident[r] == 0
            continue
        k, _ = K.cell_key(one, CAM, lp)
        home, fp = hashing.cell_identity(k, 12)
        idt = (int(home[0]), int(fp[0]))
        q, _ = K.quantize_radiance(one[6:9])
        s = table.setdefault(idt, [0, 0, 0, 0])
        for ch in range(3):
            s[ch] += int(q[ch, 0])
        s[3] += 1
        assert int(ident[r]) == (idt[0] << 24 | idt[1])
    assert len(table) == c.live_count()
    for row, idt in enumerate(c.ids):
        s = table[(int(idt) >> 24, int(idt) & 0xFFFFFF)]
        assert list(c.sums[row]) == s[:3] and c.count[row] == s[3]
    # every identity is found, and appears once
    assert np.unique(c.ids).size == c.ids.size
    assert np.all(c.find(ident[ident > 0]) >= 0)


def test_split_batches_equal_one_batch():
    rng = np.random.default_rng(12)
    n = 2000
    rec = np.zeros((13, n), np.float32)
    rec[0:3] = rng.uniform(-1, 1, (3, n)).astype(np.float32)
    rec[3:6] = np.array([0, 1, 0], np.float32)[:, None]
    rec[6:9] = rng.uniform(0, 1, (3, n)).astype(np.float32)
    rec[9] = 1.0
    a, b = _cache(), _cache()
    a.update(rec, 0, CAM, FOV, W, H)
    b.update(rec[:, :700], 0, CAM, FOV, W, H)
    b.update(rec[:, 700:], 0, CAM, FOV, W, H)
    assert np.array_equal(a.ids, b.ids) and np.array_equal(a.sums, b.sums) and np.array_equal(a.count, b.count)
    a.resolve(0)
    b.resolve(0)
    assert np.array_equal(a.value, b.value)
