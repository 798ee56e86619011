"""Pins for oracle/key.py: the cell descriptor (Sections 2.2.1, 2.2.2), the
distance LOD against Algorithm 6 written with logarithms, and the fixed-point
quantiser, on boundary cases where a dropped term, a wrong rounding or a
swapped axis would show."""
import math

import numpy as np

from oracle import key as K

F32 = np.float32


def _rec(pos, nrm=(0, 0, 1), ln=1.0, rad=(1, 1, 1), d=(0, 0, -1)):
    pos = np.asarray(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    rec = np.zeros((13, n), np.float32)
    rec[0:3] = pos.T
    rec[3:6] = np.broadcast_to(np.asarray(nrm, np.float32), (n, 3)).T
    rec[6:9] = np.broadcast_to(np.asarray(rad, np.float32), (n, 3)).T
    rec[9] = ln
    rec[10:13] = np.broadcast_to(np.asarray(d, np.float32), (n, 3)).T
    return rec


def _fields(key):
    key = int(key)
    m = (1 << 19) - 1
    return dict(lod=key >> 61, leak=(key >> 60) & 1, dir=(key >> 57) & 7,
                qx=(key >> 38) & m, qy=(key >> 19) & m, qz=key & m)


LP = K.lod_params(0.05, 4, math.radians(60), 64, 64)


def test_distance_scale_algorithm6():
    # 1080p, 60 degrees: max(1/H, H/W^2) = 1/1080
    ds = K.distance_scale(math.radians(60.0), 1920, 1080)
    assert abs(ds - math.tan(math.radians(60.0) * 8.0 / 1080.0)) < 1e-15
    # a portrait view switches to the H/W^2 branch
    ds2 = K.distance_scale(1.0, 100, 400)
    assert abs(ds2 - math.tan(8.0 * 400.0 / 100.0 ** 2)) < 1e-15


def test_lod_matches_log2_definition_away_from_thresholds():
    # lod = clamp(floor(log2(cell_size(d) / s0)), 0, L-1), cell_size(d) = distance_scale * d
    fov, W, H = math.radians(60.0), 1920, 1080
    lp = K.lod_params(0.05, 4, fov, W, H)
    ds = K.distance_scale(fov, W, H)
    rng = np.random.default_rng(0)
    d = rng.uniform(0.1, 120.0, 5000)
    dirs = rng.normal(size=(5000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pos = (dirs * d[:, None]).astype(np.float32)
    _, lod = K.cell_key(_rec(pos), (0, 0, 0), lp)
    want = np.clip(np.floor(np.log2(ds * np.linalg.norm(pos.astype(np.float64), axis=1) / 0.05)), 0, 3)
    ratio = ds * np.linalg.norm(pos.astype(np.float64), axis=1) / 0.05
    away = np.abs(np.log2(ratio) - np.round(np.log2(ratio))) > 1e-5
    assert np.all(lod[away] == want[away])


def test_lod_threshold_is_inclusive():
    # exactly at d^2 = T_0 the point is at LOD 1; one float below it stays at LOD 0
    t0 = float(LP.thresholds[0])
    x = F32(math.sqrt(t0))
    while F32(x * x) < LP.thresholds[0]:
        x = np.nextafter(x, F32(np.inf))
    while F32(np.nextafter(x, F32(0)) ** 2) >= LP.thresholds[0]:
        x = np.nextafter(x, F32(0))
    _, lod = K.cell_key(_rec([[x, 0, 0], [np.nextafter(x, F32(0)), 0, 0]]), (0, 0, 0), LP)
    assert list(lod) == [1, 0]


def test_distance_is_float32_in_fixed_order():
    # d2 = (dx*dx + dy*dy) + dz*dz, each op rounded to float32: compare with an exact rational check
    rng = np.random.default_rng(5)
    pos = rng.uniform(-3, 3, (2000, 3)).astype(np.float32)
    cam = np.array([0.1, -0.2, 0.3], np.float32)
    _, lod = K.cell_key(_rec(pos), cam, LP)
    d = (pos - cam).astype(np.float32)
    d2 = F32(F32(d[:, 0] * d[:, 0]) + F32(d[:, 1] * d[:, 1])) + F32(d[:, 2] * d[:, 2])
    want = (d2[:, None] >= LP.thresholds[None, :3]).sum(axis=1)
    assert np.all(lod == want)


def test_position_quantisation_floor_and_wrap():
    s0 = float(LP.side[0])
    inv = float(LP.inv_side[0])
    assert inv == float(F32(1.0 / F32(0.05)))
    # LOD 0 needs d^2 < T_0: stay close to the camera at (0,0,0)
    pts = [[0.1, -0.01, -0.0], [0.05, 0.0999, -0.05]]
    key, lod = K.cell_key(_rec(pts), (0, 0, 0), LP)
    assert list(lod) == [0, 0]
    f0, f1 = _fields(key[0]), _fields(key[1])
    assert f0["qx"] == int(math.floor(float(F32(F32(0.1) * F32(inv)))))
    assert f0["qy"] == (1 << 19) - 1          # floor(-0.2) = -1 wraps to 0x7FFFF
    assert f0["qz"] == 0                      # -0.0 quantises to 0
    assert f1["qx"] == int(math.floor(float(F32(F32(0.05) * F32(inv)))))
    assert f1["qz"] == (1 << 19) - 1
    # side at LOD l is s0 * 2^l and its inverse inv0 * 2^-l
    assert np.all(LP.side == F32(s0) * F32(2.0) ** np.arange(4, dtype=np.float32))
    assert np.all(LP.inv_side == F32(inv) * F32(0.5) ** np.arange(4, dtype=np.float32))


def test_direction_code_dominant_axis_sign_and_ties():
    nrm = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
           (0.6, 0.6, 0.2), (0.1, -0.7, -0.7), (-0.0, 0.0, 0.0), (0.577, 0.577, 0.577)]
    rec = _rec(np.zeros((len(nrm), 3)), nrm=np.zeros(3))
    rec[3:6] = np.asarray(nrm, np.float32).T
    key, _ = K.cell_key(rec, (5, 5, 5), LP)
    codes = [_fields(k)["dir"] for k in key]
    # ties: x beats y beats z; the sign bit decides, so -0.0 counts as negative
    assert codes == [0, 1, 2, 3, 4, 5, 0, 3, 1, 0]


def test_ray_direction_descriptor_uses_outgoing_direction():
    rec = _rec(np.zeros((2, 3)), d=(0, 0, -1))
    rec[10:13, 1] = (0.9, 0.1, 0.0)
    key, _ = K.cell_key(rec, (5, 5, 5), LP, key_dir=K.KEY_DIR_RAY)
    assert [_fields(k)["dir"] for k in key] == [4, 1]  # -(0,0,-1) = +z; -(0.9,..) = -x


def test_leak_bit_compares_ray_length_with_cell_side():
    s = float(LP.side[0])
    rec = _rec(np.zeros((3, 3)) + 0.01)
    rec[9] = [np.nextafter(F32(s), F32(0)), s, 10.0]
    key, lod = K.cell_key(rec, (0, 0, 0), LP)
    assert list(lod) == [0, 0, 0]
    assert [_fields(k)["leak"] for k in key] == [1, 0, 0]


def test_hit_mask():
    rec = _rec(np.zeros((5, 3)))
    rec[9] = [1.0, np.inf, -1.0, np.nan, 0.0]
    rec[0, 4] = np.nan
    assert list(K.record_is_hit(rec)) == [True, False, False, False, False]


def test_quantiser_rounds_half_even_and_clamps():
    u = 2.0 ** -24
    rad = np.array([[0.5 * u, 1.5 * u, 2.5 * u, 1.0, -1.0, np.nan, 1e9, 32768.0]], np.float32)
    q, bad = K.quantize_radiance(np.repeat(rad, 3, axis=0))
    assert list(q[0]) == [0, 2, 2, 1 << 24, 0, 0, 32768 << 24, 32768 << 24]
    assert list(bad) == [False, False, False, False, True, True, True, False]
