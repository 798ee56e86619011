"""Pins for oracle/tiles.py (two-level world cache, Section 2.2.3): the tile descriptor's geometry
(in-plane floor division by 8 with negative coordinates, the main axis from the direction, the cell
index), a dense patch brute-forced into exactly its tiles, level-0 values equal to the plain
cache's cells record by record (same quantised cell, so the same samples and blend), MIP closed
forms (constant field, a single live cell, a hand-averaged 2x2 block), the level rule, and an
expired cell leaving its tile's levels at the resolve that evicts it."""
import math

import numpy as np

from oracle import key as K
from oracle import tiles as T
from oracle.cache import OracleCache
import workload as wl

LP = K.lod_params(0.05, 4, math.radians(60), 1920, 1080)  # every point below sits at LOD 0


def _rec(pos, nrm, rad=(1.0, 1.0, 1.0), ln=1.0):
    pos = np.asarray(pos, np.float32).reshape(-1, 3)
    n = pos.shape[0]
    rec = np.zeros((13, n), np.float32)
    rec[0:3] = pos.T
    rec[3:6] = np.broadcast_to(np.asarray(nrm, np.float32), (n, 3)).T
    rec[6:9] = np.broadcast_to(np.asarray(rad, np.float32), (n, 3)).T
    rec[9] = ln
    return rec


def _fields(key):
    key = int(key)
    return dict(lod=key >> 61, leak=(key >> 60) & 1, dir=(key >> 57) & 7, tu=(key >> 35) & 0xFFFF,
                tv=(key >> 19) & 0xFFFF, w=key & ((1 << 19) - 1))


def test_tile_key_geometry_per_main_axis():
    s = 0.05
    # cell coordinates (qx, qy, qz) = (13, -1, 4): normal +z -> plane (x, y), main axis z
    p = np.array([[13.5 * s, -0.5 * s, 4.5 * s]])
    for nrm, (u, v, w), code in (((0, 0, 1), (13, -1, 4), 4), ((1, 0, 0), (-1, 4, 13), 0),
                                 ((0, -1, 0), (13, 4, -1), 3)):
        key, cell, lod = T.tile_key(_rec(p, nrm), (0.0, 0.0, 0.0), LP)
        f = _fields(key[0])
        assert lod[0] == 0 and f["dir"] == code
        assert f["tu"] == (u >> 3) & 0xFFFF and f["tv"] == (v >> 3) & 0xFFFF and f["w"] == w & ((1 << 19) - 1)
        assert cell[0] == (u & 7) + 8 * (v & 7)
    # -1 lies in tile -1 (0xFFFF) at cell 7
    key, cell, _ = T.tile_key(_rec([[-0.5 * s, 0.5 * s, 0.0]], (0, 0, 1)), (0, 0, 0), LP)
    assert _fields(key[0])["tu"] == 0xFFFF and cell[0] == 7


def test_dense_patch_fills_exactly_its_tiles():
    # a 16 x 16 block of cells on the plane z = const, one record per cell, aligned on tiles
    s = 0.05
    i, j = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    pos = np.stack([(i.reshape(-1) + 0.5) * s, (j.reshape(-1) + 0.5) * s, np.full(256, 0.3)], axis=1)
    tc = T.OracleTileCache(10)
    cid, tid, cell, hit = tc.identities(_rec(pos, (0, 0, 1)), (0, 0, 0), math.radians(60), 1920, 1080)
    assert hit.all()
    assert np.unique(tid).size == 4 and np.unique(cid).size == 256
    for t in np.unique(tid):
        assert np.array_equal(np.sort(cell[tid == t]), np.arange(64))


def test_level0_values_equal_plain_cache_cells():
    """Tile + cell index names the same quantised cell as the plain descriptor: record by record the
    two caches return the same blended value over several frames."""
    frames = wl.make_frames(1, frames=3)
    tc = T.OracleTileCache(14, min_samples=1)
    oc = OracleCache(16)
    for fr in frames:
        cam = fr.camera
        ids_t = tc.update(fr.records, fr.frame, cam.pos, cam.fov_y, cam.width, cam.height)
        ids_c = oc.update(fr.records, fr.frame, cam.pos, cam.fov_y, cam.width, cam.height)
        tc.resolve(fr.frame)
        oc.resolve(fr.frame)
        vt, lv, ft = tc.radiance(ids_t)
        vc, fc = oc.radiance(ids_c)
        assert np.array_equal(ft, fc)
        assert (lv[ft] == 0).all()  # min_samples 1: every resolved cell answers at level 0
        np.testing.assert_allclose(vt[ft], vc[fc], rtol=1e-15)
        assert tc.cells.ids.size == oc.ids.size


def test_mips_of_constant_field_and_of_a_single_cell():
    s = 0.05
    i, j = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    pos = np.stack([(i.reshape(-1) + 0.5) * s, (j.reshape(-1) + 0.5) * s, np.full(64, 0.3)], axis=1)
    tc = T.OracleTileCache(10, min_samples=1000)
    rec = _rec(pos, (0, 0, 1), rad=(0.25, 0.5, 2.0))
    cid = tc.update(rec, 0, (0, 0, 0), math.radians(60), 1920, 1080)
    tc.resolve(0)
    vals, n, has = tc.mips[int(cid[0]) >> 6]
    assert has.all() and np.allclose(vals, [0.25, 0.5, 2.0], rtol=0, atol=1e-12)
    assert list(n[[0, 64, 80, 84]]) == [1, 4, 16, 64]
    # not enough samples anywhere: the 1x1 level answers
    v, lv, f = tc.radiance(cid[:3])
    assert f.all() and (lv == 3).all()
    # one live cell: every ancestor equals it
    tc1 = T.OracleTileCache(10)
    c1 = tc1.update(_rec(pos[10:11], (0, 0, 1), rad=(3.0, 1.0, 0.5)), 0, (0, 0, 0), math.radians(60), 1920, 1080)
    tc1.resolve(0)
    vals, n, has = tc1.mips[int(c1[0]) >> 6]
    cell = int(c1[0]) & 63
    for lv in range(4):
        k = int(T.mip_index(cell, lv))
        assert has[k] and np.allclose(vals[k], [3.0, 1.0, 0.5]) and n[k] == 1
    assert has.sum() == 4


def test_mip_box_filter_and_level_rule_by_hand():
    # cells (0,0), (1,0), (0,1) of a tile with 1, 2 and 5 samples, values 1, 2, 6: level-1 cell 0 =
    # mean (1 + 2 + 6) / 3 = 3 over 8 samples
    s = 0.05
    cells = [(0, 0, 1, 1.0), (1, 0, 2, 2.0), (0, 1, 5, 6.0)]
    pos, rad = [], []
    for (i, j, k, v) in cells:
        pos += [((i + 0.5) * s, (j + 0.5) * s, 0.3)] * k
        rad += [v] * k
    rec = _rec(pos, (0, 0, 1))
    rec[6:9] = np.asarray(rad, np.float32)[None, :]
    tc = T.OracleTileCache(10, min_samples=5)
    cid = tc.update(rec, 0, (0, 0, 0), math.radians(60), 1920, 1080)
    tc.resolve(0)
    vals, n, has = tc.mips[int(cid[0]) >> 6]
    assert np.allclose(vals[64], 3.0) and n[64] == 8
    v, lv, f = tc.radiance(cid)
    # the 5-sample cell answers itself, the others climb to level 1 (8 >= 5)
    for r in range(cid.size):
        want = 0 if (int(cid[r]) & 63) == 8 else 1
        assert lv[r] == want
    assert np.allclose(v[lv == 1], 3.0) and np.allclose(v[lv == 0], 6.0)


def test_expired_cell_leaves_the_levels_of_its_tile():
    # cells A = (0, 0) and B = (1, 0) of one tile; B is hit in frame 0 only, A in every frame.
    # B is evicted at the resolve of frame 8 (8 untouched frames, E = 8): from then on the tile's
    # levels are A alone, with A's sample count, and B no longer answers.
    s = 0.05
    a = ((0.5 * s, 0.5 * s, 0.3),)
    b = ((1.5 * s, 0.5 * s, 0.3),)
    tc = T.OracleTileCache(10, min_samples=1000)
    fov = math.radians(60)
    ca = tc.update(_rec(a, (0, 0, 1), rad=(1.0, 1.0, 1.0)), 0, (0, 0, 0), fov, 1920, 1080)
    cb = tc.update(_rec(b, (0, 0, 1), rad=(5.0, 5.0, 5.0)), 0, (0, 0, 0), fov, 1920, 1080)
    tc.resolve(0)
    tile = int(ca[0]) >> 6
    assert int(cb[0]) >> 6 == tile
    vals, n, has = tc.mips[tile]
    assert np.allclose(vals[64], 3.0) and n[64] == 2  # level 1 holds both cells: (1 + 5) / 2
    for f in range(1, 9):
        tc.update(_rec(a, (0, 0, 1), rad=(1.0, 1.0, 1.0)), f, (0, 0, 0), fov, 1920, 1080)
        tc.resolve(f)
        vals, n, has = tc.mips[tile]
        if f < 8:  # B is still live: it keeps its value in the levels
            assert np.allclose(vals[64], 3.0) and n[64] == f + 2
    cell_a = int(ca[0]) & 63
    for lv in range(4):
        k = int(T.mip_index(cell_a, lv))
        assert has[k] and np.allclose(vals[k], 1.0) and n[k] == 9
    assert has.sum() == 4
    v, lv, found = tc.radiance(np.array([ca[0], cb[0]], np.uint64))
    assert found[0] and not found[1] and np.allclose(v[0], 1.0)
