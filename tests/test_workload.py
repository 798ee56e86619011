"""The seeded workload generator is deterministic and self-consistent."""
import numpy as np

import workload as wl


def test_frames_are_deterministic():
    a = wl.make_frame(1, 1)
    b = wl.make_frame(1, 1)
    assert np.array_equal(a.records, b.records, equal_nan=True)
    assert np.array_equal(a.gbuffer, b.gbuffer)


def test_records_layout_and_hits_lie_on_boxes():
    fr = wl.make_frame(1, 0)
    rec = fr.records
    assert rec.shape == (13, 64 * 256)
    hit = np.isfinite(rec[9]) & (rec[9] >= 0)
    sc = wl.make_scene(1)
    # every hit point lies on the surface of some box, on the face its normal names
    t, box, face = wl.scene.trace(sc.bmin, sc.bmax, rec[0:3, hit].T - rec[10:13, hit].T * 1e-3, rec[10:13, hit].T)
    assert np.all(box >= 0)
    assert np.abs(t - 1e-3).max() < 1e-4
    nrm = rec[3:6, hit]
    assert np.all(np.abs(nrm).sum(axis=0) == 1.0)
    # normals face the incoming ray
    assert np.all((nrm * rec[10:13, hit]).sum(axis=0) < 0)


def test_halton_jitter_in_tile():
    for f in range(64):
        jx, jy = wl.halton_jitter(f)
        assert 0 <= jx < 8 and 0 <= jy < 8
