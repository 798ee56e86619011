"""One frame of the path, in the paper's pass order: probe spawn, world-cache
update at the probe rays' hit points, resolve (blend + decay), query of the
cached radiance for every probe ray, probe irradiance, per-pixel
interpolation (Sections 2.1.1, 2.2, 2.1.4, 2.4).

`frame` is any object with the fields of a seeded workload frame: camera
(pos, fwd, right, up, fov_y, width, height), gbuffer (H, W, 4), records
(13, R) and rays_per_probe.
"""
from __future__ import annotations

import numpy as np

from . import probes
from .cache import OracleCache


def ray_radiance(cache: OracleCache, rec, ident, env=(0.0, 0.0, 0.0)):
    """Radiance and sample flag of each probe ray after resolve: the cell's value for a hit,
    the environment for a miss (infinite ray length), no sample otherwise."""
    ln = rec[9]
    hit = ident != 0
    miss = np.isposinf(ln)
    rad, found = cache.radiance(ident)
    rad[~found] = 0.0
    rad[miss] = np.asarray(env, np.float64)
    has = (hit & found) | miss
    return rad, has


def run_frame(cache: OracleCache, frame, f: int | None = None, env=(0.0, 0.0, 0.0)):
    f = frame.frame if f is None else f
    cam = frame.camera
    sp = probes.spawn(frame.gbuffer, cam, f)
    ident = cache.update(frame.records, f, cam.pos, cam.fov_y, cam.width, cam.height)
    sums = cache.sums.copy(), cache.count.copy(), cache.ids.copy()
    cache.resolve(f)
    rad, has = ray_radiance(cache, frame.records, ident, env)
    P = sp["valid"].size
    rpp = frame.rays_per_probe
    coeffs = probes.integrate(sp["valid"], sp["nrm"], rad.reshape(P, rpp, 3), has.reshape(P, rpp))
    irr, flag, diag = probes.interpolate(frame.gbuffer, cam, sp, coeffs)
    return dict(spawn=sp, ident=ident, pre_resolve=sums, ray_rad=rad, ray_has=has, sh=coeffs,
                irr=irr, flag=flag, diag=diag)
