"""Pins for oracle/hemioct.py and oracle/sh.py.

* Cell moments against closed forms: each cell is a spherical quadrilateral
  (its corners joined by great-circle arcs, since the octahedral map sends
  straight segments to geodesics), whose solid angle, first moment (Arvo 1995)
  and second moment (Stokes on the sphere: 3 int w w^T = Omega I +
  sum_edges n_e (int_e w ds)^T) have closed forms.
* Hemisphere totals: 2 pi, (0, 0, pi), (2 pi / 3) I.
* SH basis against scipy's spherical harmonics; A_l against Legendre
  quadrature of the clamped cosine; the whole probe projection against
  brute-force quadrature in spherical coordinates through the inverse map;
  uniform radiance L -> irradiance pi L at the probe normal.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as ss

from oracle import hemioct, probes, sh


def _corners(c):
    u0, v0 = hemioct.cell_bounds(c)
    h = hemioct.CELL_W
    uv = [(u0, v0), (u0 + h, v0), (u0 + h, v0 + h), (u0, v0 + h)]
    return [hemioct.uv_to_dir(u, v) for (u, v) in uv]


def _polygon_moments(verts):
    verts = [np.asarray(v, float) for v in verts]
    cen = sum(verts)
    area = sum(np.cross(verts[k], verts[(k + 1) % len(verts)]) for k in range(len(verts)))
    if np.dot(area, cen) < 0:  # make the order counter-clockwise seen from outside
        verts = verts[::-1]
    n = len(verts)
    omega = 0.0
    for k in range(1, n - 1):  # triangle fan, Van Oosterom & Strackee
        a, b, c = verts[0], verts[k], verts[k + 1]
        num = np.dot(a, np.cross(b, c))
        den = 1.0 + np.dot(a, b) + np.dot(b, c) + np.dot(c, a)
        omega += 2.0 * math.atan2(num, den)
    m1 = np.zeros(3)
    m2 = omega * np.eye(3)
    for k in range(n):
        a, b = verts[k], verts[(k + 1) % n]
        cr = np.cross(a, b)
        th = math.atan2(np.linalg.norm(cr), np.dot(a, b))
        ne = cr / np.linalg.norm(cr)
        m1 += 0.5 * th * ne
        cdir = (b - a * math.cos(th)) / math.sin(th)
        e = a * math.sin(th) + cdir * (1.0 - math.cos(th))
        m2 += np.outer(e, ne)
    m2 /= 3.0
    return omega, m1, 0.5 * (m2 + m2.T)


def test_cell_moments_match_spherical_polygon_closed_forms():
    omega, m1, m2 = hemioct.moments()
    for c in range(64):
        o, a, b = _polygon_moments(_corners(c))
        assert abs(omega[c] - o) < 1e-13
        assert np.abs(m1[c] - a).max() < 1e-13
        assert np.abs(m2[c] - b).max() < 1e-13


def test_hemisphere_totals():
    omega, m1, m2 = hemioct.moments()
    assert abs(omega.sum() - 2 * math.pi) < 1e-13
    assert np.abs(m1.sum(0) - [0, 0, math.pi]).max() < 1e-13
    assert np.abs(m2.sum(0) - 2 * math.pi / 3 * np.eye(3)).max() < 1e-13


def test_quadrature_converged():
    a = hemioct.cell_moments(n=16, sub=2)
    b = hemioct.cell_moments(n=24, sub=3)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-14


def test_uv_map_covers_upper_hemisphere_and_inverts():
    rng = np.random.default_rng(0)
    u, v = rng.uniform(-1, 1, (2, 10000))
    w = hemioct.uv_to_dir(u, v)
    assert np.all(w[:, 2] >= -1e-15)
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0)
    # inverse: p = w / (|wx|+|wy|+wz); u = x + y, v = x - y
    p = w / np.abs(w).sum(axis=1, keepdims=True)
    assert np.allclose(p[:, 0] + p[:, 1], u) and np.allclose(p[:, 0] - p[:, 1], v)


def _real_sh_scipy(l, m, w):
    theta = np.arccos(np.clip(w[..., 2], -1, 1))
    phi = np.arctan2(w[..., 1], w[..., 0])
    if hasattr(ss, "sph_harm_y"):
        Y = ss.sph_harm_y(l, abs(m), theta, phi)
    else:  # older scipy argument order: (m, l, azimuth, polar)
        Y = ss.sph_harm(abs(m), l, phi, theta)
    if m > 0:
        return math.sqrt(2) * (-1) ** m * Y.real
    if m < 0:
        return math.sqrt(2) * (-1) ** m * Y.imag
    return Y.real


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(1)
    w = rng.normal(size=(500, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    Y = sh.basis(w)
    lm = [(0, 0), (1, -1), (1, 0), (1, 1), (2, -2), (2, -1), (2, 0), (2, 1), (2, 2)]
    for k, (l, m) in enumerate(lm):
        assert np.abs(Y[:, k] - _real_sh_scipy(l, m, w)).max() < 1e-12, (l, m)


def test_cosine_lobe_coefficients():
    # A_l = 2 pi int_0^1 P_l(t) t dt (Funk-Hecke eigenvalue of the clamped cosine)
    for l in range(3):
        val, _ = si.quad(lambda t: ss.eval_legendre(l, t) * t, 0.0, 1.0, epsabs=1e-14)
        assert abs(2 * math.pi * val - sh.A_HAT[l]) < 1e-12


def _unit(v):
    v = np.asarray(v, float)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_uniform_radiance_gives_pi_L():
    rng = np.random.default_rng(2)
    nrm = _unit(rng.normal(size=(40, 3)))
    nrm[:6] = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    L = np.array([0.3, 1.0, 7.0])
    rad = np.broadcast_to(L, (40, 64, 3))
    coeffs = probes.integrate(np.ones(40, bool), nrm, rad, np.ones((40, 64), bool))
    E = sh.irradiance(coeffs, nrm)
    assert np.abs(E - math.pi * L).max() < 1e-12 * 7.0
    # the L2 zonal term of a hemisphere step around the normal vanishes; L0 + L1 give pi L / 2 each
    Y = sh.basis(nrm)
    e0 = sh.A_HAT[0] * Y[:, 0:1] * coeffs[:, 0, :]
    assert np.abs(e0 - math.pi * L / 2).max() < 1e-12 * 7.0


def _cell_of_dir_local(w):
    p = w / np.abs(w).sum(axis=-1, keepdims=True)
    u, v = p[..., 0] + p[..., 1], p[..., 0] - p[..., 1]
    i = np.clip(np.floor((u + 1) * 4), 0, 7).astype(int)
    j = np.clip(np.floor((v + 1) * 4), 0, 7).astype(int)
    return 8 * j + i


def test_projection_matches_bruteforce_sphere_quadrature():
    rng = np.random.default_rng(3)
    nrm = _unit(rng.normal(size=(3,)))
    L = rng.uniform(0, 2, (64, 3))
    coeffs = probes.integrate(np.ones(1, bool), nrm[None], L[None], np.ones((1, 64), bool))[0]
    # midpoint rule on (theta, phi) over the whole sphere, radiance looked up through the inverse map
    nt, nph = 1200, 2400
    th = (np.arange(nt) + 0.5) * math.pi / nt
    ph = (np.arange(nph) + 0.5) * 2 * math.pi / nph
    T, PH = np.meshgrid(th, ph, indexing="ij")
    w = np.stack([np.sin(T) * np.cos(PH), np.sin(T) * np.sin(PH), np.cos(T)], axis=-1)
    dA = np.sin(T) * (math.pi / nt) * (2 * math.pi / nph)
    t, b = hemioct.onb(nrm)
    loc = np.stack([w @ t, w @ b, w @ nrm], axis=-1)
    up = loc[..., 2] > 0
    cell = _cell_of_dir_local(loc)
    f = np.where(up[..., None], L[cell], 0.0)
    Y = sh.basis(w)
    brute = np.einsum("ij,ijk,ijc->kc", dA, Y, f)
    assert np.abs(brute - coeffs).max() < 2e-3 * np.abs(coeffs).max()


def test_onb_is_orthonormal_right_handed():
    rng = np.random.default_rng(4)
    n = _unit(rng.normal(size=(1000, 3)))
    n[:6] = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    t, b = hemioct.onb(n)
    for x, y in ((t, b), (t, n), (b, n)):
        assert np.abs((x * y).sum(1)).max() < 1e-12
    assert np.allclose(np.cross(t, b), n, atol=1e-12)
