"""Hemispherical octahedral 8x8 probe cells (Section 2.1).

The paper stores each probe's incoming radiance over the oriented hemisphere
in an 8x8 atlas through an octahedral mapping (Cigolle et al. 2014).  This
reading uses the hemi-octahedral form: (u, v) in [-1, 1]^2,
x = (u + v)/2, y = (u - v)/2, z = 1 - |x| - |y|, direction = (x, y, z)/|.|,
in the probe's local frame (tangent, bitangent, normal).  Cell c = 8 j + i
covers u in [-1 + i/4, -1 + (i+1)/4] and v in [-1 + j/4, -1 + (j+1)/4].

Solid angle in (u, v): on the face of the octahedron the point is
p = (x, y, 1-|x|-|y|) and d(omega) = dx dy / |p|^3 = du dv / (2 |p|^3).

Cell moments (solid angle, first and second moments of the direction) are
integrated numerically with tensor Gauss-Legendre rules.  The integrand is
smooth inside a face and only has kinks on x = 0 (u = -v) and y = 0
(u = v); those lines run corner to corner through the diagonal cells, which
are therefore split into two triangles (collapsed Gauss-Legendre rule on
each), so every piece is smooth.
"""
from __future__ import annotations

import numpy as np

CELLS = 64
CELL_W = 0.25


def uv_to_dir(u, v):
    """Local unit direction(s) of hemi-octahedral coordinates."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    x = 0.5 * (u + v)
    y = 0.5 * (u - v)
    z = 1.0 - np.abs(x) - np.abs(y)
    n = np.sqrt(x * x + y * y + z * z)
    return np.stack([x / n, y / n, z / n], axis=-1)


def jacobian(u, v):
    """d(omega) / (du dv) = 1 / (2 |p|^3)."""
    x = 0.5 * (np.asarray(u, np.float64) + v)
    y = 0.5 * (np.asarray(u, np.float64) - v)
    z = 1.0 - np.abs(x) - np.abs(y)
    r2 = x * x + y * y + z * z
    return 0.5 / (r2 * np.sqrt(r2))


def cell_bounds(c: int):
    i, j = c & 7, c >> 3
    return -1.0 + i * CELL_W, -1.0 + j * CELL_W


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w  # on [0, 1]


def _square_rule(u0, v0, h, n, sub):
    t, w = _gl(n)
    us, vs, ws = [], [], []
    hs = h / sub
    for a in range(sub):
        for b in range(sub):
            uu = u0 + (a + t) * hs
            vv = v0 + (b + t) * hs
            U, V = np.meshgrid(uu, vv, indexing="ij")
            W = np.outer(w, w) * hs * hs
            us.append(U.ravel()); vs.append(V.ravel()); ws.append(W.ravel())
    return np.concatenate(us), np.concatenate(vs), np.concatenate(ws)


def _triangle_rule(A, B, C, n, sub):
    """Collapsed (Duffy) Gauss-Legendre rule on triangle ABC, refined by 4^k midpoint splits."""
    tris = [(np.asarray(A, float), np.asarray(B, float), np.asarray(C, float))]
    for _ in range(sub):
        nt = []
        for (a, b, c) in tris:
            ab, bc, ca = 0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)
            nt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = nt
    t, w = _gl(n)
    S, T = np.meshgrid(t, t, indexing="ij")
    WS = np.outer(w, w)
    us, vs, ws = [], [], []
    for (a, b, c) in tris:
        # x = a + s (b - a) + s t (c - b), |J| = s |det(b - a, c - b)|
        det = abs((b[0] - a[0]) * (c[1] - b[1]) - (b[1] - a[1]) * (c[0] - b[0]))
        P = a[None, None, :] + S[..., None] * (b - a)[None, None, :] + (S * T)[..., None] * (c - b)[None, None, :]
        us.append(P[..., 0].ravel()); vs.append(P[..., 1].ravel()); ws.append((WS * S * det).ravel())
    return np.concatenate(us), np.concatenate(vs), np.concatenate(ws)


def cell_rule(c: int, n: int = 16, sub: int = 2):
    """Quadrature nodes (u, v) and weights (du dv measure) covering cell c."""
    u0, v0 = cell_bounds(c)
    h = CELL_W
    on_diag = abs(u0 - v0) < 1e-12                 # the line u = v crosses it corner to corner
    on_anti = abs(u0 + v0 + h) < 1e-12             # the line u = -v crosses it corner to corner
    if on_diag:
        a, b, cc, d = (u0, v0), (u0 + h, v0), (u0 + h, v0 + h), (u0, v0 + h)
        r1 = _triangle_rule(a, b, cc, n, sub)
        r2 = _triangle_rule(a, cc, d, n, sub)
    elif on_anti:
        a, b, cc, d = (u0, v0), (u0 + h, v0), (u0 + h, v0 + h), (u0, v0 + h)
        r1 = _triangle_rule(a, b, d, n, sub)
        r2 = _triangle_rule(b, cc, d, n, sub)
    else:
        return _square_rule(u0, v0, h, n, 2 ** sub)
    return tuple(np.concatenate([p, q]) for p, q in zip(r1, r2))


def cell_moments(n: int = 16, sub: int = 2):
    """Per cell: solid angle (64,), first moment (64, 3), second moment (64, 3, 3), local frame."""
    omega = np.zeros(CELLS)
    m1 = np.zeros((CELLS, 3))
    m2 = np.zeros((CELLS, 3, 3))
    for c in range(CELLS):
        u, v, w = cell_rule(c, n, sub)
        wj = w * jacobian(u, v)
        d = uv_to_dir(u, v)
        omega[c] = wj.sum()
        m1[c] = (wj[:, None] * d).sum(axis=0)
        m2[c] = np.einsum("k,ki,kj->ij", wj, d, d)
    return omega, m1, m2


_CACHE = {}


def moments():
    """Cached cell moments at the default rule."""
    if "m" not in _CACHE:
        _CACHE["m"] = cell_moments()
    return _CACHE["m"]


def onb(n):
    """Tangent and bitangent of unit normals (Duff et al. 2017, 'Building an orthonormal
    basis, revisited'), float64: the probe's local frame is (t, b, n)."""
    n = np.asarray(n, np.float64)
    sign = np.where(np.signbit(n[..., 2]), -1.0, 1.0)
    a = -1.0 / (sign + n[..., 2])
    b = n[..., 0] * n[..., 1] * a
    t = np.stack([1.0 + sign * n[..., 0] * n[..., 0] * a, sign * b, -sign * n[..., 0]], axis=-1)
    bb = np.stack([b, sign + n[..., 1] * n[..., 1] * a, -n[..., 1]], axis=-1)
    return t, bb
