"""Three-band real spherical harmonics and cosine-lobe convolution (Section 2.4.2).

The paper projects each probe's radiance onto the first three SH bands and
obtains irradiance as the dot product of the projected radiance with the
analytically projected clamped cosine lobe (Ramamoorthi & Hanrahan 2001):
E(n) = sum_lm A_l L_lm Y_lm(n), with A_0 = pi, A_1 = 2 pi / 3, A_2 = pi / 4.

Basis order (l, m): (0,0) (1,-1) (1,0) (1,1) (2,-2) (2,-1) (2,0) (2,1) (2,2),
Y = c0; c1 y; c1 z; c1 x; c2 xy; c2 yz; c3 (3z^2 - 1); c2 xz; c4 (x^2 - y^2),
c0 = 1/(2 sqrt(pi)), c1 = sqrt(3/(4 pi)), c2 = sqrt(15/pi)/2,
c3 = sqrt(5/pi)/4, c4 = sqrt(15/pi)/4.

Because every basis function is a polynomial of degree <= 2 in the
direction, the projection of a radiance field only needs its zeroth, first
and second direction moments: S0 = int L, S1 = int L w, S2 = int L w w^T.
"""
from __future__ import annotations

import math

import numpy as np

C0 = 0.5 / math.sqrt(math.pi)
C1 = math.sqrt(3.0 / (4.0 * math.pi))
C2 = 0.5 * math.sqrt(15.0 / math.pi)
C3 = 0.25 * math.sqrt(5.0 / math.pi)
C4 = 0.25 * math.sqrt(15.0 / math.pi)
A_HAT = (math.pi, 2.0 * math.pi / 3.0, math.pi / 4.0)
BAND = (0, 1, 1, 1, 2, 2, 2, 2, 2)


def basis(w):
    """Y_lm at unit directions w (..., 3) -> (..., 9)."""
    w = np.asarray(w, np.float64)
    x, y, z = w[..., 0], w[..., 1], w[..., 2]
    return np.stack([np.full_like(x, C0), C1 * y, C1 * z, C1 * x, C2 * x * y, C2 * y * z,
                     C3 * (3.0 * z * z - 1.0), C2 * x * z, C4 * (x * x - y * y)], axis=-1)


def project_moments(S0, S1, S2):
    """SH coefficients (..., 9, ch) from moments S0 (..., ch), S1 (..., 3, ch), S2 (..., 3, 3, ch)."""
    x, y, z = 0, 1, 2
    c = [C0 * S0,
         C1 * S1[..., y, :], C1 * S1[..., z, :], C1 * S1[..., x, :],
         C2 * S2[..., x, y, :], C2 * S2[..., y, z, :], C3 * (3.0 * S2[..., z, z, :] - S0),
         C2 * S2[..., x, z, :], C4 * (S2[..., x, x, :] - S2[..., y, y, :])]
    return np.stack(c, axis=-2)


def irradiance(coeffs, n):
    """E(n) = sum_lm A_l L_lm Y_lm(n); coeffs (..., 9, ch), n (..., 3) -> (..., ch)."""
    y = basis(n)
    a = np.array([A_HAT[b] for b in BAND])
    return np.einsum("...k,...kc->...c", y * a, coeffs)
