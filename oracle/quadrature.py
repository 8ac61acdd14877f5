"""Seven-point, degree-5 Gaussian rule on a triangle (oracle, test infrastructure).

The Galerkin integrals (lambda_i, O lambda_j) of Sec. III are evaluated with
this rule on the test and on the source triangle.  The points and weights are
the classical Radon/Strang-Fix degree-5 rule, written here from its closed
form (barycentric coordinates built from sqrt(15)).
"""
from __future__ import annotations

import math

import numpy as np


def rule7():
    """Barycentric points (7,3) and weights (7,) summing to 1."""
    s = math.sqrt(15.0)
    a1 = (6.0 - s) / 21.0
    b1 = 1.0 - 2.0 * a1
    a2 = (6.0 + s) / 21.0
    b2 = 1.0 - 2.0 * a2
    w1 = (155.0 - s) / 1200.0
    w2 = (155.0 + s) / 1200.0
    bary = np.array(
        [
            [1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0],
            [b1, a1, a1],
            [a1, b1, a1],
            [a1, a1, b1],
            [b2, a2, a2],
            [a2, b2, a2],
            [a2, a2, b2],
        ]
    )
    w = np.array([9.0 / 40.0, w1, w1, w1, w2, w2, w2])
    return bary, w


def points(tri_verts):
    """Quadrature points of triangles given as (..., 3, 3) vertex arrays -> (..., 7, 3)."""
    bary, _ = rule7()
    return np.einsum("qk,...kd->...qd", bary, tri_verts)
