"""Pins of the oracle's quadrature rule and closed-form triangle integrals.

The 7-point rule is checked against exact monomial integrals on the reference
triangle; the closed-form integrals of R^-1, R, (rho'-rho)R^q, grad R^-1 and
grad R are checked against brute-force polar integration around the
projection of the observation point (adaptive radial quadrature), including
the principal value of grad(1/R) for points on the triangle's own plane.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import potentials, quadrature


def test_rule7_weights_and_points():
    bary, w = quadrature.rule7()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(bary.sum(axis=1), 1.0, atol=1e-15)
    assert np.all(bary > 0)


def test_rule7_exact_to_degree5_only():
    bary, w = quadrature.rule7()
    x, y = bary[:, 1], bary[:, 2]
    # reference triangle (0,0),(1,0),(0,1) has area 1/2: int x^a y^b = a! b! / (a+b+2)!
    for deg in range(0, 7):
        worst = 0.0
        for a in range(deg + 1):
            b = deg - a
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            approx = 0.5 * np.sum(w * x ** a * y ** b)
            worst = max(worst, abs(approx - exact) / exact)
        if deg <= 5:
            assert worst < 1e-14, (deg, worst)
        else:
            assert worst > 1e-6, "rule should not be exact at degree 6"


TRI = np.array([[0.1, -0.2, 0.05], [1.3, 0.1, 0.2], [0.4, 0.9, -0.1]])


def _frame(tv):
    n = np.cross(tv[1] - tv[0], tv[2] - tv[0])
    n /= np.linalg.norm(n)
    return n


def _brute(r, tv, h_zero=False):
    """Polar integration around rho over the signed sub-triangles (rho, V_i, V_i+1)."""
    n = _frame(tv)
    h = 0.0 if h_zero else float(np.dot(n, r - tv[0]))
    rho = r - h * n
    out = {k: 0.0 for k in ("S_m1", "S_1")}
    out.update({k: np.zeros(3) for k in ("V_m1", "V_1", "G_m3", "G_1")})
    gl_x, gl_w = np.polynomial.legendre.leggauss(48)
    for i in range(3):
        A, B = tv[i], tv[(i + 1) % 3]
        a, b = A - rho, B - rho
        la, lb = np.linalg.norm(a), np.linalg.norm(b)
        if la < 1e-14 or lb < 1e-14:
            continue
        ea = a / la
        sgn = np.sign(np.dot(np.cross(a, b), n))
        if sgn == 0:
            continue
        e_perp = np.cross(n, ea) * sgn            # rotation direction toward b
        theta_max = math.atan2(np.dot(b, e_perp), np.dot(b, ea))
        # distance to the line AB along direction u(theta)
        d = B - A
        for panel in range(4):
            t0, t1 = panel * theta_max / 4, (panel + 1) * theta_max / 4
            for xg, wg in zip(gl_x, gl_w):
                th = 0.5 * (t1 - t0) * xg + 0.5 * (t1 + t0)
                wt = 0.5 * (t1 - t0) * wg * sgn
                u = math.cos(th) * ea + math.sin(th) * e_perp
                # solve rho + s u = A + t d (in plane) for s
                M = np.stack([u, -d], axis=1)
                s_max = np.linalg.lstsq(M, A - rho, rcond=None)[0][0]
                R = lambda s: math.sqrt(s * s + h * h)
                q = lambda f: quad(f, 0.0, s_max, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
                i_sm1 = q(lambda s: s / R(s))
                i_s1 = q(lambda s: s * R(s))
                i_v1 = q(lambda s: s * s / R(s))
                i_v3 = q(lambda s: s * s * R(s))
                out["S_m1"] += wt * i_sm1
                out["S_1"] += wt * i_s1
                out["V_m1"] += wt * i_v1 * u
                out["V_1"] += wt * i_v3 * u
                if h == 0.0:
                    g_in = math.log(s_max)              # finite part of int ds/s
                    g_n = 0.0
                else:
                    g_in = q(lambda s: s * s / R(s) ** 3)
                    g_n = q(lambda s: s / R(s) ** 3)
                out["G_m3"] += wt * (g_in * u - h * g_n * n)
                out["G_1"] += wt * (-i_v1 * u + h * i_sm1 * n)
    return out


CASES = [
    ("above_inside", lambda tv, n: tv.mean(axis=0) + 0.3 * n, False),
    ("above_outside", lambda tv, n: tv[1] + 0.4 * (tv[1] - tv[0]) + 0.2 * n, False),
    ("close_above", lambda tv, n: 0.2 * tv[0] + 0.5 * tv[1] + 0.3 * tv[2] + 1e-3 * n, False),
    ("inplane_outside", lambda tv, n: tv[2] + 0.5 * (tv[2] - tv[0]) + 0.3 * (tv[1] - tv[0]), True),
    ("inplane_inside_pv", lambda tv, n: 0.25 * tv[0] + 0.35 * tv[1] + 0.4 * tv[2], True),
]


@pytest.mark.parametrize("name,make,inplane", CASES, ids=[c[0] for c in CASES])
def test_closed_forms_match_polar_brute_force(name, make, inplane):
    tv = TRI
    n = _frame(tv)
    r = make(tv, n)
    got = potentials.triangle_integrals(r[None], tv[None], n[None], inplane=np.array([inplane]))
    ref = _brute(r, tv, h_zero=inplane)
    for key in ("S_m1", "S_1", "V_m1", "V_1", "G_m3", "G_1"):
        g = np.asarray(got[key][0], dtype=float)
        e = np.asarray(ref[key], dtype=float)
        scale = max(np.max(np.abs(e)), 1e-3)
        assert np.max(np.abs(g - e)) <= 1e-9 * scale, (key, g, e)


def test_solid_angle_limit_inside():
    # just above an interior point the normal part of int grad(1/R) tends to -2 pi n
    tv = TRI
    n = _frame(tv)
    r = tv.mean(axis=0) + 1e-9 * n
    got = potentials.triangle_integrals(r[None], tv[None], n[None])
    assert abs(np.dot(got["G_m3"][0], n) + 2 * math.pi) < 1e-6
