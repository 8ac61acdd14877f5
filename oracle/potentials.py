"""Closed-form integrals over a flat triangle (oracle, test infrastructure).

The operators of Sec. II carry a principal value (D, D*) and a finite part
(N).  In a Galerkin code these singular kernels are tamed by singularity
extraction: the leading terms of the small-R expansion of the kernel,

    e^{-jkR}/(4 pi R) = 1/(4 pi R) - k^2 R/(8 pi) + smooth,

are integrated over the source triangle in closed form and only the smooth
remainder goes to quadrature.  This module provides those closed forms for an
observation point r and a flat triangle T with unit normal n:

    S_m1 = int_T 1/R dS'                 S_1  = int_T R dS'
    V_m1 = int_T (rho'-rho)/R dS'        V_1  = int_T (rho'-rho) R dS'
    G_m3 = int_T grad_r (1/R) dS'        G_1  = int_T grad_r R dS'

with rho the projection of r on the plane of T and h = n.(r - v0) its signed
height.  They follow from the divergence and gradient theorems in the plane,
which turn every surface integral into line integrals I_q = int_edge R^q dl
(q = -1, 1, 3) plus, for 1/R and grad(1/R), the solid angle Omega subtended by
T (the classical results of Wilton et al. 1984 and Graglia 1993):

    (q+2) int R^q = q h^2 int R^{q-2} + sum_i t_i I_i^q
    int (rho'-rho) R^q = 1/(q+2) sum_i m_i I_i^{q+2}
    h^2 int R^-3 = |h| Omega

where m_i is the outward in-plane unit normal of edge i and t_i the signed
distance from rho to the line of edge i.  For h = 0 with rho inside T (a
triangle interacting with itself) the normal part of G_m3 is the Cauchy
principal value, i.e. zero.
"""
from __future__ import annotations

import numpy as np


def _line_integrals(lm, lp, r0sq):
    """I^-1, I^1, I^3 of R = sqrt(l^2 + R0^2) over l in [lm, lp] (vectorised)."""
    rm = np.sqrt(lm * lm + r0sq)
    rp = np.sqrt(lp * lp + r0sq)
    with np.errstate(divide="ignore", invalid="ignore"):
        f1 = np.log((rp + lp) / (rm + lm))            # lm >= 0: no cancellation
        f2 = np.log((rm - lm) / (rp - lp))            # lp <= 0
        f3 = np.log((rp + lp) * (rm - lm) / r0sq)     # lm < 0 < lp
    im1 = np.where(lm >= 0.0, f1, np.where(lp <= 0.0, f2, f3))
    i1 = 0.5 * (lp * rp - lm * rm + r0sq * im1)
    i3 = 0.25 * (lp * rp ** 3 - lm * rm ** 3) + 0.75 * r0sq * i1
    return im1, i1, i3, rm, rp


def triangle_integrals(r, tv, normal, inplane=None):
    """Closed-form integrals for observation points r (P,3) and triangles tv (P,3,3).

    ``normal`` (P,3) is the unit normal of each triangle, consistent with its
    counter-clockwise vertex order.  ``inplane`` (P,) bool forces h = 0 (used
    when r lies on the triangle itself).  Returns a dict with S_m1, S_1 (P,),
    V_m1, V_1, G_m3, G_1 (P,3).
    """
    r = np.asarray(r, dtype=np.float64)
    tv = np.asarray(tv, dtype=np.float64)
    n = np.asarray(normal, dtype=np.float64)
    h = np.einsum("pd,pd->p", n, r - tv[:, 0, :])
    if inplane is not None:
        h = np.where(inplane, 0.0, h)
    rho = r - h[:, None] * n
    ah = np.abs(h)
    s_m1 = np.zeros(len(r))
    sum_t_i1 = np.zeros(len(r))
    omega = np.zeros(len(r))
    v_m1 = np.zeros_like(r)
    v_1 = np.zeros_like(r)
    g_in = np.zeros_like(r)
    for i in range(3):
        va = tv[:, i, :]
        vb = tv[:, (i + 1) % 3, :]
        e = vb - va
        lhat = e / np.linalg.norm(e, axis=1, keepdims=True)
        mhat = np.cross(lhat, n)
        lm = np.einsum("pd,pd->p", va - rho, lhat)
        lp = np.einsum("pd,pd->p", vb - rho, lhat)
        t = np.einsum("pd,pd->p", va - rho, mhat)
        r0sq = t * t + h * h
        im1, i1, i3, rm, rp = _line_integrals(lm, lp, r0sq)
        # an edge whose line passes through rho (t = 0) adds nothing to the t-weighted sums
        im1_t = np.where(t == 0.0, 0.0, im1)
        s_m1 += t * im1_t
        sum_t_i1 += t * i1
        with np.errstate(divide="ignore", invalid="ignore"):
            a_p = np.arctan(t * lp / (r0sq + ah * rp))
            a_m = np.arctan(t * lm / (r0sq + ah * rm))
        om = np.where(r0sq + ah * np.minimum(rp, rm) > 0.0, a_p - a_m, 0.0)
        omega += np.nan_to_num(om)
        v_m1 += mhat * i1[:, None]
        v_1 += mhat * (i3 / 3.0)[:, None]
        g_in -= mhat * im1[:, None]
    s_m1 = s_m1 - ah * omega
    s_1 = (h * h * s_m1 + sum_t_i1) / 3.0
    g_m3 = g_in - (np.sign(h) * omega)[:, None] * n
    g_1 = -v_m1 + (h * s_m1)[:, None] * n
    return {"S_m1": s_m1, "S_1": s_1, "V_m1": v_m1, "V_1": v_1, "G_m3": g_m3, "G_1": g_1, "h": h, "rho": rho}
