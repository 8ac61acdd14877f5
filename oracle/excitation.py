"""Plane-wave right-hand sides (oracle, test infrastructure).

The tested incident fields of Eq. 8's right-hand side and the two relations
after it, (lambda_i, E^inc) and (lambda_i, H^inc), on RWG bases:

    e_m = int f_m . E_inc dS,      h_m = int f_m . H_inc dS,
    E_inc(r) = e0 exp(-j k0 khat.r),   H_inc = khat x E_inc / eta0,

evaluated with the 7-point rule.  The library's normalised right-hand side is
b = [e ; eta0 h] (``eta0 h`` needs no impedance value).
"""
from __future__ import annotations

import numpy as np

from . import quadrature
from .rwg import RWG


def rhs_planewave(rwg: RWG, k0: float, khat, e0):
    """Normalised RHS b (2ne,) or (2ne,nrhs) for one or several plane waves."""
    khat = np.atleast_2d(np.asarray(khat, dtype=np.float64))
    e0 = np.atleast_2d(np.asarray(e0, dtype=np.complex128))
    single = khat.shape[0] == 1 and np.ndim(e0) == 2 and e0.shape[0] == 1
    tv = rwg.verts[rwg.tris]
    bary, w = quadrature.rule7()
    pts = np.einsum("qk,tkd->tqd", bary, tv)                       # (nt,7,3)
    wts = rwg.area[:, None] * w[None, :]
    coef = rwg.tri_sign * rwg.length[rwg.tri_edge] / (2.0 * rwg.area[:, None])   # (nt,3)
    f = coef[:, None, :, None] * (pts[:, :, None, :] - tv[:, None, :, :])          # (nt,7,i,3)
    ne = rwg.ne
    out = np.zeros((2 * ne, len(khat)), dtype=np.complex128)
    for r in range(len(khat)):
        phase = np.exp(-1j * k0 * np.einsum("tqd,d->tq", pts, khat[r]))
        E = phase[:, :, None] * e0[r][None, None, :]                # (nt,7,3)
        H = np.cross(khat[r][None, None, :], E)                     # eta0 * H_inc
        eloc = np.einsum("tq,tqid,tqd->ti", wts, f, E)
        hloc = np.einsum("tq,tqid,tqd->ti", wts, f, H)
        np.add.at(out[:ne, r], rwg.tri_edge.ravel(), eloc.ravel())
        np.add.at(out[ne:, r], rwg.tri_edge.ravel(), hloc.ravel())
    return out[:, 0] if single else out
