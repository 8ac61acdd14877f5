"""Absorbed, extinguished and scattered power (oracle, test infrastructure).

The dosimetric output the paper aims at (Sec. I: the energy absorbed by the
tissue; Sec. IV: the field scattered by the skin sample).  With J = n x H and
M = E x n on the outward-oriented surface, E_t = n x M, and the power flowing
into the body is

    P_abs = -1/2 Re oint (E x H*).n dS = 1/2 Re oint (n x M).J* dS
          = 1/2 Re  J^H X M,          X[m,n] = int f_m . (n x f_n) dS,

the extinguished power is P_ext = 1/2 Re oint (E_inc.J* + H_inc*.M) dS, and the
scattered power is the far-field flux 1/(2 eta0) oint |E_far|^2 dOmega with

    E_far(rhat) = (j k0/(4 pi)) [ rhat x L - eta0 N_t ],
    N = int J e^{j k0 rhat.r'} dS',  L = int M e^{j k0 rhat.r'} dS'.

In the library's normalised unknowns x = [eta0 J ; M] and b = [e ; eta0 h]
every power carries the same factor 1/(2 eta0); the functions here return
efficiencies Q = P / (pi a^2 |E0|^2 / (2 eta0)), in which eta0 cancels.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import quadrature
from .rwg import RWG


def _basis_at_points(rwg: RWG):
    tv = rwg.verts[rwg.tris]
    bary, w = quadrature.rule7()
    pts = np.einsum("qk,tkd->tqd", bary, tv)
    wts = rwg.area[:, None] * w[None, :]
    coef = rwg.tri_sign * rwg.length[rwg.tri_edge] / (2.0 * rwg.area[:, None])
    f = coef[:, None, :, None] * (pts[:, :, None, :] - tv[:, None, :, :])   # (nt,7,i,3)
    return pts, wts, f


def twisted_gram_local(rwg: RWG):
    """Per-triangle 3x3 blocks X_t[i,j] = int_t f_i . (n x f_j) dS (exact: degree 2)."""
    pts, wts, f = _basis_at_points(rwg)
    nf = np.cross(rwg.normal[:, None, None, :], f)                    # (nt,7,j,3)
    return np.einsum("tq,tqid,tqjd->tij", wts, f, nf)


def twisted_gram(rwg: RWG):
    """Sparse X (ne x ne)."""
    loc = twisted_gram_local(rwg)
    rows = np.broadcast_to(rwg.tri_edge[:, :, None], loc.shape).ravel()
    cols = np.broadcast_to(rwg.tri_edge[:, None, :], loc.shape).ravel()
    return sp.coo_matrix((loc.ravel(), (rows, cols)), shape=(rwg.ne, rwg.ne)).tocsr()


def gram_local(rwg: RWG):
    """Per-triangle 3x3 blocks of the Gram matrix G[m,n] = int f_m . f_n (after Eq. 8)."""
    pts, wts, f = _basis_at_points(rwg)
    return np.einsum("tq,tqid,tqjd->tij", wts, f, f)


def absorbed(rwg: RWG, x):
    """Re(xJ^H X xM) = 2 eta0 P_abs (x normalised, shape (2ne,))."""
    ne = rwg.ne
    X = twisted_gram(rwg)
    return float(np.real(np.vdot(x[:ne], X @ x[ne:])))


def absorbed_density(rwg: RWG, x):
    """Per-triangle 2 eta0 * (absorbed power / area), shape (nt,)."""
    ne = rwg.ne
    loc = twisted_gram_local(rwg)
    xj = x[:ne][rwg.tri_edge]
    xm = x[ne:][rwg.tri_edge]
    p = np.real(np.einsum("ti,tij,tj->t", np.conj(xj), loc, xm))
    return p / rwg.area


def extinguished(rwg: RWG, x, b):
    """Re(xJ^H bJ + bM^H xM) = 2 eta0 P_ext."""
    ne = rwg.ne
    return float(np.real(np.vdot(x[:ne], b[:ne]) + np.vdot(b[ne:], x[ne:])))


def scattered(rwg: RWG, k0: float, x, n_theta: int = 64, n_phi: int = 128):
    """oint |E_far|^2 dOmega = 2 eta0 P_sca, product Gauss-Legendre x uniform grid."""
    ne = rwg.ne
    pts, wts, f = _basis_at_points(rwg)
    Jq = np.einsum("ti,tiqd->tqd", x[:ne][rwg.tri_edge], f.transpose(0, 2, 1, 3))   # eta0 J at points
    Mq = np.einsum("ti,tiqd->tqd", x[ne:][rwg.tri_edge], f.transpose(0, 2, 1, 3))
    P = pts.reshape(-1, 3)
    Jw = (Jq * wts[:, :, None]).reshape(-1, 3)
    Mw = (Mq * wts[:, :, None]).reshape(-1, 3)
    ct, wt = np.polynomial.legendre.leggauss(n_theta)
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    st = np.sqrt(1.0 - ct * ct)
    total = 0.0
    for it in range(n_theta):
        rhat = np.stack([st[it] * np.cos(phi), st[it] * np.sin(phi), np.full(n_phi, ct[it])], axis=1)
        ph = np.exp(1j * k0 * (rhat @ P.T))                           # (n_phi, npts)
        N = ph @ Jw
        L = ph @ Mw
        Nt = N - np.sum(rhat * N, axis=1, keepdims=True) * rhat
        E = (1j * k0 / (4.0 * math.pi)) * (np.cross(rhat, L) - Nt)
        total += wt[it] * (2.0 * math.pi / n_phi) * np.sum(np.abs(E) ** 2)
    return float(total)


def efficiencies(rwg: RWG, k0: float, x, b, radius: float, e0_norm: float = 1.0):
    """Q_ext, Q_abs, Q_sca of the normalised solution (cross sections over pi a^2)."""
    den = math.pi * radius ** 2 * e0_norm ** 2
    return {
        "ext": extinguished(rwg, x, b) / den,
        "abs": absorbed(rwg, x) / den,
        "sca": scattered(rwg, k0, x) / den,
    }
