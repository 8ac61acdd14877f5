"""Gradient of the absorbed power with respect to excitation weights (oracle,
test infrastructure: imported only by tests and the benchmark's baseline).

The paper computes no gradients; this is the plain definition the adjoint path
of the library must reproduce.  With the absorbed power of the dosimetric output
(Sec. I; see power.absorbed)

    P(x) = Re(xJ^H X xM) = x^H H x,      H = 1/2 [[0, X], [X^T, 0]]  (X real),

and the excitation a weighted sum of right-hand sides, b = Bm w, x = Z^-1 b, the
power is a Hermitian quadratic form in the weights,

    P(w) = w^H Q w,      Q = (Z^-1 Bm)^H H (Z^-1 Bm),

so its gradient with respect to conj(w) is Q w -- written out here with a dense
LU solve and no adjoint system.  Parity of this function is pinned in the tests
by central finite differences of P(w) and by the Hermitian structure of Q.

The gradient with respect to the interior permittivity is taken by central
differences of the dense solution (absorbed_eps_gradient), pinned in the tests by
the lossless limit (P = 0 for every real eps_r, so dP/d Re eps_r = 0 there and
dP/d Im eps_r < 0) and by the Mie series of the sphere (same derivative of the
absorption efficiency, to the discretisation error).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import power
from .rwg import RWG


def hermitian_form(rwg: RWG):
    """Sparse H = 1/2 [[0, X], [X^T, 0]] with P_abs(x) = x^H H x."""
    X = power.twisted_gram(rwg)
    return 0.5 * sp.bmat([[None, X], [X.T, None]], format="csr")


def weight_form(rwg: RWG, Z, Bm):
    """Dense Q = (Z^-1 Bm)^H H (Z^-1 Bm) (nw x nw, Hermitian)."""
    Y = np.linalg.solve(Z, Bm)
    return Y.conj().T @ (hermitian_form(rwg) @ Y)


def absorbed_and_weight_gradient(rwg: RWG, Z, Bm, w):
    """(P(w), dP/d conj(w)) for b = Bm w, from the dense form Q."""
    Q = weight_form(rwg, Z, Bm)
    w = np.asarray(w, dtype=np.complex128)
    return float(np.real(np.vdot(w, Q @ w))), Q @ w


def absorbed_eps_gradient(rwg: RWG, k0: float, eps_r: complex, b, h: float = 1e-6):
    """(dP/d Re eps_r, dP/d Im eps_r) of P = Re(xJ^H X xM), x = Z(eps_r)^-1 b, by
    central differences of the dense LU solution (the plain definition; b does not
    depend on eps_r: the excitation lives in the exterior medium)."""
    from . import operators

    def p_of(e):
        Z = operators.pmchwt_matrix(rwg, k0, e)
        return power.absorbed(rwg, np.linalg.solve(Z, b))

    d_re = (p_of(eps_r + h) - p_of(eps_r - h)) / (2 * h)
    d_im = (p_of(eps_r + 1j * h) - p_of(eps_r - 1j * h)) / (2 * h)
    return np.array([d_re, d_im])
