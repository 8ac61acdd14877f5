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
