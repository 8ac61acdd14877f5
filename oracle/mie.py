"""Mie series of a homogeneous sphere (oracle pin, test infrastructure).

A closed-form solution against which the whole discrete chain (RWG, operators,
PMCHWT signs, right-hand side, powers) is checked.  Textbook form (Bohren and
Huffman, ch. 4) with Riccati-Bessel functions psi_n(z) = z j_n(z) and
xi_n(z) = z h_n^(1)(z), in that book's e^{-i w t} convention: a permittivity
eps_r written for e^{+j w t} (Im eps_r <= 0, Eq. 5) enters as the relative
index m = sqrt(conj(eps_r) conj(mu_r)).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _psi(n, z):
    return z * spherical_jn(n, z)


def _dpsi(n, z):
    return spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)


def _xi(n, x):
    return x * (spherical_jn(n, x) + 1j * spherical_yn(n, x))


def _dxi(n, x):
    h = spherical_jn(n, x) + 1j * spherical_yn(n, x)
    dh = spherical_jn(n, x, derivative=True) + 1j * spherical_yn(n, x, derivative=True)
    return h + x * dh


def coefficients(x: float, m: complex, nmax: int | None = None):
    """Scattering coefficients a_n, b_n (n = 1..nmax) for size parameter x and index m (mu_r = 1)."""
    if nmax is None:
        nmax = int(math.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0)) + 10
    n = np.arange(1, nmax + 1)
    mx = m * x
    px, dpx = _psi(n, x), _dpsi(n, x)
    pm, dpm = _psi(n, mx), _dpsi(n, mx)
    xx, dxx = _xi(n, x), _dxi(n, x)
    a = (m * pm * dpx - px * dpm) / (m * pm * dxx - xx * dpm)
    b = (pm * dpx - m * px * dpm) / (pm * dxx - m * xx * dpm)
    return n, a, b


def efficiencies_eps(x: float, eps_r_ejwt: complex):
    """Q_ext, Q_sca, Q_abs for a sphere of size x = k0 a and permittivity given for e^{+j w t}."""
    m = np.sqrt(np.conj(complex(eps_r_ejwt)))
    return efficiencies(x, m)


def efficiencies(x: float, m: complex):
    n, a, b = coefficients(x, m)
    qext = 2.0 / x ** 2 * float(np.sum((2 * n + 1) * np.real(a + b)))
    qsca = 2.0 / x ** 2 * float(np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2)))
    return {"ext": qext, "sca": qsca, "abs": qext - qsca}
