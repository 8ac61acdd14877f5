"""Mie series of a homogeneous sphere (oracle pin, test infrastructure).

A closed-form solution against which the whole discrete chain (RWG, operators,
PMCHWT signs, right-hand side, powers) is checked.  Textbook form (Bohren and
Huffman, ch. 4) with Riccati-Bessel functions psi_n(z) = z j_n(z) and
xi_n(z) = z h_n^(1)(z), in that book's e^{-i w t} convention: a permittivity
eps_r written for e^{+j w t} (Im eps_r <= 0, Eq. 6) enters as the relative
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


def _chi(n, z):
    return -z * spherical_yn(n, z)


def _dchi(n, z):
    return -(spherical_yn(n, z) + z * spherical_yn(n, z, derivative=True))


def coated_coefficients(x_core: float, x_shell: float, m_core: complex, m_shell: complex, nmax: int | None = None):
    """Scattering coefficients a_n, b_n of a sphere with a concentric coating (mu_r = 1).

    x_core = k r_core and x_shell = k r_shell are the size parameters of the two
    interfaces, m_core and m_shell the relative indices (e^{-i w t}).  The radial
    function of each region is a combination of Riccati-Bessel functions of
    that region's argument m k r: psi in the core, psi and chi = -z y_n in the
    coating, psi - s xi outside (s = a_n or b_n).  Tangential E and H are
    continuous at both interfaces, which for mu_r = 1 reads (derivatives taken
    with respect to each function's own argument)
        electric (a_n) modes:  u' continuous and m u continuous,
        magnetic (b_n) modes:  u  continuous and m u' continuous,
    the textbook coated-sphere problem (Aden and Kerker 1951; Bohren and
    Huffman, Sec. 8.1).  The four conditions per mode and order are solved as a
    4 x 4 linear system; m_core = m_shell gives the homogeneous sphere.
    """
    if nmax is None:
        nmax = int(math.ceil(x_shell + 4.0 * x_shell ** (1.0 / 3.0) + 2.0)) + 10
    n_all = np.arange(1, nmax + 1)
    a = np.zeros(nmax, dtype=np.complex128)
    b = np.zeros(nmax, dtype=np.complex128)
    m1, m2 = complex(m_core), complex(m_shell)
    x, y = float(x_core), float(x_shell)
    for i, n in enumerate(n_all):
        p1, dp1 = _psi(n, m1 * x), _dpsi(n, m1 * x)
        p2x, dp2x = _psi(n, m2 * x), _dpsi(n, m2 * x)
        c2x, dc2x = _chi(n, m2 * x), _dchi(n, m2 * x)
        p2y, dp2y = _psi(n, m2 * y), _dpsi(n, m2 * y)
        c2y, dc2y = _chi(n, m2 * y), _dchi(n, m2 * y)
        py, dpy = _psi(n, y), _dpsi(n, y)
        xy, dxy = _xi(n, y), _dxi(n, y)
        # unknowns (alpha, beta, gamma, s): core psi, coating psi and chi, scattered xi
        elec = np.array([
            [dp1, -dp2x, -dc2x, 0.0],
            [m1 * p1, -m2 * p2x, -m2 * c2x, 0.0],
            [0.0, dp2y, dc2y, dxy],
            [0.0, m2 * p2y, m2 * c2y, xy],
        ], dtype=np.complex128)
        rhs_a = np.array([0.0, 0.0, dpy, py], dtype=np.complex128)
        magn = np.array([
            [p1, -p2x, -c2x, 0.0],
            [m1 * dp1, -m2 * dp2x, -m2 * dc2x, 0.0],
            [0.0, p2y, c2y, xy],
            [0.0, m2 * dp2y, m2 * dc2y, dxy],
        ], dtype=np.complex128)
        rhs_b = np.array([0.0, 0.0, py, dpy], dtype=np.complex128)
        # column scaling keeps the system well conditioned when chi grows
        for M, r, out in ((elec, rhs_a, a), (magn, rhs_b, b)):
            sc = 1.0 / np.maximum(np.abs(M).max(axis=0), 1e-300)
            sol = np.linalg.solve(M * sc[None, :], r)
            out[i] = sol[3] * sc[3]
    return n_all, a, b


def coated_efficiencies(x_core: float, x_shell: float, m_core: complex, m_shell: complex):
    """Q_ext, Q_sca, Q_abs of the coated sphere, normalised by the outer cross-section."""
    n, a, b = coated_coefficients(x_core, x_shell, m_core, m_shell)
    y = float(x_shell)
    qext = 2.0 / y ** 2 * float(np.sum((2 * n + 1) * np.real(a + b)))
    qsca = 2.0 / y ** 2 * float(np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2)))
    return {"ext": qext, "sca": qsca, "abs": qext - qsca}


def coated_efficiencies_eps(k0: float, r_core: float, r_shell: float, eps_core_ejwt: complex,
                            eps_shell_ejwt: complex):
    """Coated-sphere efficiencies with permittivities given for e^{+j w t} (Im eps <= 0)."""
    m1 = np.sqrt(np.conj(complex(eps_core_ejwt)))
    m2 = np.sqrt(np.conj(complex(eps_shell_ejwt)))
    return coated_efficiencies(k0 * r_core, k0 * r_shell, m1, m2)
