"""Pins of oracle/gradient.py: the weight gradient of the absorbed power against
central finite differences of P(w) (computed by forward solves only, with
power.absorbed), and the Hermitian structure of the weight form Q."""
import numpy as np
import pytest

import workloads as W
from oracle import excitation as E
from oracle import gradient as G
from oracle import operators as O
from oracle import power as P
from oracle import rwg as R

K0, EPS = 2.0, 3.2 - 1.9j


@pytest.fixture(scope="module")
def case():
    v, t = W.icosphere(1)
    g = R.build(v, t)
    Z = O.pmchwt_matrix(g, K0, EPS)
    khat, e0 = W.plane_wave_batch(4, seed=2)
    Bm = np.stack([E.rhs_planewave(g, K0, khat[i], e0[i]) for i in range(4)], axis=1)
    w = W.complex_normal(4, seed=3) / 8.0
    return g, Z, Bm, w


def _p(g, Z, Bm, w):
    return P.absorbed(g, np.linalg.solve(Z, Bm @ w))


def test_weight_form_is_hermitian_and_matches_power(case):
    g, Z, Bm, w = case
    Q = G.weight_form(g, Z, Bm)
    assert np.abs(Q - Q.conj().T).max() <= 1e-12 * np.abs(Q).max()
    p, _ = G.absorbed_and_weight_gradient(g, Z, Bm, w)
    assert abs(p - _p(g, Z, Bm, w)) <= 1e-12 * abs(p)
    # absorbed power of a lossy body is positive for any excitation
    assert np.linalg.eigvalsh(Q).min() > 0


def test_weight_gradient_matches_finite_differences(case):
    g, Z, Bm, w = case
    _, grad = G.absorbed_and_weight_gradient(g, Z, Bm, w)
    h = 1e-6
    fd = np.zeros(len(w), dtype=np.complex128)
    for i in range(len(w)):
        e = np.zeros(len(w))
        e[i] = 1.0
        dre = (_p(g, Z, Bm, w + h * e) - _p(g, Z, Bm, w - h * e)) / (2 * h)
        dim = (_p(g, Z, Bm, w + 1j * h * e) - _p(g, Z, Bm, w - 1j * h * e)) / (2 * h)
        fd[i] = dre + 1j * dim          # = 2 dP/d conj(w_i)
    assert np.abs(2 * grad - fd).max() <= 1e-7 * np.abs(fd).max()


def test_planted_sign_error_is_caught(case):
    """A gradient taken with the non-conjugate Wirtinger derivative (a plausible
    slip) fails the finite-difference pin."""
    g, Z, Bm, w = case
    _, grad = G.absorbed_and_weight_gradient(g, Z, Bm, w)
    h = 1e-6
    e = np.zeros(len(w))
    e[0] = 1.0
    dim = (_p(g, Z, Bm, w + 1j * h * e) - _p(g, Z, Bm, w - 1j * h * e)) / (2 * h)
    assert abs(2 * np.conj(grad[0]).imag - dim) > 1e-3 * abs(dim)


def test_eps_gradient_lossless_limit():
    """At a real permittivity the body absorbs nothing for every real eps_r, so
    dP/d Re eps_r = 0 up to the discretisation error of P_abs (the discrete
    absorbed power of a lossless body is small but not zero); adding loss
    (Im eps_r < 0 under e^{+jwt}) raises the absorption, so dP/d Im eps_r < 0."""
    v, t = W.icosphere(1)
    g = R.build(v, t)
    b = E.rhs_planewave(g, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    d = G.absorbed_eps_gradient(g, K0, 3.2 + 0.0j, b)
    scale = abs(d[1])
    assert scale > 0
    assert abs(d[0]) <= 2e-2 * scale
    assert d[1] < 0


def test_eps_gradient_matches_mie_series():
    """dQ_abs/d eps_r of the discretised sphere (k0 a = 2) against the Mie
    series' derivative (central differences of the series): the error shrinks
    from 80 to 320 triangles and is within 10 % at 320 (discretisation-limited,
    like Q_abs itself)."""
    from oracle import mie

    eps = 3.2 - 1.9j
    h = 1e-6
    qm = lambda e: mie.efficiencies_eps(K0, e)["abs"]  # noqa: E731
    ref = np.array([(qm(eps + h) - qm(eps - h)) / (2 * h), (qm(eps + 1j * h) - qm(eps - 1j * h)) / (2 * h)])
    errs = []
    for level in (1, 2):
        v, t = W.icosphere(level)
        g = R.build(v, t)
        b = E.rhs_planewave(g, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
        d = G.absorbed_eps_gradient(g, K0, eps, b, h=1e-5) / np.pi  # efficiency per unit eps (radius 1)
        errs.append(np.abs(d - ref).max() / np.abs(ref).max())
    assert errs[1] < errs[0]
    assert errs[1] <= 0.10, errs
