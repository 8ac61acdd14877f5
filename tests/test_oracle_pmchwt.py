"""Whole-chain pins of the oracle: Mie series, energy balance, lossless limit.

The dense PMCHWT solve of a homogeneous lossy sphere (k0 a = 2,
eps_r = 3.2 - 1.9j) is compared with the Mie series; the error must fall as the
icosphere is refined (discretisation-limited, a few percent at 320 triangles).
Signs and conventions of every block (T, K, the right-hand side, the power
functionals) are fixed by this comparison.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import excitation as E
from oracle import mie
from oracle import operators as O
from oracle import power as P
from oracle import rwg as R

K0 = 2.0
EPS = 3.2 - 1.9j


def _solve(level, eps=EPS, k0=K0):
    v, t = W.icosphere(level)
    g = R.build(v, t)
    Z = O.pmchwt_matrix(g, k0, eps)
    b = E.rhs_planewave(g, k0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    x = np.linalg.solve(Z, b)
    return g, x, b


@pytest.fixture(scope="module")
def results():
    out = {}
    for level in (1, 2, 3):
        g, x, b = _solve(level)
        out[level] = P.efficiencies(g, K0, x, b, radius=1.0)
    return out


def test_mie_convergence(results):
    ref = mie.efficiencies_eps(K0, EPS)
    errs = {q: [abs(results[l][q] - ref[q]) / ref[q] for l in (1, 2, 3)] for q in ("ext", "abs", "sca")}
    for q, e in errs.items():
        assert e[0] > e[1] > e[2], (q, e)
        assert e[1] < 0.05, (q, e)
        assert e[2] < 0.02, (q, e)


def test_energy_balance_improves(results):
    bal = [abs(results[l]["ext"] - results[l]["abs"] - results[l]["sca"]) / results[l]["ext"] for l in (1, 2, 3)]
    assert bal[0] > bal[2]
    assert bal[2] < 5e-3


def test_lossless_sphere_absorbs_nothing():
    g, x, b = _solve(2, eps=3.2)
    q = P.efficiencies(g, K0, x, b, radius=1.0)
    ref = mie.efficiencies_eps(K0, 3.2)
    assert abs(q["abs"]) < 0.02 * q["ext"]
    assert abs(q["ext"] - ref["ext"]) / ref["ext"] < 0.05


def test_absorbed_density_sums_to_total():
    g, x, b = _solve(1)
    dens = P.absorbed_density(g, x)
    assert abs(np.sum(dens * g.area) - P.absorbed(g, x)) < 1e-12 * abs(P.absorbed(g, x))


def test_twisted_gram_antisymmetric():
    v, t = W.icosphere(1)
    g = R.build(v, t)
    X = P.twisted_gram(g).toarray()
    assert np.abs(X + X.T).max() < 1e-15 * np.abs(X).max()


def test_rhs_static_limit_closed_form():
    # k0 -> 0: e_m = E0 . int f_m = E0 . (l/2) [(c+ - p+) - (c- - p-)]
    v, t = W.icosphere(1)
    g = R.build(v, t)
    e0 = np.array([0.3, -0.2, 0.9])
    b = E.rhs_planewave(g, 0.0, [0.0, 0.0, 1.0], e0)
    cen = v[t].mean(axis=1)
    intf = 0.5 * g.length[:, None] * ((cen[g.tplus] - v[g.pplus]) - (cen[g.tminus] - v[g.pminus]))
    assert np.abs(b[:g.ne] - intf @ e0).max() < 1e-14


def test_mie_series_limits():
    # Rayleigh limit of a small sphere
    x, eps = 0.01, 2.5 - 0.8j
    m = np.sqrt(np.conj(eps))
    q = mie.efficiencies(x, m)
    al = (m ** 2 - 1) / (m ** 2 + 2)
    assert abs(q["sca"] - 8.0 / 3.0 * x ** 4 * abs(al) ** 2) / q["sca"] < 1e-3
    assert abs(q["abs"] - 4 * x * al.imag) / q["abs"] < 1e-3
    # lossless: nothing absorbed
    q = mie.efficiencies(3.0, 1.5)
    assert abs(q["ext"] - q["sca"]) < 1e-12
    # large absorbing sphere: extinction paradox, Q_ext -> 2 with the x^(-2/3) edge term
    q200 = mie.efficiencies(200.0, 1.3 + 0.2j)["ext"]
    q800 = mie.efficiencies(800.0, 1.3 + 0.2j)["ext"]
    assert 2.0 < q800 < q200
    for x, qq in ((200.0, q200), (800.0, q800)):
        assert 1.5 < (qq - 2.0) * x ** (2.0 / 3.0) < 2.2
