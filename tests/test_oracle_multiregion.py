"""Pins of the multi-region oracle: the coated-sphere series and the layered PMCHWT system.

The coated-sphere coefficients (interface conditions solved order by order)
are pinned by three limits that reduce them to the homogeneous-sphere series:
equal indices, a vanishing core and a vanishing coating (the last one checks
the inner interface with two different indices), and by energy conservation
of a lossless coated sphere.  The dense layered PMCHWT solve is then pinned to
the coated-sphere series (k0 a = 2, shell eps 3.2 - 1.9j, core eps 2.5 - 1.2j,
core radius a / 2): the error must fall as both icospheres are refined.  An
inner interface between two copies of one medium must be transparent (the
homogeneous-sphere series), and one surface between regions 0 and 1 must
give the single-body matrix.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mie
from oracle import multiregion as MR
from oracle import operators as O
from oracle import power as P
from oracle import rwg as R

K0 = 2.0
EPS_SHELL = 3.2 - 1.9j
EPS_CORE = 2.5 - 1.2j
EPS3 = [1.0, EPS_SHELL, EPS_CORE]


def _two_layer(level_outer, level_inner, radius_inner=0.5):
    (vo, to), (vi, ti) = W.concentric_spheres(level_outer, 1.0, level_inner, radius_inner)
    v, t, s = MR.union_mesh([(vo, to), (vi, ti)])
    g = R.build(v, t)
    regions = np.where(s[:, None] == 0, np.array([0, 1]), np.array([1, 2]))
    return g, regions


def _efficiencies(g, regions, eps_core, k0=K0):
    Z = MR.pmchwt_regions(g, regions, k0, [1.0, EPS_SHELL, eps_core])
    b = MR.rhs_planewave(g, regions, k0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    x = np.linalg.solve(Z, b)
    return P.efficiencies(g, k0, MR.exterior_currents(g, regions, x), b, radius=1.0)


def test_coated_equal_indices_is_homogeneous():
    m = np.sqrt(np.conj(EPS_SHELL))
    n, a, b = mie.coefficients(2.0, m)
    _, a2, b2 = mie.coated_coefficients(1.0, 2.0, m, m, nmax=len(n))
    assert np.abs(a - a2).max() < 1e-13
    assert np.abs(b - b2).max() < 1e-13


def test_coated_vanishing_core_and_vanishing_coating():
    m_core = np.sqrt(np.conj(EPS_CORE))
    m_shell = np.sqrt(np.conj(EPS_SHELL))
    n, a_s, b_s = mie.coefficients(2.0, m_shell)
    _, a0, b0 = mie.coated_coefficients(1e-4, 2.0, m_core, m_shell, nmax=len(n))
    assert np.abs(a0 - a_s).max() < 1e-10 and np.abs(b0 - b_s).max() < 1e-10
    # a coating of thickness d -> 0 leaves the core-material sphere, with an O(d) error
    _, a_c, b_c = mie.coefficients(2.0, m_core)
    errs = []
    for d in (1e-3, 1e-5):
        _, a1, b1 = mie.coated_coefficients(2.0 - d, 2.0, m_core, m_shell, nmax=len(n))
        errs.append(max(np.abs(a1 - a_c).max(), np.abs(b1 - b_c).max()))
    assert errs[0] < 1e-3 and errs[1] < 1e-5
    assert 50 < errs[0] / errs[1] < 200


def test_coated_lossless_conserves_energy():
    q = mie.coated_efficiencies(1.0, 3.0, 1.7, 1.3)
    assert q["ext"] > 0.5
    assert abs(q["ext"] - q["sca"]) < 1e-12 * q["ext"]


def test_one_surface_is_the_single_body_matrix():
    v, t = W.icosphere(1)
    g = R.build(v, t)
    regions = np.tile([0, 1], (g.nt, 1))
    Z = MR.pmchwt_regions(g, regions, K0, [1.0, EPS_SHELL])
    Z1 = O.pmchwt_matrix(g, K0, EPS_SHELL)
    assert np.abs(Z - Z1).max() < 1e-13 * np.abs(Z1).max()


def test_region_boundaries_and_reciprocity():
    g, regions = _two_layer(1, 0)
    ne_outer = 30 * 4
    # region 0 sees the outer surface from its normal side, region 2 the inner one from
    # behind, region 1 both (the outer one from behind)
    for r, lo, hi, sg in ((0, 0, ne_outer, 1.0), (2, ne_outer, g.ne, -1.0)):
        sub, edges, sigma = MR.region_boundary(g, regions, r)
        assert np.array_equal(edges, np.arange(lo, hi)) and np.all(sigma == sg)
    sub, edges, sigma = MR.region_boundary(g, regions, 1)
    assert np.array_equal(edges, np.arange(g.ne))
    assert np.all(sigma[:ne_outer] == -1.0) and np.all(sigma[ne_outer:] == 1.0)
    assert np.array_equal(sub.edges, g.edges)
    # Z^T = J Z J with J = diag(I, -I), each region's T and K being symmetric: exactly
    # for the regular pairs between the surfaces (an inner sphere of radius 0.3 has
    # no near-singular pair with the outer one), to the 7-point outer rule's error
    # for the singular pairs on each surface
    g, regions = _two_layer(2, 0, radius_inner=0.3)
    Z = MR.pmchwt_regions(g, regions, K0, [1.0, EPS_SHELL, EPS_CORE])
    J = np.concatenate([np.ones(g.ne), -np.ones(g.ne)])
    D = Z.T - J[:, None] * Z * J[None, :]
    na = 30 * 16
    ia = np.r_[0:na, g.ne:g.ne + na]
    ib = np.r_[na:g.ne, g.ne + na:2 * g.ne]
    assert np.abs(D[np.ix_(ia, ib)]).max() < 1e-13 * np.abs(Z).max()
    assert np.linalg.norm(D) < 5e-3 * np.linalg.norm(Z)


def test_exterior_normals_must_point_out():
    g, regions = _two_layer(1, 0)
    flipped = regions[:, ::-1].copy()
    with pytest.raises(ValueError):
        MR.exterior_mask(g, flipped)


@pytest.fixture(scope="module")
def coated_results():
    ref = mie.coated_efficiencies_eps(K0, 0.5, 1.0, EPS_CORE, EPS_SHELL)
    out = {}
    for lo, li in ((2, 1), (3, 2)):
        g, regions = _two_layer(lo, li)
        q = _efficiencies(g, regions, EPS_CORE)
        out[(lo, li)] = {k: abs(q[k] - ref[k]) / ref[k] for k in ("ext", "abs", "sca")}
    return out


def test_layered_solve_converges_to_coated_series(coated_results):
    coarse, fine = coated_results[(2, 1)], coated_results[(3, 2)]
    for q in ("ext", "abs", "sca"):
        assert fine[q] < coarse[q], (q, coarse, fine)
        assert coarse[q] < 0.06, (q, coarse)
        assert fine[q] < 0.02, (q, fine)


def test_interface_between_equal_media_is_transparent():
    g, regions = _two_layer(2, 1)
    q = _efficiencies(g, regions, EPS_SHELL)
    ref = mie.efficiencies_eps(K0, EPS_SHELL)
    for k in ("ext", "abs", "sca"):
        assert abs(q[k] - ref[k]) / ref[k] < 0.06, (k, q, ref)


def test_rows_on_the_fly_equal_dense():
    g, regions = _two_layer(2, 1)
    Z = MR.pmchwt_regions(g, regions, K0, [1.0, EPS_SHELL, EPS_CORE])
    x = W.complex_normal(2 * g.ne, seed=4)
    rows = np.random.default_rng(5).choice(2 * g.ne, 24, replace=False)
    got = MR.pmchwt_regions_rows_apply(g, regions, K0, [1.0, EPS_SHELL, EPS_CORE], x, rows)
    ref = Z[rows] @ x
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_layered_weight_gradient_by_finite_differences():
    g, regions = _two_layer(1, 0)
    Z = MR.pmchwt_regions(g, regions, K0, [1.0, EPS_SHELL, EPS_CORE])
    kh, e0 = W.plane_wave_batch(3, seed=2)
    Bm = MR.rhs_planewave(g, regions, K0, kh, e0)
    w = W.complex_normal(3, seed=6)
    p, grad = MR.absorbed_and_weight_gradient(g, regions, Z, Bm, w)
    xe = MR.exterior_currents(g, regions, np.linalg.solve(Z, Bm @ w))
    assert abs(p - P.absorbed(g, xe)) < 1e-12 * abs(p)
    h = 1e-6
    for i in range(3):
        d = np.zeros(3, dtype=np.complex128)
        d[i] = h
        fd_re = (MR.absorbed_and_weight_gradient(g, regions, Z, Bm, w + d)[0]
                 - MR.absorbed_and_weight_gradient(g, regions, Z, Bm, w - d)[0]) / (2 * h)
        fd_im = (MR.absorbed_and_weight_gradient(g, regions, Z, Bm, w + 1j * d)[0]
                 - MR.absorbed_and_weight_gradient(g, regions, Z, Bm, w - 1j * d)[0]) / (2 * h)
        # dP/d conj(w) = (dP/d Re w + j dP/d Im w) / 2
        assert abs(0.5 * (fd_re + 1j * fd_im) - grad[i]) < 1e-6 * np.abs(grad).max()


def test_coated_sphere_workload_is_the_union_of_its_surfaces():
    v, t, regions = W.coated_sphere(2, 1.0, 1, 0.5)
    (vo, to), (vi, ti) = W.concentric_spheres(2, 1.0, 1, 0.5)
    v2, t2, s2 = MR.union_mesh([(vo, to), (vi, ti)])
    assert np.array_equal(v, v2) and np.array_equal(t, t2)
    assert np.array_equal(regions, np.where(s2[:, None] == 0, np.array([0, 1]), np.array([1, 2])))


def test_coated_sphere_golden_against_series():
    """The stored dense solution of the 19,200-unknown coated sphere (k0 a = 6) is
    within its discretisation error of the coated-sphere series."""
    import os

    d = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "coated_sphere_oracle.npz"))
    q = mie.coated_efficiencies_eps(float(d["k0"]), float(d["radii"][1]), float(d["radii"][0]),
                                    complex(d["eps"][2]), complex(d["eps"][1]))
    assert np.allclose(d["mie"], [q["ext"], q["abs"], q["sca"]], rtol=1e-12)
    a2 = np.pi * float(d["radii"][0]) ** 2
    for key, ref in (("p_ext", q["ext"]), ("p_abs", q["abs"]), ("p_sca", q["sca"])):
        assert abs(float(d[key]) / a2 - ref) / ref < 0.01, key
    assert d["x"].shape == (19200,)


def test_layered_eps_gradient_lossless_limit():
    """Lossless coating and core: the body absorbs nothing for every real eps of
    either region, so dP/d Re eps = 0 up to the discretisation error of P_abs, and
    adding loss to either region raises the absorption (dP/d Im eps < 0)."""
    g, regions = _two_layer(1, 0)
    b = MR.rhs_planewave(g, regions, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    for r in (1, 2):
        d = MR.absorbed_eps_gradient(g, regions, K0, [1.0, 3.2, 2.5], r, b, h=1e-5)
        assert d[1] < 0, r
        assert abs(d[0]) <= 2e-2 * abs(d[1]), (r, d)


def test_layered_eps_gradient_matches_coated_series():
    """dQ_abs/d eps of the coating and of the core against the coated-sphere
    series' derivatives (central differences of the series): the error shrinks
    from 100 to 400 triangles and is within 10 % at 400."""
    h = 1e-6
    eps = list(EPS3)

    def q_abs(r, e):
        ee = list(eps)
        ee[r] = e
        return mie.coated_efficiencies_eps(K0, 0.5, 1.0, ee[2], ee[1])["abs"]

    errs = {1: [], 2: []}
    for lo, li in ((1, 0), (2, 1)):
        g, regions = _two_layer(lo, li)
        b = MR.rhs_planewave(g, regions, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
        for r in (1, 2):
            e = eps[r]
            ref = np.array([(q_abs(r, e + h) - q_abs(r, e - h)) / (2 * h),
                            (q_abs(r, e + 1j * h) - q_abs(r, e - 1j * h)) / (2 * h)])
            d = MR.absorbed_eps_gradient(g, regions, K0, eps, r, b, h=1e-5) / np.pi
            errs[r].append(np.abs(d - ref).max() / np.abs(ref).max())
    for r in (1, 2):
        assert errs[r][1] < errs[r][0], errs
        assert errs[r][1] <= 0.10, errs


def test_planted_media_swap_fails_the_coated_series(monkeypatch):
    """Assigning the core's medium to the coating and vice versa (a plausible slip in
    the region bookkeeping) moves the efficiencies far outside the discretisation
    error of the coated-sphere pin."""
    g, regions = _two_layer(2, 1)
    ref = mie.coated_efficiencies_eps(K0, 0.5, 1.0, EPS_CORE, EPS_SHELL)
    good = _efficiencies(g, regions, EPS_CORE)
    orig = MR.region_media

    def swapped(k0, eps_r, mu_r=None):
        m = orig(k0, eps_r, mu_r)
        return [m[0], m[2], m[1]]

    monkeypatch.setattr(MR, "region_media", swapped)
    bad = _efficiencies(g, regions, EPS_CORE)
    e_good = max(abs(good[q] - ref[q]) / ref[q] for q in ("ext", "abs", "sca"))
    e_bad = max(abs(bad[q] - ref[q]) / ref[q] for q in ("ext", "abs", "sca"))
    assert e_good < 0.06 and e_bad > 3 * e_good, (e_good, e_bad)
