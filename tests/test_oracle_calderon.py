"""Pins of the oracle's Calderon preconditioner (oracle/calderon.py), each against a
fact fixed outside the construction:

  * the barycentric refinement is a closed, consistently oriented mesh of six
    equal-area children per triangle on the same flat faces;
  * the coarse RWG functions written in the fine basis equal the coarse
    functions pointwise (exact representation);
  * the BC functions' radial fluxes equal the closed form l_e (1/2 - i/N), with
    i counted by angle around the vertex in the tangent plane (independent of
    the least-norm solve that builds them), and their divergence is +-l_e/N per
    fine triangle on the two dual cells and zero elsewhere;
  * the mixed Gram matrix is well conditioned under refinement, while the
    rotated RWG-RWG pairing is antisymmetric;
  * the preconditioned PMCHWT operator Z P has a condition number and a GMRES
    iteration count that stay flat from 80 to 320 triangles while those of Z
    grow by about the h^-2 of a first-kind operator (the Calderon property of
    Sec. III carried to the 3-D PMCHWT operator), and with G^-1 in place of G^-T,
    a plausible slip, the condition number grows again."""
import numpy as np
import pytest

import workloads as W
from oracle import calderon as CA
from oracle import operators as O
from oracle import rwg as R

EPS = 3.2 - 1.9j
_cache = {}


def ref(level):
    if level not in _cache:
        v, t = W.icosphere(level)
        _cache[level] = CA.refine(R.build(v, t))
    return _cache[level]


def test_refinement_is_a_closed_mesh_of_equal_children():
    r = ref(1)
    c, f = r.coarse, r.fine
    assert f.nt == 6 * c.nt and f.ne == 6 * c.ne and len(f.verts) == len(c.verts) + c.ne + c.nt
    assert np.allclose(f.area, c.area[r.parent] / 6.0, rtol=1e-12)
    assert np.allclose(f.normal, c.normal[r.parent], atol=1e-12)
    # every fine vertex lies on the plane of its parent
    for tau in range(f.nt):
        T = r.parent[tau]
        d = f.verts[f.tris[tau]] - c.verts[c.tris[T, 0]]
        assert np.abs(d @ c.normal[T]).max() < 1e-12


def test_coarse_rwg_is_exact_in_the_fine_basis():
    r = ref(1)
    c, f = r.coarse, r.fine
    rng = np.random.default_rng(0)
    for tau in range(0, f.nt, 7):
        T = int(r.parent[tau])
        bary = rng.dirichlet(np.ones(3), size=4)
        pts = bary @ f.verts[f.tris[tau]]
        vals, ks = CA.fine_basis_on_triangle(f, tau, pts)
        for m in c.tri_edge[T]:
            want = R.eval_basis(c, int(m), T, pts)
            got = sum(r.R[k, m] * vals[i] for i, k in enumerate(ks))
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def _vertex_normal(r, v):
    f = r.fine
    taus = np.nonzero(f.tris[:, 0] == v)[0]
    n = (f.normal[taus] * f.area[taus, None]).sum(0)
    return n / np.linalg.norm(n), taus


@pytest.mark.parametrize("level", [1, 2])
def test_bc_radial_fluxes_follow_the_closed_form(level):
    r = ref(level)
    c, f = r.coarse, r.fine
    nv = len(c.verts)
    for e in range(0, c.ne, 5 if level == 1 else 37):
        tri = list(c.tris[c.tplus[e]])
        i = [j for j in range(3) if {tri[j], tri[(j + 1) % 3]} == set(c.edges[e])][0]
        a, b = tri[i], tri[(i + 1) % 3]
        for v, sgn in ((a, -1.0), (b, 1.0)):  # ccw fluxes: sink cell +, source cell -
            nvec, taus = _vertex_normal(r, v)
            N = len(taus)
            d0 = f.verts[nv + e] - c.verts[v]
            radial = [k for k in range(f.ne) if v in f.edges[k]]
            assert len(radial) == N
            ang = []
            for k in radial:
                w = f.verts[f.edges[k].sum() - v] - c.verts[v]
                ang.append(np.arctan2(np.cross(d0, w) @ nvec, d0 @ w) % (2 * np.pi))
            order = np.argsort(ang)
            assert ang[order[0]] < 1e-9  # the radial edge along e itself comes first
            for idx, j in enumerate(order):
                k = radial[j]
                w = f.verts[f.edges[k].sum() - v] - c.verts[v]
                pm = f.verts[f.pminus[k]] - c.verts[v]
                ccw_side_minus = np.cross(w, pm) @ nvec > 0
                flux = r.C[k, e] * f.length[k] * (1.0 if ccw_side_minus else -1.0)
                want = 0.0 if idx == 0 else sgn * c.length[e] * (0.5 - idx / N)
                assert abs(flux - want) <= 1e-12 * c.length[e], (e, v, idx, flux, want)


def test_bc_divergence_is_constant_per_triangle_on_the_two_cells():
    r = ref(1)
    c, f = r.coarse, r.fine
    for e in range(c.ne):
        charge = np.zeros(f.nt)
        for tau in range(f.nt):
            for s in range(3):
                k = f.tri_edge[tau, s]
                charge[tau] += r.C[k, e] * f.length[k] * f.tri_sign[tau, s]
        a, b = c.edges[e]
        for v in (a, b):
            cell = f.tris[:, 0] == v
            q = charge[cell]
            assert np.allclose(q, q[0], atol=1e-13) and abs(abs(q.sum()) - c.length[e]) < 1e-12
        assert np.abs(charge[(f.tris[:, 0] != a) & (f.tris[:, 0] != b)]).max() < 1e-13
        assert abs(charge.sum()) < 1e-12


def test_mixed_gram_is_well_conditioned_and_rwg_pairing_antisymmetric():
    conds = []
    for level in (1, 2):
        r = ref(level)
        G = CA.mixed_gram(r)
        conds.append(np.linalg.cond(G))
        assert np.all(np.diag(G) > 0)
        Gf = CA.fine_rotated_gram(r.fine)
        rr = r.R.T @ Gf @ r.R  # <n x f_m, f_n> on the coarse RWG functions
        assert np.abs(rr + rr.T).max() <= 1e-12 * np.abs(rr).max()
    assert max(conds) < 5.0 and conds[1] < 1.3 * conds[0], conds


def _gmres_iterations(A, b):
    import scipy.sparse.linalg as sla

    count = [0]

    def cb(_):
        count[0] += 1

    sla.gmres(A, b, rtol=1e-6, restart=400, maxiter=2000, callback=cb, callback_type="pr_norm")
    return count[0]


def test_preconditioned_pmchwt_is_bounded_under_refinement():
    k0 = 2.0
    rows = []
    for level in (1, 2):
        r = ref(level)
        Z = O.pmchwt_matrix(r.coarse, k0, EPS)
        G = CA.mixed_gram(r)
        Zbc = CA.pmchwt_bc(r, k0, EPS)
        P = CA.preconditioner(G, Zbc)
        b = W.complex_normal(Z.shape[0], seed=1)
        z = np.zeros_like(G)
        Gb = np.block([[G, z], [z, G]])
        Pbad = -np.linalg.solve(Gb, Zbc @ np.linalg.inv(Gb))  # G^-1 where G^-T belongs
        rows.append((np.linalg.cond(Z), np.linalg.cond(Z @ P), np.linalg.cond(Z @ Pbad),
                     _gmres_iterations(Z, b), _gmres_iterations(Z @ P, b)))
    (cz1, cp1, cb1, iz1, ip1), (cz2, cp2, cb2, iz2, ip2) = rows
    print(rows)
    assert cz2 > 3.0 * cz1                      # Z: h^-2 growth (factor 4 per level)
    assert cp2 < 1.2 * cp1 and cp2 < 10.0       # Z P: bounded
    assert iz2 > 1.5 * iz1 and ip2 <= ip1 + 2   # iterations: growing vs flat
    assert ip2 < 0.3 * iz2
    assert cb2 > 1.5 * cb1                      # with the slip the growth comes back
