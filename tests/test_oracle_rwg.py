"""Pins of the oracle's RWG edge table and mesh validation."""
import numpy as np
import pytest

import workloads as W
from oracle import power, quadrature, rwg as R


@pytest.mark.parametrize("level", [0, 1, 2])
def test_counts_and_order(level):
    v, t = W.icosphere(level)
    g = R.build(v, t)
    assert g.nt == 20 * 4 ** level
    assert g.ne == 3 * g.nt // 2
    key = g.edges[:, 0] * (len(v) + 1) + g.edges[:, 1]
    assert np.all(np.diff(key) > 0)                     # lexicographic, no duplicates
    assert np.all(g.tplus < g.tminus)
    # outward normals on a sphere centred at 0
    cen = v[t].mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", g.normal, cen) > 0)


def test_basis_properties():
    v, t = W.icosphere(1)
    g = R.build(v, t)
    bary, w = quadrature.rule7()
    for n in range(g.ne):
        # zero net charge: int div f = l - l = 0; and int over T+ of div f = l
        assert abs(g.length[n] / g.area[g.tplus[n]] * g.area[g.tplus[n]] - g.length[n]) < 1e-15
        # normal component across the shared edge is continuous and equals 1
        a, b = g.verts[g.edges[n, 0]], g.verts[g.edges[n, 1]]
        for s in (0.2, 0.5, 0.8):
            p = (1 - s) * a + s * b
            fp = R.eval_basis(g, n, g.tplus[n], p)
            fm = R.eval_basis(g, n, g.tminus[n], p)
            # in-plane unit vector of T+ perpendicular to the edge pointing away from p+
            tang = (b - a) / np.linalg.norm(b - a)
            mp = np.cross(tang, g.normal[g.tplus[n]])
            if np.dot(mp, p - g.verts[g.pplus[n]]) < 0:
                mp = -mp
            mm = np.cross(tang, g.normal[g.tminus[n]])
            if np.dot(mm, g.verts[g.pminus[n]] - p) < 0:
                mm = -mm
            assert abs(np.dot(fp, mp) - 1.0) < 1e-12
            assert abs(np.dot(fm, mm) - 1.0) < 1e-12


def test_gram_diagonal_closed_form():
    # int_T |r - p|^2 dS = A/6 (|e1|^2 + e1.e2 + |e2|^2) with e1, e2 the edges leaving p
    v, t = W.icosphere(1)
    g = R.build(v, t)
    loc = power.gram_local(g)
    for tri in range(g.nt):
        for i in range(3):
            p = g.verts[g.tris[tri, i]]
            e1 = g.verts[g.tris[tri, (i + 1) % 3]] - p
            e2 = g.verts[g.tris[tri, (i + 2) % 3]] - p
            l = g.length[g.tri_edge[tri, i]]
            A = g.area[tri]
            exact = (l / (2 * A)) ** 2 * A / 6 * (e1 @ e1 + e1 @ e2 + e2 @ e2)
            assert abs(loc[tri, i, i] - exact) < 1e-14 * max(1.0, exact)


def test_mesh_errors():
    v, t = W.icosphere(1)
    with pytest.raises(R.MeshError):
        R.build(v, t[1:])                               # open surface
    bad = t.copy()
    bad[3] = bad[3][[0, 2, 1]]
    with pytest.raises(R.MeshError):
        R.build(v, bad)                                 # inconsistent orientation
    vz = v.copy()
    tz = t.copy()
    vz[tz[0, 2]] = 0.5 * (vz[tz[0, 0]] + vz[tz[0, 1]])  # collapse a triangle
    with pytest.raises(R.MeshError):
        R.build(vz, tz)
    with pytest.raises(R.MeshError):
        R.build(v, np.zeros((0, 3), dtype=np.int32))


def test_box_mesh_closed():
    v, t = W.box_mesh(2.0, 1.5, 0.5, 4, 3, 2)
    g = R.build(v, t)
    assert g.nt == 4 * (4 * 3 + 4 * 2 + 3 * 2)
    cen = v[t].mean(axis=1) - np.array([1.0, 0.75, 0.25])
    assert np.all(np.einsum("ij,ij->i", g.normal, cen) > 0)
