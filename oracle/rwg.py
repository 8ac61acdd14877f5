"""Mesh -> RWG edge table (oracle, test infrastructure).

Sec. III expands the surface currents in piecewise-linear bases lambda_i on a
mesh of the boundary.  On a triangulated closed surface the 3-D counterpart is
the Rao-Wilton-Glisson function of an interior edge n shared by triangles
T+ and T-:

    f_n(r) = +l_n / (2 A+) (r - p+)   on T+,     div f_n = +l_n / A+
    f_n(r) = -l_n / (2 A-) (r - p-)   on T-,     div f_n = -l_n / A-

with p+/- the vertex of T+/- opposite the edge.  Conventions fixed here:
  * edges are numbered in lexicographic order of (min vertex, max vertex);
  * T+ is the adjacent triangle with the smaller index;
  * the mesh must be closed, two-manifold, consistently oriented (every edge
    traversed in opposite directions by its two triangles) with no
    degenerate triangle (twice its area <= 1e-12 x its longest edge squared);
    otherwise ``MeshError`` is raised.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


class MeshError(ValueError):
    pass


@dataclass
class RWG:
    verts: np.ndarray      # (nv,3) float64
    tris: np.ndarray       # (nt,3) int64
    edges: np.ndarray      # (ne,2) vertex indices, edges[:,0] < edges[:,1]
    tplus: np.ndarray      # (ne,) triangle T+
    tminus: np.ndarray     # (ne,) triangle T-
    pplus: np.ndarray      # (ne,) free vertex of T+
    pminus: np.ndarray     # (ne,) free vertex of T-
    length: np.ndarray     # (ne,) edge length
    area: np.ndarray       # (nt,) triangle area
    normal: np.ndarray     # (nt,3) unit outward normal
    tri_edge: np.ndarray   # (nt,3) edge opposite local vertex i
    tri_sign: np.ndarray   # (nt,3) +1 if the triangle is T+ of that edge, -1 if T-

    @property
    def ne(self) -> int:
        return len(self.edges)

    @property
    def nt(self) -> int:
        return len(self.tris)

    def midpoints(self) -> np.ndarray:
        """Edge midpoints (ne,3), computed as (v0 + v1) * 0.5."""
        return (self.verts[self.edges[:, 0]] + self.verts[self.edges[:, 1]]) * 0.5


def build(verts, tris) -> RWG:
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    nt = len(tris)
    if verts.ndim != 2 or verts.shape[1] != 3 or tris.ndim != 2 or tris.shape[1] != 3:
        raise MeshError("verts must be (nv,3) and tris (nt,3)")
    if nt == 0:
        raise MeshError("empty mesh")
    if tris.min() < 0 or tris.max() >= len(verts):
        raise MeshError("triangle index out of range")
    if np.any(tris[:, 0] == tris[:, 1]) or np.any(tris[:, 1] == tris[:, 2]) or np.any(tris[:, 0] == tris[:, 2]):
        raise MeshError("degenerate triangle (repeated vertex)")
    p0, p1, p2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    cr = np.cross(p1 - p0, p2 - p0)
    dbl = np.linalg.norm(cr, axis=1)
    lmax2 = np.max(np.stack([np.sum((p1 - p0) ** 2, 1), np.sum((p2 - p1) ** 2, 1), np.sum((p0 - p2) ** 2, 1)]), axis=0)
    if np.any(dbl <= 1e-12 * lmax2):
        raise MeshError("zero-area triangle (twice the area <= 1e-12 x longest edge squared)")
    area = 0.5 * dbl
    normal = cr / dbl[:, None]

    # directed half-edges: local vertex i is opposite the edge (v[i+1], v[i+2])
    occ = {}
    for t in range(nt):
        for i in range(3):
            a = int(tris[t, (i + 1) % 3])
            b = int(tris[t, (i + 2) % 3])
            key = (a, b) if a < b else (b, a)
            occ.setdefault(key, []).append((t, i, a < b))
    keys = sorted(occ.keys())
    ne = len(keys)
    edges = np.array(keys, dtype=np.int64)
    tplus = np.empty(ne, np.int64)
    tminus = np.empty(ne, np.int64)
    pplus = np.empty(ne, np.int64)
    pminus = np.empty(ne, np.int64)
    tri_edge = np.empty((nt, 3), np.int64)
    tri_sign = np.empty((nt, 3), np.int64)
    for e, key in enumerate(keys):
        uses = occ[key]
        if len(uses) != 2:
            raise MeshError(f"edge {key} is shared by {len(uses)} triangles (mesh not closed two-manifold)")
        (ta, ia, fa), (tb, ib, fb) = uses
        if fa == fb:
            raise MeshError(f"edge {key} has inconsistent orientation")
        if ta == tb:
            raise MeshError(f"edge {key} used twice by triangle {ta}")
        if tb < ta:
            ta, ia, tb, ib = tb, ib, ta, ia
        tplus[e], tminus[e] = ta, tb
        pplus[e], pminus[e] = tris[ta, ia], tris[tb, ib]
        tri_edge[ta, ia], tri_sign[ta, ia] = e, 1
        tri_edge[tb, ib], tri_sign[tb, ib] = e, -1
    length = np.linalg.norm(verts[edges[:, 1]] - verts[edges[:, 0]], axis=1)
    return RWG(verts, tris, edges, tplus, tminus, pplus, pminus, length, area, normal, tri_edge, tri_sign)


def eval_basis(rwg: RWG, n: int, tri: int, r: np.ndarray) -> np.ndarray:
    """Value of f_n at points r (..,3) lying on triangle ``tri`` (zero off its support)."""
    if tri == rwg.tplus[n]:
        return (rwg.length[n] / (2.0 * rwg.area[tri])) * (r - rwg.verts[rwg.pplus[n]])
    if tri == rwg.tminus[n]:
        return -(rwg.length[n] / (2.0 * rwg.area[tri])) * (r - rwg.verts[rwg.pminus[n]])
    return np.zeros_like(r)
